"""GPU checks of the batched cosmologies entry point (cov_batch_snr).

The batch captures the cosmology-dependent step once, into the body of a
graph "while" node, and runs the other cosmologies as one graph launch (a
loop on the device); every cosmology's data vector and cumulative S/N must
equal those of the plain calls (cov_update, cov_spectra, cov_assemble,
cov_snr) for that cosmology, to 1e-10 relative, with and without the
launch-configuration tuning (the reference handle uses the contraction and
Cholesky kernels the tuner kept), in both precisions.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1812_07437_gb300 import native as N  # noqa: E402
from paper_1812_07437_gb300 import workloads  # noqa: E402

DEV = "cuda:0"
TOL = 1e-10


def _fisher_points(k):
    """Fiducial and +-1% steps in two parameters: a Fisher-style set."""
    out = [dict(workloads.FIDUCIAL)]
    for p in ("Om", "sigma8", "w0", "ns"):
        for s in (+1, -1):
            c = dict(workloads.FIDUCIAL)
            c[p] *= 1.0 + 0.01 * s
            out.append(c)
    return out[:k]


def _plain(h, cosmo, precision):
    D = torch.zeros(h.M, dtype=torch.float64, device=DEV)
    C = torch.zeros(h.M, h.M, dtype=torch.float64, device=DEV)
    h.update(cosmo)
    h.spectra(D)
    h.assemble(C, N.COV_TERMS_ALL, precision)
    snr = np.stack([h.snr(C, D, w) for w in (N.COV_WHICH_P, N.COV_WHICH_B, N.COV_WHICH_JOINT)])
    return D.cpu().numpy(), snr


def _rel(a, b):
    m = np.isfinite(b)
    assert np.array_equal(m, np.isfinite(a))
    return float(np.max(np.abs(a[m] / b[m] - 1.0))) if m.any() else 0.0


@pytest.mark.parametrize("name,precision,tune", [("mid_3bin", N.COV_SPLIT_BF16, True),
                                                 ("mid_2bin", N.COV_FP64, False),
                                                 ("cfg2_5bin", N.COV_SPLIT_BF16, True)])
def test_batch_equals_plain_calls(name, precision, tune):
    from paper_1812_07437_gb300.handle import Handle
    cos = _fisher_points(5)
    h = Handle(workloads.get(name))
    snr, D, info = h.batch_snr(cos, precision=precision, with_D=True, tune=tune)
    assert info["replay_ms"] > 0 and info["capture_ms"] > 0
    assert info["single_launch"] == 1
    if tune:
        assert all(t > 0 for t in info["candidate_ms"])
    ref = Handle(workloads.get(name), tc_kernel=N.COV_TC_SINGLE if info["tc_kernel"] == 0 else N.COV_TC_AUTO,
                 chol_kernel=info["chol_kernel"])
    for k, c in enumerate(cos):
        Dk, sk = _plain(ref, c, precision)
        assert np.max(np.abs(D[k] / Dk - 1.0)) <= TOL, k
        for w in range(3):
            assert _rel(snr[k, w], sk[w]) <= TOL, (k, w)
    # different cosmologies give different results
    assert not np.allclose(snr[0, 2], snr[1, 2])
    h.close()
    ref.close()
