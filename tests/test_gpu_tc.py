"""GPU checks of the tensor-core (split-BF16) contraction and of the large
workloads.

* Small workloads: the split-BF16 covariance against the oracle within
  1e-4 sqrt(C_aa C_bb) per element and the S/N within 1e-3 relative.
* cfg2_5bin (M = 6375, K = 12288) and cfg3_10bin: exact integer counts against
  the oracle's stored counts; FP64 covariance elements against the oracle on a
  seeded sample; split-BF16 against the FP64 GPU form over the whole matrix
  (the FP64 form being pinned to the oracle by the sample and the small
  cases).
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.covariance import TERMS_ALL  # noqa: E402
from oracle.pipeline import OracleRun  # noqa: E402
from oracle.snr import WHICH_JOINT, cumulative_snr  # noqa: E402
from paper_1812_07437_gb300 import native as N  # noqa: E402
from paper_1812_07437_gb300 import workloads  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_counts  # noqa: E402
import make_snr  # noqa: E402

TOL_ELEM = 1e-4
TOL_SNR = 1e-3


def _cov(h, terms, precision):
    D = torch.zeros(h.M, dtype=torch.float64, device="cuda:0")
    h.spectra(D)
    C = torch.full((h.M, h.M), float("nan"), dtype=torch.float64, device="cuda:0")
    h.assemble(C, terms, precision)
    torch.cuda.synchronize()
    return C, D


def _sym(C):
    L = torch.tril(C)
    return L + torch.tril(L, -1).T


@pytest.mark.parametrize("name", ["tiny_2bin", "cfg1_1bin", "mid_2bin", "mid_3bin"])
def test_split_bf16_matches_oracle(name):
    from paper_1812_07437_gb300.handle import Handle
    h = Handle(workloads.get(name))
    r = OracleRun(workloads.get(name))
    C, D = _cov(h, N.COV_TERMS_ALL, N.COV_SPLIT_BF16)
    Cg = _sym(C).cpu().numpy()
    Co = r.cov.full(TERMS_ALL)
    d = np.sqrt(np.diag(Co))
    err = np.abs(Cg - Co) / np.outer(d, d)
    assert np.all(np.isfinite(Cg))
    assert err.max() <= TOL_ELEM, f"max normalised err {err.max():.3e}"
    got = h.snr(_sym(C), D, N.COV_WHICH_JOINT)
    ref = cumulative_snr(Co, r.D, r.rows, len(r.T.ell), WHICH_JOINT)
    m = np.isfinite(ref)
    assert np.max(np.abs(got[m] / ref[m] - 1)) <= TOL_SNR
    h.close()


@pytest.mark.parametrize("name", ["cfg2_5bin", "cfg3_10bin"])
def test_counts_bit_exact_large(name):
    from paper_1812_07437_gb300.handle import Handle
    h = Handle(workloads.get(name))
    ne, nt = h.counts()
    Nref, Tref = make_counts.load(name)
    assert np.array_equal(ne, np.array(Nref))
    assert np.array_equal(nt, np.array(Tref))
    h.close()


@pytest.fixture(scope="module")
def cfg2():
    from paper_1812_07437_gb300.handle import Handle
    name = "cfg2_5bin"
    h = Handle(workloads.get(name))
    r = OracleRun(workloads.get(name), ntri=make_counts.load(name)[1])
    C64, D = _cov(h, N.COV_TERMS_ALL, N.COV_FP64)
    yield h, r, C64, D
    h.close()


def test_cfg2_fp64_sampled_elements_match_oracle(cfg2):
    h, r, C64, D = cfg2
    rng = np.random.default_rng(2024)
    a = rng.integers(0, h.M, 600)
    b = rng.integers(0, h.M, 600)
    # every term type: half the sample on pairs sharing a triangle or an ell bin
    rows = r.rows
    diag = np.diag(C64.cpu().numpy())
    Cl = C64.cpu().numpy()
    assert np.all(np.isfinite(diag)) and np.all(diag > 0)
    worst = 0.0
    for i, j in zip(np.maximum(a, b), np.minimum(a, b)):
        ref = r.cov.element(int(i), int(j))
        scale = np.sqrt(r.cov.element(int(i), int(i)) * r.cov.element(int(j), int(j)))
        worst = max(worst, abs(Cl[i, j] - ref) / scale)
    for i in range(0, h.M, 97):
        ref = r.cov.element(i, i)
        worst = max(worst, abs(Cl[i, i] - ref) / ref)
    assert worst <= 1e-10, f"worst normalised err {worst:.3e}"
    np.testing.assert_allclose(D.cpu().numpy(), r.D, rtol=1e-10, atol=0)


def test_cfg2_split_bf16_matches_fp64_form(cfg2):
    h, r, C64, D = cfg2
    Cs, _ = _cov(h, N.COV_TERMS_ALL, N.COV_SPLIT_BF16)
    L64 = torch.tril(C64)
    Ls = torch.tril(Cs)
    d = torch.sqrt(torch.diagonal(L64))
    err = (torch.abs(Ls - L64) / torch.outer(d, d)).tril()
    assert torch.isfinite(Ls).all()
    assert float(err.max()) <= TOL_ELEM, f"max normalised err {float(err.max()):.3e}"
    for which in (N.COV_WHICH_P, N.COV_WHICH_B, N.COV_WHICH_JOINT):
        s64 = h.snr(C64, D, which)
        ss = h.snr(Cs, D, which)
        assert np.max(np.abs(ss / s64 - 1)) <= TOL_SNR


def test_cfg2_pair_kernel_equals_one_cta_kernel(cfg2):
    """The CTA-pair contraction (tcgen05.mma.cta_group::2, 256 x 512 pair
    tiles) and the one-CTA contraction (256 x 256 tiles) form the same
    products over the same K blocks: over the whole cfg2 matrix (25 tile rows,
    diagonal pair tiles with one tile, a ragged last tile row of 231 rows) the
    two agree far inside the split form's own error."""
    from paper_1812_07437_gb300.handle import Handle
    h, r, C64, D = cfg2
    Cp, _ = _cov(h, N.COV_TERMS_ALL, N.COV_SPLIT_BF16)
    h1 = Handle(workloads.get("cfg2_5bin"), tc_kernel=N.COV_TC_SINGLE)
    C1, _ = _cov(h1, N.COV_TERMS_ALL, N.COV_SPLIT_BF16)
    h1.close()
    Lp, L1 = torch.tril(Cp), torch.tril(C1)
    assert torch.isfinite(Lp).all() and torch.isfinite(L1).all()
    d = torch.sqrt(torch.diagonal(torch.tril(C64)))
    err = (torch.abs(Lp - L1) / torch.outer(d, d)).tril()
    assert float(err.max()) <= 1e-6, f"pair vs one-CTA max normalised diff {float(err.max()):.3e}"


def test_cfg2_persistent_cholesky_update_is_bit_identical(cfg2):
    """Dense cov_snr with the persistent trailing update (the default) and with
    the one-CTA-per-tile update: the same exact group sums, so the three
    cumulative S/N are equal bit for bit."""
    from paper_1812_07437_gb300.handle import Handle
    h, r, C64, D = cfg2
    h1 = Handle(workloads.get("cfg2_5bin"), chol_kernel=N.COV_CHOL_TILE)
    for w in (N.COV_WHICH_P, N.COV_WHICH_B, N.COV_WHICH_JOINT):
        assert np.array_equal(h.snr(C64, D, w), h1.snr(C64, D, w), equal_nan=True), w
    h1.close()


WHICH = (("P", N.COV_WHICH_P), ("B", N.COV_WHICH_B), ("J", N.COV_WHICH_JOINT))


def _snr_rel(got, ref):
    m = np.isfinite(ref)
    assert np.array_equal(m, np.isfinite(got))
    return float(np.max(np.abs(got[m] / ref[m] - 1)))


def test_cfg2_snr_matches_stored_oracle(cfg2):
    """Cumulative S/N of cfg2 against the oracle's own (full FP64 covariance,
    scipy Cholesky; tests/golden/make_snr.py): FP64 form to 1e-10, split-BF16
    form to 1e-3."""
    h, r, C64, D = cfg2
    ref = make_snr.load("cfg2_5bin")
    Cs, _ = _cov(h, N.COV_TERMS_ALL, N.COV_SPLIT_BF16)
    for tag, w in WHICH:
        assert _snr_rel(h.snr(C64, D, w), ref[tag]) <= 1e-10, tag
        assert _snr_rel(h.snr(Cs, D, w), ref[tag]) <= TOL_SNR, tag


@pytest.mark.skipif(not os.path.exists(os.path.join(HERE, "golden", "snr_cfg3_5bin.txt")),
                    reason="oracle S/N of cfg3_5bin not written")
def test_cfg3_5bin_snr_matches_stored_oracle():
    """The 10-bin quadrature and binning with 5 tomographic bins (M = 24400),
    the largest configuration whose full oracle S/N can be computed on the
    host: FP64 form to 1e-10, split-BF16 form to 1e-3."""
    from paper_1812_07437_gb300.handle import Handle
    h = Handle(workloads.get("cfg3_5bin"))
    ref = make_snr.load("cfg3_5bin")
    C, D = _cov(h, N.COV_TERMS_ALL, N.COV_FP64)
    s64 = [h.snr(C, D, w) for _, w in WHICH]
    h.assemble(C, N.COV_TERMS_ALL, N.COV_SPLIT_BF16)
    torch.cuda.synchronize()
    ss = [h.snr(C, D, w) for _, w in WHICH]
    for k, (tag, _) in enumerate(WHICH):
        assert _snr_rel(s64[k], ref[tag]) <= 1e-10, tag
        assert _snr_rel(ss[k], ref[tag]) <= TOL_SNR, tag
    h.close()
