"""GPU checks of the serving loop (cov_server_*): continuous batching.

* Each request's S/N is the same alone (one slot, one request at a time) and
  in a mix (several slots, every request submitted at once, kernels of
  different requests overlapping on the GPU): within 1e-10 relative.
* A served request equals the same covariance + S/N computed directly with a
  handle (cov_init, cov_spectra, cov_assemble, cov_snr), within 1e-10.
* Requests overlap in time and reuse resident state for a repeated binning;
  the reserved bytes stay within the budget.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1812_07437_gb300 import native as N  # noqa: E402
from paper_1812_07437_gb300 import workloads  # noqa: E402

TOL = 1e-10


def _mix():
    out = []
    for k, name in enumerate(["mid_3bin", "tiny_2bin", "mid_2bin", "cfg1_1bin", "tiny_2bin", "mid_3bin",
                              "cfg2_5bin"]):
        c = dict(workloads.FIDUCIAL)
        c["sigma8"] *= 1.0 + 0.02 * ((k % 3) - 1)
        c["Om"] *= 1.0 + 0.01 * (k % 2)
        out.append(workloads.get(name, cosmology=c))
    return out


def _rel(a, b):
    m = np.isfinite(b)
    assert np.array_equal(m, np.isfinite(a))
    return float(np.max(np.abs(a[m] / b[m] - 1.0))) if m.any() else 0.0


@pytest.fixture(scope="module")
def alone():
    from paper_1812_07437_gb300.server import Server
    s = Server(n_slots=1, precision=N.COV_SPLIT_BF16)
    res = []
    for wl in _mix():
        i = s.submit(wl)
        info, snr = s.wait(i, timeout=300.0)
        assert info["state"] == N.COV_REQ_DONE, s.error(i)
        res.append(snr)
    s.close()
    return res


def test_results_same_alone_and_in_the_mix(alone):
    from paper_1812_07437_gb300.server import Server
    s = Server(n_slots=4, precision=N.COV_SPLIT_BF16)
    ids = [s.submit(wl) for wl in _mix()]
    infos = []
    for k, i in enumerate(ids):
        info, snr = s.wait(i, timeout=300.0)
        assert info["state"] == N.COV_REQ_DONE, s.error(i)
        infos.append(info)
        for w in range(3):
            assert _rel(snr[w], alone[k][w]) <= TOL, (k, w)
    st = s.stats()
    s.close()
    assert st["max_running"] >= 2
    # at least two requests ran at overlapping times
    spans = sorted((x["t_start"], x["t_done"]) for x in infos)
    assert any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1))
    assert st["peak_reserved"] <= st["budget"]


def test_served_equals_direct_handle(alone):
    from paper_1812_07437_gb300.handle import Handle
    wl = _mix()[0]
    h = Handle(wl)
    D = torch.zeros(h.M, dtype=torch.float64, device="cuda:0")
    C = torch.zeros(h.M, h.M, dtype=torch.float64, device="cuda:0")
    h.spectra(D)
    h.assemble(C, N.COV_TERMS_ALL, N.COV_SPLIT_BF16)
    for w in range(3):
        assert _rel(alone[0][w], h.snr(C, D, w)) <= TOL
    h.close()


def test_repeated_binning_reuses_resident_state():
    from paper_1812_07437_gb300.server import Server
    s = Server(n_slots=1, precision=N.COV_SPLIT_BF16)
    a = s.submit(workloads.get("mid_2bin"))
    b = s.submit(workloads.get("mid_2bin", cosmology=dict(workloads.FIDUCIAL, sigma8=0.85)))
    ia, sa = s.wait(a, timeout=120.0)
    ib, sb = s.wait(b, timeout=120.0)
    assert ia["reused"] == 0 and ib["reused"] == 1
    assert not np.allclose(sa[2], sb[2])  # a different cosmology gives a different S/N
    s.close()
