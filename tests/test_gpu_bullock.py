"""GPU parity of the Bullock et al. median concentration (Sec. 5.4) and of the
paper's own set-up against the FP64 oracle, through the C ABI.

* tiny_2bin with the Bullock median (model B): tables, spectra, every
  covariance term and the S/N to 1e-10.
* paper_2bin: the paper's cosmology, 14 ell bins on [10, 5000], m_min = 1e9,
  Bullock median with the lognormal scatter (model A, 4 nodes), M = 818 rows
  (four 256-row tiles, ragged tail): the same bar in FP64, 1e-4 per element
  and 1e-3 on the S/N in the split-BF16 form.  Its exact triangle counts come
  from the oracle's stored file (tests/golden/make_counts.py).
* paper_2bin_full: the same set-up at the paper-replica quadrature, its
  cumulative S/N against the oracle's stored curve (tests/golden/make_snr.py).
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.covariance import TERM_1H, TERM_BBPT, TERM_G, TERM_PB, TERM_SSC, TERMS_ALL  # noqa: E402
from oracle.pipeline import OracleRun  # noqa: E402
from oracle.snr import WHICH_B, WHICH_JOINT, WHICH_P, cumulative_snr  # noqa: E402
from paper_1812_07437_gb300 import native as N  # noqa: E402
from paper_1812_07437_gb300 import workloads  # noqa: E402

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_counts  # noqa: E402

TOL = 1e-10
_O, _H = {}, {}


def _wl(name):
    if name == "tiny_2bin":
        return workloads.get(name, bins=dict(conc_model=N.COV_CONC_BULLOCK))
    return workloads.get(name)


def oracle(name):
    if name not in _O:
        ntri = make_counts.load(name)[1] if name.startswith("paper") else None
        _O[name] = OracleRun(_wl(name), ntri=ntri)
    return _O[name]


def handle(name):
    from paper_1812_07437_gb300.handle import Handle
    if name not in _H:
        _H[name] = Handle(_wl(name), device=0)
    return _H[name]


def close(got, ref, rtol=TOL, floor=1e-13):
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    assert got.shape == ref.shape
    scale = np.max(np.abs(ref)) if ref.size else 0.0
    err = np.abs(got - ref)
    ok = err <= rtol * np.abs(ref) + floor * scale
    assert np.all(ok), f"max rel err {np.max(err / (np.abs(ref) + floor * scale + 1e-300)):.3e}"


def _cov(h, terms, precision=N.COV_FP64):
    D = torch.zeros(h.M, dtype=torch.float64, device="cuda:0")
    h.spectra(D)
    C = torch.full((h.M, h.M), float("nan"), dtype=torch.float64, device="cuda:0")
    h.assemble(C, terms, precision)
    torch.cuda.synchronize()
    L = torch.tril(C).cpu().numpy()
    return L + np.tril(L, -1).T, D


CASES = ["tiny_2bin", "paper_2bin"]




@pytest.mark.parametrize("name", CASES)
def test_collapse_epoch_tables_and_spectra(name):
    h, r = handle(name), oracle(name)
    T = r.T
    close(h.table("collapse_a"), T.a_c, 1e-11)
    close(h.table("growth"), T.D, 1e-12)
    close(h.table("U"), T.U, 1e-11, 1e-13)
    ne, nt = h.counts()
    assert np.array_equal(ne, r.Nmodes) and np.array_equal(nt, r.Ntri)
    D = torch.zeros(h.M, dtype=torch.float64, device="cuda:0")
    h.spectra(D)
    torch.cuda.synchronize()
    for t in ("P3", "RP3", "B3", "B1h3", "Ps", "B1h"):
        close(h.table(t), getattr(r.S, t))
    close(h.table("RB3"), r.S.RB3, TOL, 1e-12)
    close(D.cpu().numpy(), r.D)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("terms", [TERM_G, TERM_1H, TERM_BBPT, TERM_PB, TERM_SSC, TERMS_ALL])
def test_covariance_terms_match_oracle(name, terms):
    h, r = handle(name), oracle(name)
    Cg, _ = _cov(h, terms)
    Co = r.cov.full(terms)
    d = np.sqrt(np.diag(r.cov.full(TERMS_ALL) if terms != TERMS_ALL else Co))
    err = np.abs(Cg - Co) / np.outer(d, d)
    assert np.all(np.isfinite(Cg))
    assert err.max() <= TOL, f"{name} terms={terms}: max normalised err {err.max():.3e}"


@pytest.mark.parametrize("name", CASES)
def test_snr_matches_oracle_both_precisions(name):
    h, r = handle(name), oracle(name)
    Co = r.cov.full(TERMS_ALL)
    d = np.sqrt(np.diag(Co))
    n_ell = len(r.T.ell)
    for precision, ctol, stol in ((N.COV_FP64, TOL, TOL), (N.COV_SPLIT_BF16, 1e-4, 1e-3)):
        Cg, D = _cov(h, TERMS_ALL, precision)
        assert np.max(np.abs(Cg - Co) / np.outer(d, d)) <= ctol
        Ct = torch.tensor(Cg, device="cuda:0")
        for which, ow in ((N.COV_WHICH_P, WHICH_P), (N.COV_WHICH_B, WHICH_B), (N.COV_WHICH_JOINT, WHICH_JOINT)):
            got = h.snr(Ct, D, which)
            ref = cumulative_snr(Co, r.D, r.rows, n_ell, ow)
            m = np.isfinite(ref)
            assert np.array_equal(m, np.isfinite(got))
            assert np.max(np.abs(got[m] / ref[m] - 1)) <= stol, (precision, which)


def test_paper_set_up_at_full_quadrature_matches_stored_oracle_snr():
    """The paper's 2-bin set-up at the quadrature of the paper-replica runs
    (N_chi = 128, N_M = 96, Bullock median, M = 818): cumulative S/N of P, B and
    the joint vector in the FP64 form against the oracle's stored curve
    (tests/golden/make_snr.py) to 1e-10."""
    import make_snr
    from paper_1812_07437_gb300.handle import Handle
    h = Handle(workloads.get("paper_2bin_full"))
    ref = make_snr.load("paper_2bin_full")
    C, D = _cov(h, N.COV_TERMS_ALL, N.COV_FP64)
    Ct = torch.tensor(C, device="cuda:0")
    for tag, w in (("P", N.COV_WHICH_P), ("B", N.COV_WHICH_B), ("J", N.COV_WHICH_JOINT)):
        got, r = h.snr(Ct, D, w), ref[tag]
        m = np.isfinite(r)
        assert np.array_equal(m, np.isfinite(got)) and np.max(np.abs(got[m] / r[m] - 1)) <= TOL, tag
    h.close()
