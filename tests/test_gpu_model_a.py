"""GPU parity of the concentration scatter ("model A", Eq. LogNormC) against
the FP64 oracle, through the C ABI.

Same bar as the model-B parity tests: tables, spectra and every covariance
term to 1e-10 (|dC_ab| <= 1e-10 sqrt(C_aa C_bb)), S/N to relative 1e-10 in the
FP64 form; the split-BF16 tensor-core form to 1e-4 per element and 1e-3 on the
S/N.  A rule of one concentration node is model B bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import halo  # noqa: E402
from oracle.covariance import TERM_1H, TERM_BBPT, TERM_G, TERM_PB, TERM_SSC, TERMS_ALL  # noqa: E402
from oracle.pipeline import OracleRun  # noqa: E402
from oracle.snr import WHICH_B, WHICH_JOINT, WHICH_P, cumulative_snr  # noqa: E402
from paper_1812_07437_gb300 import native as N  # noqa: E402
from paper_1812_07437_gb300 import workloads  # noqa: E402

TOL = 1e-10
CASES = {"tiny_2bin": 8, "mid_2bin": 4}  # workload -> concentration nodes
_O, _H = {}, {}


def _wl(name, n_conc=None):
    return workloads.get(name, bins=dict(n_conc=CASES[name] if n_conc is None else n_conc,
                                         sigma_lnc=workloads.SIGMA_LNC))


def oracle(name):
    if name not in _O:
        _O[name] = OracleRun(_wl(name))
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


@pytest.mark.parametrize("name", list(CASES))
def test_tables_and_spectra_match_oracle(name):
    h, r = handle(name), oracle(name)
    T, nc = r.T, CASES[name]
    s, w = halo.conc_rule(nc, workloads.SIGMA_LNC)
    close(h.table("conc_offsets"), s, 1e-13, 1e-15)
    close(h.table("conc_weights"), w, 1e-12, 1e-15)
    close(h.table("mass"), np.repeat(T.m, nc), 1e-14)
    close(h.table("f"), np.repeat(T.f, nc, axis=1), 1e-11)
    close(h.table("b1"), np.repeat(T.b1, nc, axis=1), 1e-11)
    close(h.table("b2"), np.repeat(T.b2, nc, axis=1), 1e-10, 1e-12)
    close(h.table("U"), T.U, 1e-11, 1e-13)
    D = torch.zeros(h.M, dtype=torch.float64, device="cuda:0")
    h.spectra(D)
    torch.cuda.synchronize()
    for t in ("P3", "RP3", "B3", "B1h3", "Ps", "B1h"):
        close(h.table(t), getattr(r.S, t))
    close(h.table("RB3"), r.S.RB3, TOL, 1e-12)
    close(D.cpu().numpy(), r.D)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("terms", [TERM_G, TERM_1H, TERM_BBPT, TERM_PB, TERM_SSC, TERMS_ALL])
def test_covariance_terms_match_oracle(name, terms):
    h, r = handle(name), oracle(name)
    Cg, _ = _cov(h, terms)
    Co = r.cov.full(terms)
    d = np.sqrt(np.diag(r.cov.full(TERMS_ALL) if terms != TERMS_ALL else Co))
    err = np.abs(Cg - Co) / np.outer(d, d)
    assert np.all(np.isfinite(Cg))
    assert err.max() <= TOL, f"{name} terms={terms}: max normalised err {err.max():.3e}"


@pytest.mark.parametrize("name", list(CASES))
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


def test_one_concentration_node_is_model_b_bitwise():
    from paper_1812_07437_gb300.handle import Handle
    hb = Handle(workloads.get("tiny_2bin"))
    h1 = Handle(_wl("tiny_2bin", n_conc=1))
    for t in ("mass", "f", "b1", "b2", "U"):
        assert np.array_equal(h1.table(t), hb.table(t)), t
    for precision in (N.COV_FP64, N.COV_SPLIT_BF16):
        Cb, Db = _cov(hb, TERMS_ALL, precision)
        C1, D1 = _cov(h1, TERMS_ALL, precision)
        assert np.array_equal(Cb, C1) and torch.equal(Db, D1)
    hb.close()
    h1.close()


def test_largest_rule_and_zero_width():
    """The largest concentration rule the API takes (32 nodes): the rule and the
    data vector against the oracle; a zero-width lognormal (sigma_lnc = 0, all
    nodes at the median) reproduces model B to rounding."""
    from paper_1812_07437_gb300.handle import Handle
    wl = workloads.get("tiny_2bin", bins=dict(n_conc=32, sigma_lnc=workloads.SIGMA_LNC))
    h, r = Handle(wl), OracleRun(wl)
    s, w = halo.conc_rule(32, workloads.SIGMA_LNC)
    close(h.table("conc_offsets"), s, 1e-13, 1e-15)
    close(h.table("conc_weights"), w, 1e-12, 1e-15)
    D = torch.zeros(h.M, dtype=torch.float64, device="cuda:0")
    h.spectra(D)
    torch.cuda.synchronize()
    close(D.cpu().numpy(), r.D)
    h.close()
    hb = Handle(workloads.get("tiny_2bin"))
    h0 = Handle(workloads.get("tiny_2bin", bins=dict(n_conc=8, sigma_lnc=0.0)))
    Cb, Db = _cov(hb, TERMS_ALL)
    C0, D0 = _cov(h0, TERMS_ALL)
    d = np.sqrt(np.diag(Cb))
    assert np.max(np.abs(C0 - Cb) / np.outer(d, d)) <= 1e-13
    assert torch.max(torch.abs(D0 / Db - 1)).item() <= 1e-13
    hb.close()
    h0.close()
