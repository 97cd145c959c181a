"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (FP64 path): tables, spectra and every covariance term agree to
1e-10, the covariance measured as |dC_ab| <= 1e-10 sqrt(C_aa C_bb); integer
counts are bit-exact; S/N agrees to relative 1e-10.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.covariance import TERM_1H, TERM_BBPT, TERM_G, TERM_PB, TERM_SSC, TERMS_ALL  # noqa: E402
from oracle.pipeline import OracleRun  # noqa: E402
from oracle.snr import WHICH_B, WHICH_JOINT, WHICH_P, cumulative_snr  # noqa: E402
from paper_1812_07437_gb300 import native as N  # noqa: E402
from paper_1812_07437_gb300 import workloads  # noqa: E402

TOL = 1e-10
_ORACLES = {}
_HANDLES = {}


def oracle(name):
    if name not in _ORACLES:
        _ORACLES[name] = OracleRun(workloads.get(name))
    return _ORACLES[name]


def handle(name):
    from paper_1812_07437_gb300.handle import Handle
    if name not in _HANDLES:
        _HANDLES[name] = Handle(workloads.get(name), device=0)
    return _HANDLES[name]


def close(got, ref, rtol=TOL, floor=1e-13):
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    assert got.shape == ref.shape
    scale = np.max(np.abs(ref)) if ref.size else 0.0
    err = np.abs(got - ref)
    ok = err <= rtol * np.abs(ref) + floor * scale
    assert np.all(ok), f"max rel err {np.max(err / (np.abs(ref) + floor * scale + 1e-300)):.3e}"


SMALL = ["tiny_2bin", "cfg1_1bin", "mid_2bin"]


@pytest.mark.parametrize("name", ["tiny_2bin", "cfg1_1bin"])
def test_tables_match_oracle(name):
    h, r = handle(name), oracle(name)
    T = r.T
    close(h.table("chi"), T.chi, 1e-14)
    close(h.table("wchi"), T.wchi, 1e-13)
    close(h.table("z"), T.z, 1e-13)
    close(h.table("growth"), T.D, 1e-12)
    close(h.table("mass"), T.m, 1e-14)
    close(h.table("f"), T.f, 1e-11)
    close(h.table("b1"), T.b1, 1e-11)
    close(h.table("b2"), T.b2, 1e-10, 1e-12)
    close(h.table("U"), T.U, 1e-11, 1e-13)
    close(h.table("Plin"), T.Pl, 1e-12)
    close(h.table("dPlin"), T.dPl, 1e-10, 1e-12)
    close(h.table("W"), T.W, 1e-11, 1e-14)
    close(h.table("zedges"), T.zedges, 1e-14)
    close(h.table("sigw2"), T.sigW2, 1e-11)


@pytest.mark.parametrize("name", SMALL)
def test_counts_bit_exact(name):
    h, r = handle(name), oracle(name)
    ne, nt = h.counts()
    assert np.array_equal(ne, r.Nmodes)
    assert np.array_equal(nt, r.Ntri)


@pytest.mark.parametrize("name", ["tiny_2bin", "cfg1_1bin"])
def test_spectra_match_oracle(name):
    h, r = handle(name), oracle(name)
    D = torch.zeros(h.M, dtype=torch.float64, device="cuda:0")
    h.spectra(D)
    torch.cuda.synchronize()
    S = r.S
    close(h.table("P3"), S.P3)
    close(h.table("RP3"), S.RP3)
    close(h.table("B3"), S.B3)
    close(h.table("RB3"), S.RB3, TOL, 1e-12)
    close(h.table("B1h3"), S.B1h3)
    close(h.table("Ps"), S.Ps)
    close(h.table("B1h"), S.B1h)
    close(D.cpu().numpy(), r.D)


def _gpu_cov(h, terms, precision=N.COV_FP64):
    D = torch.zeros(h.M, dtype=torch.float64, device="cuda:0")
    h.spectra(D)
    C = torch.full((h.M, h.M), float("nan"), dtype=torch.float64, device="cuda:0")
    h.assemble(C, terms, precision)
    torch.cuda.synchronize()
    L = torch.tril(C).cpu().numpy()
    return L + np.tril(L, -1).T, D


@pytest.mark.parametrize("name", SMALL)
@pytest.mark.parametrize("terms", [TERM_G, TERM_1H, TERM_BBPT, TERM_PB, TERM_SSC, TERMS_ALL])
def test_covariance_terms_match_oracle(name, terms):
    h, r = handle(name), oracle(name)
    Cg, _ = _gpu_cov(h, terms)
    Co = r.cov.full(terms)
    Call = r.cov.full(TERMS_ALL) if terms != TERMS_ALL else Co
    d = np.sqrt(np.diag(Call))
    err = np.abs(Cg - Co) / np.outer(d, d)
    assert np.all(np.isfinite(Cg))
    assert err.max() <= TOL, f"{name} terms={terms}: max normalised err {err.max():.3e}"


@pytest.mark.parametrize("name", SMALL)
def test_snr_matches_oracle(name):
    h, r = handle(name), oracle(name)
    Cg, D = _gpu_cov(h, TERMS_ALL)
    Ct = torch.tensor(Cg, device="cuda:0")
    Co = r.cov.full(TERMS_ALL)
    n_ell = len(r.T.ell)
    for which, ow in ((N.COV_WHICH_P, WHICH_P), (N.COV_WHICH_B, WHICH_B), (N.COV_WHICH_JOINT, WHICH_JOINT)):
        got = h.snr(Ct, D, which)
        ref = cumulative_snr(Co, r.D, r.rows, n_ell, ow)
        m = np.isfinite(ref)
        assert np.array_equal(m, np.isfinite(got))
        assert np.max(np.abs(got[m] / ref[m] - 1)) <= TOL


def test_not_positive_definite_reported():
    h = handle("tiny_2bin")
    D = torch.ones(h.M, dtype=torch.float64, device="cuda:0")
    C = torch.eye(h.M, dtype=torch.float64, device="cuda:0")
    C[1, 0] = 3.0  # |C_10| > sqrt(C_00 C_11): indefinite
    with pytest.raises(N.CovError) as e:
        h.snr(C, D, N.COV_WHICH_JOINT)
    assert e.value.code == N.COV_ERR_NOT_PD
    # the handle stays usable afterwards
    Cg, D2 = _gpu_cov(h, TERM_G)
    assert np.all(np.isfinite(Cg))


def test_update_cosmology_matches_fresh_init():
    from paper_1812_07437_gb300.handle import Handle
    wl = workloads.get("tiny_2bin")
    cos2 = dict(wl["cosmology"], Om=0.3, sigma8=0.8)
    h = Handle(wl)
    h.update(cos2)
    wl2 = workloads.get("tiny_2bin", cosmology=cos2)
    h2 = Handle(wl2)
    C1, _ = _gpu_cov(h, TERMS_ALL)
    C2, _ = _gpu_cov(h2, TERMS_ALL)
    assert np.array_equal(C1, C2)
    h.close()
    h2.close()
