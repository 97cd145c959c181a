"""GPU parity of the exact BB+PT couplings (COV_COUPLING_EXACT; App. B, Eq.
CovBB) against the oracle (oracle/coupling.py).

* The integer Gram matrices of the leg counts are bit-exact: whole matrices on
  small binnings, sha256 digests plus diagonals and row sums on the
  cfg2_5bin and cfg3_10bin binnings (tests/golden/coupling_*.txt, written by
  make_coupling.py from the oracle alone).
* The covariance with the exact couplings matches the oracle's to 1e-10
  (normalised) term by term, and its S/N to 1e-10; the handle's couplings
  leave every other term unchanged (bit-identical to a COV_COUPLING_MODES
  handle), and BB+PT differs from it.
"""
import hashlib
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import coupling as cpl  # noqa: E402
from oracle.covariance import TERM_1H, TERM_BBPT, TERM_G, TERM_PB, TERM_SSC, TERMS_ALL  # noqa: E402
from oracle.pipeline import OracleRun  # noqa: E402
from oracle.snr import WHICH_B, WHICH_JOINT, WHICH_P, cumulative_snr  # noqa: E402
from paper_1812_07437_gb300 import native as N  # noqa: E402
from paper_1812_07437_gb300 import workloads  # noqa: E402

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
import make_coupling  # noqa: E402

TOL = 1e-10
_OR = {}
_H = {}


def oracle(name):
    if name not in _OR:
        _OR[name] = OracleRun(workloads.get(name), coupling="exact")
    return _OR[name]


def handle(name, coupling=N.COV_COUPLING_EXACT):
    from paper_1812_07437_gb300.handle import Handle
    key = (name, coupling)
    if key not in _H:
        _H[key] = Handle(workloads.get(name), device=0, coupling=coupling)
    return _H[key]


def _cov(h, terms):
    D = torch.zeros(h.M, dtype=torch.float64, device="cuda:0")
    h.spectra(D)
    C = torch.full((h.M, h.M), float("nan"), dtype=torch.float64, device="cuda:0")
    h.assemble(C, terms, N.COV_FP64)
    torch.cuda.synchronize()
    L = torch.tril(C).cpu().numpy()
    return L + np.tril(L, -1).T, D


@pytest.mark.parametrize("name", ["tiny_2bin", "cfg1_1bin"])
def test_gram_matrices_bit_exact(name):
    h, r = handle(name), oracle(name)
    cols, _ = cpl.columns(r.tris, len(r.Nmodes))
    for A in range(len(r.Nmodes)):
        gc, gG = h.coupling_gram(A)
        assert [tuple(c) for c in gc.tolist()] == cols[A]
        assert np.array_equal(gG, r.G[A])


@pytest.mark.parametrize("name", ["cfg2_5bin", "cfg3_10bin"])
def test_gram_matrices_bit_exact_benchmark_binnings(name):
    from paper_1812_07437_gb300.handle import Handle
    gold = make_coupling.load(name)
    # the couplings depend on the binning only: a coarse quadrature keeps the
    # handle's tables small
    wl = workloads.get(name, bins=dict(workloads.get(name)["bins"], n_chi=16, n_mass=12))
    h = Handle(wl, device=0, coupling=N.COV_COUPLING_EXACT)
    try:
        assert sorted(gold) == list(range(wl["bins"]["n_ell"]))
        for A, (sha, rows) in gold.items():
            gc, gG = h.coupling_gram(A)
            assert [tuple(c) for c in gc.tolist()] == [(y, z) for y, z, _, _ in rows]
            assert np.array_equal(np.diag(gG), [g for _, _, g, _ in rows])
            assert [sum(int(v) for v in row) for row in gG] == [s for _, _, _, s in rows]
            assert hashlib.sha256(np.ascontiguousarray(gG, dtype="<i8").tobytes()).hexdigest() == sha
    finally:
        h.close()


@pytest.mark.parametrize("name", ["tiny_2bin", "cfg1_1bin"])
@pytest.mark.parametrize("terms", [TERM_BBPT, TERMS_ALL])
def test_exact_coupling_covariance_matches_oracle(name, terms):
    h, r = handle(name), oracle(name)
    Cg, _ = _cov(h, terms)
    Co = r.cov.full(terms)
    Call = r.cov.full(TERMS_ALL) if terms != TERMS_ALL else Co
    d = np.sqrt(np.diag(Call))
    err = np.abs(Cg - Co) / np.outer(d, d)
    assert np.all(np.isfinite(Cg))
    assert err.max() <= TOL, f"{name} terms={terms}: max normalised err {err.max():.3e}"


@pytest.mark.parametrize("name", ["tiny_2bin", "cfg1_1bin"])
def test_exact_coupling_snr_matches_oracle(name):
    h, r = handle(name), oracle(name)
    Cg, D = _cov(h, TERMS_ALL)
    Ct = torch.tensor(Cg, device="cuda:0")
    Co = r.cov.full(TERMS_ALL)
    n_ell = len(r.T.ell)
    for which, ow in ((N.COV_WHICH_P, WHICH_P), (N.COV_WHICH_B, WHICH_B), (N.COV_WHICH_JOINT, WHICH_JOINT)):
        got = h.snr(Ct, D, which)
        ref = cumulative_snr(Co, r.D, r.rows, n_ell, ow)
        m = np.isfinite(ref)
        assert np.array_equal(m, np.isfinite(got))
        assert np.max(np.abs(got[m] / ref[m] - 1)) <= TOL


def test_only_the_bbpt_term_changes():
    name = "tiny_2bin"
    he, hm = handle(name), handle(name, N.COV_COUPLING_MODES)
    for terms in (TERM_G, TERM_1H, TERM_PB, TERM_SSC):
        Ce, _ = _cov(he, terms)
        Cm, _ = _cov(hm, terms)
        assert np.array_equal(Ce, Cm)
    Ce, _ = _cov(he, TERM_BBPT)
    Cm, _ = _cov(hm, TERM_BBPT)
    m = Cm != 0
    assert np.array_equal(m, Ce != 0)
    rel = np.abs(Ce[m] / Cm[m] - 1.0)
    assert 1e-4 < rel.max() < 0.3


def test_gram_requires_exact_handle():
    hm = handle("tiny_2bin", N.COV_COUPLING_MODES)
    with pytest.raises(N.CovError) as e:
        hm.coupling_gram(0)
    assert e.value.code == N.COV_ERR_INVALID
