"""Pins of the oracle's spectra, covariance terms and S/N (CPU only)."""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.special import j1

from oracle import cosmology as cz
from oracle import spectra as sp
from oracle.covariance import TERM_1H, TERM_BBPT, TERM_G, TERM_PB, TERM_SSC, TERMS_ALL, Covariance
from oracle.snr import WHICH_B, WHICH_JOINT, WHICH_P, cumulative_snr
from paper_1812_07437_gb300 import workloads


def test_halo_integrals_k_to_zero():
    """u -> 1 as k -> 0, so I_n^0 -> sum omega f~ (m/rho)^n and I_1^1 -> 1 (Eq. ImunuHalos)."""
    wl = workloads.get("tiny_2bin", bins=dict(ell_min=1e-4, ell_max=2e-4))
    T = sp.Tables(wl)
    for n in range(0, len(T.chi), 5):
        for mu in (1, 2, 3, 4, 6):
            ref = np.sum(T.om * T.f[n] * T.mr ** mu)
            assert T.I([0] * mu, mu, 0, n) == pytest.approx(ref, rel=1e-9)
        assert T.I([1], 1, 1, n) == pytest.approx(1.0, rel=1e-9)


def test_bpt_equilateral_and_homogeneity():
    """Tree-level B^PT: equilateral with constant P gives 12/7 P^2; for P ~ k^n
    sum_i dB/dln k_i = 2 n B (homogeneity), which pins the finite difference."""
    assert sp.bpt_from(1.0, 1.0, 1.0, 2.0, 2.0, 2.0) == pytest.approx(12.0 / 7.0 * 4.0, rel=1e-14)
    # squeezed-limit symmetry: F2 is symmetric in its two legs
    assert sp.F2(0.3, 0.7, 0.2) == pytest.approx(sp.F2(0.7, 0.3, 0.2), rel=1e-15)
    cos = workloads.FIDUCIAL
    amp = cz.plin_amplitude(cos)
    ks = [0.11, 0.17, 0.2]
    total = sum(sp.dbpt_dlnk(ks, 1.0, amp, cos, i) for i in range(3))
    lam = 1e-3
    f = lambda s: sp.bpt_from(*(k * math.exp(s) for k in ks),
                              *(float(cz.plin(k * math.exp(s), 1.0, amp, cos)) for k in ks))
    direct = (-f(2 * lam) + 8 * f(lam) - 8 * f(-lam) + f(-2 * lam)) / (12 * lam)
    assert total == pytest.approx(direct, rel=1e-8)


def test_sigma_w2_adaptive_quadrature():
    cos = workloads.FIDUCIAL
    amp = cz.plin_amplitude(cos)
    theta = math.acos(1 - 2 * 0.36)
    for chi in (50.0, 1500.0):
        got = sp.sigma_w2(np.array([chi]), np.array([1.0]), theta, amp, cos)[0]
        f = lambda le: (math.exp(le) ** 2 * (j1(math.exp(le) * chi * theta) / (math.exp(le) * chi * theta)) ** 2
                        * float(cz.plin(math.exp(le), 1.0, amp, cos)))
        ref = 4 / (2 * math.pi) * integrate.quad(f, sp.LNEPS_MIN, sp.LNEPS_MAX, limit=5000, epsrel=1e-10)[0]
        assert got == pytest.approx(ref, rel=1e-4)  # the fixed 4096-node rule under-resolves the far oscillating tail at ~1e-5


def test_gauss_constant_power(oracle_tiny):
    """Constant P^s = c: equilateral 6 c^3 Omega/N_tri, isosceles 2x, scalene 1x, PP 2c^2/N."""
    r = oracle_tiny
    cov = Covariance(r.T, r.S, r.rows, r.tris, r.Nmodes, r.Ntri)
    c = 3.0e-9
    cov.S = type("S", (), {})()
    cov.S.Ps = np.full_like(r.S.Ps, c)
    rows = r.rows
    seen = set()
    for a, row in enumerate(rows):
        if row[0] == "P":
            assert cov.gauss(row, row) == pytest.approx(2 * c * c / r.Nmodes[row[1]], rel=1e-14)
            continue
        a_, b_, c_ = row[2]
        kind = "eq" if a_ == b_ == c_ else ("iso" if (a_ == b_ or b_ == c_) else "sca")
        if kind in seen:
            continue
        seen.add(kind)
        mult = dict(eq=6, iso=2, sca=1)[kind]
        assert cov.gauss(row, row) == pytest.approx(mult * c ** 3 * r.T.omega / r.Ntri[row[1]], rel=1e-14)
    assert seen == {"eq", "iso", "sca"}


def _set_partitions_two_blocks(items):
    """All splits of ``items`` into two non-empty blocks (unordered)."""
    items = list(items)
    first, rest = items[0], items[1:]
    out = []
    for r in range(0, len(rest) + 1):
        for comb in itertools.combinations(rest, r):
            blk = [first] + list(comb)
            other = [x for x in rest if x not in comb]
            if other:
                out.append((blk, other))
    return out


def _wick_reference(r, row1, row2):
    """BB+PT or PB term by enumerating every connected 2-block split of the
    legs (Wick decomposition of the 6- or 5-point function, Appendix B)."""
    S, T = r.S, r.T
    cov = r.cov
    tri_index = {tuple(t): i for i, t in enumerate(r.tris)}

    def legs(row, tag):
        if row[0] == "P":
            return [(tag, 0, row[1], row[2][0]), (tag, 1, row[1], row[2][1])]
        return [(tag, x, row[2][x], row[3][x]) for x in range(3)]

    L = legs(row1, "u") + legs(row2, "p")
    total = 0.0
    for A, B in _set_partitions_two_blocks(L):
        if not all({l[0] for l in blk} == {"u", "p"} for blk in (A, B)):
            continue  # a block inside one estimator is the disconnected mean
        sizes = sorted((len(A), len(B)))
        small = A if len(A) <= len(B) else B
        big = B if small is A else A
        if sizes == [3, 3]:
            # each 3-block closes only if its lone leg matches a leg of the other estimator
            lone = [l for l in A if sum(1 for x in A if x[0] == l[0]) == 1][0]
            mate = [l for l in B if sum(1 for x in B if x[0] == l[0]) == 1][0]
            if lone[2] != mate[2]:
                continue
            vals = []
            for blk in (A, B):
                key = tuple(sorted(l[2] for l in blk))
                t = tri_index[key]
                tom = [l[3] for l in blk]
                vals.append(S.B1h[t, tom[0], tom[1], tom[2]])
            total += vals[0] * vals[1] / r.Nmodes[lone[2]]
        elif sizes == [2, 4] or sizes == [2, 3]:
            if small[0][2] != small[1][2]:
                continue
            b = small[0][2]
            pst = S.Ps[b, small[0][3], small[1][3]]
            if len(big) == 4:
                total += pst * cov.polyspec_1h([l[2] for l in big], [l[3] for l in big]) / r.Nmodes[b]
            else:
                key = tuple(sorted(l[2] for l in big))
                t = tri_index[key]
                tom = [l[3] for l in big]
                total += pst * S.B1h[t, tom[0], tom[1], tom[2]] / r.Nmodes[b]
    return total


def test_bbpt_pb_match_wick_enumeration(oracle_tiny):
    r = oracle_tiny
    rng = np.random.default_rng(7)
    rows = r.rows
    b_rows = [a for a, x in enumerate(rows) if x[0] == "B"]
    p_rows = [a for a, x in enumerate(rows) if x[0] == "P"]
    checked = 0
    for _ in range(400):
        a, b = rng.choice(b_rows), rng.choice(b_rows)
        ref = _wick_reference(r, rows[a], rows[b])
        got = r.cov.bbpt(rows[a], rows[b])
        assert got == pytest.approx(ref, rel=1e-12, abs=1e-300)
        checked += ref != 0.0
    for _ in range(200):
        a, b = rng.choice(p_rows), rng.choice(b_rows)
        ref = _wick_reference(r, rows[a], rows[b])
        assert r.cov.pb(rows[a], rows[b]) == pytest.approx(ref, rel=1e-12, abs=1e-300)
        assert r.cov.pb(rows[b], rows[a]) == pytest.approx(ref, rel=1e-12, abs=1e-300)
        checked += ref != 0.0
    assert checked > 100


def test_covariance_symmetric_pd_and_block_forms(oracle_tiny):
    r = oracle_tiny
    C = r.cov.full(TERMS_ALL)
    assert np.allclose(C, C.T, rtol=1e-13, atol=0)
    d = np.sqrt(np.diag(C))
    assert np.linalg.eigvalsh(C / np.outer(d, d)).min() > 0
    rng = np.random.default_rng(3)
    C1 = r.cov.one_halo_block()
    F = r.cov.ssc_rows()
    Cs = F @ F.T
    for _ in range(200):
        a, b = rng.integers(0, r.M, 2)
        e = r.cov.element_terms(a, b)
        scale = math.sqrt(C[a, a] * C[b, b])
        assert abs(e[TERM_1H] - C1[a, b]) <= 1e-13 * scale
        assert abs(e[TERM_SSC] - Cs[a, b]) <= 1e-13 * scale
        assert abs(sum(e.values()) - C[a, b]) <= 1e-13 * scale
    # the 1-halo and SSC blocks are Gram matrices: Cauchy-Schwarz holds
    for blk in (C1, Cs):
        dd = np.sqrt(np.clip(np.diag(blk), 0, None))
        assert np.all(np.abs(blk) <= np.outer(dd, dd) * (1 + 1e-12) + 1e-300)


def test_snr_closed_forms(oracle_tiny):
    r = oracle_tiny
    rows, D = r.rows, r.D
    n_ell = len(r.T.ell)
    diag = np.abs(D) * 0.1 + 1e-20
    C = np.diag(diag ** 2)
    s = cumulative_snr(C, D, rows, n_ell, WHICH_JOINT)
    assert s[-1] == pytest.approx(math.sqrt(np.sum(D ** 2 / diag ** 2)), rel=1e-13)
    Cfull = r.cov.full(TERMS_ALL)
    sj = cumulative_snr(Cfull, D, rows, n_ell, WHICH_JOINT)
    assert sj[-1] == pytest.approx(math.sqrt(D @ np.linalg.solve(Cfull, D)), rel=1e-9)
    assert np.all(np.diff(sj) >= -1e-12)
    assert np.all(cumulative_snr(Cfull, 2 * D, rows, n_ell, WHICH_P) ==
                  pytest.approx(2 * cumulative_snr(Cfull, D, rows, n_ell, WHICH_P), rel=1e-12))
    # P and B alone never exceed the joint S/N
    sp_ = cumulative_snr(Cfull, D, rows, n_ell, WHICH_P)
    sb = cumulative_snr(Cfull, D, rows, n_ell, WHICH_B)
    assert sp_[-1] <= sj[-1] * (1 + 1e-12) and sb[-1] <= sj[-1] * (1 + 1e-12)
    # block-diagonal Gauss-only covariance: joint S/N^2 = P S/N^2 + B S/N^2
    Cg = r.cov.full(TERM_G)
    a = cumulative_snr(Cg, D, rows, n_ell, WHICH_JOINT)[-1] ** 2
    b = cumulative_snr(Cg, D, rows, n_ell, WHICH_P)[-1] ** 2 + cumulative_snr(Cg, D, rows, n_ell, WHICH_B)[-1] ** 2
    assert a == pytest.approx(b, rel=1e-11)
