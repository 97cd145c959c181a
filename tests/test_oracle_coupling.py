"""Pins of the exact BB+PT couplings (oracle/coupling.py; App. B, Eq. CovBB).

* Per-point leg counts n_{A|YZ}(q) by FFT convolution equal a direct
  enumeration of p in Y, and are constant on the orbits of the square's
  symmetry group (the lattice and the annuli are invariant under it).
* The Gram entries equal the definition written as a count over explicit
  lattice triangles: the number of pairs (t, t'), t of triangle bin tau and
  t' of tau', whose leg x and leg y are the same lattice mode (and the same
  count with opposite modes).
* Summed over q, each column gives N_tri exactly (so the PB coupling is 1/N(A)
  exactly), for every leg of every triangle.
* Cauchy-Schwarz: G_cc N(A) >= N_tri^2, equality iff n is constant over A; a
  thin annulus A with wide, well-closed Y and Z gives kappa N(A) close to 1
  (the paper's continuum prefactor).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import counts as cnt
from oracle import coupling as cpl

# three small annuli (squared radii in lattice units) and every bin triple
# they close
S_LO = np.array([4, 20, 45], dtype=np.int64)
S_HI = np.array([20, 45, 80], dtype=np.int64)


def _triangles():
    out = []
    for a, b, c in itertools.combinations_with_replacement(range(3), 3):
        if cnt.triangle_count_bruteforce(S_LO, S_HI, a, b, c) > 0:
            out.append((a, b, c))
    return out


def _lattice_triangles(tri):
    """All ordered lattice triangles (q1, q2, q3) of a bin triple, q3 = -q1-q2,
    as an array [n, 3, 2]."""
    a, b, c = tri
    ax, ay = cpl.annulus_points(S_LO, S_HI, a)
    bx, by = cpl.annulus_points(S_LO, S_HI, b)
    out = []
    for x1, y1 in zip(ax, ay):
        x3, y3 = -x1 - bx, -y1 - by
        s = x3 * x3 + y3 * y3
        m = (s >= S_LO[c]) & (s < S_HI[c])
        for x2, y2, xx, yy in zip(bx[m], by[m], x3[m], y3[m]):
            out.append(((x1, y1), (x2, y2), (xx, yy)))
    return np.array(out, dtype=np.int64).reshape(-1, 3, 2)


def test_leg_counts_fft_equals_enumeration_and_orbit_symmetry():
    lc = cpl.LegCounts(S_LO, S_HI)
    for A, Y, Z in itertools.product(range(3), repeat=3):
        if Y > Z:
            continue
        fft = lc.counts(A, [(Y, Z)])[(Y, Z)]
        brute = cpl.leg_counts_bruteforce(S_LO, S_HI, A, Y, Z)
        assert np.array_equal(fft, brute)
        # n(q) is the same on the orbit of q under the 8 symmetries of the square
        qx, qy = cpl.annulus_points(S_LO, S_HI, A)
        where = {(int(x), int(y)): i for i, (x, y) in enumerate(zip(qx, qy))}
        for i, (x, y) in enumerate(zip(qx, qy)):
            for gx, gy in ((y, x), (-x, y), (x, -y), (-y, -x), (-x, -y), (y, -x), (-y, x)):
                assert brute[where[(int(gx), int(gy))]] == brute[i]


def test_gram_equals_count_of_triangle_pairs_sharing_a_mode():
    tris = _triangles()
    assert len(tris) >= 6
    cols, col, G = cpl.grams(S_LO, S_HI, tris)
    lat = {t: _lattice_triangles(tri) for t, tri in enumerate(tris)}
    ntri = [len(lat[t]) for t in range(len(tris))]
    assert ntri == [cnt.triangle_count_bruteforce(S_LO, S_HI, *tri) for tri in tris]
    kappa = cpl.kappa_table(col, G, ntri, tris)
    checked = 0
    for t1, t2 in itertools.product(range(len(tris)), repeat=2):
        for x, y in itertools.product(range(3), repeat=2):
            A = tris[t1][x]
            if tris[t2][y] != A:
                continue
            # modes of leg x of every triangle of t1, leg y of every triangle of t2
            v1, n1 = np.unique(lat[t1][:, x, :], axis=0, return_counts=True)
            v2, n2 = np.unique(lat[t2][:, y, :], axis=0, return_counts=True)
            c2 = {tuple(v): n for v, n in zip(v2.tolist(), n2.tolist())}
            same = sum(n * c2.get(tuple(v), 0) for v, n in zip(v1.tolist(), n1.tolist()))
            opposite = sum(n * c2.get((-v[0], -v[1]), 0) for v, n in zip(v1.tolist(), n1.tolist()))
            g = int(G[A][col[t1][x], col[t2][y]])
            assert g == same == opposite
            assert kappa(t1, x, t2, y) == float(same) / (float(ntri[t1]) * float(ntri[t2]))
            checked += 1
    assert checked > 50


def test_column_sums_are_the_triangle_counts():
    tris = _triangles()
    lc = cpl.LegCounts(S_LO, S_HI)
    cols, col = cpl.columns(tris, 3)
    for t, tri in enumerate(tris):
        ntri = cnt.triangle_count_bruteforce(S_LO, S_HI, *tri)
        for x in range(3):
            A = tri[x]
            n = lc.counts(A, [cols[A][col[t][x]]])[cols[A][col[t][x]]]
            # (so the PB coupling, sum_q n(q) / (N(A) N_tri), is 1 / N(A) exactly)
            assert int(n.sum()) == ntri


def test_cauchy_schwarz_and_thin_annulus_limit():
    tris = _triangles()
    cols, col, G = cpl.grams(S_LO, S_HI, tris)
    Ntri = cnt.triangle_counts(S_LO, S_HI, tris)
    N = cnt.mode_counts(S_LO, S_HI)
    for t, tri in enumerate(tris):
        for x in range(3):
            A = tri[x]
            assert int(G[A][col[t][x], col[t][x]]) * int(N[A]) >= int(Ntri[t]) ** 2
    # a thin annulus (|q| in [100, 102)) between two wide ones that close
    # comfortably around it: n(q) nearly constant, kappa N(A) -> 1
    s_lo = np.array([100 ** 2, 60 ** 2, 90 ** 2], dtype=np.int64)
    s_hi = np.array([102 ** 2, 80 ** 2, 110 ** 2], dtype=np.int64)
    tri = [(0, 1, 2)]
    cols, col, G = cpl.grams(s_lo, s_hi, tri, bins=[0])
    ntri = int(cnt.triangle_counts(s_lo, s_hi, tri)[0])
    NA = int(cnt.mode_counts(s_lo, s_hi)[0])
    kN = float(G[0][0, 0]) * NA / (float(ntri) ** 2)
    assert 1.0 <= kN < 1.01
    # and a nearly degenerate closure (|q3| >= 100 needs |q1|, |q2| near 60 and
    # nearly parallel): n(q) vanishes on the inner part of A, far from 1
    s_lo = np.array([40 ** 2, 40 ** 2, 100 ** 2], dtype=np.int64)
    s_hi = np.array([60 ** 2, 60 ** 2, 120 ** 2], dtype=np.int64)
    cols, col, G = cpl.grams(s_lo, s_hi, [(0, 1, 2)], bins=[0])
    ntri = int(cnt.triangle_counts(s_lo, s_hi, [(0, 1, 2)])[0])
    NA = int(cnt.mode_counts(s_lo, s_hi)[0])
    assert float(G[0][0, 0]) * NA / (float(ntri) ** 2) > 1.4


@pytest.fixture(scope="module")
def tiny():
    from oracle.pipeline import OracleRun
    from paper_1812_07437_gb300 import workloads
    return OracleRun(workloads.get("tiny_2bin"), coupling="exact")


def test_exact_coupling_on_a_workload(tiny):
    """tiny_2bin: every column sums to its N_tri; kappa >= 1/N(A) on the
    diagonal (Cauchy-Schwarz); the covariance stays positive definite and the
    BB+PT term moves by a few per cent."""
    from oracle.covariance import TERM_BBPT
    r = tiny
    lc = cpl.LegCounts(r.s_lo, r.s_hi)
    cols, col = cpl.columns(r.tris, len(r.Nmodes))
    for t, tri in enumerate(r.tris):
        for x in range(3):
            A = tri[x]
            c = cols[A][col[t][x]]
            assert int(lc.counts(A, [c])[c].sum()) == int(r.Ntri[t])
            assert r.cov.kappa(t, x, t, x) * r.Nmodes[A] >= 1.0
    C = r.cov.full()
    np.linalg.cholesky(C)
    from oracle.covariance import Covariance
    plain = Covariance(r.T, r.S, r.rows, r.tris, r.Nmodes, r.Ntri)
    b = [k for k, row in enumerate(r.rows) if row[0] == "B"]
    e = np.array([r.cov.element_terms(i, j)[TERM_BBPT] for i in b[:12] for j in b[:12]])
    p = np.array([plain.element_terms(i, j)[TERM_BBPT] for i in b[:12] for j in b[:12]])
    m = p != 0
    rel = np.abs(e[m] / p[m] - 1.0)
    assert rel.max() < 0.2 and rel.max() > 1e-4
    assert math.isfinite(float(rel.max()))
