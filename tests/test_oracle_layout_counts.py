"""Pins of the oracle's data-vector layout and integer counts (CPU only)."""
import math
import os

import numpy as np
import pytest

from oracle import counts as cnt
from oracle.layout import closed_triangles, data_layout, tomo_triples
from oracle.survey import ell_bins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


def test_paper_vector_sizes():
    """Sec. 5: 14 ell bins on [10, 5000] give the printed P, B and joint sizes."""
    _, centres, _ = ell_bins(14, 10.0, 5000.0)
    for nt, n_p, n_b, n_j in _read_rows("paper_vector_sizes.txt"):
        rows, tris = data_layout(centres, int(nt))
        got_p = sum(1 for r in rows if r[0] == "P")
        assert got_p == n_p
        assert len(rows) - got_p == n_b
        if n_j > 0:
            assert len(rows) == n_j
    assert len(closed_triangles(centres)) == 130


def test_tomo_reduction_counts():
    for nt in (1, 2, 3, 5, 10):
        assert len(tomo_triples((0, 1, 2), nt)) == nt ** 3
        assert len(tomo_triples((1, 1, 2), nt)) == nt * nt * (nt + 1) // 2
        assert len(tomo_triples((0, 2, 2), nt)) == nt * nt * (nt + 1) // 2
        assert len(tomo_triples((3, 3, 3), nt)) == nt * (nt + 1) * (nt + 2) // 6


def test_layout_order():
    """Sec. 5: P first (ell slow, i<=j, j fast); B triples with l_b fastest, l_c slowest."""
    _, centres, _ = ell_bins(6, 10.0, 5000.0)
    rows, tris = data_layout(centres, 2)
    assert rows[0] == ("P", 0, (0, 0)) and rows[1] == ("P", 0, (0, 1)) and rows[3] == ("P", 1, (0, 0))
    for (a, b, c), (a2, b2, c2) in zip(tris, tris[1:]):
        assert (c, a, b) < (c2, a2, b2)
    first_b = [r for r in rows if r[0] == "B"][:3]
    assert [r[3] for r in first_b] == [(0, 0, 0), (0, 0, 1), (0, 1, 1)]


def _small_thresholds():
    # ell_f = 1 lattice, bins in squared radius (inclusive low, exclusive high)
    s_lo = np.array([25, 100, 300, 700], dtype=np.int64)
    s_hi = np.array([100, 300, 700, 1600], dtype=np.int64)
    return s_lo, s_hi


def test_mode_counts_bruteforce():
    s_lo, s_hi = _small_thresholds()
    got = cnt.mode_counts(s_lo, s_hi)
    for b in range(len(s_lo)):
        n = 0
        R = math.isqrt(int(s_hi[b]))
        for x in range(-R, R + 1):
            for y in range(-R, R + 1):
                if s_lo[b] <= x * x + y * y < s_hi[b]:
                    n += 1
        assert got[b] == n


def test_triangle_counts_fft_equals_bruteforce():
    """Exact N_tri of the FFT route against pair enumeration on tiny bins."""
    s_lo, s_hi = _small_thresholds()
    tris = [(0, 0, 0), (0, 0, 1), (0, 1, 1), (0, 1, 2), (1, 1, 2), (1, 2, 3), (2, 2, 3), (3, 3, 3), (0, 2, 2)]
    got = cnt.triangle_counts(s_lo, s_hi, tris)
    for t, (a, b, c) in enumerate(tris):
        assert got[t] == cnt.triangle_count_bruteforce(s_lo, s_hi, a, b, c), (a, b, c)


def test_triangle_counts_symmetric_in_legs():
    """#{n1 in A, n2 in B, n1+n2 in C} is invariant under any leg permutation."""
    s_lo, s_hi = _small_thresholds()
    perms = [(0, 1, 2), (1, 0, 2), (1, 2, 0), (2, 1, 0), (0, 2, 1), (2, 0, 1)]
    vals = cnt.triangle_counts(s_lo, s_hi, perms)
    assert len(set(int(v) for v in vals)) == 1


def test_mode_counts_continuum_limit():
    """N(l^b) -> 2 l Delta l f_sky for bins much wider than ell_f (Eq. PSest text)."""
    edges, centres, widths = ell_bins(8, 200.0, 3000.0)
    ell_f, s_lo, s_hi = cnt.lattice_thresholds(edges, 0.36)
    N = cnt.mode_counts(s_lo, s_hi)
    approx = 2.0 * centres * widths * 0.36
    assert np.all(np.abs(N / approx - 1.0) < 0.01)


def test_triangle_counts_continuum_limit():
    """Exact N_tri against the continuum measure for wide, well-closed bins."""
    edges, centres, widths = ell_bins(4, 300.0, 1200.0)
    ell_f, s_lo, s_hi = cnt.lattice_thresholds(edges, 0.36)
    tris = [(1, 1, 1), (2, 2, 3), (1, 2, 2)]
    got = cnt.triangle_counts(s_lo, s_hi, tris)
    omega = 4 * math.pi * 0.36
    for t, (a, b, c) in enumerate(tris):
        ref = cnt.ntri_continuum(centres[a], centres[b], centres[c], widths[a], widths[b], widths[c], omega)
        assert abs(got[t] / ref - 1.0) < 0.08, (a, b, c, got[t], ref)


def test_thresholds_edges():
    edges, centres, _ = ell_bins(5, 10.0, 100.0)
    ell_f, s_lo, s_hi = cnt.lattice_thresholds(edges, 0.36)
    assert ell_f == pytest.approx(2 * math.pi / math.sqrt(4 * math.pi * 0.36), rel=1e-15)
    for b in range(5):
        assert ell_f * math.sqrt(s_lo[b]) >= edges[b]
        assert ell_f * math.sqrt(s_lo[b] - 1) < edges[b]
        assert np.all(s_hi[:-1] == s_lo[1:])
    assert ell_f * math.sqrt(s_hi[-1] - 1) <= edges[-1] < ell_f * math.sqrt(s_hi[-1])
