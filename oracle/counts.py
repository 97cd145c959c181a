"""Integer mode and triangle counts (oracle, exact integers).

Modes live on the lattice ell_f * (n_x, n_y), (n_x, n_y) in Z^2 without the
origin (Sec. 3.2.2, equation after Eq. PSest).  The paper's two statements
ell_f = 2 pi / Theta_sky and N(ell^b) ~ 2 ell Delta ell f_sky do not agree; the
reading taken here is ell_f = 2 pi / sqrt(Omega_sky), for which the number of
lattice points in an annulus is ~ Omega ell Delta ell / (2 pi) =
2 ell Delta ell f_sky, i.e. N(ell^b) counts lattice points (not +- pairs).

Bin membership uses integer squared radii s = n_x^2 + n_y^2:
  s_lo[b] = ceil((lo_b / ell_f)^2)   (inclusive lower edge)
  s_hi[b] = s_lo[b+1]                (exclusive upper edge),
  s_hi[last] = floor((ell_max/ell_f)^2) + 1 (the last bin is closed).

N(ell^b)  = #{n : s_lo[b] <= |n|^2 < s_hi[b]}                 (Eq. PSest)
N_tri(abc) = #{(n1, n2) : n1 in A_a, n2 in A_b, n1 + n2 in A_c}
            (the first equality of the N_tri definition in Appendix B; the
            printed continuum approximation there is garbled and is used
            only as a loose check).

N_tri is evaluated as sum_{n in A_c} (1_{A_a} * 1_{A_b})(n), with the lattice
convolution taken by FFT on a periodic grid of side L >= 3R + 1 (no alias
reaches |n| <= R) and rounded to the nearest integer; a brute-force pair
enumeration is kept for tiny bins.
"""
import math

import numpy as np
import scipy.fft as sfft


def lattice_thresholds(ell_edges, f_sky):
    omega = 4.0 * math.pi * f_sky
    ell_f = 2.0 * math.pi / math.sqrt(omega)
    nb = len(ell_edges) - 1
    s_lo = []
    for b in range(nb):
        x = ell_edges[b] / ell_f
        s_lo.append(int(math.ceil(x * x)))
    x = ell_edges[nb] / ell_f
    s_top = int(math.floor(x * x)) + 1
    s_hi = s_lo[1:] + [s_top]
    return ell_f, np.array(s_lo, dtype=np.int64), np.array(s_hi, dtype=np.int64)


def _grid_radius(s_hi):
    return math.isqrt(int(max(s_hi)) - 1)


def mode_counts(s_lo, s_hi):
    """N(ell^b) by direct enumeration of every lattice point of radius <= R."""
    R = _grid_radius(s_hi)
    v = np.arange(-R, R + 1, dtype=np.int64)
    s = (v[:, None] ** 2 + v[None, :] ** 2).ravel()
    out = np.zeros(len(s_lo), dtype=np.int64)
    for b in range(len(s_lo)):
        out[b] = np.count_nonzero((s >= s_lo[b]) & (s < s_hi[b]))
    return out


def _annulus_points(slo, shi):
    R = math.isqrt(int(shi) - 1)
    v = np.arange(-R, R + 1, dtype=np.int64)
    X, Y = np.meshgrid(v, v, indexing="xy")
    s = X * X + Y * Y
    m = (s >= slo) & (s < shi)
    return X[m], Y[m]


def triangle_count_bruteforce(s_lo, s_hi, a, b, c):
    """Pair enumeration over A_a x A_b (tiny bins only)."""
    xa, ya = _annulus_points(s_lo[a], s_hi[a])
    xb, yb = _annulus_points(s_lo[b], s_hi[b])
    total = 0
    for x1, y1 in zip(xa, ya):
        sx = x1 + xb
        sy = y1 + yb
        s = sx * sx + sy * sy
        total += int(np.count_nonzero((s >= s_lo[c]) & (s < s_hi[c])))
    return total


def triangle_counts(s_lo, s_hi, triangles, workers=None):
    """N_tri for every (a, b, c) in ``triangles`` via FFT lattice convolution."""
    R = _grid_radius(s_hi)
    L = sfft.next_fast_len(3 * R + 1)
    v = np.arange(-R, R + 1, dtype=np.int64)
    X, Y = np.meshgrid(v, v, indexing="xy")
    S = X * X + Y * Y
    iy = np.mod(Y, L)
    ix = np.mod(X, L)

    def indicator(b):
        g = np.zeros((L, L))
        m = (S >= s_lo[b]) & (S < s_hi[b])
        g[iy[m], ix[m]] = 1.0
        return g, m

    spectra = {}
    masks = {}
    needed = sorted({t[0] for t in triangles} | {t[1] for t in triangles} | {t[2] for t in triangles})
    for b in needed:
        g, m = indicator(b)
        masks[b] = m
        spectra[b] = sfft.rfft2(g, workers=workers)
    by_pair = {}
    for idx, (a, b, c) in enumerate(triangles):
        by_pair.setdefault((a, b), []).append((idx, c))
    out = np.zeros(len(triangles), dtype=np.int64)
    worst = 0.0
    for (a, b), items in by_pair.items():
        conv = sfft.irfft2(spectra[a] * spectra[b], s=(L, L), workers=workers)
        for idx, c in items:
            vals = conv[iy[masks[c]], ix[masks[c]]]
            r = np.rint(vals)
            worst = max(worst, float(np.max(np.abs(vals - r))) if vals.size else 0.0)
            out[idx] = int(np.sum(r.astype(np.int64)))
    assert worst < 1e-3, f"FFT convolution not integral to 1e-3 (worst {worst})"
    return out


def ntri_continuum(la, lb, lc, da, db, dc, omega):
    """Continuum limit of N_tri for wide bins (loose check only).

    Lattice density Omega/(2 pi)^2; the measure of (ell1, ell2) with |ell1| in
    bin a, |ell2| in bin b and |ell1+ell2| in bin c is
    8 pi la lb lc da db dc / lambda, lambda = sqrt(2la^2lb^2 + 2lb^2lc^2 +
    2lc^2la^2 - la^4 - lb^4 - lc^4).
    """
    lam2 = 2 * la * la * lb * lb + 2 * lb * lb * lc * lc + 2 * lc * lc * la * la - la ** 4 - lb ** 4 - lc ** 4
    dens = omega / (2.0 * math.pi) ** 2
    return dens * dens * 8.0 * math.pi * la * lb * lc * da * db * dc / math.sqrt(lam2)
