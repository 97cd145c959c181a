"""Survey geometry (oracle, FP64): Sec. 2, Eq. ShotNoise, Appendix A.

* Source distribution n(z) ~ z^2 exp(-(z/z0)^alpha), alpha = 1.5 (Appendix A).
* Equipopulated tomographic edges: each bin holds 1/n_t of int n(z) dz over
  [z_min, z_max]; the CDF is closed form for alpha = 1.5
  (int z^2 e^{-(z/z0)^1.5} dz ~ 1 - (1+x) e^{-x}, x = (z/z0)^1.5); edges by
  bisection to machine precision.
* Optional Gaussian photo-z scatter sigma_0 (1+z): n_i(z) = n(z) P_i(z) with
  P_i the probability that z_ph falls in [z_lo, z_hi) (reading: galaxies
  scattered outside [z_min, z_max] are dropped); without scatter P_i is the
  bin indicator (paper Sec. 2 ignores photo-z).
* Lensing kernel (Eqs. KernelLensing1, LensEff):
  W_i(chi) = 3/2 Om H0^2 (1+z) chi int_{z}^{z_max} dz_s n_i(z_s)
             (chi(z_s) - chi)/chi(z_s), n_i normalised to unit integral.
  Quadrature rule: [z(chi), z_max] split at the tomographic edges inside it,
  64-node Gauss-Legendre on each piece; the n_i normalisation uses the same
  rule on [z_min, z_max].
* ell bins (Sec. 3.2.1, Appendix A): edges ell_min (ell_max/ell_min)^(b/n_ell),
  centre = (lo+hi)/2 (symmetric interval), width = hi - lo.
* Shot noise (Eq. ShotNoise): sigma_e^2 / nbar_i with nbar_i = n_gal / n_t
  per steradian.
"""
import math

import numpy as np
from scipy.special import erf

from .cosmology import C_OVER_H0, H0, E, _leggauss, gl_nodes

N_ZS = 64
N_GL_CHI = 64
ARCMIN2_PER_SR = (10800.0 / math.pi) ** 2


def chi_of_z_vec(z, cosmo):
    """Vectorised chi(z) with the 64-node Gauss-Legendre rule on [0, z]."""
    z = np.asarray(z, dtype=np.float64)
    x, w = _leggauss(N_GL_CHI)
    zz = 0.5 * z[..., None] * (x + 1.0)
    return C_OVER_H0 * 0.5 * z * np.sum(w / E(zz, cosmo), axis=-1)


def nz_shape(z, nz):
    z = np.asarray(z, dtype=np.float64)
    return z * z * np.exp(-(z / nz["z0"]) ** nz["alpha"])


def _cdf_unnorm(z, nz):
    assert nz["alpha"] == 1.5, "closed-form CDF is written for alpha = 1.5"
    x = (z / nz["z0"]) ** 1.5
    return 1.0 - (1.0 + x) * math.exp(-x)


def tomo_edges(nz):
    """Equipopulated edges z_0 = z_min < ... < z_nt = z_max (bisection)."""
    nt = nz["n_tomo"]
    zmin, zmax = nz["zmin"], nz["zmax"]
    g0 = _cdf_unnorm(zmin, nz)
    g1 = _cdf_unnorm(zmax, nz)
    edges = [zmin]
    for e in range(1, nt):
        target = e / nt
        lo, hi = zmin, zmax
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if mid <= lo or mid >= hi:
                break
            if (_cdf_unnorm(mid, nz) - g0) / (g1 - g0) < target:
                lo = mid
            else:
                hi = mid
        edges.append(0.5 * (lo + hi))
    edges.append(zmax)
    return np.array(edges)


def bin_selection(z, i, edges, sigma0):
    """P_i(z): probability that a source at true z is assigned to bin i."""
    z = np.asarray(z, dtype=np.float64)
    lo, hi = edges[i], edges[i + 1]
    if sigma0 == 0.0:
        last = i == len(edges) - 2
        sel = (z >= lo) & ((z <= hi) if last else (z < hi))
        return sel.astype(np.float64)
    s = math.sqrt(2.0) * sigma0 * (1.0 + z)
    return 0.5 * (erf((hi - z) / s) - erf((lo - z) / s))


def _pieces(a, b, edges):
    pts = [a] + [e for e in edges if a < e < b] + [b]
    return list(zip(pts[:-1], pts[1:]))


def bin_norms(nz, edges):
    """N_i = int n(z) P_i(z) dz on [z_min, z_max] (same piecewise rule)."""
    out = np.zeros(nz["n_tomo"])
    for (a, b) in _pieces(nz["zmin"], nz["zmax"], edges):
        x, w = gl_nodes(N_ZS, a, b)
        for i in range(nz["n_tomo"]):
            out[i] += np.sum(w * nz_shape(x, nz) * bin_selection(x, i, edges, nz["photoz_sigma0"]))
    return out


def lensing_kernels(chi_nodes, z_nodes, nz, cosmo, edges=None):
    """W_i(chi_n) for all tomographic bins i and line-of-sight nodes n."""
    if edges is None:
        edges = tomo_edges(nz)
    norms = bin_norms(nz, edges)
    nt = nz["n_tomo"]
    W = np.zeros((nt, len(chi_nodes)))
    pref = 1.5 * cosmo["Om"] * H0 * H0
    for n, (chi, z) in enumerate(zip(chi_nodes, z_nodes)):
        if z >= nz["zmax"]:
            continue
        acc = np.zeros(nt)
        for (a, b) in _pieces(z, nz["zmax"], edges):
            zs, w = gl_nodes(N_ZS, a, b)
            chis = chi_of_z_vec(zs, cosmo)
            geo = w * nz_shape(zs, nz) * (chis - chi) / chis
            for i in range(nt):
                acc[i] += np.sum(geo * bin_selection(zs, i, edges, nz["photoz_sigma0"]))
        W[:, n] = pref * (1.0 + z) * chi * acc / norms
    return W


def ell_bins(n_ell, ell_min, ell_max):
    """Log-spaced edges, centres (lo+hi)/2 and widths hi-lo."""
    r = ell_max / ell_min
    edges = np.array([ell_min * math.pow(r, b / n_ell) for b in range(n_ell + 1)])
    return edges, 0.5 * (edges[:-1] + edges[1:]), edges[1:] - edges[:-1]


def sky(f_sky):
    """Omega_sky = 4 pi f_sky, Theta_sky with Omega = 2 pi (1 - cos Theta)."""
    omega = 4.0 * math.pi * f_sky
    theta = math.acos(1.0 - 2.0 * f_sky)
    return omega, theta


def shot_noise(nz):
    """sigma_e^2 / nbar_i for each tomographic bin (Eq. ShotNoise)."""
    nbar = nz["n_gal_arcmin2"] * ARCMIN2_PER_SR / nz["n_tomo"]
    return np.full(nz["n_tomo"], nz["sigma_e"] ** 2 / nbar)
