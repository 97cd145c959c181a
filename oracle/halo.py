"""Halo model ingredients (oracle, FP64): Sec. 4 of the paper.

* Sheth-Tormen mass function f_m(m) = dn/dm with nu = (delta_c/sigma)^2
  (Sec. 4.5, Eq. BoundinMass context).  Parameters q = 0.707, p = 0.3,
  A from the normalisation int f(nu) dnu = 1; delta_c = 1.686.
* Peak-background-split biases b1, b2 (Sec. 4.2.1, Eq. TidalKernel context):
  Lagrangian b_n^L = (1/G) d^n G/d delta_b^n with delta_c -> delta_c - delta_b
  in G(nu) = nu f(nu), then the spherical-collapse Eulerian mapping
  b1 = 1 + b1^L, b2 = (8/21) b1^L + b2^L.
* Regularisation at m_min (Eq. effectiveMasBias): a delta of weight alpha_0 at
  the first mass node and the node-0 biases replaced by alpha_1, alpha_2 so
  that the discrete consistency relations (Eq. BoundinMass) hold exactly.
* Concentration: Duffy et al. (2008) mean-density fit c = 10.14
  (m / 2e12)^-0.081 (1+z)^-1.01 with r_200m = (3m/(4 pi 200 rho_com))^(1/3);
  or the Bullock et al. (2001) median the paper uses (Sec. 5.4):
  c_bar = K a(z) / a_c with nu(F m, a_c) = 1, i.e. the collapse epoch a_c at
  which D(a_c) sigma(F m, z=0) = delta_c (D(1) = 1), F = 0.01, K = 4.0.  a_c
  is the root of the growth ODE's solution on [1e-3, 100]; where F m has not
  collapsed by a = 100 (the growth is then within 0.4% of its asymptote) a_c
  is taken as 100.  No floor: where F m collapses late the median falls far
  below 1 (to ~0.01 for a_c = 100), which the profile below handles.
* NFW Fourier profile u(k, m, c), u(0) = 1: the truncated NFW density
  rho ~ 1/(y (1 + y)^2), y = r/r_s, r <= r_vir = c r_s, transformed with the
  kernel sin(kr)/(kr) and divided by its mass.  For c >= 1 the closed form in
  sine/cosine integrals; for c < 1, where that form divides terms that cancel
  to O(c^2) by ln(1+c) - c/(1+c) ~ c^2/2, the defining integral itself in
  t = r/r_vir: u = int_0^1 w(t) sinc(K t) dt / int_0^1 w(t) dt with
  w(t) = t/(1 + c t)^2 and K = k r_vir, both integrals on one composite
  16-point Gauss-Legendre rule of ceil(K/(2 pi)) equal panels (at least one):
  every panel spans at most one period of sin(K t) and w is analytic well
  beyond [0, 1] for c < 1, so the rule is exact to rounding.
* Concentration scatter (Eq. LogNormC, the paper's "model A"): ln c is
  normal about ln c_bar(m, z) with sigma_lnc (0.18 in the paper).  The c
  integral of Eq. ImunuHalos is taken with an N_c-point Gauss-Hermite rule
  in x = (ln c - ln c_bar)/sigma_lnc: nodes c_j = c_bar exp(sigma_lnc x_j),
  weights w_j of the standard normal density (sum w_j = 1).  N_c <= 1 is the
  delta-function p(c) of "model B" (c = c_bar, weight 1).

Mass rule: N_M nodes m_q log-spaced over [m_min, m_max] (both included),
trapezoid weights in ln m: omega_q = dlnm * m_q * (1/2 at both ends), so that
int dm g(m) ~ sum_q omega_q g(m_q).
"""
import math

import numpy as np
from numpy.polynomial.hermite_e import hermegauss
from scipy.optimize import brentq
from scipy.special import sici

from . import cosmology as cz

ST_Q = 0.707
ST_P = 0.3
DELTA_C = 1.686
DUFFY_A = 10.14
DUFFY_B = -0.081
DUFFY_C = -1.01
DUFFY_MPIVOT = 2.0e12
DELTA_VIR = 200.0
BULLOCK_F = 0.01
BULLOCK_K = 4.0
NFW_C_INTEGRAL = 1.0  # below this concentration u is the quadrature of its defining integral
A_COLLAPSE_MAX = 100.0
CONC_DUFFY = 0
CONC_BULLOCK = 1


def st_amplitude():
    """A such that int_0^inf f(nu) dnu = 1: A = 1/(1 + 2^-p Gamma(1/2-p)/sqrt(pi))."""
    return 1.0 / (1.0 + 2.0 ** (-ST_P) * math.gamma(0.5 - ST_P) / math.sqrt(math.pi))


def st_G(nu):
    """Multiplicity G(nu) = nu f(nu) of Sheth & Tormen."""
    nu = np.asarray(nu, dtype=np.float64)
    qn = ST_Q * nu
    return st_amplitude() * np.sqrt(qn / (2.0 * math.pi)) * (1.0 + qn ** (-ST_P)) * np.exp(-0.5 * qn)


def st_dlnG_dnu(nu):
    qn = ST_Q * nu
    return 0.5 / nu - ST_P / (nu * (1.0 + qn ** ST_P)) - 0.5 * ST_Q


def st_d2lnG_dnu2(nu):
    qn = ST_Q * nu
    return -0.5 / nu ** 2 + ST_P * (1.0 + (ST_P + 1.0) * qn ** ST_P) / (nu ** 2 * (1.0 + qn ** ST_P) ** 2)


def st_biases(nu):
    """Eulerian (b1, b2) from the peak-background split of G(nu)."""
    nu = np.asarray(nu, dtype=np.float64)
    a = st_dlnG_dnu(nu)
    ap = st_d2lnG_dnu2(nu)
    b1L = -2.0 * nu * a / DELTA_C
    b2L = (a * a + ap) * 4.0 * nu * nu / DELTA_C ** 2 + a * 2.0 * nu / DELTA_C ** 2
    return 1.0 + b1L, (8.0 / 21.0) * b1L + b2L


def mass_nodes(n_mass, m_min, m_max):
    """Log-spaced nodes and trapezoid weights in ln m (includes both ends)."""
    dl = math.log(m_max / m_min) / (n_mass - 1)
    m = m_min * np.exp(dl * np.arange(n_mass))
    om = dl * m
    om[0] *= 0.5
    om[-1] *= 0.5
    return m, om


def mass_function(m, sigma, dlnsigma_dlnm, rho):
    """f_m(m) = dn/dm = (rho/m^2) G(nu) d ln nu / d ln m, nu = (delta_c/sigma)^2."""
    nu = (DELTA_C / sigma) ** 2
    return rho / m ** 2 * st_G(nu) * (-2.0 * dlnsigma_dlnm), nu


def regularise(m, om, fm, b1, b2, rho):
    """Eq. effectiveMasBias on the discrete mass rule (one redshift).

    Returns (f~, b1~, b2~): alpha_0 folded into node 0 so that
    sum omega (m/rho) f~ = 1, and node-0 biases alpha_1, alpha_2 so that the
    beta = 1 sum is 1 and the beta = 2 sum is 0 (Eq. BoundinMass).
    """
    mr = m / rho
    s0 = np.sum(om * mr * fm)
    alpha0 = (1.0 - s0) / mr[0]
    ft = fm.copy()
    ft[0] = fm[0] + alpha0 / om[0]
    den = om[0] * mr[0] * ft[0]
    a1 = (1.0 - np.sum(om[1:] * mr[1:] * fm[1:] * b1[1:])) / den
    a2 = (0.0 - np.sum(om[1:] * mr[1:] * fm[1:] * b2[1:])) / den
    b1t = b1.copy()
    b2t = b2.copy()
    b1t[0] = a1
    b2t[0] = a2
    return ft, b1t, b2t


def concentration(m, z):
    """Duffy et al. (2008) c(m, z) for the 200 x mean-density mass definition."""
    return DUFFY_A * (np.asarray(m) / DUFFY_MPIVOT) ** DUFFY_B * (1.0 + z) ** DUFFY_C


def collapse_epoch(sigma_Fm, cosmo):
    """a_c with D(a_c) sigma(F m, 0) = delta_c for each sigma(F m, 0) (D(1) = 1),
    D from the growth ODE (cosmology.growth's RK4 rule carried to a_c), by
    Brent's method in ln a; A_COLLAPSE_MAX where no root lies below it, the
    start of the growth rule where the root lies before it."""
    d1 = cz._growth_raw(1.0, cosmo)
    dmax = cz._growth_raw(A_COLLAPSE_MAX, cosmo) / d1
    dmin = cz._growth_raw(cz.A_INIT, cosmo) / d1
    out = []
    for s in np.atleast_1d(sigma_Fm):
        target = DELTA_C / s
        if dmax <= target:
            out.append(A_COLLAPSE_MAX)
            continue
        if dmin >= target:  # collapsed before the growth rule starts (never for m >= 1e2 Msun/h)
            out.append(cz.A_INIT)
            continue
        g = lambda lna: cz._growth_raw(math.exp(lna), cosmo) / d1 - target
        out.append(math.exp(brentq(g, math.log(cz.A_INIT), math.log(A_COLLAPSE_MAX), xtol=1e-15, rtol=9e-16,
                                   maxiter=200)))
    return np.array(out)


def bullock_concentration(a_c, z):
    """Bullock et al. (2001) median c_bar = K a(z) / a_c (Sec. 5.4)."""
    return BULLOCK_K / ((1.0 + z) * np.asarray(a_c))


def conc_rule(n_conc, sigma_lnc):
    """Offsets s_j = sigma_lnc x_j of ln c from ln c_bar and weights w_j of
    the concentration integral: x_j, w_j Gauss-Hermite for the standard
    normal density (numpy's hermegauss weights / sqrt(2 pi)); n_conc <= 1
    gives the single offset 0 with weight 1 (model B)."""
    if n_conc <= 1:
        return np.zeros(1), np.ones(1)
    x, w = hermegauss(n_conc)
    return x * sigma_lnc, w / math.sqrt(2.0 * math.pi)


def r_vir(m, rho):
    return (3.0 * np.asarray(m) / (4.0 * math.pi * DELTA_VIR * rho)) ** (1.0 / 3.0)


def nfw_u(k, m, z, rho, c=None):
    """Normalised Fourier transform u(k|m, c) of a truncated NFW profile
    (c defaults to the median concentration c_bar(m, z)).

    c >= 1: u = [sin x (Si((1+c)x) - Si(x)) - sin(cx)/((1+c)x)
                 + cos x (Ci((1+c)x) - Ci(x))] / (ln(1+c) - c/(1+c)),  x = k r_s,
    with scipy.special.sici as the Si/Ci step.  c < 1: nfw_u_integral.
    """
    if c is None:
        c = concentration(m, z)
    k = np.asarray(k, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    k, m, c = np.broadcast_arrays(k, m, c)
    scalar = k.ndim == 0
    k, m, c = np.atleast_1d(k), np.atleast_1d(m), np.atleast_1d(c)
    rv = r_vir(m, rho)
    out = np.empty(k.shape)
    big = c >= NFW_C_INTEGRAL
    if np.any(big):
        cb = c[big]
        x = k[big] * rv[big] / cb
        si1, ci1 = sici(x)
        si2, ci2 = sici((1.0 + cb) * x)
        num = np.sin(x) * (si2 - si1) - np.sin(cb * x) / ((1.0 + cb) * x) + np.cos(x) * (ci2 - ci1)
        out[big] = num / (np.log(1.0 + cb) - cb / (1.0 + cb))
    for idx in zip(*np.nonzero(~big)):
        out[idx] = nfw_u_integral(float(k[idx] * rv[idx]), float(c[idx]))
    return float(out[0]) if scalar else out


_GL16 = np.polynomial.legendre.leggauss(16)


def nfw_u_integral(K, c):
    """u = int_0^1 w(t) sinc(K t) dt / int_0^1 w(t) dt, w(t) = t/(1 + c t)^2:
    the truncated NFW transform with r = t r_vir (K = k r_vir), on the
    composite 16-point Gauss-Legendre rule of ceil(K/(2 pi)) panels."""
    P = max(1, int(math.ceil(K / (2.0 * math.pi))))
    x, w = _GL16
    t = ((np.arange(P)[:, None] + 0.5 * (x[None, :] + 1.0)) / P).ravel()
    wt = np.tile(w, P) * (0.5 / P) * t / (1.0 + c * t) ** 2
    Kt = K * t
    return float(np.sum(wt * np.sin(Kt) / Kt) / np.sum(wt))
