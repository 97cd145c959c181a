"""Background cosmology and linear matter power spectrum (oracle, FP64).

Flat w0-CDM with c = 1, lengths in Mpc/h, masses in Msun/h (paper Sec. 1,
last paragraph).  The linear spectrum is the Eisenstein & Hu (1998) no-wiggle
fit normalised to sigma_8 (the paper leaves P_lin unspecified).

Discrete rules (shared as a written specification with the CUDA side, not as
code):
  * chi(z) = (1/H0) int_0^z dz'/E(z') with a 64-node Gauss-Legendre rule on
    [0, z].
  * z(chi) by Newton iteration on chi(z) - chi = 0 until the step is below
    1e-15 (1+z).
  * growth D(a): RK4 with exactly 1024 equal steps in ln a from a = 1e-3
    (D = a, dD/dln a = a) to the target a; D is divided by the same
    integration carried to a = 1.
  * sigma(R) and d sigma^2/dR: 4096-node Gauss-Legendre rule in ln k on
    [ln 1e-5, ln 1e3] (k in h/Mpc); the top-hat window uses its Taylor series
    below x = 0.5.
"""
import functools
import math

import numpy as np

C_OVER_H0 = 2997.92458          # Mpc/h
H0 = 1.0 / C_OVER_H0            # h/Mpc, c = 1
RHO_CRIT0 = 2.77536627e11       # (Msun/h) / (Mpc/h)^3

N_GL_CHI = 64
N_RK4 = 1024
A_INIT = 1.0e-3
N_K_SIGMA = 4096
LNK_MIN = math.log(1.0e-5)
LNK_MAX = math.log(1.0e3)
X_SERIES_TOPHAT = 0.5


@functools.lru_cache(maxsize=None)
def _leggauss(n):
    return np.polynomial.legendre.leggauss(n)


def gl_nodes(n, a, b):
    """Gauss-Legendre nodes and weights on [a, b] (numpy.leggauss as a step)."""
    x, w = _leggauss(n)
    half = 0.5 * (b - a)
    return a + half * (x + 1.0), half * w


def E(z, cosmo):
    """H(z)/H0 for a flat universe with a constant dark-energy w0."""
    om = cosmo["Om"]
    ode = 1.0 - om
    zp1 = 1.0 + np.asarray(z, dtype=np.float64)
    return np.sqrt(om * zp1 ** 3 + ode * zp1 ** (3.0 * (1.0 + cosmo["w0"])))


def chi_of_z(z, cosmo):
    """Comoving distance chi(z) in Mpc/h (Eq. kappa uses chi(z))."""
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    out = np.empty_like(z)
    for i, zi in enumerate(z):
        x, w = gl_nodes(N_GL_CHI, 0.0, zi)
        out[i] = C_OVER_H0 * np.sum(w / E(x, cosmo))
    return out


def z_of_chi(chi, cosmo):
    """Invert chi(z) by Newton iteration (d chi/dz = 1/H)."""
    chi = np.atleast_1d(np.asarray(chi, dtype=np.float64))
    out = np.empty_like(chi)
    for i, c in enumerate(chi):
        z = c * H0
        for _ in range(100):
            f = chi_of_z(z, cosmo)[0] - c
            step = f * H0 * E(z, cosmo)
            z = z - step
            if abs(step) < 1e-15 * (1.0 + z):
                break
        out[i] = z
    return out


def _growth_rhs(lna, y, cosmo):
    a = math.exp(lna)
    om = cosmo["Om"]
    ode = 1.0 - om
    w = cosmo["w0"]
    em = om * a ** -3
    ed = ode * a ** (-3.0 * (1.0 + w))
    e2 = em + ed
    dlnh = 0.5 * (-3.0 * em - 3.0 * (1.0 + w) * ed) / e2
    om_a = em / e2
    d, dp = y
    return np.array([dp, -(2.0 + dlnh) * dp + 1.5 * om_a * d])


def _growth_raw(a_target, cosmo):
    x0 = math.log(A_INIT)
    x1 = math.log(a_target)
    h = (x1 - x0) / N_RK4
    y = np.array([A_INIT, A_INIT])
    x = x0
    for _ in range(N_RK4):
        k1 = _growth_rhs(x, y, cosmo)
        k2 = _growth_rhs(x + 0.5 * h, y + 0.5 * h * k1, cosmo)
        k3 = _growth_rhs(x + 0.5 * h, y + 0.5 * h * k2, cosmo)
        k4 = _growth_rhs(x + h, y + h * k3, cosmo)
        y = y + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        x = x + h
    return y[0]


def growth(z, cosmo):
    """Linear growth D(z)/D(0) from the linear growth ODE in ln a."""
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    d0 = _growth_raw(1.0, cosmo)
    return np.array([_growth_raw(1.0 / (1.0 + zi), cosmo) / d0 for zi in z])


def eh_nowiggle_T(k, cosmo):
    """Eisenstein & Hu (1998) zero-baryon-oscillation transfer function.

    k in h/Mpc.  Sound horizon, alpha_Gamma, Gamma_eff and the L0/C0 fit as
    published in that paper (its Eqs. 26 and 28-31).
    """
    k = np.asarray(k, dtype=np.float64)
    h = cosmo["h"]
    om = cosmo["Om"]
    ob = cosmo["Ob"]
    omh2 = om * h * h
    obh2 = ob * h * h
    fb = ob / om
    theta = cosmo["Tcmb"] / 2.7
    s = 44.5 * math.log(9.83 / omh2) / math.sqrt(1.0 + 10.0 * obh2 ** 0.75)
    alpha = 1.0 - 0.328 * math.log(431.0 * omh2) * fb + 0.38 * math.log(22.3 * omh2) * fb * fb
    ks = k * h * s
    gamma_eff = om * h * (alpha + (1.0 - alpha) / (1.0 + (0.43 * ks) ** 4))
    q = k * theta * theta / gamma_eff
    L0 = np.log(2.0 * math.e + 1.8 * q)
    C0 = 14.2 + 731.0 / (1.0 + 62.5 * q)
    return L0 / (L0 + C0 * q * q)


def tophat_W(x):
    """Fourier transform of a spherical top-hat, 3 (sin x - x cos x)/x^3."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = x < X_SERIES_TOPHAT
    xs = x[small]
    x2 = xs * xs
    acc = np.zeros_like(xs)
    for n in range(6, -1, -1):
        c = 3.0 * (-1) ** n * (2 * n + 2) / math.factorial(2 * n + 3)
        acc = acc * x2 + c
    out[small] = acc
    xl = x[~small]
    out[~small] = 3.0 * (np.sin(xl) - xl * np.cos(xl)) / xl ** 3
    return out


def tophat_dW(x):
    """dW/dx of the top-hat window."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = x < X_SERIES_TOPHAT
    xs = x[small]
    x2 = xs * xs
    acc = np.zeros_like(xs)
    for n in range(7, 0, -1):
        c = 3.0 * (-1) ** n * (2 * n + 2) / math.factorial(2 * n + 3)
        acc = acc * x2 + 2 * n * c
    out[small] = acc * xs
    xl = x[~small]
    out[~small] = 3.0 * ((xl * xl - 3.0) * np.sin(xl) + 3.0 * xl * np.cos(xl)) / xl ** 4
    return out


def _sigma_k_rule():
    lnk, w = gl_nodes(N_K_SIGMA, LNK_MIN, LNK_MAX)
    return np.exp(lnk), w


def _sigma2_unnormalised(R, cosmo):
    """int dlnk k^3 k^ns T^2 / (2 pi^2) W(kR)^2 for unit amplitude."""
    k, w = _sigma_k_rule()
    d2 = k ** 3 * k ** cosmo["ns"] * eh_nowiggle_T(k, cosmo) ** 2 / (2.0 * math.pi ** 2)
    R = np.atleast_1d(R)
    return np.array([np.sum(w * d2 * tophat_W(k * r) ** 2) for r in R])


def plin_amplitude(cosmo):
    """Amplitude A of P_lin(k, 0) = A k^ns T(k)^2 fixed by sigma_8."""
    return cosmo["sigma8"] ** 2 / _sigma2_unnormalised(8.0, cosmo)[0]


def plin(k, z_growth, amp, cosmo):
    """P_lin(k, z) = A k^ns T(k)^2 D(z)^2 (D passed in as z_growth)."""
    k = np.asarray(k, dtype=np.float64)
    return amp * k ** cosmo["ns"] * eh_nowiggle_T(k, cosmo) ** 2 * z_growth ** 2


def dplin_dlnk(k, z_growth, amp, cosmo, h=1.0e-3):
    """dP_lin/dln k by the fourth-order central difference with step h in ln k."""
    k = np.asarray(k, dtype=np.float64)
    f = lambda s: plin(k * math.exp(s), z_growth, amp, cosmo)
    return (-f(2 * h) + 8.0 * f(h) - 8.0 * f(-h) + f(-2 * h)) / (12.0 * h)


def rho_mean(cosmo):
    """Comoving mean matter density rho_com (paper Eq. P1halos)."""
    return RHO_CRIT0 * cosmo["Om"]


def sigma_and_dlnsigma_dlnm(m, amp, cosmo):
    """sigma(m, z=0) and d ln sigma / d ln m for Lagrangian radius R(m).

    R = (3 m / (4 pi rho_mean))^(1/3); d ln sigma/d ln m = (R/6) (d sigma^2/dR)/sigma^2.
    """
    m = np.atleast_1d(np.asarray(m, dtype=np.float64))
    rho = rho_mean(cosmo)
    R = (3.0 * m / (4.0 * math.pi * rho)) ** (1.0 / 3.0)
    k, w = _sigma_k_rule()
    d2 = amp * k ** 3 * k ** cosmo["ns"] * eh_nowiggle_T(k, cosmo) ** 2 / (2.0 * math.pi ** 2)
    sig2 = np.empty_like(m)
    dsig2 = np.empty_like(m)
    for i, r in enumerate(R):
        x = k * r
        Wx = tophat_W(x)
        sig2[i] = np.sum(w * d2 * Wx * Wx)
        dsig2[i] = np.sum(w * d2 * 2.0 * Wx * tophat_dW(x) * k)
    return np.sqrt(sig2), (R / 6.0) * dsig2 / sig2
