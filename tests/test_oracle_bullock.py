"""Pins of the oracle's Bullock et al. median concentration (Sec. 5.4):
c_bar = K a(z) / a_c with nu(F m, a_c) = 1, i.e. D(a_c) sigma(F m, 0) = delta_c.

The collapse epoch is a root of the growth ODE's solution; these checks fix it
against the closed form of an Einstein-de Sitter universe (D = a), against the
integral form of the LCDM growth factor (Heath 1977) past a = 1, and against
the limits of the rule.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import cosmology as cz
from oracle import halo
from oracle.spectra import Tables
from paper_1812_07437_gb300 import workloads

COSMO = workloads.PAPER_COSMOLOGY


def test_collapse_epoch_einstein_de_sitter_closed_form():
    """D(a) = a when Omega_m = 1, so a_c = delta_c / sigma(F m, 0)."""
    eds = dict(COSMO, Om=1.0)
    sig = np.array([1.7, 2.5, 4.0, 7.0, 0.9, 0.2])
    ac = halo.collapse_epoch(sig, eds)
    np.testing.assert_allclose(ac, halo.DELTA_C / sig, rtol=1e-9)


def test_collapse_epoch_against_integral_growth_past_today():
    """D(a_c) sigma = delta_c with D from H(a) int da/(a H)^3, a_c on both sides of a = 1."""
    om = COSMO["Om"]
    H = lambda x: math.sqrt(om * x ** -3 + 1.0 - om)
    heath = lambda a: H(a) * integrate.quad(lambda x: 1.0 / (x * H(x)) ** 3, 0.0, a, epsabs=0, epsrel=1e-13)[0]
    sig = np.array([5.0, 3.0, 1.9, 1.6, 1.4, 1.3])
    ac = halo.collapse_epoch(sig, COSMO)
    assert ac.min() < 1.0 < ac.max() < halo.A_COLLAPSE_MAX
    for s, a in zip(sig, ac):
        assert heath(a) / heath(1.0) * s == pytest.approx(halo.DELTA_C, rel=2e-7)


def test_collapse_epoch_limits():
    """No root below a = 100: capped there; a root before the growth rule starts: its start."""
    ac = halo.collapse_epoch(np.array([1e-3, 1e5]), COSMO)
    assert ac[0] == halo.A_COLLAPSE_MAX and ac[1] == cz.A_INIT


def test_bullock_median_monotone_and_normalised():
    """c_bar = K a / a_c (Sec. 5.4, no floor): it falls with mass wherever F m
    collapses before a = 100 and is flat where the collapse epoch is capped,
    scales as a(z) everywhere, and equals K at the collapse epoch."""
    wl = workloads.get("tiny_2bin", cosmology=dict(COSMO), bins=dict(conc_model=halo.CONC_BULLOCK, m_min=1e9))
    T = Tables(wl)
    c0 = T.cbar(0)
    free = T.a_c < halo.A_COLLAPSE_MAX
    assert free.sum() >= 6 and np.all(np.diff(c0[free]) < 0) and np.all(np.diff(c0) <= 0)
    capped = ~free
    if capped.any():
        np.testing.assert_allclose(c0[capped], halo.BULLOCK_K / ((1 + T.z[0]) * halo.A_COLLAPSE_MAX), rtol=1e-15)
    assert c0.min() < 1.0  # the median leaves c >= 1 for the late-collapsing masses
    for n in (3, 9):  # proportional to a(z)
        cn = T.cbar(n)
        np.testing.assert_allclose(cn * (1 + T.z[n]), c0 * (1 + T.z[0]), rtol=1e-15)
    ac = T.a_c[3]
    assert halo.bullock_concentration(ac, 1.0 / ac - 1.0) == pytest.approx(halo.BULLOCK_K, rel=1e-14)
    # F m is the collapsing mass at a_c: sigma(F m, a_c) = delta_c
    sigF, _ = cz.sigma_and_dlnsigma_dlnm(halo.BULLOCK_F * T.m[3], T.amp, T.cosmo)
    assert cz.growth(1.0 / ac - 1.0, T.cosmo)[0] * sigF[0] == pytest.approx(halo.DELTA_C, rel=1e-12)


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
def test_nfw_profile_against_adaptive_quadrature_down_to_small_concentration():
    """u(k|m, c) against adaptive quadrature of its definition (the truncated
    NFW density transformed with sin(kr)/(kr), divided by its mass), from
    c = 5 down to c = 0.01, k from the linear regime to k_max = 50 h/Mpc:
    |du| <= 1e-12 |u| + 1e-15 on both sides of the switch at c = 1 (the
    closed form's error grows like eps/c^2 below it, the defining integral's
    does not)."""
    rho = cz.rho_mean(workloads.FIDUCIAL)
    m = 1e16
    rv = halo.r_vir(m, rho)
    for c in (5.0, 1.0, 0.9, 0.3, 0.1, 0.04, 0.01):
        for k in (0.05, 1.0, 10.0, 50.0):
            rs = rv / c
            prof = lambda r: 1.0 / ((r / rs) * (1 + r / rs) ** 2)
            norm = integrate.quad(lambda r: 4 * math.pi * r * r * prof(r), 0, rv, epsrel=2e-14, limit=200)[0]
            ft = integrate.quad(lambda r: 4 * math.pi * r * r * prof(r) * math.sin(k * r) / (k * r), 0, rv,
                                limit=8000, epsrel=2e-14, epsabs=0)[0]
            u = ft / norm
            got = float(halo.nfw_u(k, m, 0.0, rho, c))
            assert abs(got - u) <= 1e-12 * abs(u) + 1e-15, (c, k, got, u)


def test_nfw_profile_forms_agree_at_the_switch():
    """At c = 1 the closed form (well conditioned there) and the quadrature of
    the defining integral give the same u to rounding, at every K = k r_vir
    the tables reach (up to k_max r_vir(1e16) ~ 260): 1e-14, the closed form's own
    rounding near K -> 0, where u -> 1."""
    rho = cz.rho_mean(workloads.FIDUCIAL)
    for m in (1e10, 1e13, 1e16):
        for k in np.geomspace(1e-3, 50.0, 12):
            K = k * halo.r_vir(m, rho)
            assert abs(halo.nfw_u_integral(K, 1.0) - halo.nfw_u(k, m, 0.0, rho, 1.0)) <= 1e-14, (m, k)
