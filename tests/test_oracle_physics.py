"""Pins of the oracle's background, halo and survey functions (CPU only).

Each check compares against something the paper or the mathematics fixes
independently of the oracle code: adaptive quadrature of the defining
integral, closed forms, printed values, or limits.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import cosmology as cz
from oracle import halo, survey
from paper_1812_07437_gb300 import workloads

COSMO = workloads.FIDUCIAL
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_chi_matches_adaptive_quadrature():
    for z in (0.1, 1.0, 2.5, 3.0):
        ref = cz.C_OVER_H0 * integrate.quad(lambda x: 1.0 / cz.E(x, COSMO), 0.0, z, epsabs=0, epsrel=1e-13)[0]
        assert cz.chi_of_z(z, COSMO)[0] == pytest.approx(ref, rel=1e-13)
    chi = cz.chi_of_z(np.array([0.3, 1.7]), COSMO)
    assert np.allclose(cz.z_of_chi(chi, COSMO), [0.3, 1.7], rtol=1e-14, atol=0)


def test_growth_lcdm_integral_form():
    """For w = -1 the growth factor is D ~ H(a) int_0^a da'/(a' H)^3 (Heath 1977)."""
    def heath(a):
        H = lambda x: math.sqrt(COSMO["Om"] * x ** -3 + 1.0 - COSMO["Om"])
        return H(a) * integrate.quad(lambda x: 1.0 / (x * H(x)) ** 3, 0.0, a, epsabs=0, epsrel=1e-13)[0]
    zs = np.array([0.0, 0.5, 1.5, 3.0])
    ref = np.array([heath(1 / (1 + z)) for z in zs]) / heath(1.0)
    assert np.allclose(cz.growth(zs, COSMO), ref, rtol=2e-7, atol=0)
    eds = dict(COSMO, Om=1.0)
    assert np.allclose(cz.growth(zs, eds), 1.0 / (1.0 + zs), rtol=1e-10)


def test_eh_nowiggle_limits():
    assert cz.eh_nowiggle_T(1e-6, COSMO) == pytest.approx(1.0, abs=1e-4)
    T = cz.eh_nowiggle_T(np.logspace(-4, 2, 200), COSMO)
    assert np.all(np.diff(T) < 0)
    # large-k limit: T ~ ln(q)/q^2, so the log slope tends to -2 from above
    k1, k2 = 1e3, 2e3
    slope = math.log(cz.eh_nowiggle_T(k2, COSMO) / cz.eh_nowiggle_T(k1, COSMO)) / math.log(k2 / k1)
    assert -2.0 < slope < -1.8


def test_tophat_series_matches_closed_form():
    x = np.array([0.3, 0.49, 0.5, 0.51, 0.7])
    direct = 3 * (np.sin(x) - x * np.cos(x)) / x ** 3
    assert np.allclose(cz.tophat_W(x), direct, rtol=1e-14)
    ddirect = 3 * ((x * x - 3) * np.sin(x) + 3 * x * np.cos(x)) / x ** 4
    assert np.allclose(cz.tophat_dW(x), ddirect, rtol=1e-12)
    h = 1e-5
    xs = np.array([1e-3, 0.2])
    fd = (cz.tophat_W(xs + h) - cz.tophat_W(xs - h)) / (2 * h)
    assert np.allclose(cz.tophat_dW(xs), fd, rtol=1e-7, atol=1e-12)


def test_sigma8_normalisation_and_sigma_quadrature():
    amp = cz.plin_amplitude(COSMO)
    s, dl = cz.sigma_and_dlnsigma_dlnm(4.0 * math.pi / 3.0 * 8.0 ** 3 * cz.rho_mean(COSMO), amp, COSMO)
    assert s[0] == pytest.approx(COSMO["sigma8"], rel=1e-12)
    # adaptive quadrature of sigma^2(R) for R = 1 Mpc/h
    R = 1.0
    f = lambda lk: amp * math.exp(lk) ** (3 + COSMO["ns"]) * cz.eh_nowiggle_T(math.exp(lk), COSMO) ** 2 \
        / (2 * math.pi ** 2) * cz.tophat_W(np.array([math.exp(lk) * R]))[0] ** 2
    ref = integrate.quad(f, cz.LNK_MIN, cz.LNK_MAX, limit=2000, epsabs=0, epsrel=1e-12)[0]
    m = 4.0 * math.pi / 3.0 * R ** 3 * cz.rho_mean(COSMO)
    s, dl = cz.sigma_and_dlnsigma_dlnm(m, amp, COSMO)
    assert s[0] ** 2 == pytest.approx(ref, rel=1e-9)
    # d ln sigma / d ln m against a finite difference of sigma
    e = 1e-4
    sp, _ = cz.sigma_and_dlnsigma_dlnm(m * math.exp(e), amp, COSMO)
    sm, _ = cz.sigma_and_dlnsigma_dlnm(m * math.exp(-e), amp, COSMO)
    assert dl[0] == pytest.approx((math.log(sp[0]) - math.log(sm[0])) / (2 * e), rel=1e-6)


def test_st_normalisation():
    """int_0^inf f(nu) d nu = 1 (consistency relation, Eq. BoundinMass, beta = 0)."""
    val = integrate.quad(lambda nu: halo.st_G(nu) / nu, 0, np.inf, limit=500, epsrel=1e-12)[0]
    assert val == pytest.approx(1.0, rel=1e-9)


def test_st_biases_peak_background_split():
    """b1, b2 against finite differences of G(nu) with delta_c -> delta_c - delta_b."""
    sigma = np.array([0.4, 0.9, 1.6, 3.0])
    dc = halo.DELTA_C
    G = lambda d: halo.st_G(((dc - d) / sigma) ** 2)
    h = 1e-3
    g0 = G(0.0)
    d1 = (-G(2 * h) + 8 * G(h) - 8 * G(-h) + G(-2 * h)) / (12 * h) / g0
    d2 = (-G(2 * h) + 16 * G(h) - 30 * g0 + 16 * G(-h) - G(-2 * h)) / (12 * h * h) / g0
    b1, b2 = halo.st_biases((dc / sigma) ** 2)
    assert np.allclose(b1, 1.0 + d1, rtol=1e-6)
    assert np.allclose(b2, 8.0 / 21.0 * d1 + d2, rtol=1e-5, atol=1e-6)
    # published Sheth-Tormen linear bias
    nu = (dc / sigma) ** 2
    qn = halo.ST_Q * nu
    st_b1 = 1 + (qn - 1) / dc + 2 * halo.ST_P / (dc * (1 + qn ** halo.ST_P))
    assert np.allclose(b1, st_b1, rtol=1e-14)


def test_bias_consistency_continuum():
    """int b1 f dnu = 1 and int b2 f dnu = 0 over all masses (Eq. BoundinMass)."""
    f1 = lambda nu: halo.st_biases(nu)[0] * halo.st_G(nu) / nu
    f2 = lambda nu: halo.st_biases(nu)[1] * halo.st_G(nu) / nu
    assert integrate.quad(f1, 0, np.inf, limit=500, epsrel=1e-11)[0] == pytest.approx(1.0, rel=1e-8)
    assert abs(integrate.quad(f2, 0, np.inf, limit=500, epsrel=1e-11)[0]) < 1e-8


def test_regularisation_discrete_sums(oracle_cfg1):
    """Eq. BoundinMass holds exactly on the discrete mass rule after Eq. effectiveMasBias."""
    T = oracle_cfg1.T
    for n in range(0, len(T.chi), 7):
        w = T.om * T.mr * T.f[n]
        assert np.sum(w) == pytest.approx(1.0, abs=1e-14)
        assert np.sum(w * T.b1[n]) == pytest.approx(1.0, abs=1e-14)
        assert abs(np.sum(w * T.b2[n])) < 1e-14


def test_nfw_u_against_direct_fourier_transform():
    """u(k|m) = int_0^rvir 4 pi r^2 rho_NFW(r) sin(kr)/(kr) dr / m."""
    rho = cz.rho_mean(COSMO)
    for m, z, k in ((1e12, 0.5, 0.3), (1e14, 0.0, 2.0), (1e11, 1.5, 20.0), (1e15, 1.0, 5e-3)):
        c = halo.concentration(m, z)
        rv = halo.r_vir(m, rho)
        rs = rv / c
        prof = lambda r: 1.0 / ((r / rs) * (1 + r / rs) ** 2)
        norm = integrate.quad(lambda r: 4 * math.pi * r * r * prof(r), 0, rv, epsrel=1e-13)[0]
        ft = integrate.quad(lambda r: 4 * math.pi * r * r * prof(r) * math.sin(k * r) / (k * r), 0, rv,
                            limit=2000, epsrel=1e-13, epsabs=0)[0]
        assert halo.nfw_u(k, m, z, rho) == pytest.approx(ft / norm, rel=1e-9, abs=1e-12)
    assert halo.nfw_u(1e-7, 1e13, 0.0, rho) == pytest.approx(1.0, abs=1e-10)


def test_equipopulated_bins():
    nz = workloads.get("cfg2_5bin")["nz"]
    edges = survey.tomo_edges(nz)
    tot = integrate.quad(lambda z: survey.nz_shape(z, nz), nz["zmin"], nz["zmax"], epsrel=1e-13)[0]
    for i in range(nz["n_tomo"]):
        part = integrate.quad(lambda z: survey.nz_shape(z, nz), edges[i], edges[i + 1], epsrel=1e-13)[0]
        assert part / tot == pytest.approx(1.0 / nz["n_tomo"], rel=1e-10)


def test_paper_printed_edges_loose():
    """Appendix A / Sec. 5.1 printed edges, reproduced to the ~1e-2 the text allows."""
    with open(os.path.join(GOLDEN, "paper_tomo_edges.txt")) as fh:
        rows = [[float(x) for x in l.split()] for l in fh if l.strip() and not l.startswith("#")]
    for row in rows:
        nt = int(row[0])
        nz = dict(n_tomo=nt, z0=0.9 / math.sqrt(2), alpha=1.5, zmin=0.001, zmax=2.5, photoz_sigma0=0.0,
                  n_gal_arcmin2=30.0, sigma_e=0.3)
        assert np.max(np.abs(survey.tomo_edges(nz) - np.array(row[1:]))) < 0.015


def test_lensing_kernel_adaptive_quadrature():
    """Eqs. KernelLensing1 and LensEff against adaptive quadrature (no photo-z)."""
    nz = workloads.get("mid_2bin")["nz"]
    edges = survey.tomo_edges(nz)
    chis = cz.chi_of_z(np.array([0.2, 0.7, 1.4]), COSMO)
    zs = cz.z_of_chi(chis, COSMO)
    W = survey.lensing_kernels(chis, zs, nz, COSMO, edges)
    for i in range(2):
        norm = integrate.quad(lambda z: survey.nz_shape(z, nz), edges[i], edges[i + 1], epsrel=1e-13)[0]
        for n, (chi, z) in enumerate(zip(chis, zs)):
            lo = max(z, edges[i])
            if lo >= edges[i + 1]:
                assert W[i, n] == 0.0
                continue
            integ = integrate.quad(lambda x: survey.nz_shape(x, nz) * (cz.chi_of_z(x, COSMO)[0] - chi)
                                   / cz.chi_of_z(x, COSMO)[0], lo, edges[i + 1], epsrel=1e-11)[0]
            ref = 1.5 * COSMO["Om"] * cz.H0 ** 2 * (1 + z) * chi * integ / norm
            assert W[i, n] == pytest.approx(ref, rel=1e-9)


def test_shot_noise_value():
    nz = workloads.get("cfg2_5bin")["nz"]
    nbar = 30.0 * (180 * 60 / math.pi) ** 2 / 5
    assert np.allclose(survey.shot_noise(nz), 0.09 / nbar, rtol=1e-15)
