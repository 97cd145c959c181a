"""Pins of the oracle's concentration scatter ("model A", Eq. LogNormC).

The oracle takes the c integral of Eq. ImunuHalos on a Gauss-Hermite rule in
ln c.  These checks fix it against what the paper and the mathematics give
independently of that rule: adaptive quadrature over c of the lognormal
density as the paper writes it, the closed-form lognormal moments, the
delta-function limit (model B), and the regularisation identities on the
enlarged node set.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import cosmology as cz
from oracle import halo
from oracle.pipeline import OracleRun
from paper_1812_07437_gb300 import workloads

COSMO = workloads.FIDUCIAL
SIG = workloads.SIGMA_LNC


def _p_lognormal(c, cbar, sig):
    """p(c, m) of Eq. LogNormC: lognormal in c about the median cbar."""
    return math.exp(-(math.log(c) - math.log(cbar)) ** 2 / (2 * sig * sig)) / (c * math.sqrt(2 * math.pi * sig * sig))


def _avg_quad(g, cbar, sig):
    """int dc p(c) g(c) by adaptive quadrature over c (eight widths each side)."""
    lo, hi = cbar * math.exp(-8 * sig), cbar * math.exp(8 * sig)
    return integrate.quad(lambda c: _p_lognormal(c, cbar, sig) * g(c), lo, hi, epsabs=0, epsrel=1e-13,
                          limit=400)[0]


def _avg_rule(g, cbar, n_conc, sig):
    s, w = halo.conc_rule(n_conc, sig)
    return float(sum(wj * g(cbar * math.exp(sj)) for sj, wj in zip(s, w)))


def test_conc_rule_lognormal_moments():
    """<c^p> = cbar^p exp(p^2 sigma^2 / 2) for a lognormal (closed form), to
    within the Gauss-Hermite remainder n!/(2n)! f^(2n) (f = exp(p sigma x))."""
    for n_conc in (4, 8, 12):
        for p in (1, 2, -1, 3):
            got = _avg_rule(lambda c: c ** p, 7.0, n_conc, SIG)
            a = abs(p) * SIG
            bound = math.factorial(n_conc) / math.factorial(2 * n_conc) * a ** (2 * n_conc) * math.exp(2 * a * a)
            assert got == pytest.approx(7.0 ** p * math.exp(p * p * SIG * SIG / 2), rel=max(bound, 5e-16))
    s, w = halo.conc_rule(8, SIG)
    assert np.sum(w) == pytest.approx(1.0, abs=1e-15)
    assert np.all(w > 0) and np.allclose(s, -s[::-1], atol=1e-15)


def test_conc_rule_average_of_u_against_density_quadrature():
    """sum_j w_j u(k|m, c_j) = int dc p(c, m) u(k|m, c), p from Eq. LogNormC."""
    rho = cz.rho_mean(COSMO)
    for m, z, k in ((1e12, 0.5, 0.3), (1e14, 0.0, 2.0), (1e11, 1.5, 20.0), (1e15, 1.0, 5e-3), (3e13, 0.7, 8.0)):
        cbar = halo.concentration(m, z)
        for power in (1, 2, 3):
            g = lambda c: float(halo.nfw_u(k, m, z, rho, c)) ** power
            ref = _avg_quad(g, cbar, SIG)
            assert _avg_rule(g, cbar, 16, SIG) == pytest.approx(ref, rel=1e-10, abs=1e-14)
    # with 8 nodes (the parity workloads' rule) the rule error stays below 1e-7
    cbar = halo.concentration(1e14, 0.3)
    g = lambda c: float(halo.nfw_u(3.0, 1e14, 0.3, rho, c)) ** 2
    assert _avg_rule(g, cbar, 8, SIG) == pytest.approx(_avg_quad(g, cbar, SIG), rel=1e-7)


def test_single_node_and_vanishing_width_are_model_b():
    """n_conc = 1 is model B exactly; sigma_lnc -> 0 tends to it."""
    base = OracleRun(workloads.get("tiny_2bin"))
    one = OracleRun(workloads.get("tiny_2bin", bins=dict(n_conc=1, sigma_lnc=SIG)))
    assert np.array_equal(one.T.U[..., 0], base.T.U[..., 0])
    assert np.array_equal(one.D, base.D)
    narrow = OracleRun(workloads.get("tiny_2bin", bins=dict(n_conc=6, sigma_lnc=1e-9)))
    np.testing.assert_allclose(narrow.D, base.D, rtol=1e-13)
    Cb = base.cov.full()
    Cn = narrow.cov.full()
    scale = np.sqrt(np.outer(np.diag(Cb), np.diag(Cb)))
    assert np.max(np.abs(Cn - Cb) / scale) < 1e-12


@pytest.fixture(scope="module")
def model_a():
    return OracleRun(workloads.get("tiny_2bin", bins=dict(n_conc=8, sigma_lnc=SIG)))


def test_halo_integral_against_density_quadrature(model_a):
    """I_mu^0 at one node: the mass rule times int dc p(c) prod u by quadrature."""
    T = model_a.T
    n = len(T.chi) // 2
    for legs in ([0, 0], [1, 3], [0, 2, 4], [2, 2, 2, 4]):
        if not T.legs_valid(legs, n):
            continue
        mu = len(legs)
        cbar = halo.concentration(T.m, T.z[n])
        tot = 0.0
        for q in range(len(T.m)):
            g = lambda c: float(np.prod([halo.nfw_u(T.k[b, n], T.m[q], T.z[n], T.rho, c) for b in legs]))
            tot += T.om[q] * T.f[n, q] * T.mr[q] ** mu * _avg_quad(g, cbar[q], SIG)
        assert T.I(legs, mu, 0, n) == pytest.approx(tot, rel=1e-7)


def test_regularisation_holds_with_scatter(model_a):
    """Eq. BoundinMass on the (mass, concentration) node set: the c weights sum to 1."""
    T = model_a.T
    for n in range(0, len(T.chi), 5):
        w = (T.om * T.mr * T.f[n])[:, None] * T.wc[None, :]
        assert np.sum(w) == pytest.approx(1.0, abs=1e-14)
        assert np.sum(w * T.b1[n][:, None]) == pytest.approx(1.0, abs=1e-14)
        assert abs(np.sum(w * T.b2[n][:, None])) < 1e-14


def test_block_form_equals_element_form_with_scatter(model_a):
    """F diag(g) F^T over (n, q, j) = the per-element 1-halo sums."""
    C = model_a.cov.one_halo_block()
    M = model_a.M
    rng = np.random.default_rng(7)
    for a, b in rng.integers(0, M, size=(40, 2)):
        ref = model_a.cov.one_halo(model_a.rows[a], model_a.rows[b])
        assert C[a, b] == pytest.approx(ref, rel=1e-12, abs=1e-300)


def test_scatter_changes_one_halo_more_than_spectra(model_a):
    """The scatter moves the 1-halo covariance by more than the data vector
    (the paper's Sec. 5.4 finding: percent-level on P and B, tens of percent on
    the bispectrum covariance); both move."""
    base = OracleRun(workloads.get("tiny_2bin"))
    dD = np.max(np.abs(model_a.D / base.D - 1.0))
    d1h = np.max(np.abs(np.diag(model_a.cov.one_halo_block()) / np.diag(base.cov.one_halo_block()) - 1.0))
    assert 1e-4 < dD < 0.1
    assert d1h > dD
