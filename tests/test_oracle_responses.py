"""Pins of the oracle's halo-model bispectrum and responses (Eqs. B2halos,
B3halos, PowerHMResp, BispHMResp, RespP, RespB) and of the super-sample term
(Eq. WLSSCflatskyLimber), each against what the mathematics fixes
independently of the oracle's own formulas (CPU only):

* the power-spectrum response to a long mode equals the angle-averaged
  squeezed limit of the tree-level bispectrum (a perturbation-theory identity,
  evaluated here numerically from the textbook F2 kernel), which fixes the
  47/21 and -1/3 of Eq. RespP;
* as k -> 0 the profiles go to 1, the halo integrals to closed discrete sums
  over the mass rule and P_lin to a power law of slope n_s; with the biases
  of the tables perturbed so that I_1^1 != 1 and I_1^2 != 0, every term of
  B^HM and of both responses is then a number computed here by hand from
  those sums (equilateral F2 = 2/7, B_PT = 12/7 P^2, B_G2 = -9/2 P^2,
  S2(-1/2) = -1/12, sum_i dB_PT/dln k_i = 2 n B_PT by homogeneity), so a
  wrong coefficient, a dropped cyclic term or a swapped bias index fails;
* B^HM and its response are symmetric in the three legs (the cyclic sums are
  complete);
* the super-sample term, with responses replaced by analytic functions of
  chi, is the continuous chi integral of Eq. WLSSCflatskyLimber (adaptive
  quadrature against the oracle's Gauss-Legendre sum).
"""
import math
import types

import numpy as np
import pytest

from oracle import cosmology as cz
from oracle import spectra as sp
from oracle import survey
from oracle.covariance import Covariance
from oracle.layout import data_layout
from paper_1812_07437_gb300 import workloads


# ---------------------------------------------------------------- squeezed limit
def _f2_vec(a, b):
    na, nb = np.linalg.norm(a), np.linalg.norm(b)
    mu = float(np.dot(a, b)) / (na * nb)
    return 5.0 / 7.0 + 0.5 * mu * (na / nb + nb / na) + 2.0 / 7.0 * mu * mu


def _squeezed_response(k, n, q=1e-4):
    """lim_{q->0} < B_tree(k1, k2, q) >_angle / P(q) / P(k) for P ~ k^n, with
    k1 + k2 + q = 0, |k1| = k, averaged over the angle between k1 and q."""
    P = lambda x: x ** n
    x, w = np.polynomial.legendre.leggauss(96)
    tot = 0.0
    for mu, wi in zip(x, w):
        k1 = np.array([0.0, 0.0, k])
        qv = q * k * np.array([math.sqrt(1.0 - mu * mu), 0.0, mu])
        k2 = -(k1 + qv)
        n1, n2, nq = np.linalg.norm(k1), np.linalg.norm(k2), np.linalg.norm(qv)
        B = (2 * _f2_vec(k1, k2) * P(n1) * P(n2) + 2 * _f2_vec(k2, qv) * P(n2) * P(nq)
             + 2 * _f2_vec(qv, k1) * P(nq) * P(n1))
        tot += 0.5 * wi * B / P(nq)
    return tot / P(k)


class _Stub:
    """The attributes resp_p3d reads, with chosen halo integrals and P_lin."""

    def __init__(self, P, dP, i11, i21):
        self.valid = np.ones((1, 1), dtype=bool)
        self.Pl = np.array([[P]])
        self.dPl = np.array([[dP]])
        self._i = {(1, 1): i11, (2, 1): i21}

    def I(self, legs, mu, beta, n):
        return self._i[(mu, beta)]


@pytest.mark.parametrize("n", [-1.0, -1.5, -2.2])
def test_power_response_is_the_squeezed_tree_bispectrum(n):
    """Eq. RespP: with I_1^1 = 1 and no 1-halo part, the response of P^HM is the
    tree-level response, which must equal the squeezed bispectrum limit."""
    k = 0.37
    P = k ** n
    got = sp.resp_p3d(_Stub(P, n * P, 1.0, 0.0), 0, 0)
    assert got / P == pytest.approx(_squeezed_response(k, n), rel=1e-7, abs=0)
    # the halo factors: the linear response scales with (I_1^1)^2, the 1-halo part adds I_2^1
    g2 = sp.resp_p3d(_Stub(P, n * P, 1.3, 0.25), 0, 0)
    assert g2 == pytest.approx(1.69 * got + 0.25, rel=1e-14, abs=0)


# ---------------------------------------------------------------- k -> 0 limits
@pytest.fixture(scope="module")
def k0():
    """Tables at l ~ 1e-6 (k <~ 1e-7 h/Mpc: u = 1 to ~1e-14 and P_lin = A k^n_s D^2
    with a log-slope within ~1e-9 of n_s) with the biases perturbed: b1 -> 1.1 b1 (I_1^1 = 1.1), b2 -> b2 + 0.3
    (I_1^2 = 0.3), which switches on every term of B^HM and the responses."""
    wl = workloads.get("tiny_2bin", bins=dict(ell_min=1e-6, ell_max=2e-6))
    T = sp.Tables(wl)
    T.b1 = 1.1 * T.b1
    T.b2 = T.b2 + 0.3
    return T


def _sums(T, n):
    s = lambda bb, mu: float(np.sum(T.om * T.f[n] * bb * T.mr ** mu))
    one = np.ones_like(T.mr)
    return dict(I11=s(T.b1[n], 1), I12=s(T.b2[n], 1), I21=s(T.b1[n], 2), I22=s(T.b2[n], 2),
                I30=s(one, 3), I31=s(T.b1[n], 3))


def test_k0_sums_are_the_perturbed_consistency_relations(k0):
    T = k0
    for n in (0, 7, 15):
        S = _sums(T, n)
        assert S["I11"] == pytest.approx(1.1, rel=1e-12, abs=0)
        assert S["I12"] == pytest.approx(0.3, rel=1e-12, abs=0)
        for legs, mu, beta, key in (([0], 1, 1, "I11"), ([0], 1, 2, "I12"), ([0, 0], 2, 1, "I21"),
                                    ([0, 0], 2, 2, "I22"), ([0, 0, 0], 3, 0, "I30"), ([0, 0, 0], 3, 1, "I31")):
            assert T.I(legs, mu, beta, n) == pytest.approx(S[key], rel=1e-10, abs=0)  # u = 1 - O((k r_vir)^2)


class _Tri:
    """The attributes bhm3d and resp_b3d read, for three legs of equal k with
    chosen halo integrals (keyed by mu, beta) and a power-law P_lin."""

    def __init__(self, k, A, ns, ints):
        self.k = np.full((1, 1), k)
        self.Pl = np.full((1, 1), A * k ** ns)
        self.dPl = ns * self.Pl
        self.valid = np.ones((1, 1), dtype=bool)
        self.D = np.ones(1)
        self.amp = A
        self.cosmo = dict(ns=ns)
        self._i = ints

    def legs_valid(self, legs, n):
        return True

    def I(self, legs, mu, beta, n):
        return self._i[(mu, beta)]


@pytest.mark.parametrize("ns", [-1.5, -2.0])
def test_equilateral_bispectrum_and_responses_closed_forms(monkeypatch, ns):
    """Eqs. B1halo + B2halos + B3halos, PowerHMResp + RespP, BispHMResp + RespB
    at three equal legs (mu = -1/2 on every pair), P_lin = A k^n (P ~ 6, so the
    P^2 terms weigh as much as the others) and halo integrals of distinct values:
    every coefficient and the count of every cyclic term shows."""
    monkeypatch.setattr(cz, "plin", lambda k, Dg, amp, cosmo: amp * np.asarray(k) ** cosmo["ns"] * Dg * Dg)
    i11, i12, i21, i22, i30, i31 = 1.1, 0.3, 0.7, 0.45, 0.2, 0.35
    T = _Tri(0.3, 1.0, ns, {(1, 1): i11, (1, 2): i12, (2, 1): i21, (2, 2): i22, (3, 0): i30, (3, 1): i31})
    P = T.Pl[0, 0]
    rlin = (47.0 / 21.0 - ns / 3.0) * P
    bhm = (i30 + 3 * i11 * i21 * P + i11 ** 3 * (12.0 / 7.0) * P * P + 3 * i11 * i11 * i12 * P * P
           + 3 * (4.0 / 7.0) * i11 * i11 * (-1.0 / 12.0) * P * P * (1.0 - i11))
    assert sp.bhm3d(T, (0, 0, 0), 0) == pytest.approx(bhm, rel=1e-12, abs=0)
    assert sp.resp_p3d(T, 0, 0) == pytest.approx(i11 * i11 * rlin + i21, rel=1e-12, abs=0)
    rbpt = (433.0 / 126.0 * 12.0 / 7.0 + 5.0 / 126.0 * (-4.5) - 2.0 * ns / 3.0 * 12.0 / 7.0) * P * P
    resp_b = i11 ** 3 * rbpt + 3 * i11 * i22 * P + 3 * i11 * i21 * rlin + i31
    assert sp.resp_b3d(T, (0, 0, 0), 0) == pytest.approx(resp_b, rel=1e-9, abs=0)


@pytest.mark.parametrize("n", [0, 9, 15])
def test_k0_tables_reduce_to_the_closed_forms(k0, n):
    """The same closed forms on the real tables as k -> 0 (u = 1, the halo
    integrals the discrete sums of the mass rule, P_lin a power law)."""
    T = k0
    ns = T.cosmo["ns"]
    S = _sums(T, n)
    b = 1
    P = T.Pl[b, n]
    assert T.dPl[b, n] == pytest.approx(ns * P, rel=1e-9, abs=0)
    i11, i12, i21, i22, i30, i31 = (S[k] for k in ("I11", "I12", "I21", "I22", "I30", "I31"))
    rlin = (47.0 / 21.0 - ns / 3.0) * P
    bhm = (i30 + 3 * i11 * i21 * P + i11 ** 3 * (12.0 / 7.0) * P * P + 3 * i11 * i11 * i12 * P * P
           + 3 * (4.0 / 7.0) * i11 * i11 * (-1.0 / 12.0) * P * P * (1.0 - i11))
    assert sp.bhm3d(T, (b, b, b), n) == pytest.approx(bhm, rel=1e-9, abs=0)
    assert sp.resp_p3d(T, b, n) == pytest.approx(i11 * i11 * rlin + i21, rel=1e-9, abs=0)
    rbpt = (433.0 / 126.0 * 12.0 / 7.0 + 5.0 / 126.0 * (-4.5) - 2.0 * ns / 3.0 * 12.0 / 7.0) * P * P
    resp_b = i11 ** 3 * rbpt + 3 * i11 * i22 * P + 3 * i11 * i21 * rlin + i31
    assert sp.resp_b3d(T, (b, b, b), n) == pytest.approx(resp_b, rel=1e-8, abs=0)


def test_bispectrum_and_response_symmetric_in_the_legs():
    """Scalene triangles at l ~ 100-800 (u != 1, P_lin not a power law): every
    ordering of the three legs gives the same B^HM and response."""
    T = sp.Tables(workloads.get("tiny_2bin"))
    T.b2 = T.b2 + 0.2  # the b2 term on
    for tri in ((0, 1, 2), (1, 2, 3), (0, 2, 2)):
        for n in (4, 11):
            ref_b, ref_r = sp.bhm3d(T, tri, n), sp.resp_b3d(T, tri, n)
            assert ref_b != 0.0 and ref_r != 0.0
            for p in ((1, 2, 0), (2, 0, 1), (0, 2, 1), (2, 1, 0), (1, 0, 2)):
                t2 = tuple(tri[i] for i in p)
                assert sp.bhm3d(T, t2, n) == pytest.approx(ref_b, rel=1e-12, abs=0)
                assert sp.resp_b3d(T, t2, n) == pytest.approx(ref_r, rel=1e-7, abs=0)


# ---------------------------------------------------------------- super-sample term
def test_ssc_is_the_continuous_chi_integral():
    """Eq. WLSSCflatskyLimber: C_ssc = int dchi T_a T_b R_a R_b sigma_W^2 with
    T = chi^(2 - 2n) prod W.  Responses replaced by analytic functions of chi
    (P rows: a constant per ell bin; B rows: a constant times (chi/chi_max)^4,
    which keeps the B integrands finite at chi -> 0), kernels with photo-z
    scatter (smooth in chi): the oracle's Gauss-Legendre sum over 96 nodes
    against adaptive quadrature of the continuous integral."""
    wl = workloads.get("tiny_2bin", bins=dict(n_chi=96))
    T = sp.Tables(wl)
    rows, tris = data_layout(T.ell, wl["nz"]["n_tomo"])
    chimax = T.chimax
    cP = {b: 1.0 + 0.3 * b for b in range(len(T.ell))}
    cB = {t: 0.5 + 0.1 * t for t in range(len(tris))}
    S = types.SimpleNamespace(
        RP3=np.array([cP[b] * (T.chi / chimax) ** 2 for b in range(len(T.ell))]),
        RB3=np.array([cB[t] * (T.chi / chimax) ** 4 for t in range(len(tris))]))
    cov = Covariance(T, S, rows, tris, np.ones(len(T.ell)), np.ones(len(tris)))
    zed = survey.tomo_edges(wl["nz"])
    # the continuous integrand on an independent composite rule (40 panels of
    # 16 Gauss-Legendre nodes on [0, chi_max]): kernels and sigma_W^2 evaluated
    # at each of its 640 points
    x, w = np.polynomial.legendre.leggauss(16)
    P = 40
    chis = ((np.arange(P)[:, None] + 0.5 * (x[None, :] + 1.0)) * chimax / P).ravel()
    wts = np.tile(w, P) * 0.5 * chimax / P
    zs = cz.z_of_chi(chis, T.cosmo)
    Wc = survey.lensing_kernels(chis, zs, wl["nz"], T.cosmo, zed)
    s2 = sp.sigma_w2(chis, cz.growth(zs, T.cosmo), T.theta, T.amp, T.cosmo)

    def continuous(r1, r2):
        val = wts * s2
        for r in (r1, r2):
            tom = r[2] if r[0] == "P" else r[3]
            val = val * chis ** (2 - 2 * len(tom)) * np.prod([Wc[t] for t in tom], axis=0)
            val = val * (cP[r[1]] * (chis / chimax) ** 2 if r[0] == "P" else cB[r[1]] * (chis / chimax) ** 4)
        return float(np.sum(val))

    iP = [a for a, r in enumerate(rows) if r[0] == "P"]
    iB = [a for a, r in enumerate(rows) if r[0] == "B"]
    for a, b in ((iP[0], iP[0]), (iP[-1], iP[2]), (iB[3], iP[1]), (iB[-1], iB[5]), (iB[10], iB[10])):
        got = cov.ssc(rows[a], rows[b])
        ref = continuous(rows[a], rows[b])
        assert got == pytest.approx(ref, rel=5e-6, abs=0), (rows[a], rows[b])
