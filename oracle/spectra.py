"""Halo-model tables, 3D polyspectra, responses and Limber projection (oracle).

Paper sections followed:
  * Eq. nProjection: P^(n)_{i1..in} = int dchi chi^(2-2n) prod_i W_i P3D(l/chi).
  * Eq. ImunuHalos: I_mu^beta(k1..k_mu) = int dm b_beta (m/rho)^mu f_m
    int dc p(c, m) prod u(k_i, m, c).  With bins["n_conc"] >= 2 the inner
    integral is the lognormal of Eq. LogNormC ("model A", sigma_lnc =
    bins["sigma_lnc"]) on the Gauss-Hermite rule of halo.conc_rule; else p(c)
    is a delta function at the median ("model B") and the inner integral is a
    single evaluation.  The m_min regularisation is set on the mass rule
    alone: its halos at m_min carry the same concentration scatter.
  * Eq. PspHMtot2: P^HM = I_2^0 + (I_1^1)^2 P_lin.
  * Eqs. B1halo, B2halos, B3halos, BspHMtot: B^HM = B^1h + B^2h + B^3h with the
    tree-level B^PT, F2 kernel, b2 term and the tidal term
    4/7 I_1^1 I_1^1 S2 P P (1 - I_1^1(k3)) taken as printed.
  * Eq. General1h: 1-halo n-point function = I_n^0 (used by the covariance).
  * Eqs. PowerHMResp, BispHMResp, RespP, RespB: responses to a long mode,
    with dI_mu^beta/d delta_b read as I_mu^(beta+1) and the "P_lin(k)" of the
    I_2^2 term read as P_lin(k1).  B_G2 = 2 sum_cyc (mu_ab^2 - 1) P_a P_b.
  * Eq. Mask and the sigma_W^2 equation of Appendix B:
    sigma_W^2(chi) = 4 int d^2eps/(2 pi)^2 [J1(eps chi Theta)/(eps chi Theta)]^2
    P_lin(eps, z(chi)) with a 4096-node Gauss-Legendre rule in ln eps on
    [ln 1e-5, ln 1e3].
  * k_max = 50 h/Mpc (Sec. 4.5): a 3D polyspectrum or response at a
    line-of-sight node is set to zero when any of its legs has l/chi > k_max.

Line-of-sight rule: N_chi Gauss-Legendre nodes on [0, chi(z_max)].
"""
import math

import numpy as np
from scipy.special import j1

from . import cosmology as cz
from . import halo
from . import survey

N_EPS = 4096
LNEPS_MIN = math.log(1.0e-5)
LNEPS_MAX = math.log(1.0e3)
FD_H = 1.0e-3


class Tables:
    """Every per-node table the path needs for one workload."""

    def __init__(self, wl):
        cosmo, nz, bins = wl["cosmology"], wl["nz"], wl["bins"]
        self.cosmo, self.nz, self.bins = cosmo, nz, bins
        self.rho = cz.rho_mean(cosmo)
        self.omega, self.theta = survey.sky(bins["f_sky"])
        # line of sight
        self.chimax = cz.chi_of_z(nz["zmax"], cosmo)[0]
        self.chi, self.wchi = cz.gl_nodes(bins["n_chi"], 0.0, self.chimax)
        self.z = cz.z_of_chi(self.chi, cosmo)
        self.D = cz.growth(self.z, cosmo)
        self.amp = cz.plin_amplitude(cosmo)
        # ell bins
        self.ell_edges, self.ell, self.dell = survey.ell_bins(bins["n_ell"], bins["ell_min"], bins["ell_max"])
        # mass rule and halo tables
        self.m, self.om = halo.mass_nodes(bins["n_mass"], bins["m_min"], bins["m_max"])
        self.mr = self.m / self.rho
        sig0, dlns = cz.sigma_and_dlnsigma_dlnm(self.m, self.amp, cosmo)
        # median concentration rule (Duffy fit, or the Bullock et al. median of Sec. 5.4)
        self.conc_model = int(bins.get("conc_model", halo.CONC_DUFFY))
        if self.conc_model == halo.CONC_BULLOCK:
            sigF, _ = cz.sigma_and_dlnsigma_dlnm(halo.BULLOCK_F * self.m, self.amp, cosmo)
            self.a_c = halo.collapse_epoch(sigF, cosmo)
        nchi, nm = bins["n_chi"], bins["n_mass"]
        self.f = np.empty((nchi, nm))
        self.b1 = np.empty((nchi, nm))
        self.b2 = np.empty((nchi, nm))
        for n in range(nchi):
            fm, nu = halo.mass_function(self.m, self.D[n] * sig0, dlns, self.rho)
            b1, b2 = halo.st_biases(nu)
            self.f[n], self.b1[n], self.b2[n] = halo.regularise(self.m, self.om, fm, b1, b2, self.rho)
        # Limber wavenumbers, validity, profiles and linear spectra
        nl = bins["n_ell"]
        self.k = self.ell[:, None] / self.chi[None, :]
        self.valid = self.k <= bins["k_max"]
        # concentration rule: U[b, n, q, j] = u(l_b/chi_n, m_q, c_bar exp(s_j))
        self.cs, self.wc = halo.conc_rule(int(bins.get("n_conc", 0)), float(bins.get("sigma_lnc", 0.0)))
        nc = len(self.wc)
        self.U = np.zeros((nl, nchi, nm, nc))
        self.Pl = np.zeros((nl, nchi))
        self.dPl = np.zeros((nl, nchi))
        for b in range(nl):
            for n in range(nchi):
                if self.valid[b, n]:
                    cbar = self.cbar(n)
                    for j in range(nc):
                        self.U[b, n, :, j] = halo.nfw_u(self.k[b, n], self.m, self.z[n], self.rho,
                                                        cbar * math.exp(self.cs[j]))
                    self.Pl[b, n] = cz.plin(self.k[b, n], self.D[n], self.amp, cosmo)
                    self.dPl[b, n] = cz.dplin_dlnk(self.k[b, n], self.D[n], self.amp, cosmo, FD_H)
        # survey kernels and noise
        self.zedges = survey.tomo_edges(nz)
        self.W = survey.lensing_kernels(self.chi, self.z, nz, cosmo, self.zedges)
        self.noise = survey.shot_noise(nz)
        self.sigW2 = sigma_w2(self.chi, self.D, self.theta, self.amp, cosmo)

    def cbar(self, n):
        """Median concentration of every mass node at line-of-sight node n."""
        if self.conc_model == halo.CONC_BULLOCK:
            return halo.bullock_concentration(self.a_c, self.z[n])
        return halo.concentration(self.m, self.z[n])

    # -- halo integrals -------------------------------------------------
    def I(self, legs, mu, beta, n):
        """I_mu^beta at node n for the ell bins in ``legs`` (Eq. ImunuHalos):
        the sum over mass nodes q and concentration nodes j."""
        bb = (None, self.b1[n], self.b2[n])[beta]
        arr = self.om * self.f[n] * self.mr ** mu
        if bb is not None:
            arr = arr * bb
        arr = arr[:, None] * self.wc[None, :]
        for b in legs:
            arr = arr * self.U[b, n]
        return float(np.sum(arr))

    def legs_valid(self, legs, n):
        return all(self.valid[b, n] for b in legs)

    def proj(self, tomos, n):
        """T(i1..in; chi) = chi^(2-2n) prod W (Eq. nProjection)."""
        val = self.chi[n] ** (2 - 2 * len(tomos))
        for t in tomos:
            val *= self.W[t, n]
        return val


def sigma_w2(chi, D, theta, amp, cosmo):
    """sigma_W^2(chi) for a disk of angular radius Theta (Appendix B)."""
    lne, w = cz.gl_nodes(N_EPS, LNEPS_MIN, LNEPS_MAX)
    eps = np.exp(lne)
    p0 = cz.plin(eps, 1.0, amp, cosmo)
    out = np.empty(len(chi))
    for n, c in enumerate(chi):
        x = eps * c * theta
        win = j1(x) / x
        out[n] = 4.0 / (2.0 * math.pi) * np.sum(w * eps * eps * win * win * p0) * D[n] ** 2
    return out


# -- tree-level PT pieces ----------------------------------------------------
def _mus(k1, k2, k3):
    mu12 = (k3 * k3 - k1 * k1 - k2 * k2) / (2.0 * k1 * k2)
    mu23 = (k1 * k1 - k2 * k2 - k3 * k3) / (2.0 * k2 * k3)
    mu31 = (k2 * k2 - k3 * k3 - k1 * k1) / (2.0 * k3 * k1)
    return mu12, mu23, mu31


def F2(ka, kb, mu):
    return 5.0 / 7.0 + 0.5 * mu * (ka / kb + kb / ka) + 2.0 / 7.0 * mu * mu


def bpt_from(k1, k2, k3, P1, P2, P3):
    mu12, mu23, mu31 = _mus(k1, k2, k3)
    return (2.0 * F2(k1, k2, mu12) * P1 * P2 + 2.0 * F2(k2, k3, mu23) * P2 * P3
            + 2.0 * F2(k3, k1, mu31) * P3 * P1)


def bg2_from(k1, k2, k3, P1, P2, P3):
    mu12, mu23, mu31 = _mus(k1, k2, k3)
    return 2.0 * ((mu12 * mu12 - 1.0) * P1 * P2 + (mu23 * mu23 - 1.0) * P2 * P3
                  + (mu31 * mu31 - 1.0) * P3 * P1)


def s2(mu):
    """Tidal kernel S2 = mu^2 - 1/3 (Eq. TidalKernel)."""
    return mu * mu - 1.0 / 3.0


def dbpt_dlnk(ks, Dn, amp, cosmo, i, h=FD_H):
    """d B^PT / d ln k_i with the other two sides fixed (4th-order difference)."""
    def f(s):
        kk = list(ks)
        kk[i] = kk[i] * math.exp(s)
        P = [float(cz.plin(q, Dn, amp, cosmo)) for q in kk]
        return bpt_from(kk[0], kk[1], kk[2], P[0], P[1], P[2])
    return (-f(2 * h) + 8.0 * f(h) - 8.0 * f(-h) + f(-2 * h)) / (12.0 * h)


# -- 3D spectra at one line-of-sight node ----------------------------------
def p3d(T, b, n):
    if not T.valid[b, n]:
        return 0.0
    return T.I([b, b], 2, 0, n) + T.I([b], 1, 1, n) ** 2 * T.Pl[b, n]


def resp_p3d(T, b, n):
    if not T.valid[b, n]:
        return 0.0
    rlin = 47.0 / 21.0 * T.Pl[b, n] - T.dPl[b, n] / 3.0
    return T.I([b], 1, 1, n) ** 2 * rlin + T.I([b, b], 2, 1, n)


def b1h3d(T, tri, n):
    if not T.legs_valid(tri, n):
        return 0.0
    return T.I(list(tri), 3, 0, n)


def bhm3d(T, tri, n):
    if not T.legs_valid(tri, n):
        return 0.0
    l = list(tri)
    k = [T.k[b, n] for b in l]
    P = [T.Pl[b, n] for b in l]
    I11 = [T.I([b], 1, 1, n) for b in l]
    I12 = [T.I([b], 1, 2, n) for b in l]
    cyc = ((0, 1, 2), (1, 2, 0), (2, 0, 1))
    b1h = T.I(l, 3, 0, n)
    b2h = sum(I11[a] * T.I([l[b], l[c]], 2, 1, n) * P[a] for (a, b, c) in cyc)
    mus = _mus(k[0], k[1], k[2])  # mu12, mu23, mu31
    bpt = bpt_from(k[0], k[1], k[2], P[0], P[1], P[2])
    b3h = I11[0] * I11[1] * I11[2] * bpt
    for (a, b, c), mu in zip(cyc, mus):
        b3h += I11[a] * I11[b] * I12[c] * P[a] * P[b]
        b3h += 4.0 / 7.0 * I11[a] * I11[b] * s2(mu) * P[a] * P[b] * (1.0 - I11[c])
    return b1h + b2h + b3h


def resp_b3d(T, tri, n):
    if not T.legs_valid(tri, n):
        return 0.0
    l = list(tri)
    k = [T.k[b, n] for b in l]
    P = [T.Pl[b, n] for b in l]
    rlin = [47.0 / 21.0 * T.Pl[b, n] - T.dPl[b, n] / 3.0 for b in l]
    I11 = [T.I([b], 1, 1, n) for b in l]
    bpt = bpt_from(k[0], k[1], k[2], P[0], P[1], P[2])
    bg2 = bg2_from(k[0], k[1], k[2], P[0], P[1], P[2])
    dsum = sum(dbpt_dlnk(k, T.D[n], T.amp, T.cosmo, i) for i in range(3))
    rbpt = 433.0 / 126.0 * bpt + 5.0 / 126.0 * bg2 - dsum / 3.0
    out = I11[0] * I11[1] * I11[2] * rbpt
    for (a, b, c) in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        out += I11[a] * T.I([l[b], l[c]], 2, 2, n) * P[a]
        out += I11[a] * T.I([l[b], l[c]], 2, 1, n) * rlin[a]
    out += T.I(l, 3, 1, n)
    return out


class Spectra:
    """Per-node 3D spectra and their Limber projections for one workload."""

    def __init__(self, T, tris):
        nl, nchi, nt = len(T.ell), len(T.chi), T.nz["n_tomo"]
        self.T, self.tris = T, tris
        self.P3 = np.array([[p3d(T, b, n) for n in range(nchi)] for b in range(nl)])
        self.RP3 = np.array([[resp_p3d(T, b, n) for n in range(nchi)] for b in range(nl)])
        self.B3 = np.array([[bhm3d(T, t, n) for n in range(nchi)] for t in tris]).reshape(len(tris), nchi)
        self.RB3 = np.array([[resp_b3d(T, t, n) for n in range(nchi)] for t in tris]).reshape(len(tris), nchi)
        self.B1h3 = np.array([[b1h3d(T, t, n) for n in range(nchi)] for t in tris]).reshape(len(tris), nchi)
        w = T.wchi
        # projected spectra (Eq. nProjection with n = 2, 3); einsum is the sum
        W = T.W
        self.P = np.einsum("n,in,jn,bn->bij", w * T.chi ** -2.0, W, W, self.P3)
        # P^s with shot noise on the diagonal (Eq. ShotNoise)
        self.Ps = self.P.copy()
        for b in range(nl):
            for i in range(nt):
                self.Ps[b, i, i] += T.noise[i]
        self.B1h = np.einsum("n,in,jn,kn,tn->tijk", w * T.chi ** -4.0, W, W, W, self.B1h3)
        self.Bproj = np.einsum("n,in,jn,kn,tn->tijk", w * T.chi ** -4.0, W, W, W, self.B3)

    def data_value(self, row):
        """Expected data-vector entry: P_ij(l) or B_ijk(l_a, l_b, l_c) (no noise)."""
        if row[0] == "P":
            b, (i, j) = row[1], row[2]
            return self.P[b, i, j]
        i, j, k = row[3]
        return self.Bproj[row[1], i, j, k]
