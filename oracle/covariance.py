"""Joint P+B covariance terms (oracle, FP64): Sec. 3.2 and Appendix B.

Element-by-element forms, each the paper's expression written out:
  Gauss PP   Eq. CovPPG: delta_ll'/N(l) [P^s_ii' P^s_jj' + P^s_ij' P^s_ji'].
  Gauss BB   Appendix B: Omega/N_tri sum over the six leg permutations s of
             prod_a [bin(l_a) = bin(l'_s(a))] P^s_{t_a t'_s(a)}(l_a)
             (nonzero only for the same bin triple).
  1-halo     Eqs. CovPPNG, Ins5P, Ins6P: (1/Omega) P^(n+n')_1h of all legs,
             projected with Eq. nProjection and I^0 of Eq. General1h.
  BB + PT    Eq. CovBB: for each unprimed leg x and primed leg y in the same
             ell bin, 1/N(l_x) times
               B_{t'_y, t_rest}(tau) B_{t_x, t'_rest}(tau')  and
               P^s_{t_x t'_y}(l_x) T_{t_rest, t'_rest}(rest legs);
             the paper's prefactor 2 pi/(Omega l Delta l) is its continuum
             value of 1/N(l); the integer N(l^b) is used, as in the Gauss
             term.  B and T are the 1-halo polyspectra (Sec. 4.1).  With a
             `kappa` function (oracle/coupling.py) the exact lattice coupling
             kappa(tau, x; tau', y) replaces 1/N(l_x).
  PB         Eq. Covpb: for each leg y of the bispectrum in the bin of P,
             1/N(l) [P^s_{i t'_y} B_{j, t'_rest} + P^s_{j t'_y} B_{i, t'_rest}]
             (the printed tomographic indices are garbled; this is the Wick
             pairing of the 5-point function).
  SSC        Eq. WLSSCflatskyLimber: int dchi T_a T_b dP_a/d delta_b
             dP_b/d delta_b sigma_W^2(chi), with the projection kernel of
             Eq. nProjection (the 1/Omega of Eq. CovPP22 is not used; the
             Appendix-B form is dimensionally consistent with sigma_W^2 of
             Appendix B).

Block forms used for whole matrices: the 1-halo term as F diag(g) F^T with
F[a,(n,q,j)] = chi^(1-2 mu_a) prod W (m/rho)^mu_a prod U(c_j) and
g = w_n omega_q f~ w_j/Omega (the same sum over line-of-sight, mass and
concentration nodes, grouped per row), and the SSC term as S S^T.
"""
import itertools
import math

import numpy as np

TERM_G = 1
TERM_1H = 2
TERM_BBPT = 4
TERM_PB = 8
TERM_SSC = 16
TERMS_ALL = 31


def row_legs(row):
    return [row[1], row[1]] if row[0] == "P" else list(row[2])


def row_tomos(row):
    return list(row[2]) if row[0] == "P" else list(row[3])


class Covariance:
    def __init__(self, T, S, rows, tris, Nmodes, Ntri, kappa=None):
        self.T, self.S, self.rows, self.tris = T, S, rows, tris
        self.N = np.asarray(Nmodes, dtype=np.float64)
        self.Ntri = np.asarray(Ntri, dtype=np.float64)
        self.kappa = kappa  # exact BB+PT coupling (t, x, t', y) -> value, or None for 1/N(l)
        self._icache = {}

    # -- helpers -----------------------------------------------------------
    def I0_nodes(self, legs):
        """I^0_n(legs) at every node, zero where a leg exceeds k_max."""
        key = tuple(sorted(legs))
        if key not in self._icache:
            T = self.T
            mu = len(key)
            g = T.om[None, :] * T.f * T.mr[None, :] ** mu
            arr = g[:, :, None] * T.wc[None, None, :]
            for b in key:
                arr = arr * T.U[b]
            vals = arr.sum(axis=(1, 2))
            ok = np.all(T.valid[list(key)], axis=0)
            self._icache[key] = np.where(ok, vals, 0.0)
        return self._icache[key]

    def proj_nodes(self, tomos):
        T = self.T
        v = T.chi ** (2 - 2 * len(tomos))
        for t in tomos:
            v = v * T.W[t]
        return v

    def polyspec_1h(self, legs, tomos):
        """Projected 1-halo polyspectrum of any order (Eqs. nProjection, General1h)."""
        return float(np.sum(self.T.wchi * self.proj_nodes(tomos) * self.I0_nodes(legs)))

    # -- terms -------------------------------------------------------------
    def gauss(self, r1, r2):
        Ps = self.S.Ps
        if r1[0] == "P" and r2[0] == "P":
            if r1[1] != r2[1]:
                return 0.0
            b = r1[1]
            i, j = r1[2]
            k, l = r2[2]
            return (Ps[b, i, k] * Ps[b, j, l] + Ps[b, i, l] * Ps[b, j, k]) / self.N[b]
        if r1[0] == "B" and r2[0] == "B":
            if r1[1] != r2[1]:
                return 0.0
            bins, t1, t2 = r1[2], r1[3], r2[3]
            tot = 0.0
            for s in itertools.permutations(range(3)):
                if all(bins[a] == bins[s[a]] for a in range(3)):
                    tot += Ps[bins[0], t1[0], t2[s[0]]] * Ps[bins[1], t1[1], t2[s[1]]] * Ps[bins[2], t1[2], t2[s[2]]]
            return self.T.omega / self.Ntri[r1[1]] * tot
        return 0.0

    def one_halo(self, r1, r2):
        return self.polyspec_1h(row_legs(r1) + row_legs(r2), row_tomos(r1) + row_tomos(r2)) / self.T.omega

    def bbpt(self, r1, r2):
        if r1[0] != "B" or r2[0] != "B":
            return 0.0
        B1h, Ps = self.S.B1h, self.S.Ps
        bins1, t1 = r1[2], r1[3]
        bins2, t2 = r2[2], r2[3]
        tot = 0.0
        for x in range(3):
            for y in range(3):
                if bins1[x] != bins2[y]:
                    continue
                rx = [a for a in range(3) if a != x]
                ry = [a for a in range(3) if a != y]
                nN = self.N[bins1[x]]
                bb = B1h[r1[1], t2[y], t1[rx[0]], t1[rx[1]]] * B1h[r2[1], t1[x], t2[ry[0]], t2[ry[1]]]
                tt = self.polyspec_1h([bins1[rx[0]], bins1[rx[1]], bins2[ry[0]], bins2[ry[1]]],
                                      [t1[rx[0]], t1[rx[1]], t2[ry[0]], t2[ry[1]]])
                if self.kappa is None:
                    tot += (bb + Ps[bins1[x], t1[x], t2[y]] * tt) / nN
                else:
                    tot += (bb + Ps[bins1[x], t1[x], t2[y]] * tt) * self.kappa(r1[1], x, r2[1], y)
        return tot

    def pb(self, r1, r2):
        if r1[0] == r2[0]:
            return 0.0
        if r1[0] == "B":
            r1, r2 = r2, r1
        B1h, Ps = self.S.B1h, self.S.Ps
        b = r1[1]
        i, j = r1[2]
        bins2, t2 = r2[2], r2[3]
        tot = 0.0
        for y in range(3):
            if bins2[y] != b:
                continue
            ry = [a for a in range(3) if a != y]
            tot += (Ps[b, i, t2[y]] * B1h[r2[1], j, t2[ry[0]], t2[ry[1]]]
                    + Ps[b, j, t2[y]] * B1h[r2[1], i, t2[ry[0]], t2[ry[1]]]) / self.N[b]
        return tot

    def response_nodes(self, row):
        return self.S.RP3[row[1]] if row[0] == "P" else self.S.RB3[row[1]]

    def ssc(self, r1, r2):
        T = self.T
        v = (T.wchi * T.sigW2 * self.proj_nodes(row_tomos(r1)) * self.proj_nodes(row_tomos(r2))
             * self.response_nodes(r1) * self.response_nodes(r2))
        return float(np.sum(v))

    def element_terms(self, a, b):
        r1, r2 = self.rows[a], self.rows[b]
        return {TERM_G: self.gauss(r1, r2), TERM_1H: self.one_halo(r1, r2),
                TERM_BBPT: self.bbpt(r1, r2), TERM_PB: self.pb(r1, r2), TERM_SSC: self.ssc(r1, r2)}

    def element(self, a, b, terms=TERMS_ALL):
        vals = self.element_terms(a, b)
        return sum(v for t, v in vals.items() if terms & t)

    # -- whole matrices ----------------------------------------------------
    def full(self, terms=TERMS_ALL, elementwise_terms=None):
        """Whole M x M matrix; 1-halo and SSC by their block forms."""
        M = len(self.rows)
        C = np.zeros((M, M))
        if terms & TERM_1H:
            C += self.one_halo_block()
        if terms & TERM_SSC:
            S = self.ssc_rows()
            C += S @ S.T
        rest = terms & (TERM_G | TERM_BBPT | TERM_PB)
        if rest:
            for a in range(M):
                for b in range(a + 1):
                    r1, r2 = self.rows[a], self.rows[b]
                    v = 0.0
                    if rest & TERM_G:
                        v += self.gauss(r1, r2)
                    if rest & TERM_BBPT:
                        v += self.bbpt(r1, r2)
                    if rest & TERM_PB:
                        v += self.pb(r1, r2)
                    C[a, b] += v
                    if a != b:
                        C[b, a] += v
        return C

    def factor_rows(self):
        """F[a, (n, q, j)] of the 1-halo block form and the weights g[(n, q, j)]
        (j: concentration node; one node without scatter)."""
        T = self.T
        nchi, nm = T.f.shape
        nc = len(T.wc)
        F = np.zeros((len(self.rows), nchi * nm * nc))
        for a, r in enumerate(self.rows):
            legs, tom = row_legs(r), row_tomos(r)
            mu = len(legs)
            v = (T.chi ** (1 - 2 * mu))[:, None, None] * (T.mr ** mu)[None, :, None]
            for t in tom:
                v = v * T.W[t][:, None, None]
            for b in legs:
                v = v * T.U[b]
            ok = np.all(T.valid[legs], axis=0)
            F[a] = (v * ok[:, None, None]).ravel()
        g = (T.wchi[:, None, None] * T.om[None, :, None] * T.f[:, :, None] * T.wc[None, None, :] / T.omega).ravel()
        return F, g

    def one_halo_block(self):
        F, g = self.factor_rows()
        return (F * g[None, :]) @ F.T

    def ssc_rows(self):
        T = self.T
        S = np.zeros((len(self.rows), len(T.chi)))
        for a, r in enumerate(self.rows):
            S[a] = np.sqrt(T.wchi * T.sigW2) * self.proj_nodes(row_tomos(r)) * self.response_nodes(r)
        return S
