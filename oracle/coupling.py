"""Exact bin-averaged couplings of the BB+PT terms (oracle, exact integers):
Appendix B, Eq. CovBB and the N_tri definition.

Test infrastructure, like the rest of the oracle package (see its header).

The binned bispectrum estimator averages kappa(q1) kappa(q2) kappa(q3) over
the N_tri ordered lattice triples of a bin triple tau = (A_a, A_b, A_c) with
q1 + q2 + q3 = 0 (App. B).  In the covariance of two such estimators the
BB and PT Wick terms join one leg x of tau to one leg y of tau' (their bins
equal): the pair of triangles (t, t') contributes only when leg x of t and
leg y of t' are the same lattice mode q (up to sign; the annuli are
symmetric).  With the polyspectra constant over the bins (the paper's
approximation), each such term carries the coupling

    kappa(tau, x; tau', y) = sum_{q in A} n_{tau,x}(q) n_{tau',y}(q) / (N_tau N_tau'),

n_{tau,x}(q) = #{triangles of tau whose leg x is q} = #{p in Y : q + p in Z},
{Y, Z} the bins of the two other legs.  Summed over q alone, n gives N_tau
(each triangle has exactly one leg x), so the PB term's coupling is exactly
1/N(A); and if n were constant over A the BB+PT coupling would be 1/N(A), the
paper's 2 pi / (Omega l Delta l) in the continuum.  Here the sum is taken
exactly.

n_{A|YZ}(q) = (1_Y * 1_Z)(q), the lattice convolution of the two annulus
indicators evaluated at q (the same convolution that gives N_tri when summed
over the third annulus); it depends on the bin of the leg and the unordered
pair of the other two bins only, so one column per (A; {Y, Z}) serves every
triangle and leg with those bins.  The Gram matrix
G_A[c, c'] = sum_{q in A} n_c(q) n_c'(q) is an exact integer (below 2^63 at
l_max = 5000; asserted).
"""
import math

import numpy as np
import scipy.fft as sfft


def columns(triangles, nbins):
    """For every bin A the ordered list of columns (Y, Z), Y <= Z, such that
    sorted (A, Y, Z) is one of `triangles`; and col[t][x], the column of leg x
    of triangle t in the list of its bin."""
    cols = [[] for _ in range(nbins)]
    index = [dict() for _ in range(nbins)]
    col = []
    for tri in triangles:
        cx = []
        for x in range(3):
            A = tri[x]
            Y, Z = sorted((tri[(x + 1) % 3], tri[(x + 2) % 3]))
            if (Y, Z) not in index[A]:
                index[A][(Y, Z)] = len(cols[A])
                cols[A].append((Y, Z))
            cx.append(index[A][(Y, Z)])
        col.append(tuple(cx))
    return cols, col


def _annulus(slo, shi):
    R = math.isqrt(int(shi) - 1)
    v = np.arange(-R, R + 1, dtype=np.int64)
    X, Y = np.meshgrid(v, v, indexing="xy")
    s = X * X + Y * Y
    m = (s >= slo) & (s < shi)
    return X[m], Y[m]


def leg_counts_bruteforce(s_lo, s_hi, A, Y, Z):
    """n_{A|YZ}(q) for every lattice point q of A (in the order of
    `annulus_points`), by direct enumeration of p in Y (tiny bins only)."""
    qx, qy = _annulus(s_lo[A], s_hi[A])
    px, py = _annulus(s_lo[Y], s_hi[Y])
    out = np.zeros(len(qx), dtype=np.int64)
    for i in range(len(qx)):
        sx = qx[i] + px
        sy = qy[i] + py
        s = sx * sx + sy * sy
        out[i] = np.count_nonzero((s >= s_lo[Z]) & (s < s_hi[Z]))
    return out


def annulus_points(s_lo, s_hi, A):
    """Lattice points of bin A: s_lo[A] <= |n|^2 < s_hi[A]."""
    return _annulus(s_lo[A], s_hi[A])


class LegCounts:
    """n_{A|YZ}(q) for the points q of every bin, by FFT lattice convolution on
    a periodic grid of side L >= 3R + 1 (no alias reaches |n| <= R), rounded to
    integers (the rounding margin is asserted)."""

    def __init__(self, s_lo, s_hi, workers=None):
        self.s_lo, self.s_hi = np.asarray(s_lo), np.asarray(s_hi)
        R = math.isqrt(int(max(s_hi)) - 1)
        self.L = sfft.next_fast_len(3 * R + 1)
        self.workers = workers
        self._spec = {}
        self._pts = {}

    def points(self, A):
        if A not in self._pts:
            x, y = annulus_points(self.s_lo, self.s_hi, A)
            self._pts[A] = (x, y)
        return self._pts[A]

    def _spectrum(self, b):
        if b not in self._spec:
            L = self.L
            x, y = self.points(b)
            g = np.zeros((L, L))
            g[np.mod(y, L), np.mod(x, L)] = 1.0
            self._spec[b] = sfft.rfft2(g, workers=self.workers)
        return self._spec[b]

    def at(self, Y, Z, bins):
        """{A: n_{A|YZ}(q) over the points of A} for every A in `bins`: one
        convolution of the indicators of Y and Z, read at the points of each A."""
        L = self.L
        conv = sfft.irfft2(self._spectrum(Y) * self._spectrum(Z), s=(L, L), workers=self.workers)
        out = {}
        for A in bins:
            x, y = self.points(A)
            vals = conv[np.mod(y, L), np.mod(x, L)]
            r = np.rint(vals)
            assert vals.size == 0 or float(np.max(np.abs(vals - r))) < 1e-3
            out[A] = r.astype(np.int64)
        return out

    def counts(self, A, pairs):
        """{(Y, Z): n_{A|YZ}(q) over the points of A} for the given pairs."""
        return {(Y, Z): self.at(Y, Z, [A])[A] for Y, Z in pairs}


def grams(s_lo, s_hi, triangles, bins=None, workers=None):
    """Exact Gram matrices G_A (int64, ncol_A x ncol_A) for the bins in `bins`
    (all by default), with their columns; returns (cols, col, {A: G_A}).
    Column c of bin A has the sum over q of n_c(q) equal to N_tri of the
    triangle sorted(A, Y, Z)."""
    nb = len(s_lo)
    cols, col = columns(triangles, nb)
    want = list(range(nb)) if bins is None else list(bins)
    lc = LegCounts(s_lo, s_hi, workers=workers)
    # one convolution per pair (Y, Z), read at every bin that has that column
    users = {}
    for A in want:
        for c, yz in enumerate(cols[A]):
            users.setdefault(yz, []).append((A, c))
    Nm = {A: np.zeros((len(lc.points(A)[0]), len(cols[A])), dtype=np.int64) for A in want}
    for (Y, Z), lst in users.items():
        vals = lc.at(Y, Z, sorted({A for A, _ in lst}))
        for A, c in lst:
            Nm[A][:, c] = vals[A]
    out = {}
    for A in want:
        # G[c][c'] <= max_q n_c'(q) * sum_q n_c(q): below 2^63 the int64
        # matmul is exact; above it, Python integers
        big = int(Nm[A].max()) if Nm[A].size else 0
        tot = int(Nm[A].sum(axis=0).max()) if Nm[A].size else 0
        if big * tot < 2**63:
            out[A] = Nm[A].T @ Nm[A]
        else:
            G = Nm[A].astype(object).T @ Nm[A].astype(object)
            assert max(int(v) for v in G.ravel()) < 2**63, "Gram entries leave int64"
            out[A] = G.astype(np.int64)
    return cols, col, out


def kappa_table(col, G, Ntri, triangles):
    """kappa(t, x; t', y) as a function, from the Gram matrices and the exact
    triangle counts: G_A[col(t, x), col(t', y)] / (N_tri(t) N_tri(t')), an FP64
    division of exact integers (column col(t, x) belongs to triangle t)."""

    def kappa(t1, x, t2, y):
        A = triangles[t1][x]
        assert triangles[t2][y] == A
        return float(G[A][col[t1][x], col[t2][y]]) / (float(Ntri[t1]) * float(Ntri[t2]))

    return kappa
