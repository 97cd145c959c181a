"""Cumulative signal-to-noise (oracle, FP64): Sec. 5, Eqs. SNprim and eq:SN.

(S/N)^2(l_max) = sum over entries whose ell bins are all <= l_max of
D_i [C^-1]_ij D_j, computed for every cumulative index by a direct solve of
the selected sub-matrix (no factor re-use).  The Jacobi scaling
C' = d^-1/2 C d^-1/2, D' = d^-1/2 D (d = diag C) leaves (S/N)^2 unchanged and
is applied before the Cholesky factorisation (scipy cho_factor/cho_solve as
the steps).  Reading: "l(i), l(j) < l_max" selects entries whose largest ell
bin is at most the cumulative bin index.
"""
import numpy as np
import scipy.linalg as sla

from .layout import max_bin

WHICH_P = 0
WHICH_B = 1
WHICH_JOINT = 2


def select(rows, which):
    if which == WHICH_P:
        return [a for a, r in enumerate(rows) if r[0] == "P"]
    if which == WHICH_B:
        return [a for a, r in enumerate(rows) if r[0] == "B"]
    return list(range(len(rows)))


def cumulative_snr(C, D, rows, n_ell, which=WHICH_JOINT):
    """S/N(l_max) for l_max = bin 0 .. n_ell-1 (NaN where nothing is selected)."""
    base = select(rows, which)
    out = np.full(n_ell, np.nan)
    for c in range(n_ell):
        idx = [a for a in base if max_bin(rows[a]) <= c]
        if not idx:
            continue
        Cs = C[np.ix_(idx, idx)]
        d = np.sqrt(np.diag(Cs))
        Cp = Cs / np.outer(d, d)
        Dp = D[idx] / d
        fac = sla.cho_factor(Cp, lower=True)
        out[c] = np.sqrt(Dp @ sla.cho_solve(fac, Dp))
    return out
