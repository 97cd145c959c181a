"""Principal components of the joint covariance (oracle, FP64): Sec. 6.

Test infrastructure, like the rest of the oracle package (see its header).

* Eq. SNPCA: C_ij = sum_a S_ai S_aj lambda_a, rows of S the orthonormal
  eigenvectors v_a of C and lambda_a their eigenvalues.
* Eq. NewObs: uncorrelated observables D^_a = sum_j S_aj D_j.
* Eq. SNperEign: (S/N)^2_a = D^_a^2 / lambda_a, the variance of D^_a being
  lambda_a.
* Eq. CumulSN: cumulative (S/N)^2 over the first a_max modes, with the modes
  ordered either by increasing variance lambda_a or by decreasing (S/N)_a.
  The sum over all modes is D^T C^-1 D, the total S/N^2.

Eigen-solver.  The paper stresses that the covariance's eigenvalues span ~30
orders of magnitude and uses a closed library for them.  A QR-type FP64
eigen-solver loses every eigenvalue below ~1e-16 of the largest.  Here the
eigen-pairs come from one-sided Jacobi on the Cholesky factor (Demmel &
Veselic 1992): with C = L L^T and G = L^T, plane rotations J of pairs of
columns of G make them orthogonal, G J = U diag(sigma); then
C = G^T G = J diag(sigma^2) J^T, so lambda = sigma^2 and the eigenvectors are
the columns of J.  For a positive definite C whose unit-diagonal scaling is
well conditioned (a graded matrix, as here) this gives every eigenvalue to
high relative accuracy, however small.  Rotation of columns p, q with Gram
entries a = |g_p|^2, b = |g_q|^2, c = g_p . g_q: zeta = (b - a)/(2c),
t = sign(zeta)/(|zeta| + sqrt(1 + zeta^2)), cos = 1/sqrt(1 + t^2),
sin = t cos; a pair is left alone once |c| <= tol sqrt(a b).  Plain loops:
for the small cases of the tests.

Reading: "the fraction of modes that recovers 99% of the information" is the
smallest number of modes, taken by decreasing (S/N)_a, whose cumulative S/N
(the square root of the cumulative (S/N)^2) reaches 99% of the total S/N.
"""
import math

import numpy as np

JACOBI_TOL = 1e-15
JACOBI_MAX_SWEEPS = 60


def jacobi_eigh(C, tol=JACOBI_TOL, max_sweeps=JACOBI_MAX_SWEEPS):
    """Eigenvalues (ascending) and eigenvectors (columns) of a symmetric positive
    definite C by one-sided Jacobi on its Cholesky factor.  Returns
    (lam, V, sweeps)."""
    C = np.asarray(C, dtype=np.float64)
    n = C.shape[0]
    L = np.linalg.cholesky(C)
    G = L.T.copy()
    V = np.eye(n)
    sweeps = 0
    for sweeps in range(1, max_sweeps + 1):
        rotated = False
        for p in range(n - 1):
            for q in range(p + 1, n):
                gp, gq = G[:, p], G[:, q]
                a = float(gp @ gp)
                b = float(gq @ gq)
                c = float(gp @ gq)
                if abs(c) <= tol * math.sqrt(a * b):
                    continue
                rotated = True
                zeta = (b - a) / (2.0 * c)
                t = math.copysign(1.0, zeta) / (abs(zeta) + math.sqrt(1.0 + zeta * zeta))
                cs = 1.0 / math.sqrt(1.0 + t * t)
                sn = cs * t
                G[:, p], G[:, q] = cs * gp - sn * gq, sn * gp + cs * gq
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p], V[:, q] = cs * vp - sn * vq, sn * vp + cs * vq
        if not rotated:
            break
    lam = np.einsum("ij,ij->j", G, G)
    order = np.argsort(lam)
    return lam[order], V[:, order], sweeps


def pca_snr(C, D):
    """Eqs. SNPCA, NewObs, SNperEign for covariance C and data vector D.

    Returns a dict: lam (ascending), S (rows = eigenvectors), Dhat, snr2 (per
    mode, in the lam order), total (sum of snr2)."""
    lam, V, _ = jacobi_eigh(C)
    S = V.T
    Dhat = S @ np.asarray(D, dtype=np.float64)
    snr2 = Dhat * Dhat / lam
    return {"lam": lam, "S": S, "Dhat": Dhat, "snr2": snr2, "total": float(np.sum(snr2))}


def cumulative(snr2, order="variance"):
    """Eq. CumulSN: cumulative (S/N)^2 with the modes in the paper's two orders:
    'variance' (increasing lambda: the order pca_snr returns) or 'information'
    (decreasing (S/N)_a)."""
    snr2 = np.asarray(snr2, dtype=np.float64)
    if order == "information":
        snr2 = np.sort(snr2)[::-1]
    elif order != "variance":
        raise ValueError(order)
    return np.cumsum(snr2)


def modes_for_fraction(snr2, fraction=0.99):
    """Smallest number of modes, by decreasing (S/N)_a, whose cumulative S/N
    reaches `fraction` of the total S/N (the reading in the module header)."""
    c = cumulative(snr2, "information")
    return int(np.searchsorted(np.sqrt(c), fraction * math.sqrt(c[-1])) + 1)
