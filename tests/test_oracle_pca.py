"""Pins of the oracle's principal-component analysis (Sec. 6, Eqs. SNPCA,
NewObs, SNperEign, CumulSN).

* The one-sided Jacobi eigen-pairs agree with LAPACK's QR-based solver on
  well-conditioned matrices and reconstruct C.
* On a graded matrix whose eigenvalues span 28 orders of magnitude (the
  paper's warning) they agree with a 60-digit evaluation to high relative
  accuracy, the smallest included.
* The total over modes equals D^T C^-1 D from a Cholesky solve and the
  oracle's own cumulative S/N at the last ell bin.
* Closed forms: a diagonal C, a 2 x 2 C.
* Reordering the data vector permutes nothing but the eigenvector entries.
"""
import math

import numpy as np
import pytest
from scipy.linalg import cho_factor, cho_solve

from oracle import pca
from oracle.pipeline import OracleRun
from oracle.snr import WHICH_JOINT, cumulative_snr
from paper_1812_07437_gb300 import workloads


def _spd(n, seed, cond=30.0):
    """Seeded unit-diagonal SPD matrix with condition number about `cond`."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.geomspace(1.0, 1.0 / cond, n)) @ Q.T
    d = np.sqrt(np.diag(A))
    return A / np.outer(d, d)


def test_jacobi_agrees_with_lapack_on_well_conditioned_matrices():
    for n, seed in ((5, 1), (30, 2), (64, 3)):
        C = _spd(n, seed)
        lam, V, sweeps = pca.jacobi_eigh(C)
        ref = np.linalg.eigvalsh(C)
        np.testing.assert_allclose(lam, ref, rtol=1e-12)
        np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-13)
        np.testing.assert_allclose(V @ np.diag(lam) @ V.T, C, atol=1e-13)
        assert sweeps < 20


def test_graded_matrix_every_eigenvalue_to_high_relative_accuracy():
    """C = Sigma A Sigma with Sigma from 1 to 1e-14 (C over 28 orders):
    eigenvalues against a 60-digit symmetric eigen-solver."""
    mpmath = pytest.importorskip("mpmath")
    n = 20
    A = _spd(n, 11, cond=20.0)
    sig = np.geomspace(1.0, 1e-14, n)
    C = A * np.outer(sig, sig)
    lam, _, _ = pca.jacobi_eigh(C)
    with mpmath.workdps(60):
        E, _ = mpmath.eigsy(mpmath.matrix(C.tolist()))
        ref = np.array(sorted(float(e) for e in E))
    assert ref[0] / ref[-1] < 1e-26
    np.testing.assert_allclose(lam, ref, rtol=1e-12)


def test_closed_forms():
    # diagonal: eigenvalues the diagonal, (S/N)^2_a = D_a^2 / C_aa
    c = np.array([3.0, 1e-9, 7.0, 2e-4])
    D = np.array([1.0, -2e-5, 0.5, 3e-3])
    r = pca.pca_snr(np.diag(c), D)
    order = np.argsort(c)
    np.testing.assert_allclose(r["lam"], c[order], rtol=1e-15)
    np.testing.assert_allclose(r["snr2"], (D * D / c)[order], rtol=1e-14)
    # 2 x 2: lambda = (a + b)/2 -+ sqrt(((a - b)/2)^2 + c^2)
    a, b, cc = 2.0, 1.0, 0.6
    lam, V, _ = pca.jacobi_eigh(np.array([[a, cc], [cc, b]]))
    h = math.sqrt(((a - b) / 2) ** 2 + cc * cc)
    np.testing.assert_allclose(lam, [(a + b) / 2 - h, (a + b) / 2 + h], rtol=1e-15)
    v = V[:, 1]
    assert abs(v[1] / v[0] - cc / ((a + b) / 2 + h - b)) < 1e-14


@pytest.fixture(scope="module")
def tiny():
    return OracleRun(workloads.get("tiny_2bin"))


def test_total_over_modes_is_the_cumulative_snr(tiny):
    C = tiny.cov.full()
    r = pca.pca_snr(C, tiny.D)
    ref = float(tiny.D @ cho_solve(cho_factor(C), tiny.D))
    assert r["total"] == pytest.approx(ref, rel=1e-10)
    snr = cumulative_snr(C, tiny.D, tiny.rows, len(tiny.T.ell), WHICH_JOINT)
    assert math.sqrt(r["total"]) == pytest.approx(snr[-1], rel=1e-10)
    # Eq. SNPCA: the modes rebuild C; Eq. NewObs: D^ = S D has variance lambda
    S, lam = r["S"], r["lam"]
    d = np.sqrt(np.diag(C))
    np.testing.assert_allclose((S.T * lam) @ S / np.outer(d, d), C / np.outer(d, d), atol=1e-11)
    np.testing.assert_allclose(S @ C @ S.T, np.diag(lam), atol=1e-11 * lam.max())


def test_orders_and_fraction_reading(tiny):
    r = pca.pca_snr(tiny.cov.full(), tiny.D)
    cv = pca.cumulative(r["snr2"], "variance")
    ci = pca.cumulative(r["snr2"], "information")
    assert cv[-1] == pytest.approx(ci[-1], rel=1e-13)
    assert np.all(ci >= cv - 1e-12 * ci[-1])  # the information order dominates at every count
    k = pca.modes_for_fraction(r["snr2"], 0.99)
    assert math.sqrt(ci[k - 1]) >= 0.99 * math.sqrt(ci[-1]) > (math.sqrt(ci[k - 2]) if k > 1 else -1.0)
    # a hand-made spectrum: S/N^2 per mode 64, 16, 1 -> cumulative S/N 8, sqrt(80) = 8.944, 9
    assert pca.modes_for_fraction([1.0, 64.0, 16.0], 0.995) == 3   # 8.955 needs all three
    assert pca.modes_for_fraction([1.0, 64.0, 16.0], 0.99) == 2    # 8.91
    assert pca.modes_for_fraction([1.0, 64.0, 16.0], 8.0 / 9.0) == 1


def test_reordering_the_data_vector(tiny):
    C = tiny.cov.full()
    D = tiny.D
    perm = np.random.default_rng(5).permutation(len(D))
    a = pca.pca_snr(C, D)
    b = pca.pca_snr(C[np.ix_(perm, perm)], D[perm])
    np.testing.assert_allclose(b["lam"], a["lam"], rtol=1e-10)
    np.testing.assert_allclose(np.sort(b["snr2"]), np.sort(a["snr2"]), rtol=1e-8, atol=1e-12 * a["total"])
