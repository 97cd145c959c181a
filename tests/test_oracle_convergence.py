"""Quadrature convergence of the oracle (a bound on discretisation error, not
parity): the data vector, the variances and the cumulative S/N of a small
workload settle as the line-of-sight and mass rules are refined together
(N_chi, N_M) -> (2 N_chi, 2 N_M)."""
import numpy as np

from oracle.pipeline import OracleRun
from oracle.snr import WHICH_JOINT, cumulative_snr
from paper_1812_07437_gb300 import workloads


def _run(n_chi, n_mass):
    r = OracleRun(workloads.get("tiny_2bin", bins=dict(n_chi=n_chi, n_mass=n_mass)))
    C = r.cov.full()
    return r.D, np.diag(C), cumulative_snr(C, r.D, r.rows, len(r.T.ell), WHICH_JOINT)[-1]


def test_refining_the_quadrature_converges():
    runs = [_run(16, 12), _run(32, 24), _run(64, 48)]
    steps = []
    for a, b in zip(runs[:-1], runs[1:]):
        steps.append((np.max(np.abs(a[0] / b[0] - 1)), np.max(np.abs(a[1] / b[1] - 1)), abs(a[2] / b[2] - 1)))
    (d1, v1, s1), (d2, v2, s2) = steps
    # each doubling shrinks the change at least fourfold (measured: 47x, 19x, 97x)
    assert d2 < d1 / 4 and v2 < v1 / 4 and s2 < s1 / 4
    # at (64, 48) nodes the S/N has settled to ~1e-4 or better
    assert s2 < 1e-4 and d2 < 1e-3 and v2 < 5e-3
