"""GPU principal components of the joint covariance (Sec. 6, Eqs. SNPCA,
NewObs, SNperEign, CumulSN) against the oracle's (tests/golden/make_pca.py:
oracle covariance, oracle one-sided Jacobi), on the paper's own set-up with 1
and 2 tomographic bins (M = 144, 818; eigenvalues spanning ~23 decades).

* The oracle's own covariance through cov_pca: only the eigen-solvers differ
  (both one-sided Jacobi on the Cholesky factor, in FP64, in different pair
  orders), so every eigenvalue agrees to 1e-10 relative, the smallest
  included, the per-mode (S/N)^2 to 1e-10 of the total, and the mode counts
  for 90/95/99% of the S/N exactly.
* The whole GPU path (FP64 covariance of the handle, then cov_pca): the
  covariance itself differs from the oracle's by ~1e-12 of sqrt(C_aa C_bb)
  (the FP64 parity of the other tests), which moves an eigenvalue by up to
  that times the condition number of the unit-diagonal scaling (~1e3-1e4
  here), so eigenvalues to 1e-7 relative; the total (S/N)^2 to 1e-9 and the
  mode counts exactly.
* The cumulative forms are prefix sums of the per-mode values in the two
  orders, and their last entry is D^T C^-1 D (the S/N of cov_snr squared).
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.covariance import TERMS_ALL  # noqa: E402
from oracle.pipeline import OracleRun  # noqa: E402
from paper_1812_07437_gb300 import native as N  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_counts  # noqa: E402
import make_pca  # noqa: E402

CASES = ["paper_1bin", "paper_2bin_full"]


def _handle(name):
    from paper_1812_07437_gb300.handle import Handle
    return Handle(make_pca.workload(name))


@pytest.mark.parametrize("name", CASES)
def test_pca_on_the_oracle_covariance(name):
    ref = make_pca.load(name)
    r = OracleRun(make_pca.workload(name), ntri=make_counts.load("paper_2bin_full")[1])
    Co = r.cov.full(TERMS_ALL)
    h = _handle(name)
    dev = torch.device("cuda:0")
    C = torch.as_tensor(Co, device=dev)
    D = torch.as_tensor(r.D, device=dev)
    got = h.pca(C, D)
    assert got["converged"] == 1 and got["M"] == r.M
    lam = got["lam"]
    assert lam[0] > 0 and lam[-1] / lam[0] > 1e18  # the dynamic range the paper warns about
    np.testing.assert_allclose(lam, ref["lam"], rtol=1e-10, atol=0)
    assert np.max(np.abs(got["snr2"] - ref["snr2"])) <= 1e-10 * ref["total"]
    assert got["total_snr2"] == pytest.approx(ref["total"], rel=1e-10, abs=0)
    for f, key in ((0.90, "modes_90"), (0.95, "modes_95"), (0.99, "modes_99")):
        assert got[key] == ref["modes"][f], (f, got[key], ref["modes"][f])
    np.testing.assert_allclose(got["cum_var"], np.cumsum(got["snr2"]), rtol=1e-12, atol=0)
    np.testing.assert_allclose(got["cum_info"], np.cumsum(np.sort(got["snr2"])[::-1]), rtol=1e-12, atol=0)
    h.close()


@pytest.mark.parametrize("name", CASES)
def test_pca_of_the_gpu_covariance(name):
    ref = make_pca.load(name)
    h = _handle(name)
    dev = torch.device("cuda:0")
    D = torch.zeros(h.M, dtype=torch.float64, device=dev)
    C = torch.zeros(h.M, h.M, dtype=torch.float64, device=dev)
    h.spectra(D)
    h.assemble(C, N.COV_TERMS_ALL, N.COV_FP64)
    torch.cuda.synchronize()
    got = h.pca(C, D)
    np.testing.assert_allclose(got["lam"], ref["lam"], rtol=1e-7, atol=0)
    assert got["total_snr2"] == pytest.approx(ref["total"], rel=1e-9, abs=0)
    assert got["modes_99"] == ref["modes"][0.99]
    snr = h.snr(C, D, N.COV_WHICH_JOINT)
    assert got["cum_info"][-1] == pytest.approx(float(snr[-1]) ** 2, rel=1e-9, abs=0)
    h.close()
