"""Failure detection on the GPU without a GPU fault.

The tensor-core kernels bound every wait and report an expired one as
COV_ERR_TIMEOUT through a status word.  cov_wait_selftest runs that protocol
on a wait that has no bulk copy or MMA in flight: a kernel polls a device flag
with a host-set limit.  Preset flag: COV_OK.  A flag that nothing sets: the
wait expires after the limit, the call returns COV_ERR_TIMEOUT, and the handle
(and the CUDA context) stay usable: the next assembly gives the same
covariance as before.  A non-positive Cholesky pivot is reported as
COV_ERR_NOT_PD.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1812_07437_gb300 import native as N  # noqa: E402
from paper_1812_07437_gb300 import workloads  # noqa: E402


def _cov(h):
    D = torch.zeros(h.M, dtype=torch.float64, device="cuda:0")
    Cm = torch.zeros(h.M, h.M, dtype=torch.float64, device="cuda:0")
    h.spectra(D)
    h.assemble(Cm, N.COV_TERMS_ALL, N.COV_SPLIT_BF16)
    torch.cuda.synchronize()
    return Cm, D


def test_bounded_wait_expires_and_handle_stays_usable():
    from paper_1812_07437_gb300.handle import Handle
    h = Handle(workloads.get("tiny_2bin"))
    C0, D0 = _cov(h)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert h.L.cov_wait_selftest(h.h, 200000, 1, s) == N.COV_OK
    assert h.L.cov_wait_selftest(h.h, 200000, 0, s) == N.COV_ERR_TIMEOUT
    assert b"bounded" in h.L.cov_last_error(h.h)
    assert h.L.cov_wait_selftest(h.h, 0, 0, s) == N.COV_ERR_INVALID
    C1, D1 = _cov(h)
    assert torch.equal(torch.tril(C0), torch.tril(C1)) and torch.equal(D0, D1)
    assert h.L.cov_wait_selftest(h.h, 1000, 1, s) == N.COV_OK
    h.close()


def test_indefinite_covariance_reports_not_pd():
    from paper_1812_07437_gb300.handle import Handle
    h = Handle(workloads.get("tiny_2bin"))
    Cm, D = _cov(h)
    Cm[5, 5] = -abs(float(Cm[5, 5]))
    with pytest.raises(N.CovError) as e:
        h.snr(Cm, D, N.COV_WHICH_JOINT)
    assert e.value.code == N.COV_ERR_NOT_PD
    Cm2, D2 = _cov(h)
    snr = h.snr(Cm2, D2, N.COV_WHICH_JOINT)
    assert np.all(np.isfinite(snr[-1:]))
    h.close()
