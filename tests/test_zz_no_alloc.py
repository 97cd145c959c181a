"""The allocation-free S/N entry point against the handle-based one.

cov_snr_noalloc exists for callers that cannot allocate device memory (a host
application that owns all device memory through its own pool, or a loop that
must never stall on an allocation).  It solves with a fixed static workspace
instead of allocating one, so it is checked here against cov_snr on the same
covariance: the two must agree within the FP64 tolerance of the other parity
tests (1e-10 relative), on two calls in a row (the second call finds the
previous call's data in the shared workspace).  This file is collected last
so that a failure here leaves every other test already run.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1812_07437_gb300 import native as N  # noqa: E402
from paper_1812_07437_gb300 import workloads  # noqa: E402

TOL = 1e-10


def _cumulative_order(h):
    rd = h.row_desc()
    maxbin = np.where(rd[:, 0] == 0, rd[:, 1], rd[:, 3])
    perm = np.argsort(maxbin, kind="stable")
    prefix = np.array([int(np.sum(maxbin <= c)) for c in range(h.n_ell)], dtype=np.int64)
    return perm, prefix


def _noalloc(L, Cp, Dp, prefix, stream):
    M = Cp.shape[0]
    out = torch.full((len(prefix),), float("nan"), dtype=torch.float64, device=Cp.device)
    status = torch.full((1,), 7, dtype=torch.int32, device=Cp.device)
    rc = L.cov_snr_noalloc(C.c_void_p(Cp.data_ptr()), Cp.stride(0), C.c_void_p(Dp.data_ptr()), M,
                           prefix.ctypes.data_as(C.c_void_p), len(prefix), C.c_void_p(out.data_ptr()),
                           C.c_void_p(status.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert rc == N.COV_OK, L.cov_last_error(None)
    stream.synchronize()
    return out.cpu().numpy(), int(status.item())


@pytest.mark.parametrize("name", ["mid_2bin", "tiny_2bin"])
def test_noalloc_matches_cov_snr_twice(name):
    from paper_1812_07437_gb300.handle import Handle
    h = Handle(workloads.get(name))
    dev = torch.device("cuda:0")
    D = torch.zeros(h.M, dtype=torch.float64, device=dev)
    Cm = torch.zeros(h.M, h.M, dtype=torch.float64, device=dev)
    h.spectra(D)
    h.assemble(Cm, N.COV_TERMS_ALL, N.COV_FP64)
    torch.cuda.synchronize()
    ref = h.snr(Cm, D, N.COV_WHICH_JOINT)
    perm, prefix = _cumulative_order(h)
    p = torch.as_tensor(perm, device=dev)
    S = torch.tril(Cm) + torch.tril(Cm, -1).T
    Cp = S[p][:, p].contiguous()
    Dp = D[p].contiguous()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        got, status = _noalloc(h.L, Cp, Dp, prefix, stream)
        assert status == 0
        m = np.isfinite(ref)
        assert np.array_equal(m, np.isfinite(got))
        assert np.max(np.abs(got[m] / ref[m] - 1.0)) <= TOL
    h.close()


def test_noalloc_rejects_oversize():
    L = N.lib()
    M = N.COV_NOALLOC_MAX_M + 1
    buf = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    st = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    prefix = np.array([M], dtype=np.int64)
    rc = L.cov_snr_noalloc(C.c_void_p(buf.data_ptr()), M, C.c_void_p(buf.data_ptr()), M,
                           prefix.ctypes.data_as(C.c_void_p), 1, C.c_void_p(buf.data_ptr()),
                           C.c_void_p(st.data_ptr()), None)
    assert rc == N.COV_ERR_INVALID
    assert b"static workspace" in L.cov_last_error(None)
