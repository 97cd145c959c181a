"""The allocation-free S/N entry point against the handle-based one and the
oracle.

cov_snr_noalloc exists for callers that cannot allocate device memory (a host
application that owns all device memory through its own pool, or a loop that
must never stall on an allocation).  It solves with a fixed static workspace
instead of allocating one, so it is checked here against cov_snr on the same
covariance and against the oracle's cumulative S/N: they must agree within the
FP64 tolerance of the other parity tests (1e-10 relative), on two calls in a
row (the second call finds the previous call's data in the shared workspace).
The edge cases: the largest size the workspace takes (M = COV_NOALLOC_MAX_M,
which reaches its last entry) with a leading dimension above M, an empty
prefix (NaN), and a non-positive pivot (reported through the status word while
the call returns COV_OK).  This file is collected last so that a failure here
leaves every other test already run.
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


def test_noalloc_matches_oracle_twice():
    """The GPU's FP64 covariance of tiny_2bin, solved by cov_snr_noalloc, gives
    the oracle's cumulative S/N (oracle covariance, oracle solve)."""
    from oracle.covariance import TERMS_ALL
    from oracle.pipeline import OracleRun
    from oracle.snr import WHICH_JOINT, cumulative_snr
    from paper_1812_07437_gb300.handle import Handle
    name = "tiny_2bin"
    r = OracleRun(workloads.get(name))
    ref = cumulative_snr(r.cov.full(TERMS_ALL), r.D, r.rows, len(r.T.ell), WHICH_JOINT)
    h = Handle(workloads.get(name))
    dev = torch.device("cuda:0")
    D = torch.zeros(h.M, dtype=torch.float64, device=dev)
    Cm = torch.zeros(h.M, h.M, dtype=torch.float64, device=dev)
    h.spectra(D)
    h.assemble(Cm, N.COV_TERMS_ALL, N.COV_FP64)
    torch.cuda.synchronize()
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


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n)) / np.sqrt(n)
    s = 10.0 ** rng.uniform(-3, 3, n)
    A = (B @ B.T + 0.1 * np.eye(n)) * np.outer(s, s)
    return A, rng.standard_normal(n) * s


def _snr_ref(A, d, prefix):
    out = []
    for n in prefix:
        if n == 0:
            out.append(np.nan)
            continue
        L = np.linalg.cholesky(A[:n, :n])
        y = np.linalg.solve(L, d[:n])
        out.append(np.sqrt(y @ y))
    return np.array(out)


def test_noalloc_largest_size_padded_rows_empty_prefix():
    """M = COV_NOALLOC_MAX_M (the workspace's last entry is used) with a leading
    dimension of M + 3; an empty prefix gives NaN; two calls in a row."""
    L = N.lib()
    M = N.COV_NOALLOC_MAX_M
    A, d = _spd(M, 11)
    prefix = np.array([0, 1, 100, 1000, M - 1, M], dtype=np.int64)
    ref = _snr_ref(A, d, prefix)
    dev = torch.device("cuda:0")
    buf = torch.full((M, M + 3), float("nan"), dtype=torch.float64, device=dev)
    buf[:, :M] = torch.as_tensor(A, device=dev)
    Cp = buf[:, :M]
    assert Cp.stride(0) == M + 3
    Dp = torch.as_tensor(d, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        got, status = _noalloc(L, Cp, Dp, prefix, stream)
        assert status == 0
        assert np.isnan(got[0])
        assert np.max(np.abs(got[1:] / ref[1:] - 1.0)) <= TOL


def test_noalloc_non_positive_pivot_sets_status():
    """An indefinite matrix: the call returns COV_OK and the status word is 1."""
    L = N.lib()
    n = 40
    A, d = _spd(n, 5)
    w, V = np.linalg.eigh(A)
    w[3] = -abs(w[3])  # one negative eigenvalue
    A = (V * w) @ V.T
    A = 0.5 * (A + A.T)
    dev = torch.device("cuda:0")
    Cp = torch.as_tensor(A, device=dev).contiguous()
    Dp = torch.as_tensor(d, device=dev)
    _, status = _noalloc(L, Cp, Dp, np.array([n], dtype=np.int64), torch.cuda.current_stream())
    assert status == 1
