"""Thin PyTorch-facing wrapper around the libwlcov C ABI (marshalling only).

Device buffers are torch tensors on the handle's device; streams are torch
CUDA streams.  Every computation happens inside libwlcov's kernels.
"""
import ctypes as C

import numpy as np

from . import native as N


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Handle:
    def __init__(self, wl, device=0, hbm_budget=0, rows=N.COV_ROWS_JOINT, order=N.COV_ORDER_NATURAL,
                 tc_kernel=N.COV_TC_AUTO, chol_kernel=N.COV_CHOL_AUTO, coupling=N.COV_COUPLING_MODES):
        self.L = N.lib()
        cs, ns, bs = N.structs_from_workload(wl)
        opts = N.cov_opts(int(device), int(hbm_budget), int(rows), int(order), int(tc_kernel), int(chol_kernel),
                          int(coupling))
        h = C.c_void_p()
        N.check(self.L.cov_init(C.byref(cs), C.byref(ns), C.byref(bs), C.byref(opts), C.byref(h)))
        self.h = h
        self.wl = wl
        self.device = device
        M, nP, nB, nT = (C.c_int64() for _ in range(4))
        N.check(self.L.cov_layout(h, C.byref(M), C.byref(nP), C.byref(nB), C.byref(nT), None), h)
        self.M, self.n_P, self.n_B, self.n_tri = M.value, nP.value, nB.value, nT.value
        self.n_ell = int(wl["bins"]["n_ell"])

    def close(self):
        if self.h:
            self.L.cov_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def row_desc(self):
        out = np.zeros((self.M, 8), dtype=np.int32)
        N.check(self.L.cov_layout(self.h, None, None, None, None, out.ctypes.data_as(C.c_void_p)), self.h)
        return out

    def counts(self, stream=None):
        ne = np.zeros(self.n_ell, dtype=np.int64)
        nt = np.zeros(max(self.n_tri, 1), dtype=np.int64)
        N.check(self.L.cov_counts(self.h, ne.ctypes.data_as(C.c_void_p), nt.ctypes.data_as(C.c_void_p),
                                  _stream_ptr(stream)), self.h)
        return ne, nt[: self.n_tri]

    def coupling_gram(self, ell_bin, stream=None):
        """Columns (Y, Z) of ell bin `ell_bin` and the exact Gram matrix of
        their leg counts (int64), for a handle made with COV_COUPLING_EXACT."""
        n = C.c_int(0)
        N.check(self.L.cov_coupling_gram(self.h, int(ell_bin), C.byref(n), None, None, _stream_ptr(stream)), self.h)
        cols = np.zeros((max(n.value, 1), 2), dtype=np.int32)
        gram = np.zeros((max(n.value, 1), max(n.value, 1)), dtype=np.int64)
        N.check(self.L.cov_coupling_gram(self.h, int(ell_bin), C.byref(n), cols.ctypes.data_as(C.c_void_p),
                                         gram.ctypes.data_as(C.c_void_p), _stream_ptr(stream)), self.h)
        k = n.value
        return cols[:k], gram[:k, :k]

    def table(self, name, stream=None):
        cnt = C.c_int64()
        N.check(self.L.cov_table(self.h, name.encode(), None, C.byref(cnt), _stream_ptr(stream)), self.h)
        out = np.zeros(cnt.value, dtype=np.float64)
        N.check(self.L.cov_table(self.h, name.encode(), out.ctypes.data_as(C.c_void_p), C.byref(cnt),
                                 _stream_ptr(stream)), self.h)
        return out

    def update(self, cosmology, stream=None):
        cs = N.cov_cosmology(*(float(cosmology[k]) for k in ("Om", "Ob", "h", "ns", "sigma8", "w0", "Tcmb")))
        N.check(self.L.cov_update(self.h, C.byref(cs), _stream_ptr(stream)), self.h)

    def spectra(self, D=None, stream=None):
        ptr = C.c_void_p(D.data_ptr()) if D is not None else None
        N.check(self.L.cov_spectra(self.h, ptr, _stream_ptr(stream)), self.h)

    def assemble(self, Cmat, terms=N.COV_TERMS_ALL, precision=N.COV_FP64, stream=None):
        ldc = Cmat.stride(0)
        N.check(self.L.cov_assemble(self.h, C.c_void_p(Cmat.data_ptr()), ldc, terms, precision,
                                    _stream_ptr(stream)), self.h)

    def assemble_band(self, row0, nrows, Cout, layout=None, terms=N.COV_TERMS_ALL, precision=N.COV_SPLIT_BF16,
                      stream=None):
        """Lower part of rows [row0, row0 + nrows) into Cout.

        layout COV_LAYOUT_ROWS: Cout is 2-D with Cout[r - row0, c] (row stride >= row0 + nrows);
        COV_LAYOUT_TILES: Cout is a flat buffer of the band's 256 x 256 lower tiles."""
        if layout is None:
            layout = N.COV_LAYOUT_TILES if Cout.dim() == 1 else N.COV_LAYOUT_ROWS
        ldc = Cout.stride(0) if layout == N.COV_LAYOUT_ROWS else 0
        N.check(self.L.cov_assemble_band(self.h, int(row0), int(nrows), C.c_void_p(Cout.data_ptr()), ldc, layout,
                                         terms, precision, _stream_ptr(stream)), self.h)

    def profile(self, enable=True):
        N.check(self.L.cov_profile(self.h, 1 if enable else 0), self.h)

    def stage_times(self):
        """{stage name: (summed ms, calls)} since the last query."""
        ms = np.zeros(N.N_STAGES)
        calls = np.zeros(N.N_STAGES, dtype=np.int64)
        N.check(self.L.cov_stage_times(self.h, ms.ctypes.data_as(C.c_void_p), calls.ctypes.data_as(C.c_void_p),
                                       N.N_STAGES), self.h)
        return {self.L.cov_stage_name(i).decode(): (float(ms[i]), int(calls[i])) for i in range(N.N_STAGES)}

    def snr(self, Cmat, D, which=N.COV_WHICH_JOINT, stream=None):
        out = np.zeros(self.n_ell, dtype=np.float64)
        N.check(self.L.cov_snr(self.h, C.c_void_p(Cmat.data_ptr()), Cmat.stride(0), C.c_void_p(D.data_ptr()),
                               which, out.ctypes.data_as(C.c_void_p), _stream_ptr(stream)), self.h)
        return out

    def pca(self, Cmat, D, stream=None):
        """Principal components (Sec. 6): eigenvalues ascending, (S/N)^2 per mode in that order, cumulative
        (S/N)^2 by increasing variance and by decreasing (S/N)_a, and the info fields (dict)."""
        M = self.M
        lam, snr2, cv, ci = (np.zeros(M, dtype=np.float64) for _ in range(4))
        info = N.cov_pca_info()
        N.check(self.L.cov_pca(self.h, C.c_void_p(Cmat.data_ptr()), Cmat.stride(0), C.c_void_p(D.data_ptr()),
                               *(x.ctypes.data_as(C.c_void_p) for x in (lam, snr2, cv, ci)), C.byref(info),
                               _stream_ptr(stream)), self.h)
        d = {f: getattr(info, f) for f, _ in N.cov_pca_info._fields_}
        return {"lam": lam, "snr2": snr2, "cum_var": cv, "cum_info": ci, **d}

    def snr_tiles(self, Ct, D, stream=None):
        """In-place cumulative S/N of the handle's rows on its lower-packed tiles (cumulative-order handles)."""
        out = np.zeros(self.n_ell, dtype=np.float64)
        N.check(self.L.cov_snr_tiles(self.h, C.c_void_p(Ct.data_ptr()), C.c_void_p(D.data_ptr()),
                                     out.ctypes.data_as(C.c_void_p), _stream_ptr(stream)), self.h)
        return out

    def batch_snr(self, cosmologies, terms=N.COV_TERMS_ALL, precision=N.COV_SPLIT_BF16, with_D=False, tune=False,
                  stream=None):
        """Cumulative S/N (and optionally D) for a list of cosmology dicts.

        Returns (snr [n, 3, n_ell] in the order P, B, joint; D [n, M] or None; tuning/timing dict)."""
        n = len(cosmologies)
        arr = (N.cov_cosmology * n)(*[N.cov_cosmology(*(float(c[k]) for k in ("Om", "Ob", "h", "ns", "sigma8", "w0",
                                                                           "Tcmb"))) for c in cosmologies])
        snr = np.zeros((n, 3, self.n_ell), dtype=np.float64)
        D = np.zeros((n, self.M), dtype=np.float64) if with_D else None
        info = N.cov_batch_info()
        N.check(self.L.cov_batch_snr(self.h, arr, n, terms, precision,
                                     D.ctypes.data_as(C.c_void_p) if with_D else None, snr.ctypes.data_as(C.c_void_p),
                                     N.COV_BATCH_TUNE if tune else 0, C.byref(info), _stream_ptr(stream)), self.h)
        d = {f: getattr(info, f) for f, _ in N.cov_batch_info._fields_}
        d["candidate_ms"] = list(info.candidate_ms)
        return snr, D, d


def packed_tiles(rows):
    """Number of 256 x 256 lower tiles holding rows 0..rows-1."""
    t = (rows + 255) // 256
    return t * (t + 1) // 2
