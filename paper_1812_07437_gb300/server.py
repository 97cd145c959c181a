"""Thin wrapper around the serving entry points of libwlcov (marshalling only).

The scheduler itself (worker threads, CUDA streams, HBM-budgeted admission,
resident device state) is native code in csrc/serve.cu.
"""
import ctypes as C

import numpy as np

from . import native as N


def request_from_workload(wl):
    cs, ns, bs = N.structs_from_workload(wl)
    return N.cov_request(cs, ns, bs)


class Server:
    def __init__(self, n_slots=2, hbm_budget=0, precision=N.COV_SPLIT_BF16, terms=N.COV_TERMS_ALL, device=0,
                 max_bypass=0, dry_run_us=0):
        self.L = N.lib()
        o = N.cov_server_opts(int(device), int(n_slots), int(hbm_budget), int(precision), int(terms),
                              int(max_bypass), int(dry_run_us))
        s = C.c_void_p()
        N.check(self.L.cov_server_create(C.byref(o), C.byref(s)))
        self.s = s
        self.precision, self.terms = precision, terms

    def footprint(self, wl):
        r = request_from_workload(wl)
        M, b = C.c_int64(), C.c_size_t()
        N.check(self.L.cov_request_footprint(C.byref(r), self.precision, self.terms, C.byref(M), C.byref(b)))
        return M.value, b.value

    def submit(self, wl):
        r = request_from_workload(wl)
        i = C.c_int64()
        N.check(self.L.cov_server_submit(self.s, C.byref(r), C.byref(i)))
        return i.value

    def wait(self, rid, timeout=-1.0, n_ell=None):
        """(info dict, S/N array [3][n_ell] or None); info['state'] is a COV_REQ_* code."""
        info = N.cov_request_info()
        rc = self.L.cov_server_wait(self.s, int(rid), float(timeout), C.byref(info), None)
        if rc == N.COV_ERR_TIMEOUT:
            return self._info(info), None
        N.check(rc)
        snr = None
        if info.state == N.COV_REQ_DONE:
            out = np.zeros(3 * info.n_ell, dtype=np.float64)
            N.check(self.L.cov_server_wait(self.s, int(rid), 0.0, None, out.ctypes.data_as(C.c_void_p)))
            snr = out.reshape(3, info.n_ell)
        return self._info(info), snr

    def error(self, rid):
        return self.L.cov_server_error(self.s, int(rid)).decode()

    def stats(self):
        st = N.cov_server_stats()
        N.check(self.L.cov_server_stats_get(self.s, C.byref(st)))
        return {f: getattr(st, f) for f, _ in N.cov_server_stats._fields_}

    def clock(self):
        return self.L.cov_server_clock(self.s)

    @staticmethod
    def _info(info):
        return {f: getattr(info, f) for f, _ in N.cov_request_info._fields_}

    def close(self):
        if getattr(self, "s", None):
            self.L.cov_server_free(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
