"""ctypes binding of libwlcov (argument marshalling only).

Every function of ``include/wlcov.h`` is exposed under the same name; device
memory and streams come from PyTorch tensors / streams and are passed as raw
pointers.  There is no CPU fallback: importing this module on a machine
without the built library raises.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libwlcov.so")

COV_OK = 0
COV_ERR_INVALID = -1
COV_ERR_NOMEM = -2
COV_ERR_NOT_PD = -3
COV_ERR_TIMEOUT = -4
COV_ERR_CUDA = -5

COV_TERM_G = 1
COV_TERM_1H = 2
COV_TERM_BBPT = 4
COV_TERM_PB = 8
COV_TERM_SSC = 16
COV_TERMS_ALL = 31

COV_FP64 = 0
COV_SPLIT_BF16 = 1

COV_WHICH_P = 0
COV_WHICH_B = 1
COV_WHICH_JOINT = 2

COV_LAYOUT_ROWS = 0
COV_LAYOUT_TILES = 1

COV_ROWS_JOINT = 0
COV_ROWS_P = 1
COV_ROWS_B = 2
COV_ORDER_NATURAL = 0
COV_ORDER_CUMULATIVE = 1
COV_TC_AUTO = 0
COV_TC_SINGLE = 1
COV_CHOL_AUTO = 0
COV_CHOL_TILE = 1
COV_COUPLING_MODES = 0
COV_COUPLING_EXACT = 1

COV_CONC_DUFFY = 0
COV_CONC_BULLOCK = 1

EXPORTED = ["cov_init", "cov_update", "cov_layout", "cov_counts", "cov_spectra", "cov_assemble", "cov_snr",
            "cov_assemble_band", "cov_table", "cov_profile", "cov_stage_times", "cov_stage_name", "cov_snr_noalloc",
            "cov_last_error", "cov_free", "cov_snr_tiles", "cov_batch_snr", "cov_server_create", "cov_server_submit", "cov_server_wait",
            "cov_server_error", "cov_server_stats_get", "cov_server_clock", "cov_request_footprint",
            "cov_server_free", "cov_wait_selftest", "cov_pca", "cov_coupling_gram"]

COV_REQ_QUEUED = 0
COV_REQ_RUNNING = 1
COV_REQ_DONE = 2
COV_REQ_FAILED = 3
COV_REQ_REJECTED = 4
COV_NOALLOC_MAX_M = 2047
N_STAGES = 13
HAS_SPLIT_BF16 = True


class cov_cosmology(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("Om", "Ob", "h", "ns", "sigma8", "w0", "Tcmb")]


class cov_nz(C.Structure):
    _fields_ = [("n_tomo", C.c_int)] + [(n, C.c_double) for n in (
        "z0", "alpha", "zmin", "zmax", "photoz_sigma0", "n_gal_arcmin2", "sigma_e")]


class cov_bins(C.Structure):
    _fields_ = [("n_ell", C.c_int), ("ell_min", C.c_double), ("ell_max", C.c_double), ("f_sky", C.c_double),
                ("n_chi", C.c_int), ("n_mass", C.c_int), ("m_min", C.c_double), ("m_max", C.c_double),
                ("k_max", C.c_double), ("n_conc", C.c_int), ("sigma_lnc", C.c_double), ("conc_model", C.c_int)]


class cov_opts(C.Structure):
    _fields_ = [("device", C.c_int), ("hbm_budget", C.c_size_t), ("rows", C.c_int), ("order", C.c_int),
                ("tc_kernel", C.c_int), ("chol_kernel", C.c_int), ("coupling", C.c_int)]


COV_BATCH_TUNE = 1


COV_BATCH_CANDIDATES = 6


class cov_batch_info(C.Structure):
    _fields_ = [("tc_kernel", C.c_int), ("chol_lookahead", C.c_int),
                ("candidate_ms", C.c_double * COV_BATCH_CANDIDATES), ("tuned", C.c_int), ("pr_group", C.c_int),
                ("chol_kernel", C.c_int), ("single_launch", C.c_int), ("first_ms", C.c_double),
                ("capture_ms", C.c_double), ("replay_ms", C.c_double)]


class cov_pca_info(C.Structure):
    _fields_ = [("M", C.c_int64), ("sweeps", C.c_int), ("converged", C.c_int), ("total_snr2", C.c_double),
                ("modes_90", C.c_int), ("modes_95", C.c_int), ("modes_99", C.c_int), ("ms_cholesky", C.c_double),
                ("ms_jacobi", C.c_double)]


class cov_server_opts(C.Structure):
    _fields_ = [("device", C.c_int), ("n_slots", C.c_int), ("hbm_budget", C.c_size_t), ("precision", C.c_int),
                ("terms", C.c_uint), ("max_bypass", C.c_int), ("dry_run_us", C.c_int)]


class cov_request(C.Structure):
    _fields_ = [("cosmo", cov_cosmology), ("nz", cov_nz), ("bins", cov_bins)]


class cov_request_info(C.Structure):
    _fields_ = [("state", C.c_int), ("rc", C.c_int), ("M", C.c_int64), ("n_ell", C.c_int), ("slot", C.c_int),
                ("reused", C.c_int), ("footprint", C.c_size_t), ("t_submit", C.c_double), ("t_start", C.c_double),
                ("t_done", C.c_double)]


class cov_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("done", C.c_int64), ("failed", C.c_int64), ("rejected", C.c_int64),
                ("reserved", C.c_size_t), ("peak_reserved", C.c_size_t), ("budget", C.c_size_t),
                ("max_running", C.c_int)]


_lib = None


def lib():
    """Load libwlcov.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        i64 = C.c_int64
        L.cov_init.argtypes = [C.POINTER(cov_cosmology), C.POINTER(cov_nz), C.POINTER(cov_bins),
                               C.POINTER(cov_opts), C.POINTER(P)]
        L.cov_update.argtypes = [P, C.POINTER(cov_cosmology), P]
        L.cov_layout.argtypes = [P, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), P]
        L.cov_counts.argtypes = [P, P, P, P]
        L.cov_spectra.argtypes = [P, P, P]
        L.cov_assemble.argtypes = [P, P, i64, C.c_uint, C.c_int, P]
        L.cov_snr.argtypes = [P, P, i64, P, C.c_int, P, P]
        L.cov_assemble_band.argtypes = [P, i64, i64, P, i64, C.c_int, C.c_uint, C.c_int, P]
        L.cov_snr_tiles.argtypes = [P, P, P, P, P]
        L.cov_batch_snr.argtypes = [P, C.POINTER(cov_cosmology), C.c_int, C.c_uint, C.c_int, P, P, C.c_uint,
                                    C.POINTER(cov_batch_info), P]
        L.cov_table.argtypes = [P, C.c_char_p, P, C.POINTER(i64), P]
        L.cov_profile.argtypes = [P, C.c_int]
        L.cov_stage_times.argtypes = [P, P, P, C.c_int]
        L.cov_stage_name.argtypes = [C.c_int]
        L.cov_stage_name.restype = C.c_char_p
        L.cov_snr_noalloc.argtypes = [P, i64, P, i64, P, C.c_int, P, P, P]
        L.cov_wait_selftest.argtypes = [P, C.c_uint, C.c_int, P]
        L.cov_pca.argtypes = [P, P, i64, P, P, P, P, P, C.POINTER(cov_pca_info), P]
        L.cov_coupling_gram.argtypes = [P, C.c_int, C.POINTER(C.c_int), P, P, P]
        L.cov_last_error.argtypes = [P]
        L.cov_last_error.restype = C.c_char_p
        L.cov_free.argtypes = [P]
        L.cov_free.restype = None
        L.cov_server_create.argtypes = [C.POINTER(cov_server_opts), C.POINTER(P)]
        L.cov_server_submit.argtypes = [P, C.POINTER(cov_request), C.POINTER(i64)]
        L.cov_server_wait.argtypes = [P, i64, C.c_double, C.POINTER(cov_request_info), P]
        L.cov_server_error.argtypes = [P, i64]
        L.cov_server_error.restype = C.c_char_p
        L.cov_server_stats_get.argtypes = [P, C.POINTER(cov_server_stats)]
        L.cov_server_clock.argtypes = [P]
        L.cov_server_clock.restype = C.c_double
        L.cov_request_footprint.argtypes = [C.POINTER(cov_request), C.c_int, C.c_uint, C.POINTER(i64),
                                            C.POINTER(C.c_size_t)]
        L.cov_server_free.argtypes = [P]
        L.cov_server_free.restype = None
        for n in EXPORTED:
            if n not in ("cov_last_error", "cov_free", "cov_stage_name", "cov_server_error", "cov_server_clock",
                         "cov_server_free"):
                getattr(L, n).restype = C.c_int
        _lib = L
    return _lib


class CovError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libwlcov error {code}: {msg}")
        self.code = code


def check(rc, handle=None):
    if rc != COV_OK:
        raise CovError(rc, lib().cov_last_error(handle).decode())
    return rc


def structs_from_workload(wl):
    c = wl["cosmology"]
    nz = wl["nz"]
    b = wl["bins"]
    cs = cov_cosmology(*(float(c[k]) for k in ("Om", "Ob", "h", "ns", "sigma8", "w0", "Tcmb")))
    ns = cov_nz(int(nz["n_tomo"]), *(float(nz[k]) for k in (
        "z0", "alpha", "zmin", "zmax", "photoz_sigma0", "n_gal_arcmin2", "sigma_e")))
    bs = cov_bins(int(b["n_ell"]), float(b["ell_min"]), float(b["ell_max"]), float(b["f_sky"]), int(b["n_chi"]),
                  int(b["n_mass"]), float(b["m_min"]), float(b["m_max"]), float(b["k_max"]),
                  int(b.get("n_conc", 0)), float(b.get("sigma_lnc", 0.0)), int(b.get("conc_model", 0)))
    return cs, ns, bs
