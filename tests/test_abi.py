"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every function declared in include/wlcov.h, and rejects invalid
arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1812_07437_gb300 import native
    if not os.path.exists(native.LIB_PATH):
        from paper_1812_07437_gb300 import build
        build.build()
    return native.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "wlcov.h")).read()
    return sorted(set(re.findall(r"\b(cov_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("cov_init", "cov_spectra", "cov_assemble", "cov_snr"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1812_07437_gb300 import native
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert set(native.EXPORTED) <= set(declared_functions())


def test_invalid_arguments_rejected_on_host(lib):
    from paper_1812_07437_gb300 import native as N
    from paper_1812_07437_gb300 import workloads
    wl = workloads.get("tiny_2bin")
    cs, ns, bs = N.structs_from_workload(wl)
    h = C.c_void_p()
    bad = N.cov_nz(0, *[getattr(ns, f) for f, _ in N.cov_nz._fields_[1:]])
    rc = lib.cov_init(C.byref(cs), C.byref(bad), C.byref(bs), None, C.byref(h))
    assert rc == N.COV_ERR_INVALID and not h.value
    assert b"invalid" in lib.cov_last_error(None)
    bs2 = N.cov_bins(*[getattr(bs, f) for f, _ in N.cov_bins._fields_])
    bs2.f_sky = 1.5
    assert lib.cov_init(C.byref(cs), C.byref(ns), C.byref(bs2), None, C.byref(h)) == N.COV_ERR_INVALID
    # concentration rule: at most 32 nodes, 0 <= sigma_lnc <= 2, n_mass * n_conc <= 4096
    for n_conc, sig, n_mass in ((33, 0.18, 12), (-1, 0.18, 12), (8, -0.1, 12), (8, float("nan"), 12),
                                (8, 2.5, 12), (16, 0.18, 257)):
        bs3 = N.cov_bins(*[getattr(bs, f) for f, _ in N.cov_bins._fields_])
        bs3.n_conc, bs3.sigma_lnc, bs3.n_mass = n_conc, sig, n_mass
        assert lib.cov_init(C.byref(cs), C.byref(ns), C.byref(bs3), None, C.byref(h)) == N.COV_ERR_INVALID
        assert not h.value
    for model in (-1, 2):  # median concentration: COV_CONC_DUFFY or COV_CONC_BULLOCK
        bs4 = N.cov_bins(*[getattr(bs, f) for f, _ in N.cov_bins._fields_])
        bs4.conc_model = model
        assert lib.cov_init(C.byref(cs), C.byref(ns), C.byref(bs4), None, C.byref(h)) == N.COV_ERR_INVALID
    assert lib.cov_spectra(None, None, None) == N.COV_ERR_INVALID
    assert lib.cov_snr(None, None, 0, None, 0, None, None) == N.COV_ERR_INVALID
    assert lib.cov_assemble_band(None, 0, 256, None, 0, N.COV_LAYOUT_TILES, N.COV_TERMS_ALL, N.COV_SPLIT_BF16,
                                 None) == N.COV_ERR_INVALID
    assert lib.cov_batch_snr(None, None, 0, N.COV_TERMS_ALL, N.COV_SPLIT_BF16, None, None, 0, None,
                             None) == N.COV_ERR_INVALID
    assert lib.cov_snr_tiles(None, None, None, None, None) == N.COV_ERR_INVALID


def test_tile_layout_addressing_covers_the_lower_triangle():
    """The COV_LAYOUT_TILES map (r, c) -> offset is a bijection from the lower
    triangle of a band onto distinct slots of its tiles, and consecutive bands
    tile the whole packed matrix without gaps (host restatement of the
    documented formula, checked on a ragged size)."""
    import numpy as np
    M = 3 * 256 + 37
    nt = (M + 255) // 256

    def off(r, c, row0):
        ti, tj, t0 = r >> 8, c >> 8, row0 >> 8
        return ((ti * (ti + 1) // 2 + tj - t0 * (t0 + 1) // 2) << 16) + ((r & 255) << 8) + (c & 255)

    r, c = np.tril_indices(M)
    o = off(r, c, 0)
    assert len(np.unique(o)) == len(o)
    assert o.max() < (nt * (nt + 1) // 2) << 16
    for row0 in (256, 512):
        sel = r >= row0
        assert np.array_equal(off(r[sel], c[sel], row0) + ((row0 >> 8) * ((row0 >> 8) + 1) // 2 << 16), o[sel])
