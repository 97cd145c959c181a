"""GPU checks of the streaming band assembly (cov_assemble_band).

* A band computes exactly what the full assembly computes for its rows: on
  cfg2_5bin (M = 6375, 25 tile rows, ragged last one) every band, in both
  layouts and both precisions, equals the full matrix bit for bit.
* cfg3_10bin (10 bins, 20 ell bins, M = 181350, K = 32768), which is only
  assembled band by band: the data vector against the oracle to 1e-10;
  sampled elements of the FP64 form against the oracle to 1e-10 (normalised
  by sqrt(C_aa C_bb)); sampled split-BF16 elements against the oracle to 1e-4;
  and the split-BF16 band against the FP64 band over every element to 1e-4.
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.pipeline import OracleRun  # noqa: E402
from paper_1812_07437_gb300 import native as N  # noqa: E402
from paper_1812_07437_gb300 import workloads  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_counts  # noqa: E402

DEV = "cuda:0"
TILE = 256


def tiles_to_rows(T, row0, row1):
    """Dense rows [row0, row1) x [0, row1) (lower part, NaN above) from a tile-layout band."""
    t0, t1 = row0 // TILE, (row1 + TILE - 1) // TILE
    T = T.view(-1, TILE, TILE)
    out = torch.full((row1 - row0, row1), float("nan"), dtype=torch.float64, device=T.device)
    base = t0 * (t0 + 1) // 2
    for ti in range(t0, t1):
        r0, r1 = ti * TILE, min((ti + 1) * TILE, row1)
        for tj in range(ti + 1):
            c0, c1 = tj * TILE, min((tj + 1) * TILE, row1)
            out[r0 - row0:r1 - row0, c0:c1] = T[ti * (ti + 1) // 2 + tj - base, :r1 - r0, :c1 - c0]
    return out


def lower_mask(row0, row1, device=DEV):
    r = torch.arange(row0, row1, device=device)[:, None]
    c = torch.arange(row1, device=device)[None, :]
    return c <= r


def band_tiles(row0, row1):
    t0, t1 = row0 // TILE, (row1 + TILE - 1) // TILE
    return (t1 * (t1 + 1) // 2 - t0 * (t0 + 1) // 2) * TILE * TILE


@pytest.fixture(scope="module")
def cfg2():
    from paper_1812_07437_gb300.handle import Handle
    h = Handle(workloads.get("cfg2_5bin"))
    D = torch.zeros(h.M, dtype=torch.float64, device=DEV)
    h.spectra(D)
    yield h
    h.close()


@pytest.mark.parametrize("precision", [N.COV_SPLIT_BF16, N.COV_FP64])
def test_bands_equal_full_assembly(cfg2, precision):
    h = cfg2
    M = h.M
    C = torch.full((M, M), float("nan"), dtype=torch.float64, device=DEV)
    h.assemble(C, N.COV_TERMS_ALL, precision)
    torch.cuda.synchronize()
    # uneven band sizes: one tile row, several, and the ragged end at M
    cuts = [0, 256, 1280, 2048, 4096, 6144, M]
    for row0, row1 in zip(cuts[:-1], cuts[1:]):
        m = lower_mask(row0, row1)
        ref = C[row0:row1, :row1]
        Br = torch.full((row1 - row0, row1 + 3), float("nan"), dtype=torch.float64, device=DEV)
        h.assemble_band(row0, row1 - row0, Br, N.COV_LAYOUT_ROWS, N.COV_TERMS_ALL, precision)
        Bt = torch.full((band_tiles(row0, row1),), float("nan"), dtype=torch.float64, device=DEV)
        h.assemble_band(row0, row1 - row0, Bt, N.COV_LAYOUT_TILES, N.COV_TERMS_ALL, precision)
        torch.cuda.synchronize()
        assert torch.equal(Br[:, :row1][m], ref[m]), (row0, row1)
        assert torch.isnan(Br[:, row1:]).all()  # nothing beyond the band's columns
        assert torch.equal(tiles_to_rows(Bt, row0, row1)[m], ref[m]), (row0, row1)


def test_band_arguments_rejected(cfg2):
    h = cfg2
    buf = torch.zeros(256 * 512, dtype=torch.float64, device=DEV)
    p = buf.data_ptr()
    L = h.L
    import ctypes as C
    for row0, nrows, ldc, layout, terms in [(100, 256, 512, N.COV_LAYOUT_ROWS, N.COV_TERMS_ALL),   # unaligned start
                                            (0, 300, 512, N.COV_LAYOUT_ROWS, N.COV_TERMS_ALL),     # unaligned end
                                            (256, 256, 256, N.COV_LAYOUT_ROWS, N.COV_TERMS_ALL),   # ldc < row1
                                            (0, 256, 512, 7, N.COV_TERMS_ALL),                     # bad layout
                                            (0, 256, 512, N.COV_LAYOUT_ROWS, N.COV_TERM_SSC),      # SSC without 1H
                                            (6144, 512, 8192, N.COV_LAYOUT_ROWS, N.COV_TERMS_ALL)]:  # past M
        rc = L.cov_assemble_band(h.h, row0, nrows, C.c_void_p(p), ldc, layout, terms, N.COV_SPLIT_BF16, None)
        assert rc == N.COV_ERR_INVALID, (row0, nrows, ldc, layout, terms)


# ------------------------------------------------------------------ cfg3
@pytest.fixture(scope="module")
def cfg3():
    from paper_1812_07437_gb300.handle import Handle
    name = "cfg3_10bin"
    h = Handle(workloads.get(name))
    D = torch.zeros(h.M, dtype=torch.float64, device=DEV)
    h.spectra(D)
    r = OracleRun(workloads.get(name), ntri=make_counts.load(name)[1])
    yield h, r, D
    h.close()


def _sample(rng, row0, row1, n):
    a = rng.integers(row0, row1, n)
    b = np.array([rng.integers(0, x + 1) for x in a])
    # a share on the band's own diagonal block, where the Gaussian and
    # shared-bin product terms live
    k = n // 3
    b[:k] = np.maximum(a[:k] - rng.integers(0, 256, k), 0)
    b[k:k + 8] = a[k:k + 8]
    return a, b


def _worst(r, Cband, row0, pairs, diag_cache):
    def d(i):
        if i not in diag_cache:
            diag_cache[i] = r.cov.element(i, i)
        return diag_cache[i]
    worst = 0.0
    for a, b in zip(*pairs):
        ref = r.cov.element(int(a), int(b))
        worst = max(worst, abs(float(Cband[a - row0, b]) - ref) / np.sqrt(d(int(a)) * d(int(b))))
    return worst


def test_cfg3_data_vector_matches_oracle(cfg3):
    h, r, D = cfg3
    assert h.M == 181350
    np.testing.assert_allclose(D.cpu().numpy(), r.D, rtol=1e-10, atol=0)


@pytest.fixture(scope="module")
def cfg3_diag(cfg3):
    """Assemble the whole cfg3 matrix (split-BF16, every term) band by band into
    a reused tile buffer; keep its diagonal.  Every written value must be
    finite and every diagonal entry positive."""
    h, _, _ = cfg3
    M = h.M
    nt = (M + TILE - 1) // TILE
    step = 8
    buf = torch.empty((band_tiles((nt - step) * TILE, M),), dtype=torch.float64, device=DEV)
    diag = torch.empty(M, dtype=torch.float64, device=DEV)
    idx = torch.arange(TILE, device=DEV)
    for t0 in range(0, nt, step):
        t1 = min(t0 + step, nt)
        row0, row1 = t0 * TILE, min(t1 * TILE, M)
        n = band_tiles(row0, row1)
        buf[:n].zero_()
        h.assemble_band(row0, row1 - row0, buf[:n], N.COV_LAYOUT_TILES, N.COV_TERMS_ALL, N.COV_SPLIT_BF16)
        assert bool(torch.isfinite(buf[:n]).all()), f"non-finite value in tile rows {t0}..{t1}"
        T = buf[:n].view(-1, TILE, TILE)
        base = t0 * (t0 + 1) // 2
        for ti in range(t0, t1):
            r1 = min(TILE, M - ti * TILE)
            diag[ti * TILE:ti * TILE + r1] = T[ti * (ti + 1) // 2 + ti - base][idx[:r1], idx[:r1]]
    torch.cuda.synchronize()
    assert bool((diag > 0).all())
    return diag


def test_cfg3_bands_sampled_against_oracle(cfg3, cfg3_diag):
    h, r, _ = cfg3
    M = h.M
    rng = np.random.default_rng(31)
    diag_cache = {}
    for row0, row1 in [(0, 256), (256 * 350, 256 * 352), (256 * (M // 256), M)]:
        m = lower_mask(row0, row1)
        Bs = torch.full((band_tiles(row0, row1),), float("nan"), dtype=torch.float64, device=DEV)
        h.assemble_band(row0, row1 - row0, Bs, N.COV_LAYOUT_TILES, N.COV_TERMS_ALL, N.COV_SPLIT_BF16)
        B64 = torch.full((row1 - row0, row1), float("nan"), dtype=torch.float64, device=DEV)
        h.assemble_band(row0, row1 - row0, B64, N.COV_LAYOUT_ROWS, N.COV_TERMS_ALL, N.COV_FP64)
        torch.cuda.synchronize()
        Ss = tiles_to_rows(Bs, row0, row1)
        assert bool(torch.isfinite(Ss[m]).all()) and bool(torch.isfinite(B64[m]).all())
        pairs = _sample(rng, row0, row1, 90)
        w64 = _worst(r, B64.cpu().numpy(), row0, pairs, diag_cache)
        ws = _worst(r, Ss.cpu().numpy(), row0, pairs, diag_cache)
        assert w64 <= 1e-10, f"band {row0}: FP64 form worst normalised err {w64:.3e}"
        assert ws <= 1e-4, f"band {row0}: split-BF16 worst normalised err {ws:.3e}"
        # every element of the band: split against FP64, normalised by the
        # diagonal of the whole split matrix
        d = torch.sqrt(cfg3_diag[:row1])
        norm = torch.outer(d[row0:row1], d)
        err = ((Ss - B64).abs() / norm)[m].max()
        assert float(err) <= 1e-4, f"band {row0}: split vs FP64 max normalised err {float(err):.3e}"
        # the band's diagonal is the one the full pass stored
        rows = torch.arange(row0, row1, device=DEV)
        assert torch.equal(Ss[rows - row0, rows], cfg3_diag[row0:row1])
