"""GPU checks of the cumulative row order and the in-place S/N on lower-packed
tiles (cov_snr_tiles), the form used where the dense square does not fit.

* A handle in cumulative order (rows sorted by their largest ell bin) computes
  the same data vector and covariance as the natural order, permuted.
* cov_snr_tiles on the cumulative-order handle's packed tiles (joint, P-only
  and B-only row sets) equals cov_snr on the natural-order dense matrix, in
  the FP64 form (1e-10 relative; both run the same FP64-accurate Cholesky) and
  in the split-BF16 form.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1812_07437_gb300 import native as N  # noqa: E402
from paper_1812_07437_gb300 import workloads  # noqa: E402

DEV = "cuda:0"


def _maxbin(rd):
    return np.where(rd[:, 0] == 0, rd[:, 1], rd[:, 3])


def _perm(nat, cum):
    """Index of each cumulative-order row in the natural order."""
    key = {tuple(r): a for a, r in enumerate(nat)}
    return np.array([key[tuple(r)] for r in cum])


@pytest.mark.parametrize("name", ["mid_3bin", "cfg2_5bin"])
def test_cumulative_order_is_a_permutation(name):
    from paper_1812_07437_gb300.handle import Handle
    a = Handle(workloads.get(name))
    b = Handle(workloads.get(name), order=N.COV_ORDER_CUMULATIVE)
    rn, rc = a.row_desc(), b.row_desc()
    assert np.all(np.diff(_maxbin(rc)) >= 0)
    p = _perm(rn, rc)
    assert sorted(p.tolist()) == list(range(a.M))
    Da = torch.zeros(a.M, dtype=torch.float64, device=DEV)
    Db = torch.zeros(a.M, dtype=torch.float64, device=DEV)
    a.spectra(Da)
    b.spectra(Db)
    assert torch.equal(Db.cpu(), Da.cpu()[torch.as_tensor(p)])
    Ca = torch.zeros(a.M, a.M, dtype=torch.float64, device=DEV)
    Cb = torch.zeros(a.M, a.M, dtype=torch.float64, device=DEV)
    a.assemble(Ca, N.COV_TERMS_ALL, N.COV_FP64)
    b.assemble(Cb, N.COV_TERMS_ALL, N.COV_FP64)
    Sa = torch.tril(Ca) + torch.tril(Ca, -1).T
    Sb = torch.tril(Cb) + torch.tril(Cb, -1).T
    pt = torch.as_tensor(p, device=DEV)
    ref = Sa[pt][:, pt]
    d = torch.sqrt(torch.diagonal(ref))
    assert float(((Sb - ref).abs() / torch.outer(d, d)).max()) <= 1e-12
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [N.COV_FP64, N.COV_SPLIT_BF16])
@pytest.mark.parametrize("rows,which", [(N.COV_ROWS_JOINT, N.COV_WHICH_JOINT), (N.COV_ROWS_B, N.COV_WHICH_B),
                                        (N.COV_ROWS_P, N.COV_WHICH_P)])
def test_snr_tiles_matches_dense(rows, which, precision):
    from paper_1812_07437_gb300.handle import Handle, packed_tiles
    name = "cfg2_5bin"
    a = Handle(workloads.get(name))
    Da = torch.zeros(a.M, dtype=torch.float64, device=DEV)
    Ca = torch.zeros(a.M, a.M, dtype=torch.float64, device=DEV)
    a.spectra(Da)
    a.assemble(Ca, N.COV_TERMS_ALL, precision)
    ref = a.snr(Ca, Da, which)
    b = Handle(workloads.get(name), rows=rows, order=N.COV_ORDER_CUMULATIVE)
    Db = torch.zeros(b.M, dtype=torch.float64, device=DEV)
    b.spectra(Db)
    Ct = torch.full((packed_tiles(b.M + 1) * 65536,), float("nan"), dtype=torch.float64, device=DEV)
    b.assemble_band(0, b.M, Ct, N.COV_LAYOUT_TILES, N.COV_TERMS_ALL, precision)
    got = b.snr_tiles(Ct, Db)
    m = np.isfinite(ref)
    assert np.array_equal(m, np.isfinite(got))
    assert np.max(np.abs(got[m] / ref[m] - 1)) <= 1e-10
    a.close()
    b.close()


@pytest.mark.parametrize("rows", [N.COV_ROWS_JOINT, N.COV_ROWS_P])
def test_snr_tiles_persistent_update_is_bit_identical(rows):
    """The persistent trailing update (128 x 32 tiles moved by TMA, epilogue
    overlapping the next tile's MMAs) and the one-CTA-per-tile update form the
    same exact integer group sums: on the packed tiles of cfg2 (every other
    panel starts half-way into a 128-row block; a ragged last block) the S/N
    agree bit for bit."""
    from paper_1812_07437_gb300.handle import Handle, packed_tiles
    name = "cfg2_5bin"
    b = Handle(workloads.get(name), rows=rows, order=N.COV_ORDER_CUMULATIVE)
    c = Handle(workloads.get(name), rows=rows, order=N.COV_ORDER_CUMULATIVE, chol_kernel=N.COV_CHOL_TILE)
    Db = torch.zeros(b.M, dtype=torch.float64, device=DEV)
    b.spectra(Db)
    Ct = torch.full((packed_tiles(b.M + 1) * 65536,), float("nan"), dtype=torch.float64, device=DEV)
    b.assemble_band(0, b.M, Ct, N.COV_LAYOUT_TILES, N.COV_TERMS_ALL, N.COV_FP64)
    Ct2 = Ct.clone()
    got = b.snr_tiles(Ct, Db)
    ref = c.snr_tiles(Ct2, Db)
    assert np.array_equal(got, ref, equal_nan=True)
    # the factor itself (lower triangle, rows up to the D row) bit for bit
    T = (b.M + 1 + 255) // 256
    rr = torch.arange(256, device=DEV)
    lower_of_diag = rr[:, None] >= rr[None, :]
    A1, A2 = Ct.view(-1, 256, 256), Ct2.view(-1, 256, 256)
    for ti in range(T):
        nr = min(256, b.M + 1 - 256 * ti)
        for tj in range(ti + 1):
            k = ti * (ti + 1) // 2 + tj
            x, y = A1[k, :nr], A2[k, :nr]
            if tj == ti:
                x, y = torch.where(lower_of_diag[:nr], x, 0.0), torch.where(lower_of_diag[:nr], y, 0.0)
            # (M, M), the data row's own diagonal, is never initialised or read
            nan = torch.isnan(x)
            assert torch.equal(nan, torch.isnan(y)) and torch.equal(x[~nan], y[~nan]), (ti, tj)
    b.close()
    c.close()
