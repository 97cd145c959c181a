// Cumulative signal-to-noise (paper Sec. 5, Eqs. SNprim and eq:SN).
//
// The selected entries (P, B or the joint vector) are reordered by their
// largest ell bin (stable), Jacobi-scaled, C' = d^-1/2 C d^-1/2 and
// D' = d^-1/2 D, and written with D' as one extra last row into an FP64
// workspace.  A blocked right-looking Cholesky factorisation of the leading
// M_s x M_s block carries the extra row along, so that row ends up holding
// y = L^-1 D'.  Diagonal blocks and panel solves run in FP64 on the CUDA cores;
// the trailing updates run on the tensor cores with exact integer slicing
// (chol_tc.cu), accurate to ~2^-48 of each row's largest entry.  Because the
// leading principal block of a Cholesky factor is the factor of the leading
// principal block, (S/N)^2 for every cumulative ell_max is a prefix sum of y^2
// over the reordered entries.
#include <algorithm>

#include "common.cuh"

#define NB 64

__global__ void k_snr_pack(int64_t Ms, const int* perm, const double* C, int64_t ldc, const double* D, double* Wk,
                           int64_t ldw) {
  int64_t i = blockIdx.x;  // row of the workspace (0..Ms)
  int64_t j = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (i > Ms || j > i) return;
  if (i == Ms) {
    if (j < Ms) {
      int64_t pj = perm[j];
      Wk[i * ldw + j] = D[pj] / sqrt(C[pj * ldc + pj]);
    } else {
      Wk[i * ldw + j] = 0.0;
    }
    return;
  }
  int64_t pi = perm[i], pj = perm[j];
  int64_t hi = pi > pj ? pi : pj, lo = pi > pj ? pj : pi;
  Wk[i * ldw + j] = C[hi * ldc + lo] / sqrt(C[pi * ldc + pi] * C[pj * ldc + pj]);
}

// in-place Cholesky of the kb x kb diagonal block at (k0, k0); one block of
// 256 threads, thread (tx, ty) owns rows ty + 16 r and columns tx + 16 c
__global__ void k_potrf_diag(OutMap W, int64_t k0, int kb, int* status) {
  __shared__ double L[NB][NB + 1];
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int i = ty + 16 * r, l = tx + 16 * c;
      L[i][l] = (i < kb && l <= i) ? *W.at(k0 + i, k0 + l) : 0.0;
    }
  __shared__ double inv_sh;
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (threadIdx.x == 0) {
      double d = L[j][j];
      if (!(d > 0.0)) {
        atomicExch(status, 1);
        d = 1.0;
      }
      double r = sqrt(d);
      L[j][j] = r;
      inv_sh = 1.0 / r;  // one FP64 division per step, shared by all threads
    }
    __syncthreads();
    double inv = inv_sh;
    if (tx == (j & 15)) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int i = ty + 16 * r;
        if (i > j && i < kb) L[i][j] *= inv;
      }
    }
    __syncthreads();
    // rank-1 update of the trailing triangle j < l <= i < kb: only the active
    // elements are enumerated, so no FP64 issue slot goes to masked lanes
    int m = kb - j - 1;
    int tot = m * (m + 1) / 2;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      int ii = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
      while (ii * (ii + 1) / 2 > e) --ii;
      while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
      int ll = e - ii * (ii + 1) / 2;
      int i = j + 1 + ii, l = j + 1 + ll;
      L[i][l] -= L[i][j] * L[l][j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int i = ty + 16 * r, l = tx + 16 * c;
      if (i < kb && l <= i) *W.at(k0 + i, k0 + l) = L[i][l];
    }
}

// The same factorisation with the pivot of step j + 1 taken off the critical
// path.  Once column j is scaled, lane 0 of warp 0 applies column j to the
// next diagonal entry and takes its pivot, while warps 1-7 apply column j to
// the other active pairs.  The pairs (i, l), l <= i < 64, are enumerated
// through a table ordered by l descending, so that step j's active pairs
// (l > j) are its first (63 - j)(64 - j) / 2 entries and the next diagonal
// entry (j + 1, j + 1) is entry (62 - j)(63 - j) / 2.  Every element receives
// the same FMAs and scalings in the same order as in the plain right-looking
// loop; each step has two barriers instead of three, and its pivot runs beside
// its update.  On this part a dependent FP64 operation takes 64 cycles or more
// and one warp issues at most one FP64 instruction per 64 cycles (idle lanes
// cost the same as active ones), so the update is spread over seven warps and
// the sequential pivot chain is kept short: 1 / sqrt(d) by the reciprocal
// square root and sqrt(d) as d times it (within 2 ulp of the rounded root;
// ~430 cycles together) instead of a square root and a division (~600 + ~360).
__device__ __forceinline__ void potrf_pivot(double (*L)[NB + 1], double* inv, int j, int* status) {
  double d = L[j][j];
  if (!(d > 0.0)) {
    atomicExch(status, 1);
    d = 1.0;
  }
  const double ir = rsqrt(d);
  L[j][j] = d * ir;
  inv[j] = ir;
}

__global__ void __launch_bounds__(256) k_potrf_la(OutMap W, int64_t k0, int kb, int* status) {
  __shared__ double L[NB][NB + 1];
  __shared__ double inv[NB];
  __shared__ uint16_t pr[NB * (NB + 1) / 2];
  // pair table: l = 63, 62, ..., 0; for each l, i = l .. 63
  for (int l = 0; l < NB; ++l) {
    const int base = (NB - 1 - l) * (NB - l) / 2;  // entries before column l (columns l+1..63)
    for (int i = l + (int)threadIdx.x; i < NB; i += blockDim.x) pr[base + (i - l)] = (uint16_t)(i | (l << 8));
  }
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int i = e >> 6, l = e & 63;
    L[i][l] = (i < kb && l <= i) ? *W.at(k0 + i, k0 + l) : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) potrf_pivot(L, inv, 0, status);
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  for (int j = 0; j < kb; ++j) {
    const double s = inv[j];
    for (int i = j + 1 + (int)threadIdx.x; i < kb; i += blockDim.x) L[i][j] *= s;
    __syncthreads();
    if (warp == 0) {
      if (threadIdx.x == 0 && j + 1 < kb) {
        L[j + 1][j + 1] -= L[j + 1][j] * L[j + 1][j];
        potrf_pivot(L, inv, j + 1, status);
      }
    } else {
      const int tj = (NB - 1 - j) * (NB - j) / 2;        // active pairs: l > j
      const int skip = (NB - 2 - j) * (NB - 1 - j) / 2;  // (j + 1, j + 1): lane 0 of warp 0
      const int nt = (int)blockDim.x - 32;
      // four pairs per thread at once: their loads and FMAs overlap (one warp
      // issues one FP64 instruction per 64 cycles, the latency of each)
      for (int e0 = (int)threadIdx.x - 32; e0 < tj; e0 += 4 * nt) {
        int ii[4], ll[4];
        bool ok[4];
        double acc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int e = e0 + k * nt;
          ok[k] = e < tj && e != skip;
          const int pe = pr[ok[k] ? e : 0];
          ii[k] = pe & 255;
          ll[k] = pe >> 8;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] = fma(-L[ii[k]][j], L[ll[k]][j], L[ii[k]][ll[k]]);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (ok[k]) L[ii[k]][ll[k]] = acc[k];
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int i = e >> 6, l = e & 63;
    if (i < kb && l <= i) *W.at(k0 + i, k0 + l) = L[i][l];
  }
}

#define TRSM_ROWS 32
// rows r in [r0, r1): x L11^T = a by forward substitution, one row per lane
// (32 rows per block): every lane runs the whole recurrence of its own row in
// registers, reading L11 from shared memory by broadcast, so no FP64 issue slot
// is spent on masked lanes
__global__ void k_trsm_rows(OutMap W, int64_t k0, int kb, int64_t r0, int64_t r1) {
  __shared__ double L[NB][NB + 1];
  __shared__ double invd[NB];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    int i = e >> 6, l = e & 63;
    L[i][l] = (i < kb && l <= i) ? *W.at(k0 + i, k0 + l) : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kb; i += blockDim.x) invd[i] = 1.0 / L[i][i];
  __syncthreads();
  int64_t r = r0 + (int64_t)blockIdx.x * TRSM_ROWS + threadIdx.x;
  if (r >= r1) return;
  double* row = W.at(r, k0);  // kb <= 64 consecutive entries (k0 is a multiple of 64)
  double x[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) x[j] = (j < kb) ? row[j] : 0.0;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < kb) {
      // four independent partial sums break the FP64 dependency chain
      double v0 = x[j], v1 = 0.0, v2 = 0.0, v3 = 0.0;
#pragma unroll
      for (int l = 0; l + 3 < j; l += 4) {
        v0 -= x[l] * L[j][l];
        v1 -= x[l + 1] * L[j][l + 1];
        v2 -= x[l + 2] * L[j][l + 2];
        v3 -= x[l + 3] * L[j][l + 3];
      }
#pragma unroll
      for (int l = j & ~3; l < j; ++l) v0 -= x[l] * L[j][l];
      x[j] = ((v0 + v1) + (v2 + v3)) * invd[j];
    }
  }
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < kb) row[j] = x[j];
}

// The same solve with four lanes per row (eight rows per warp): lane q owns
// the right-hand-side entries j = q (mod 4).  Column by column, the owner of
// column l scales its entry into x_l, shuffles it to the other three lanes,
// and each lane subtracts x_l L[j][l] from its entries j > l.  Four times the
// warps of k_trsm_rows, so the FP64 latency of a row's 64-step chain is hidden
// across more rows in flight.
#define TR4_THREADS 128
__global__ void __launch_bounds__(TR4_THREADS) k_trsm_rows4(OutMap W, int64_t k0, int kb, int64_t r0, int64_t r1) {
  __shared__ double L[NB][NB + 1];
  __shared__ double invd[NB];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    int i = e >> 6, l = e & 63;
    L[i][l] = (i < kb && l <= i) ? *W.at(k0 + i, k0 + l) : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kb; i += blockDim.x) invd[i] = 1.0 / L[i][i];
  __syncthreads();
  const int lane = threadIdx.x & 31, q = lane & 3, g4 = lane & ~3;
  const int64_t r = r0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 4;
  const bool valid = r < r1;
  double* row = valid ? W.at(r, k0) : nullptr;
  double a[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) a[m] = (valid && q + 4 * m < kb) ? row[q + 4 * m] : 0.0;
#pragma unroll
  for (int l = 0; l < NB; ++l) {
    if (l >= kb) break;
    if (q == (l & 3)) a[l >> 2] *= invd[l];
    const double xl = __shfl_sync(0xffffffffu, a[l >> 2], g4 + (l & 3));
#pragma unroll
    for (int m = (l + 1) / 4; m < 16; ++m) {
      const int j = q + 4 * m;
      if (j > l) a[m] = fma(-xl, L[j][l], a[m]);
    }
  }
  if (valid) {
#pragma unroll
    for (int m = 0; m < 16; ++m)
      if (q + 4 * m < kb) row[q + 4 * m] = a[m];
  }
}

__global__ void k_snr_prefix(int64_t Ms, OutMap W, const int64_t* cnt, int nl, double* out) {
  __shared__ double sh[32];
  int c = blockIdx.x;
  int64_t n = cnt[c];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double y = *W.at(Ms, i);
    s += y * y;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[c] = (n > 0) ? sqrt(s) : nan("");
}

// Scratch of the factorisation of Ms rows (slice buffers, status words, the
// side stream of the look-ahead), allocated once and grown on demand.
static int chol_scratch(cov_handle* h, int64_t Ms, size_t* one_buf) {
  *one_buf = (wl_chol_tc_bytes(Ms + 1) + 255) / 256 * 256;
  size_t need_sc = 2 * *one_buf;
  if (need_sc > h->chol_scratch_n) {
    if (h->chol_scratch) {
      cudaFree(h->chol_scratch);
      h->allocated -= h->chol_scratch_n;
    }
    h->chol_scratch = nullptr;
    h->chol_scratch_n = 0;
    WL_CHECK(h, cudaMalloc(&h->chol_scratch, need_sc));
    h->chol_scratch_n = need_sc;
    h->allocated += need_sc;
  }
  if (!h->chol_status) WL_CHECK(h, cudaMalloc(&h->chol_status, sizeof(int)));
  return wl_side_stream(h);
}

// Blocked right-looking Cholesky of the leading Ms x Ms block of the
// workspace Wm (rows 0..Ms; row Ms carries D' along and ends up as
// y = L^-1 D'), then (S/N)^2 for every cumulative selection as the prefix
// sums of y^2 up to cnt_d[c] entries, into out_d (device, n_ell).  Outside a
// captured batch step the result is copied to h_snr and the status words are
// checked; inside one (h->deferred) both stay on the device and the status
// words accumulate over the replays.
static int factor_and_prefix(cov_handle* h, OutMap Wm, int64_t Ms, const int64_t* cnt_d, double* out_d,
                             double* h_snr, cudaStream_t s) {
  size_t one_buf = 0;
  int rc;
  if ((rc = chol_scratch(h, Ms, &one_buf))) return rc;
  if (!h->deferred) {
    WL_CHECK(h, cudaMemsetAsync(h->chol_status, 0, sizeof(int), s));
    WL_CHECK(h, cudaMemsetAsync(h->piv_status, 0, sizeof(int), s));
  }
  int* st = h->piv_status;
  int tk = wl_stage_begin(h, ST_SNR_CHOL, s);
  uint8_t* bufs[2] = {(uint8_t*)h->chol_scratch, (uint8_t*)h->chol_scratch + one_buf};
  auto panel = [&](int64_t k0, cudaStream_t st_) -> int {
    int kb = (int)std::min<int64_t>(NB, Ms - k0);
    k_potrf_la<<<1, 256, 0, st_>>>(Wm, k0, kb, st);
    int64_t r0 = k0 + kb, r1 = Ms + 1;
    if (wl_chol_fused_panel(h, Wm)) {
      WL_LAUNCH(h, "k_potrf_la");
      return wl_chol_trsm_slice(h, Wm, k0, kb, r0, r1, bufs[(k0 / NB) & 1], st_);
    }
    if (r1 > r0)
      k_trsm_rows4<<<(unsigned)(((r1 - r0) * 4 + TR4_THREADS - 1) / TR4_THREADS), TR4_THREADS, 0, st_>>>(Wm, k0, kb,
                                                                                                     r0, r1);
    WL_LAUNCH(h, "Cholesky panel kernels");
    return wl_chol_slice(h, Wm, k0, kb, r0, r1, bufs[(k0 / NB) & 1], st_);
  };
  if ((rc = panel(0, s))) return rc;
  for (int64_t k0 = 0; k0 < Ms; k0 += NB) {
    int kb = (int)std::min<int64_t>(NB, Ms - k0);
    int64_t r0 = k0 + kb, r1 = Ms + 1;
    const void* buf = bufs[(k0 / NB) & 1];
    if (r0 < Ms && h->chol_lookahead) {
      // one panel of look-ahead: the trailing update of panel p first updates
      // the 64 columns of panel p+1, then the FP64 diagonal block, panel solve
      // and slicing of panel p+1 run on the side stream while the rest of the
      // update of panel p runs here
      if ((rc = wl_chol_update(h, Wm, r0, r1, buf, 0, 1, h->chol_status, s))) return rc;
      WL_CHECK(h, cudaEventRecord(h->ev_cols, s));
      WL_CHECK(h, cudaStreamWaitEvent(h->side, h->ev_cols, 0));
      if ((rc = panel(r0, h->side))) return rc;
      WL_CHECK(h, cudaEventRecord(h->ev_panel, h->side));
      if ((rc = wl_chol_update(h, Wm, r0, r1, buf, 1, -1, h->chol_status, s))) return rc;
      WL_CHECK(h, cudaStreamWaitEvent(s, h->ev_panel, 0));
    } else if (r0 < Ms) {
      if ((rc = wl_chol_update(h, Wm, r0, r1, buf, 0, -1, h->chol_status, s))) return rc;
      if ((rc = panel(r0, s))) return rc;
    } else if (r1 > r0) {
      // only the extra D row is left below this panel
      if ((rc = wl_chol_update(h, Wm, r0, r1, buf, 0, -1, h->chol_status, s))) return rc;
    }
  }
  WL_LAUNCH(h, "Cholesky kernels");
  wl_stage_end(h, tk, s);
  tk = wl_stage_begin(h, ST_SNR_PREFIX, s);
  k_snr_prefix<<<h->nl, 256, 0, s>>>(Ms, Wm, cnt_d, h->nl, out_d);
  WL_LAUNCH(h, "k_snr_prefix");
  wl_stage_end(h, tk, s);
  if (h->deferred) return COV_OK;
  int status = 0, tstatus = 0;
  WL_CHECK(h, cudaMemcpyAsync(h_snr, out_d, sizeof(double) * h->nl, cudaMemcpyDeviceToHost, s));
  WL_CHECK(h, cudaMemcpyAsync(&status, st, sizeof(int), cudaMemcpyDeviceToHost, s));
  WL_CHECK(h, cudaMemcpyAsync(&tstatus, h->chol_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  WL_CHECK(h, cudaStreamSynchronize(s));
  if (tstatus) return wl_fail(h, COV_ERR_TIMEOUT, "Cholesky trailing update: a bounded mbarrier wait expired");
  if (status) return wl_fail(h, COV_ERR_NOT_PD, "Cholesky met a non-positive pivot");
  return COV_OK;
}

static int maxbin_of(const cov_handle* h, int64_t a) {
  return h->rowdesc[8 * a] == 0 ? h->rowdesc[8 * a + 1] : h->rowdesc[8 * a + 3];
}

// Device copies of a selection (slot 0..2: P, B, joint for the dense S/N;
// slot 3: all rows, in their cumulative order, for the packed-tile S/N): the
// reordering permutation and the prefix counts, built once per handle.
static int selection(cov_handle* h, int slot, cudaStream_t s) {
  if (h->sel[slot].ready) return COV_OK;
  std::vector<int> sel;
  for (int64_t a = 0; a < h->M; ++a) {
    int type = h->rowdesc[8 * a];
    if (slot == COV_WHICH_P && type != 0) continue;
    if (slot == COV_WHICH_B && type != 1) continue;
    sel.push_back((int)a);
  }
  if (slot < 3)
    std::stable_sort(sel.begin(), sel.end(), [&](int x, int y) { return maxbin_of(h, x) < maxbin_of(h, y); });
  int64_t Ms = (int64_t)sel.size();
  std::vector<int64_t> cnt(h->nl, 0);
  for (int c = 0; c < h->nl; ++c)
    for (int64_t i = 0; i < Ms; ++i)
      if (maxbin_of(h, sel[i]) <= c) cnt[c] = i + 1;
  auto& z = h->sel[slot];
  if (!z.perm) {
    WL_CHECK(h, cudaMalloc(&z.perm, sizeof(int) * (size_t)std::max<int64_t>(Ms, 1)));
    WL_CHECK(h, cudaMalloc(&z.cnt, sizeof(int64_t) * h->nl));
    WL_CHECK(h, cudaMalloc(&z.out, sizeof(double) * h->nl));
    h->allocated += sizeof(int) * (size_t)std::max<int64_t>(Ms, 1) + sizeof(int64_t) * h->nl + sizeof(double) * h->nl;
  }
  if (!h->piv_status) {
    WL_CHECK(h, cudaMalloc(&h->piv_status, sizeof(int)));
    WL_CHECK(h, cudaMemsetAsync(h->piv_status, 0, sizeof(int), s));
  }
  if (Ms) WL_CHECK(h, cudaMemcpyAsync(z.perm, sel.data(), sizeof(int) * Ms, cudaMemcpyHostToDevice, s));
  WL_CHECK(h, cudaMemcpyAsync(z.cnt, cnt.data(), sizeof(int64_t) * h->nl, cudaMemcpyHostToDevice, s));
  WL_CHECK(h, cudaStreamSynchronize(s));  // sel and cnt are host memory read by the copies
  z.Ms = Ms;
  z.ready = true;
  return COV_OK;
}

int wl_snr(cov_handle* h, const double* C, int64_t ldc, const double* D, int which, double* h_snr, cudaStream_t s) {
  int rc;
  if ((rc = selection(h, which, s))) return rc;
  const auto& z = h->sel[which];
  const int64_t Ms = z.Ms;
  if (Ms == 0) {
    if (h_snr)
      for (int c = 0; c < h->nl; ++c) h_snr[c] = nan("");
    return COV_OK;
  }
  // rows padded to 8 doubles: the trailing update moves FP64 tiles by TMA,
  // which needs 16-byte row strides
  int64_t ldw = (Ms + 1 + 7) / 8 * 8;
  int64_t need = ldw * (Ms + 1);
  if (need > h->work_n) {
    if (h->work) {
      cudaFree(h->work);
      h->allocated -= sizeof(double) * h->work_n;
    }
    h->work = nullptr;
    h->work_n = 0;
    if (h->budget && h->allocated + sizeof(double) * need > h->budget)
      return wl_fail(h, COV_ERR_NOMEM, "hbm_budget exceeded allocating the Cholesky workspace");
    WL_CHECK(h, cudaMalloc(&h->work, sizeof(double) * need));
    h->work_n = need;
    h->allocated += sizeof(double) * need;
  }
  h->work_ld = ldw;
  dim3 gp((unsigned)(Ms + 1), (unsigned)((Ms + 1 + 255) / 256));
  int tk = wl_stage_begin(h, ST_SNR_PACK, s);
  k_snr_pack<<<gp, 256, 0, s>>>(Ms, z.perm, C, ldc, D, h->work, ldw);
  WL_LAUNCH(h, "k_snr_pack");
  wl_stage_end(h, tk, s);
  return factor_and_prefix(h, out_rows(h->work, ldw), Ms, z.cnt, z.out, h_snr, s);
}

// In place on the lower-packed tiles (rows in cumulative order): Jacobi
// scaling of every element, D' written as row M, then the same
// factorisation.  The diagonal is saved first (the scaling overwrites it).
__global__ void k_tiles_diag(int64_t M, OutMap W, double* dg) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < M) dg[r] = *W.at(r, r);
}

// one block per 32 x 32 lower block of the leading M x M part, plus the D row
__global__ void k_tiles_scale(int64_t M, OutMap W, const double* dg, const double* D) {
  int64_t id = blockIdx.x;
  int64_t bi = (int64_t)((sqrt(8.0 * (double)id + 1.0) - 1.0) * 0.5);
  while (bi * (bi + 1) / 2 > id) --bi;
  while ((bi + 1) * (bi + 2) / 2 <= id) ++bi;
  int64_t bj = id - bi * (bi + 1) / 2;
  int64_t c = bj * 32 + threadIdx.x;
  for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
    int64_t r = bi * 32 + rr;
    if (c > r || c >= M) continue;
    if (r < M) {
      double* p = W.at(r, c);
      *p = *p / sqrt(dg[r] * dg[c]);
    } else if (r == M) {
      *W.at(r, c) = D[c] / sqrt(dg[c]);
    }
  }
}

int wl_snr_tiles(cov_handle* h, double* Ct, const double* D, double* h_snr, cudaStream_t s) {
  const int64_t M = h->M;
  int rc;
  if ((rc = selection(h, 3, s))) return rc;
  OutMap Wm = out_tiles(Ct, 0);
  double* dg = nullptr;
  WL_CHECK(h, cudaMallocAsync(&dg, sizeof(double) * M, s));
  int tk = wl_stage_begin(h, ST_SNR_PACK, s);
  k_tiles_diag<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(M, Wm, dg);
  int64_t nb = (M + 1 + 31) / 32;
  k_tiles_scale<<<(unsigned)(nb * (nb + 1) / 2), dim3(32, 8), 0, s>>>(M, Wm, dg, D);
  WL_LAUNCH(h, "k_tiles_scale");
  wl_stage_end(h, tk, s);
  WL_CHECK(h, cudaFreeAsync(dg, s));
  return factor_and_prefix(h, Wm, M, h->sel[3].cnt, h->sel[3].out, h_snr, s);
}
