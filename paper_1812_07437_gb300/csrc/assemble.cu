// Covariance assembly (paper Sec. 3.2 and Appendix B):
//  * the 1-halo contraction stores the lower triangle first (no clear pass);
//  * k_gather   BB+PT and PB product terms, element by element, added on top
//               (or stored when the 1-halo term is not requested) over the
//               32 x 32 blocks whose rows share an ell bin: every one of these
//               terms vanishes elsewhere (blocks of the remaining ~3/4 of the
//               lower triangle return at once, or store zeros);
//  * k_gauss    the Gaussian PP and BB terms, added over the diagonal blocks
//               of one ell bin (P rows) or one triangle (B rows), the sum over
//               leg permutations reduced across lanes by warp shuffles;
//  * k_gemm_lower  C = alpha A B^T + beta C on the lower triangle in FP64:
//               the 1-halo (chi, M) contraction (FP64 form), the 1-halo
//               trispectrum table of the PT term and the rank-N_chi
//               super-sample term.
#include "common.cuh"

int wl_rows_a(cov_handle* h, cudaStream_t s);
int wl_rows_t(cov_handle* h, cudaStream_t s);
int wl_rows_s(cov_handle* h, cudaStream_t s);
int wl_rows_split(cov_handle* h, int nssc, cudaStream_t s);
int wl_trows_split(cov_handle* h, cudaStream_t s);

__device__ __forceinline__ int64_t leg_pair(int L1, int L2, int nleg) {
  if (L1 > L2) {
    int t = L1;
    L1 = L2;
    L2 = t;
  }
  return (int64_t)L1 * (2 * nleg - L1 + 1) / 2 + (L2 - L1);
}

struct GatherArgs {
  int nt, nleg;
  unsigned terms;
  double omega;
  const int32_t* rd;
  const double* Ps;      // [nl][nt][nt]
  const double* B1hp;    // [ntri][nt][nt][nt]
  const double* Tmat;    // [ntrow][ntrow] lower
  int64_t ntrow;
  const double* invN;    // 1 / N(l^b)
  const double* omN;     // Omega / N_tri(t)
  const uint64_t* bmask; // ell bins present in each 32-row block
  // exact BB+PT couplings (null: 1 / N(l^b)): kappa of leg x of triangle t and
  // leg y of t' in bin A at kap[koff[A] + kcol[3 t + x] kn[A] + kcol[3 t' + y]]
  const double* kap;
  const int32_t* kcol;
  const int32_t* kn;
  const int64_t* koff;
};

// 1 / N(l^b) and Omega / N_tri(t) from the exact integer counts, once per
// assembly, so that the per-element products need no FP64 division
__global__ void k_inv_counts(int nl, int ntri, double omega, const int64_t* Nm, const int64_t* Ntri, double* invN,
                             double* omN) {
  for (int i = threadIdx.x; i < nl; i += blockDim.x) invN[i] = 1.0 / (double)Nm[i];
  for (int t = threadIdx.x; t < ntri; t += blockDim.x) omN[t] = omega / (double)Ntri[t];
}

__device__ __forceinline__ double ps(const GatherArgs& g, int b, int i, int j) {
  return g.Ps[((size_t)b * g.nt + i) * g.nt + j];
}
__device__ __forceinline__ double b1h(const GatherArgs& g, int t, int i, int j, int k) {
  return g.B1hp[(((size_t)t * g.nt + i) * g.nt + j) * g.nt + k];
}

__device__ double gather_element(const GatherArgs& g, const int32_t* ra, const int32_t* rb) {
  double v = 0.0;
  if (ra[0] == 0 && rb[0] == 0) return v;  // PP: the Gaussian term only (k_gauss)
  if (ra[0] == 1 && rb[0] == 1) {
    const int* ba = ra + 1; const int* ta = ra + 4;
    const int* bb = rb + 1; const int* tb = rb + 4;
    if (g.terms & COV_TERM_BBPT) {
      for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y) {
          if (ba[x] != bb[y]) continue;
          int x1 = (x + 1) % 3, x2 = (x + 2) % 3, y1 = (y + 1) % 3, y2 = (y + 2) % 3;
          const int A = ba[x];
          const double iN = g.kap ? g.kap[g.koff[A] + (int64_t)g.kcol[3 * ra[7] + x] * g.kn[A] + g.kcol[3 * rb[7] + y]]
                                  : g.invN[A];
          double bbv = b1h(g, ra[7], tb[y], ta[x1], ta[x2]) * b1h(g, rb[7], ta[x], tb[y1], tb[y2]);
          int64_t r1 = leg_pair(ba[x1] * g.nt + ta[x1], ba[x2] * g.nt + ta[x2], g.nleg);
          int64_t r2 = leg_pair(bb[y1] * g.nt + tb[y1], bb[y2] * g.nt + tb[y2], g.nleg);
          int64_t hi = r1 > r2 ? r1 : r2, lo = r1 > r2 ? r2 : r1;
          double tv = g.Tmat[hi * g.ntrow + lo];
          v += (bbv + ps(g, ba[x], ta[x], tb[y]) * tv) * iN;
        }
    }
    return v;
  }
  if (g.terms & COV_TERM_PB) {
    const int32_t* rp = ra[0] == 0 ? ra : rb;
    const int32_t* rq = ra[0] == 0 ? rb : ra;
    int b = rp[1], i = rp[4], j = rp[5];
    for (int y = 0; y < 3; ++y) {
      if (rq[1 + y] != b) continue;
      int y1 = (y + 1) % 3, y2 = (y + 2) % 3;
      int t = rq[7];
      v += (ps(g, b, i, rq[4 + y]) * b1h(g, t, j, rq[4 + y1], rq[4 + y2]) +
            ps(g, b, j, rq[4 + y]) * b1h(g, t, i, rq[4 + y1], rq[4 + y2])) *
           g.invN[b];
    }
  }
  return v;
}

// lower-triangle tile index -> (ti, tj), ti >= tj
__device__ __forceinline__ void tri_tile(int64_t id, int64_t* ti, int64_t* tj) {
  // an FP32 estimate (the FP64 square root costs ~600 cycles on this part),
  // corrected to the exact row by the two integer searches
  int64_t i = (int64_t)((sqrtf(8.0f * (float)id + 1.0f) - 1.0f) * 0.5f);
  if (i < 0) i = 0;
  while (i * (i + 1) / 2 > id) --i;
  while ((i + 1) * (i + 2) / 2 <= id) ++i;
  *ti = i;
  *tj = id - i * (i + 1) / 2;
}

// ell bins present in every 32-row block of the data vector (bit b: a row of
// the block has a leg in ell bin b); all bits when n_ell > 64 (no skipping)
__global__ void k_block_masks(int64_t M, int nl, const int32_t* rd, uint64_t* bm) {
  int64_t blk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (blk >= (M + 31) / 32) return;
  uint64_t m = 0;
  if (nl <= 64) {
    for (int64_t r = blk * 32; r < M && r < blk * 32 + 32; ++r) {
      const int32_t* x = rd + 8 * r;
      m |= 1ull << x[1];
      if (x[0] == 1) m |= (1ull << x[2]) | (1ull << x[3]);
    }
  } else {
    m = ~0ull;
  }
  bm[blk] = m;
}

// The BB+PT and PB products of the 32 x 32 lower block (ti, tj), rows below M
// only; added to the stored value (accumulate) or stored.  With no ell bin
// common to the two row blocks every product is zero there.
__device__ __forceinline__ void gather_block(const GatherArgs& g, int64_t M, OutMap out, int accumulate, int64_t ti,
                                             int64_t tj, int32_t* rdA, int32_t* rdB) {
  int64_t a0 = ti * 32, b0 = tj * 32;
  const bool none = (g.bmask[ti] & g.bmask[tj]) == 0;
  if (none && accumulate) return;
  int tid = threadIdx.y * 32 + threadIdx.x;
  if (!none) {
    for (int e = tid; e < 256; e += 256) {
      int r = e / 8, c = e % 8;
      rdA[e] = (a0 + r < M) ? g.rd[(a0 + r) * 8 + c] : 0;
      rdB[e] = (b0 + r < M) ? g.rd[(b0 + r) * 8 + c] : 0;
    }
  }
  __syncthreads();
  int64_t b = b0 + threadIdx.x;
  for (int rr = threadIdx.y; rr < 32; rr += 8) {
    int64_t a = a0 + rr;
    if (a >= M || b >= M || b > a) continue;
    double v = none ? 0.0 : gather_element(g, rdA + rr * 8, rdB + threadIdx.x * 8);
    double* p = out.at(a, b);
    *p = accumulate ? *p + v : v;
  }
}

// every lower block of a band (tile_off: the band's first block)
__global__ void k_gather(GatherArgs g, int64_t M, OutMap out, int accumulate, int64_t tile_off) {
  __shared__ int32_t rdA[32 * 8], rdB[32 * 8];
  int64_t ti, tj;
  tri_tile((int64_t)blockIdx.x + tile_off, &ti, &tj);
  gather_block(g, M, out, accumulate, ti, tj, rdA, rdB);
}

// only the listed blocks, those whose row blocks share an ell bin (24% of the
// lower blocks at the 10-bin workload), added to the stored values: no block
// of the grid is spent on the others
__global__ void k_gather_list(GatherArgs g, int64_t M, OutMap out, const uint32_t* __restrict__ list) {
  __shared__ int32_t rdA[32 * 8], rdB[32 * 8];
  const uint32_t pk = list[blockIdx.x];
  gather_block(g, M, out, 1, (int64_t)(pk >> 16), (int64_t)(pk & 0xFFFFu), rdA, rdB);
}

// ---- Gaussian terms on the diagonal blocks ------------------------------------
// The Gaussian PP term pairs two P rows of one ell bin, the Gaussian BB term two
// B rows of one triangle (R6: Omega / N_tri times the sum over the leg
// permutations sigma whose bins match, of prod_a P^s_{t_a t'_sigma(a)}(l_a)).
// Rows of one bin (P) or one triangle (B) are contiguous in every row order, so
// the term lives on diagonal blocks, cut into 32 x 32 sub-blocks (int4: first
// row of the segment, its length, sub-block row and column).  Eight lanes per
// element: lane q computes the product of permutation q (q < 6, zero when its
// bins do not match; PP: q < 2 for the two pairings), and three xor shuffles
// reduce the eight lanes.
__global__ void __launch_bounds__(256) k_gauss(GatherArgs g, const int4* __restrict__ blk, int64_t row0,
                                               int64_t row1, OutMap out) {
  const int4 d = blk[blockIdx.x];
  const int64_t s0 = d.x, ra0 = s0 + 32 * (int64_t)d.z, rb0 = s0 + 32 * (int64_t)d.w;
  const int64_t send = s0 + d.y;
  const int lane = threadIdx.x & 31, q = lane & 7, warp = threadIdx.x >> 5;
  const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  // 1024 elements, four per warp pass, eight warps
  for (int e0 = warp * 4; e0 < 1024; e0 += 32) {
    const int e = e0 + (lane >> 3);
    const int64_t a = ra0 + (e >> 5), b = rb0 + (e & 31);
    const bool ok = a < send && b < send && b <= a && a >= row0 && a < row1;
    double v = 0.0;
    if (ok) {
      const int32_t* x = g.rd + 8 * a;
      const int32_t* y = g.rd + 8 * b;
      if (x[0] == 0) {
        const int bn = x[1], i = x[4], j = x[5], k = y[4], l = y[5];
        if (q == 0) v = ps(g, bn, i, k) * ps(g, bn, j, l);
        if (q == 1) v = ps(g, bn, i, l) * ps(g, bn, j, k);
      } else if (q < 6) {
        const int* sg = perm[q];
        const int* ba = x + 1;
        if (ba[0] == ba[sg[0]] && ba[1] == ba[sg[1]] && ba[2] == ba[sg[2]])
          v = ps(g, ba[0], x[4], y[4 + sg[0]]) * ps(g, ba[1], x[5], y[4 + sg[1]]) * ps(g, ba[2], x[6], y[4 + sg[2]]);
      }
    }
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    if (ok && q == 0) {
      const int32_t* x = g.rd + 8 * a;
      double* p = out.at(a, b);
      *p += v * (x[0] == 0 ? g.invN[x[1]] : g.omN[x[7]]);
    }
  }
}

// ---- FP64 tiled product on the lower triangle ------------------------------
// 64 x 64 tile per block, 256 threads (4 x 4 outputs each), K slabs of 16.
#define GT 64
#define GK 16
__global__ void __launch_bounds__(256) k_gemm_lower(const double* __restrict__ A, int64_t lda,
                                                    const double* __restrict__ B, int64_t ldb, OutMap out,
                                                    int64_t n, int64_t k, double alpha, double beta,
                                                    int lower_only, int64_t ntiles_1d, int64_t tile_off) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  int64_t ti, tj;
  if (lower_only) {
    tri_tile((int64_t)blockIdx.x + tile_off, &ti, &tj);
  } else {
    ti = blockIdx.x / ntiles_1d;
    tj = blockIdx.x % ntiles_1d;
  }
  int64_t i0 = ti * GT, j0 = tj * GT;
  int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  for (int64_t k0 = 0; k0 < k; k0 += GK) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      int idx = threadIdx.x + 256 * l;
      int row = idx / GK, col = idx % GK;
      int64_t gi = i0 + row, gj = j0 + row, gk = k0 + col;
      As[col][row] = (gi < n && gk < k) ? A[gi * lda + gk] : 0.0;
      Bs[col][row] = (gj < n && gk < k) ? B[gj * ldb + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int64_t gi = i0 + ty + 16 * r, gj = j0 + tx + 16 * c;
      if (gi < n && gj < n && (!lower_only || gj <= gi)) {
        double* p = out.at(gi, gj);
        *p = alpha * acc[r][c] + (beta == 0.0 ? 0.0 : beta * *p);
      }
    }
}

int wl_gemm_lower_fp64(cov_handle* h, const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                       int64_t ldc, int64_t n, int64_t k, double alpha, double beta, bool lower_only,
                       cudaStream_t s) {
  if (n <= 0) return COV_OK;
  int64_t nt1 = (n + GT - 1) / GT;
  int64_t nblk = lower_only ? nt1 * (nt1 + 1) / 2 : nt1 * nt1;
  k_gemm_lower<<<(unsigned)nblk, 256, 0, s>>>(A, lda, B, ldb, out_rows(C, ldc), n, k, alpha, beta,
                                              lower_only ? 1 : 0, nt1, 0);
  WL_LAUNCH(h, "k_gemm_lower");
  return COV_OK;
}

// lower part of rows [out.row0, row1) of A B^T (out.row0 a multiple of 64)
static int gemm_lower_band(cov_handle* h, const double* A, int64_t lda, int64_t row1, int64_t k, double beta,
                           OutMap out, cudaStream_t s) {
  int64_t t0 = out.row0 / GT, t1 = (row1 + GT - 1) / GT;
  int64_t off = t0 * (t0 + 1) / 2;
  k_gemm_lower<<<(unsigned)(t1 * (t1 + 1) / 2 - off), 256, 0, s>>>(A, lda, A, lda, out, row1, k, 1.0, beta, 1, t1,
                                                                  off);
  WL_LAUNCH(h, "k_gemm_lower");
  return COV_OK;
}

int wl_ensure(cov_handle* h, void** p, size_t bytes, const char* what) {
  if (*p) return COV_OK;
  if (h->budget && h->allocated + bytes > h->budget)
    return wl_fail(h, COV_ERR_NOMEM, std::string("hbm_budget exceeded allocating ") + what);
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return wl_fail(h, COV_ERR_NOMEM, std::string("cudaMalloc failed for ") + what);
  }
  h->allocated += bytes;
  return COV_OK;
}
static inline int ensure(cov_handle* h, void** p, size_t bytes, const char* what) {
  return wl_ensure(h, p, bytes, what);
}

static int gather_args(cov_handle* h, unsigned terms, GatherArgs* g, cudaStream_t s) {
  int rc;
  if ((rc = ensure(h, (void**)&h->invN, sizeof(double) * h->nl, "inverse mode counts"))) return rc;
  if ((rc = ensure(h, (void**)&h->omN, sizeof(double) * (h->ntri > 0 ? h->ntri : 1), "inverse triangle counts")))
    return rc;
  const int64_t nb = (h->M + 31) / 32;
  if ((rc = ensure(h, (void**)&h->bmask, sizeof(uint64_t) * nb, "block ell-bin masks"))) return rc;
  if (!h->bmask_ready) {  // the layout does not change with the cosmology
    k_block_masks<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(h->M, h->nl, h->rowdesc_d, h->bmask);
    WL_LAUNCH(h, "k_block_masks");
    h->bmask_ready = true;
  }
  k_inv_counts<<<1, 256, 0, s>>>(h->nl, h->ntri, h->omega, h->Nmodes, h->Ntri, h->invN, h->omN);
  WL_LAUNCH(h, "k_inv_counts");
  *g = GatherArgs{h->nt,   h->nleg, terms, h->omega, h->rowdesc_d, h->Ps,   h->B1hp, h->Tmat, h->ntrow,
                  h->invN, h->omN,  h->bmask, h->kap,  h->kcol,      h->kn,   h->koff};
  return COV_OK;
}

// The 32 x 32 sub-blocks (lower part) of the diagonal blocks that hold the
// Gaussian terms: one block per run of consecutive rows of the same type and
// ell bin (P) or triangle (B).  Built once per handle from the row table and
// uploaded on the stream of the kernel that reads it.
static int gauss_blocks(cov_handle* h, cudaStream_t s) {
  if (h->gblk) return COV_OK;
  // a captured step reuses the list of its eager first run: a copy from host
  // memory cannot become part of a graph
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  WL_CHECK(h, cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return wl_fail(h, COV_ERR_INVALID, "Gaussian block list not built before stream capture");
  std::vector<int4> v;
  h->gblk_row.clear();
  const int64_t M = h->M;
  int64_t a = 0;
  while (a < M) {
    const int32_t* r = &h->rowdesc[8 * a];
    const int key = r[0] == 0 ? r[1] : r[7];
    int64_t e = a + 1;
    while (e < M && h->rowdesc[8 * e] == r[0] && (r[0] == 0 ? h->rowdesc[8 * e + 1] : h->rowdesc[8 * e + 7]) == key)
      ++e;
    const int64_t L = e - a, nb = (L + 31) / 32;
    for (int64_t bi = 0; bi < nb; ++bi)
      for (int64_t bj = 0; bj <= bi; ++bj) {
        v.push_back(make_int4((int)a, (int)L, (int)bi, (int)bj));
        h->gblk_row.push_back(a + 32 * bi);
      }
    a = e;
  }
  int rc;
  if ((rc = ensure(h, (void**)&h->gblk, sizeof(int4) * std::max<size_t>(v.size(), 1), "Gaussian block list")))
    return rc;
  // (a synchronous copy would go through the legacy default stream, which a
  // non-blocking stream does not wait for; the pageable source is staged
  // before the call returns, so v may go)
  if (!v.empty())
    WL_CHECK(h, cudaMemcpyAsync(h->gblk, v.data(), sizeof(int4) * v.size(), cudaMemcpyHostToDevice, s));
  return COV_OK;
}

// The 32 x 32 lower blocks whose two row blocks share an ell bin, in row-block
// order, packed as (ti << 16) | tj, with the index of each row block's first
// listed block on the host: the only blocks where the BB+PT and PB products
// can be non-zero.  Built once per handle from the row table (the bins of each
// row block as k_block_masks forms them) and uploaded on the stream of the
// kernel that reads it.  Layouts with more than 64 ell bins or 65536 row
// blocks keep the full grid.
static int product_blocks(cov_handle* h, cudaStream_t s) {
  if (h->plist || h->plist_off) return COV_OK;
  const int64_t M = h->M, nb = (M + 31) / 32;
  if (h->nl > 64 || nb > 65536) {
    h->plist_off = true;
    return COV_OK;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  WL_CHECK(h, cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return wl_fail(h, COV_ERR_INVALID, "product-term block list not built before stream capture");
  std::vector<uint64_t> bm((size_t)nb, 0);
  for (int64_t a = 0; a < M; ++a) {
    const int32_t* r = &h->rowdesc[8 * a];
    uint64_t m = 1ull << r[1];
    if (r[0] == 1) m |= (1ull << r[2]) | (1ull << r[3]);
    bm[(size_t)(a / 32)] |= m;
  }
  std::vector<uint32_t> v;
  h->plist_start.assign((size_t)nb + 1, 0);
  for (int64_t ti = 0; ti < nb; ++ti) {
    h->plist_start[(size_t)ti] = (int64_t)v.size();
    for (int64_t tj = 0; tj <= ti; ++tj)
      if (bm[(size_t)ti] & bm[(size_t)tj]) v.push_back((uint32_t)((ti << 16) | tj));
  }
  h->plist_start[(size_t)nb] = (int64_t)v.size();
  int rc;
  if ((rc = ensure(h, (void**)&h->plist, sizeof(uint32_t) * std::max<size_t>(v.size(), 1), "product-term block list")))
    return rc;
  if (!v.empty())
    WL_CHECK(h, cudaMemcpyAsync(h->plist, v.data(), sizeof(uint32_t) * v.size(), cudaMemcpyHostToDevice, s));
  // the pageable source is staged before the call returns, so v may go
  return COV_OK;
}

// Gaussian terms of rows [r0, r1) (added; after the contraction and k_gather)
static int gauss(cov_handle* h, const GatherArgs& g, int64_t r0, int64_t r1, OutMap out, cudaStream_t s) {
  if (!(g.terms & COV_TERM_G) || r1 <= r0) return COV_OK;
  int rc;
  if ((rc = gauss_blocks(h, s))) return rc;
  const auto& st = h->gblk_row;
  const int64_t first = std::lower_bound(st.begin(), st.end(), r0 - 31) - st.begin();
  const int64_t last = std::lower_bound(st.begin(), st.end(), r1) - st.begin();
  if (last <= first) return COV_OK;
  k_gauss<<<(unsigned)(last - first), 256, 0, s>>>(g, h->gblk + first, r0, r1, out);
  WL_LAUNCH(h, "k_gauss");
  return COV_OK;
}

// The 1-halo trispectrum table T = R R^T of the PT term (Eq. CovBB): FP64
// rows and an FP64 product, or BF16 hi/lo rows built straight from the bin
// pair signatures and the tensor-core contraction.
static int build_ttable(cov_handle* h, int precision, cudaStream_t s) {
  int rc;
  const int64_t K = h->K;
  if ((rc = ensure(h, (void**)&h->Tmat, sizeof(double) * h->ntrow * h->ntrow, "trispectrum table"))) return rc;
  if (precision == COV_FP64) {
    if ((rc = ensure(h, (void**)&h->Trows, sizeof(double) * h->ntrow * K, "trispectrum rows"))) return rc;
    int tk = wl_stage_begin(h, ST_ROWS_T, s);
    if ((rc = wl_rows_t(h, s))) return rc;
    wl_stage_end(h, tk, s);
    tk = wl_stage_begin(h, ST_SYRK_T, s);
    if ((rc = wl_gemm_lower_fp64(h, h->Trows, K, h->Trows, K, h->Tmat, h->ntrow, h->ntrow, K, 1.0, 0.0, true, s)))
      return rc;
    wl_stage_end(h, tk, s);
    return COV_OK;
  }
  size_t sb = 0;
  wl_split_bytes(h->ntrow, (int)K, &sb);
  if ((rc = ensure(h, (void**)&h->Thi, sb, "BF16 hi trispectrum rows"))) return rc;
  if ((rc = ensure(h, (void**)&h->Tlo, sb, "BF16 lo trispectrum rows"))) return rc;
  if ((rc = ensure(h, (void**)&h->Tscale, sizeof(double) * h->ntrow, "trispectrum row scales"))) return rc;
  int tk = wl_stage_begin(h, ST_ROWS_T, s);
  if ((rc = wl_trows_split(h, s))) return rc;
  wl_stage_end(h, tk, s);
  tk = wl_stage_begin(h, ST_SYRK_T, s);
  if ((rc = wl_syrk_tc_rows(h, h->Thi, h->Tlo, h->Tscale, h->ntrow, wl_kpad((int)K), out_rows(h->Tmat, h->ntrow),
                            s)))
    return rc;
  wl_stage_end(h, tk, s);
  return COV_OK;
}

int wl_assemble(cov_handle* h, double* C, int64_t ldc, unsigned terms, int precision, cudaStream_t s) {
  int rc;
  const int64_t M = h->M, K = h->K;
  bool ssc_merged = false;
  // 1. the 1-halo trispectrum table of the PT term
  if (terms & COV_TERM_BBPT)
    if ((rc = build_ttable(h, precision, s))) return rc;
  // 2. 1-halo (chi, M) contraction: the first writer of the lower triangle
  if (terms & COV_TERM_1H) {
    if (precision == COV_FP64) {
      if ((rc = ensure(h, (void**)&h->A, sizeof(double) * M * K, "FP64 factor rows"))) return rc;
      int tk = wl_stage_begin(h, ST_ROWS_A, s);
      if ((rc = wl_rows_a(h, s))) return rc;
      wl_stage_end(h, tk, s);
      tk = wl_stage_begin(h, ST_SYRK_1H, s);
      if ((rc = wl_gemm_lower_fp64(h, h->A, K, h->A, K, C, ldc, M, K, 1.0, 0.0, true, s))) return rc;
      wl_stage_end(h, tk, s);
    } else {
      // the super-sample rows ride along as N_chi extra columns: one
      // contraction gives A A^T + S S^T
      ssc_merged = (terms & COV_TERM_SSC) != 0;
      int nssc = ssc_merged ? h->nchi : 0;
      size_t sb = 0;
      wl_split_bytes(M, (int)K + h->nchi, &sb);
      if ((rc = ensure(h, (void**)&h->Ahi, sb, "BF16 hi rows"))) return rc;
      if ((rc = ensure(h, (void**)&h->Alo, sb, "BF16 lo rows"))) return rc;
      if ((rc = ensure(h, (void**)&h->Ascale, sizeof(double) * M, "row scales"))) return rc;
      if ((rc = ensure(h, (void**)&h->tc_status, sizeof(int), "status word"))) return rc;
      if ((rc = ensure(h, (void**)&h->G2, sizeof(double) * K, "row factor table"))) return rc;
      if ((rc = ensure(h, (void**)&h->G3, sizeof(double) * K, "row factor table"))) return rc;
      if ((rc = ensure(h, (void**)&h->C2, sizeof(double) * h->nchi, "row factor table"))) return rc;
      if ((rc = ensure(h, (void**)&h->C3, sizeof(double) * h->nchi, "row factor table"))) return rc;
      int tk = wl_stage_begin(h, ST_ROWS_A, s);
      if ((rc = wl_rows_split(h, nssc, s))) return rc;
      wl_stage_end(h, tk, s);
      tk = wl_stage_begin(h, ST_SYRK_1H, s);
      if ((rc = wl_syrk_tc(h, nssc, out_rows(C, ldc), s))) return rc;
      wl_stage_end(h, tk, s);
    }
  }
  // per-element product terms: initialise C when no 1-halo term ran
  GatherArgs g;
  if ((rc = gather_args(h, terms, &g, s))) return rc;
  int64_t nt32 = (M + 31) / 32;
  int tg = wl_stage_begin(h, ST_GATHER, s);
  k_gather<<<(unsigned)(nt32 * (nt32 + 1) / 2), dim3(32, 8), 0, s>>>(g, M, out_rows(C, ldc),
                                                                  (terms & COV_TERM_1H) ? 1 : 0, 0);
  WL_LAUNCH(h, "k_gather");
  if ((rc = gauss(h, g, 0, M, out_rows(C, ldc), s))) return rc;
  wl_stage_end(h, tg, s);
  // 3. super-sample term, rank N_chi (already inside the split contraction)
  if ((terms & COV_TERM_SSC) && !ssc_merged) {
    if ((rc = ensure(h, (void**)&h->Srows, sizeof(double) * M * h->nchi, "SSC rows"))) return rc;
    int tk = wl_stage_begin(h, ST_ROWS_S, s);
    if ((rc = wl_rows_s(h, s))) return rc;
    wl_stage_end(h, tk, s);
    tk = wl_stage_begin(h, ST_SYRK_SSC, s);
    if ((rc = wl_gemm_lower_fp64(h, h->Srows, h->nchi, h->Srows, h->nchi, C, ldc, M, h->nchi, 1.0, 1.0, true, s)))
      return rc;
    wl_stage_end(h, tk, s);
  }
  return COV_OK;
}

// ---- band assembly -------------------------------------------------------------
// The operands (factor rows, trispectrum table) are built once per spectra and
// precision; each band then runs the contraction and the gather over its tile
// rows only.
static int prepare_operands(cov_handle* h, unsigned terms, int precision, cudaStream_t s) {
  int rc;
  const int64_t M = h->M, K = h->K;
  if (terms & COV_TERM_BBPT)
    if ((rc = build_ttable(h, precision, s))) return rc;
  if (precision == COV_FP64) {
    if (terms & COV_TERM_1H) {
      if ((rc = ensure(h, (void**)&h->A, sizeof(double) * M * K, "FP64 factor rows"))) return rc;
      int tk = wl_stage_begin(h, ST_ROWS_A, s);
      if ((rc = wl_rows_a(h, s))) return rc;
      wl_stage_end(h, tk, s);
    }
    if (terms & COV_TERM_SSC) {
      if ((rc = ensure(h, (void**)&h->Srows, sizeof(double) * M * h->nchi, "SSC rows"))) return rc;
      int tk = wl_stage_begin(h, ST_ROWS_S, s);
      if ((rc = wl_rows_s(h, s))) return rc;
      wl_stage_end(h, tk, s);
    }
  } else if (terms & COV_TERM_1H) {
    int nssc = (terms & COV_TERM_SSC) ? h->nchi : 0;
    size_t sb = 0;
    wl_split_bytes(M, (int)K + h->nchi, &sb);
    if ((rc = ensure(h, (void**)&h->Ahi, sb, "BF16 hi rows"))) return rc;
    if ((rc = ensure(h, (void**)&h->Alo, sb, "BF16 lo rows"))) return rc;
    if ((rc = ensure(h, (void**)&h->Ascale, sizeof(double) * M, "row scales"))) return rc;
    if ((rc = ensure(h, (void**)&h->tc_status, sizeof(int), "status word"))) return rc;
    if ((rc = ensure(h, (void**)&h->G2, sizeof(double) * K, "row factor table"))) return rc;
    if ((rc = ensure(h, (void**)&h->G3, sizeof(double) * K, "row factor table"))) return rc;
    if ((rc = ensure(h, (void**)&h->C2, sizeof(double) * h->nchi, "row factor table"))) return rc;
    if ((rc = ensure(h, (void**)&h->C3, sizeof(double) * h->nchi, "row factor table"))) return rc;
    int tk = wl_stage_begin(h, ST_ROWS_A, s);
    if ((rc = wl_rows_split(h, nssc, s))) return rc;
    wl_stage_end(h, tk, s);
  }
  return COV_OK;
}

// Band assembly.  In the split form the band is cut into sub-bands of about
// equal tile counts; the contraction of sub-band k+1 (main stream) runs while
// the per-element products of sub-band k (side stream) are added, so the
// gather's FP64 work and read-modify-write traffic hide under the tensor-core
// kernel, which leaves most of each SM's issue slots and HBM bandwidth free.
int wl_assemble_band(cov_handle* h, int64_t row0, int64_t nrows, OutMap out, unsigned terms, int precision,
                     cudaStream_t s) {
  int rc;
  if (h->ops_terms != (int)terms || h->ops_precision != precision) {
    if ((rc = prepare_operands(h, terms, precision, s))) return rc;
    h->ops_terms = (int)terms;
    h->ops_precision = precision;
  }
  const int64_t row1 = row0 + nrows;
  GatherArgs g;
  if ((rc = gather_args(h, terms, &g, s))) return rc;
  const int acc = (terms & COV_TERM_1H) ? 1 : 0;
  if (acc && (terms & (COV_TERM_BBPT | COV_TERM_PB)))
    if ((rc = product_blocks(h, s))) return rc;
  auto gather = [&](int64_t r0, int64_t r1, cudaStream_t st) {
    int64_t t0 = r0 / 32, t1 = (r1 + 31) / 32;
    if (acc && h->plist) {
      const int64_t first = h->plist_start[(size_t)t0], last = h->plist_start[(size_t)t1];
      if (last > first) k_gather_list<<<(unsigned)(last - first), dim3(32, 8), 0, st>>>(g, r1, out, h->plist + first);
      return;
    }
    int64_t off = t0 * (t0 + 1) / 2;
    k_gather<<<(unsigned)(t1 * (t1 + 1) / 2 - off), dim3(32, 8), 0, st>>>(g, r1, out, acc, off);
  };
  if (precision != COV_FP64 && (terms & COV_TERM_1H)) {
    const int nssc = (terms & COV_TERM_SSC) ? h->nchi : 0;
    if ((rc = wl_side_stream(h))) return rc;
    // sub-band cuts at tile rows, about equal numbers of tiles each
    const int64_t ta = row0 / 256, tb = (row1 + 255) / 256;
    const int nsub = (int)std::min<int64_t>(8, tb - ta);
    std::vector<int64_t> cut{row0};
    const double tot = 0.5 * (double)(tb * (tb + 1) - ta * (ta + 1));
    for (int k = 1; k < nsub; ++k) {
      double want = 0.5 * (double)(ta * (ta + 1)) + tot * k / nsub;
      int64_t t = (int64_t)std::floor(std::sqrt(2.0 * want));
      int64_t r = std::min(t * 256, row1);
      if (r > cut.back()) cut.push_back(r);
    }
    if (cut.back() != row1) cut.push_back(row1);
    if ((rc = wl_tc_status_reset(h, s))) return rc;
    WL_CHECK(h, cudaEventRecord(h->ev_panel, s));  // the side stream starts after the operands
    WL_CHECK(h, cudaStreamWaitEvent(h->side, h->ev_panel, 0));
    int tk = wl_stage_begin(h, ST_SYRK_1H, s);
    for (size_t k = 0; k + 1 < cut.size(); ++k) {
      if ((rc = wl_syrk_tc_part(h, nssc, out, cut[k], cut[k + 1], s))) return rc;
      WL_CHECK(h, cudaEventRecord(h->ev_cols, s));
      WL_CHECK(h, cudaStreamWaitEvent(h->side, h->ev_cols, 0));
      int tg = wl_stage_begin(h, ST_GATHER, h->side);
      gather(cut[k], cut[k + 1], h->side);
      WL_LAUNCH(h, "k_gather");
      if ((rc = gauss(h, g, cut[k], cut[k + 1], out, h->side))) return rc;
      wl_stage_end(h, tg, h->side);
    }
    wl_stage_end(h, tk, s);
    WL_CHECK(h, cudaEventRecord(h->ev_panel, h->side));
    WL_CHECK(h, cudaStreamWaitEvent(s, h->ev_panel, 0));
    return wl_tc_status_check(h, s);
  }
  // FP64 form, or no 1-halo term: contraction, products, super-sample term in turn
  if (terms & COV_TERM_1H) {
    int tk = wl_stage_begin(h, ST_SYRK_1H, s);
    if ((rc = gemm_lower_band(h, h->A, h->K, row1, h->K, 0.0, out, s))) return rc;
    wl_stage_end(h, tk, s);
  }
  int tg = wl_stage_begin(h, ST_GATHER, s);
  gather(row0, row1, s);
  WL_LAUNCH(h, "k_gather");
  if ((rc = gauss(h, g, row0, row1, out, s))) return rc;
  wl_stage_end(h, tg, s);
  if ((terms & COV_TERM_SSC) && (terms & COV_TERM_1H)) {
    int tk = wl_stage_begin(h, ST_SYRK_SSC, s);
    if ((rc = gemm_lower_band(h, h->Srows, h->nchi, row1, h->nchi, 1.0, out, s))) return rc;
    wl_stage_end(h, tk, s);
  }
  return COV_OK;
}
