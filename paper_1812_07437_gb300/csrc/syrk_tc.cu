// Tensor-core form of the 1-halo (chi, M) contraction (paper Eqs. CovPPNG,
// Ins5P, Ins6P recast as C_1h = A A^T with A the factor rows):
//
//   * k_rows_split builds each factor row in FP64, scales it by an exact power
//     of two s_a so that its largest entry lies in [0.5, 1), and splits it into
//     two BF16 rows, hi = bf16(a / s_a), lo = bf16(a / s_a - hi).
//   * k_syrk_tc computes, per 128 x 128 lower-triangle tile, the FP32 sum
//     hi_i hi_j + hi_i lo_j + lo_i hi_j over K on the tcgen05 tensor cores
//     (kind::f16, BF16 operands, FP32 accumulator in TMEM) and adds
//     acc * s_i * s_j into the FP64 covariance.
//
// Per CTA (128 threads): warp 0 / lane 0 issues TMA loads of the four
// 128 x 64 operand tiles of a K block (hi/lo rows of tile I and of tile J,
// 128B-swizzled) into a 3-stage shared-memory ring; warp 1 / lane 0 issues the
// 12 MMAs of 128 x 128 x 16 per K block and releases each stage with
// tcgen05.commit; after the last block all four warps read the accumulator
// from TMEM (tcgen05.ld 32x32b) and write the tile.  Every wait on an mbarrier
// is bounded: on expiry the kernel raises a status word, stops issuing work,
// waits (bounded) for its own copies, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"

#define TC_BM 128
#define TC_BN 128
#define TC_BK 64
#define TC_STAGES 3
#define TC_TILE_BYTES (TC_BM * TC_BK * 2)           // 16 KB per operand tile
#define TC_STAGE_BYTES (4 * TC_TILE_BYTES)          // hi_I, lo_I, hi_J, lo_J
#define TC_SMEM (TC_STAGES * TC_STAGE_BYTES + 1024) // + alignment slack
#define TC_SPIN_LIMIT (1u << 22)

// ---------------------------------------------------------------- row split
__global__ void k_rows_split(int64_t M, int nchi, int nm, int Kp, double inv_omega, double rho, const int32_t* rd,
                             const double* chi, const double* wchi, const double* W, const double* m,
                             const double* om, const double* f, const double* U, __nv_bfloat16* hi,
                             __nv_bfloat16* lo, double* rscale) {
  __shared__ double sh[32];
  int64_t a = blockIdx.x;
  if (a >= M) return;
  const int32_t* r = rd + 8 * a;
  int K = nchi * nm;
  int mu = (r[0] == 0) ? 2 : 3;
  auto value = [&](int kk) -> double {
    int n = kk / nm, q = kk % nm;
    double mr = m[q] / rho, ch = chi[n];
    double v = sqrt(wchi[n] * om[q] * f[kk] * inv_omega);
    v *= (mu == 2) ? 1.0 / (ch * ch * ch) : 1.0 / (ch * ch * ch * ch * ch);
    v *= (mu == 2) ? mr * mr : mr * mr * mr;
    v *= W[r[4] * nchi + n] * W[r[5] * nchi + n];
    v *= U[((size_t)r[1] * nchi + n) * nm + q] * U[((size_t)r[2] * nchi + n) * nm + q];
    if (mu == 3) v *= W[r[6] * nchi + n] * U[((size_t)r[3] * nchi + n) * nm + q];
    return v;
  };
  double mx = 0.0;
  for (int kk = threadIdx.x; kk < K; kk += blockDim.x) mx = fmax(mx, fabs(value(kk)));
  // block max via the sum helper's layout
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (threadIdx.x == 0) sh[0] = t;
  }
  __syncthreads();
  mx = sh[0];
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);
  double inv = ldexp(1.0, -ex);
  for (int kk = threadIdx.x; kk < Kp; kk += blockDim.x) {
    double x = (kk < K) ? value(kk) * inv : 0.0;
    __nv_bfloat16 h = __float2bfloat16_rn((float)x);
    __nv_bfloat16 l = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
    hi[a * Kp + kk] = h;
    lo[a * Kp + kk] = l;
  }
  if (threadIdx.x == 0) rscale[a] = ldexp(1.0, ex);
}

// split already-built FP64 rows X[rows][K] into scaled BF16 hi/lo rows [rows][Kp]
__global__ void k_split_rows(const double* X, int64_t rows, int K, int Kp, __nv_bfloat16* hi, __nv_bfloat16* lo,
                             double* rscale) {
  __shared__ double sh[32];
  int64_t a = blockIdx.x;
  if (a >= rows) return;
  const double* x = X + a * K;
  double mx = 0.0;
  for (int kk = threadIdx.x; kk < K; kk += blockDim.x) mx = fmax(mx, fabs(x[kk]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (threadIdx.x == 0) sh[0] = t;
  }
  __syncthreads();
  mx = sh[0];
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);
  double inv = ldexp(1.0, -ex);
  for (int kk = threadIdx.x; kk < Kp; kk += blockDim.x) {
    double v = (kk < K) ? x[kk] * inv : 0.0;
    __nv_bfloat16 h = __float2bfloat16_rn((float)v);
    __nv_bfloat16 l = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
    hi[a * Kp + kk] = h;
    lo[a * Kp + kk] = l;
  }
  if (threadIdx.x == 0) rscale[a] = ldexp(1.0, ex);
}

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ uint32_t mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok;
}

// bounded wait; false when the limit expired or another role raised the status
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status) {
  for (uint32_t i = 0; i < TC_SPIN_LIMIT; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 1023u) == 1023u && *abort_flag) return false;
  }
  *abort_flag = 1;
  atomicExch(status, 1);
  return false;
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);        // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                        // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                        // SWIZZLE_128B
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// instruction descriptor: kind::f16, BF16 x BF16 -> FP32, both K-major, M = 128, N = 128
__device__ __forceinline__ uint32_t idesc_bf16_128x128() {
  uint32_t d = 0;
  d |= 1u << 4;                 // D format FP32
  d |= 1u << 7;                 // A format BF16
  d |= 1u << 10;                // B format BF16
  d |= (uint32_t)(TC_BN >> 3) << 17;
  d |= (uint32_t)(TC_BM >> 4) << 24;
  return d;
}

__device__ __forceinline__ void tri_tile_tc(int64_t id, int64_t* ti, int64_t* tj) {
  int64_t i = (int64_t)((sqrt(8.0 * (double)id + 1.0) - 1.0) * 0.5);
  while (i * (i + 1) / 2 > id) --i;
  while ((i + 1) * (i + 2) / 2 <= id) ++i;
  *ti = i;
  *tj = id - i * (i + 1) / 2;
}

__global__ void __launch_bounds__(128, 1)
    k_syrk_tc(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo, int64_t M,
              int nk, const double* __restrict__ rscale, double* C, int64_t ldc, int* status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[TC_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[TC_STAGES];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;

  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t ti, tj;
  tri_tile_tc(blockIdx.x, &ti, &tj);
  int row_i = (int)(ti * TC_BM), row_j = (int)(tj * TC_BN);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&acc_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(TC_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  uint32_t tmem = tmem_base_sh;

  if (warp == 0 && lane == 0) {
    // TMA producer
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      int s = kb % TC_STAGES;
      uint32_t ph = (uint32_t)(kb / TC_STAGES) & 1u;
      if (!mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag, status)) break;
      issued = kb + 1;
      uint8_t* st = smem + (size_t)s * TC_STAGE_BYTES;
      mbar_expect_tx(&full_bar[s], TC_STAGE_BYTES);
      int kc = kb * TC_BK;
      tma_load_2d(&map_hi, &full_bar[s], st + 0 * TC_TILE_BYTES, kc, row_i);
      tma_load_2d(&map_lo, &full_bar[s], st + 1 * TC_TILE_BYTES, kc, row_i);
      tma_load_2d(&map_hi, &full_bar[s], st + 2 * TC_TILE_BYTES, kc, row_j);
      tma_load_2d(&map_lo, &full_bar[s], st + 3 * TC_TILE_BYTES, kc, row_j);
    }
    if (abort_flag) {
      // drain: wait (bounded) until the copies of the last ring of stages have landed
      for (int kb = issued - TC_STAGES < 0 ? 0 : issued - TC_STAGES; kb < issued; ++kb) {
        uint32_t ph = (uint32_t)(kb / TC_STAGES) & 1u;
        for (uint32_t i = 0; i < TC_SPIN_LIMIT && !mbar_try(&full_bar[kb % TC_STAGES], ph); ++i) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = idesc_bf16_128x128();
    bool ok = true;
    for (int kb = 0; kb < nk && ok; ++kb) {
      int s = kb % TC_STAGES;
      uint32_t ph = (uint32_t)(kb / TC_STAGES) & 1u;
      if (!mbar_wait(&full_bar[s], ph, &abort_flag, status)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t st = smem_u32(smem + (size_t)s * TC_STAGE_BYTES);
      uint32_t a_hi = st, a_lo = st + TC_TILE_BYTES, b_hi = st + 2 * TC_TILE_BYTES, b_lo = st + 3 * TC_TILE_BYTES;
#pragma unroll
      for (int k = 0; k < TC_BK / 16; ++k) {
        uint32_t off = k * 32;  // 16 BF16 along K inside the 128-byte swizzle row
        uint32_t first = (kb == 0 && k == 0) ? 0u : 1u;
        umma_bf16(tmem, umma_desc_sw128(a_hi + off), umma_desc_sw128(b_hi + off), idesc, first);
        umma_bf16(tmem, umma_desc_sw128(a_hi + off), umma_desc_sw128(b_lo + off), idesc, 1u);
        umma_bf16(tmem, umma_desc_sw128(a_lo + off), umma_desc_sw128(b_hi + off), idesc, 1u);
      }
      umma_commit(&empty_bar[s]);
    }
    umma_commit(&acc_bar);
  }
  __syncwarp();
  // epilogue: all four warps (warp w owns TMEM lanes 32w .. 32w+31)
  bool have = mbar_wait(&acc_bar, 0u, &abort_flag, status);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (have && !abort_flag) {
    int64_t gi = (int64_t)row_i + warp * 32 + lane;
    double si = (gi < M) ? rscale[gi] : 0.0;
#pragma unroll 1
    for (int c = 0; c < TC_BN / 32; ++c) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
      if (gi < M) {
        double* crow = C + gi * ldc;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          int64_t gj = (int64_t)row_j + c * 32 + jj;
          if (gj < M && gj <= gi) crow[gj] += (double)v[jj] * si * rscale[gj];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN));
  }
}

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

static int make_map(cov_handle* h, CUtensorMap* map, void* base, int64_t rows, int64_t kp) {
  auto fn = encode_fn();
  if (!fn) return wl_fail(h, COV_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
  cuuint32_t box[2] = {TC_BK, TC_BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return wl_fail(h, COV_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return COV_OK;
}

static inline int kpad(int K) { return (K + TC_BK - 1) / TC_BK * TC_BK; }

int wl_split_bytes(int64_t M, int K, size_t* bytes) {
  *bytes = (size_t)M * kpad(K) * 2;
  return COV_OK;
}

int wl_rows_split(cov_handle* h, cudaStream_t s) {
  double rho = WL_RHO_CRIT0 * h->cosmo.Om;
  k_rows_split<<<(unsigned)h->M, 256, 0, s>>>(h->M, h->nchi, h->nm, kpad(h->K), 1.0 / h->omega, rho, h->rowdesc_d,
                                               h->chi, h->wchi, h->W, h->m, h->om, h->f, h->U,
                                               (__nv_bfloat16*)h->Ahi, (__nv_bfloat16*)h->Alo, (double*)h->Ascale);
  WL_LAUNCH(h, "k_rows_split");
  return COV_OK;
}

// C (lower, FP64) += (hi + lo)(hi + lo)^T scaled, without the lo lo^T term
int wl_syrk_tc_rows(cov_handle* h, const void* hi, const void* lo, const double* rscale, int64_t rows, int Kp,
                    double* C, int64_t ldc, cudaStream_t s) {
  CUtensorMap mhi, mlo;
  int rc;
  if ((rc = make_map(h, &mhi, (void*)hi, rows, Kp))) return rc;
  if ((rc = make_map(h, &mlo, (void*)lo, rows, Kp))) return rc;
  static bool attr = false;
  if (!attr) {
    WL_CHECK(h, cudaFuncSetAttribute(k_syrk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    attr = true;
  }
  if (!h->tc_status) WL_CHECK(h, cudaMalloc(&h->tc_status, sizeof(int)));
  int64_t nt = (rows + TC_BM - 1) / TC_BM;
  int64_t nblk = nt * (nt + 1) / 2;
  WL_CHECK(h, cudaMemsetAsync(h->tc_status, 0, sizeof(int), s));
  k_syrk_tc<<<(unsigned)nblk, 128, TC_SMEM, s>>>(mhi, mlo, rows, Kp / TC_BK, rscale, C, ldc, h->tc_status);
  WL_LAUNCH(h, "k_syrk_tc");
  int st = 0;
  WL_CHECK(h, cudaMemcpyAsync(&st, h->tc_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  WL_CHECK(h, cudaStreamSynchronize(s));
  if (st) return wl_fail(h, COV_ERR_TIMEOUT, "tensor-core contraction: a bounded mbarrier wait expired");
  return COV_OK;
}

int wl_syrk_tc(cov_handle* h, double* C, int64_t ldc, cudaStream_t s) {
  return wl_syrk_tc_rows(h, h->Ahi, h->Alo, h->Ascale, h->M, kpad(h->K), C, ldc, s);
}

int wl_split_rows(cov_handle* h, const double* X, int64_t rows, int K, void* hi, void* lo, double* rscale,
                  cudaStream_t s) {
  k_split_rows<<<(unsigned)rows, 256, 0, s>>>(X, rows, K, kpad(K), (__nv_bfloat16*)hi, (__nv_bfloat16*)lo, rscale);
  WL_LAUNCH(h, "k_split_rows");
  return COV_OK;
}
