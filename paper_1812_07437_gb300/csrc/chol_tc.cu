// FP64-accurate trailing update of the blocked Cholesky on the tcgen05 tensor
// cores (the S/N solve of the paper's Sec. 5, Eq. eq:SN), by exact integer
// slicing in the manner of Ozaki, Ogita & Oishi (2012):
//
//   * k_chol_slice: every panel row x (kb <= 64 FP64 entries) is scaled by an
//     exact power of two 2^-e (e from its largest entry) and cut into
//     S = 6 fixed-point slices, x 2^-e = sum_t d_t 2^(-7-8t), d_t integers in
//     [-128, 128] stored exactly as BF16; the residual is below 2^-48 of the row
//     maximum.  The digits are the balanced base-256 digits of the integer
//     X = RN(x 2^(47 - e)), taken by integer operations from the bits of x.
//   * k_chol_update: per 128 x 64 lower tile of the trailing matrix, the
//     products d_t(i) . d_u(j) over the panel's K = 64 are exact in FP32
//     (|d d| <= 2^14, 64 terms -> 2^20), and so are their sums over the pairs
//     with equal t + u = g (at most 6 pairs -> < 2^23).  21 pairs (t + u <= 5) x
//     4 K steps of tcgen05.mma (kind::f16, M = 128, N = 64) accumulate into six
//     TMEM accumulators, one per g; the epilogue recombines them exactly in
//     int64, v = 2^(e_i + e_j - 54) sum_g acc_g 2^(8 (5 - g)), converts once to
//     FP64 and subtracts v from the FP64 trailing matrix (coalesced stores; the
//     tile was copied to shared memory during the MMAs).
//
// One CTA (128 threads) per lower tile (no blocks for tiles above the
// diagonal): warp 0 / lane 0 loads the 6 I-slices
// (128 x 64) and 6 J-slices (64 x 64) with TMA (128B swizzle) in one stage,
// warp 1 / lane 0 issues the MMAs, all four warps run the epilogue.  Waits are
// bounded (status word, COV_ERR_TIMEOUT).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"

#define CS_S 6                                   // slices per entry
#define CS_BI 128                                // tile rows
#define CS_BJ 64                                 // tile columns
#define CS_K 64                                  // panel width
#define CS_IBYTES (CS_BI * CS_K * 2)             // 16 KB per I slice tile
#define CS_JBYTES (CS_BJ * CS_K * 2)             // 8 KB per J slice tile
#define CS_STAGE (CS_S * (CS_IBYTES + CS_JBYTES))  // 144 KB
#define CS_CTILE (CS_BI * CS_BJ * 8)             // 64 KB FP64 trailing tile
#define CS_SMEM (CS_STAGE + CS_CTILE + 1024)
#define CS_SPIN (1u << 22)

// X = RN(x 2^(47 - e)) (ties to even) for |x| < 2^e, by integer operations on
// the bits of x (x = m 2^(E' - 1075), m the 53-bit significand): |X| <= 2^47.
// The FP64 pipe of this part is narrow, and any exact digit scheme of the
// same X gives the same slices' value.
__device__ __forceinline__ long long slice_int(double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FFu);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
  const int sh = 1028 + e - (E ? E : 1);  // X = RN(m / 2^sh); sh >= 6 unless the row holds only subnormals
  unsigned long long q;
  if (sh <= 0) {
    q = m << (-sh < 63 ? -sh : 63);
  } else if (sh >= 64) {
    q = 0;
  } else {
    q = m >> sh;
    const unsigned long long rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
  }
  return (b >> 63) ? -(long long)q : (long long)q;
}

// BF16 bits of an integer |d| <= 255 (exact: at most 8 significant bits)
__device__ __forceinline__ unsigned short bf16_bits_of_int(int d) {
  if (d == 0) return 0;
  const unsigned a = (unsigned)(d < 0 ? -d : d);
  const int p = 31 - __clz((int)a);  // leading bit
  const unsigned bits = ((unsigned)(127 + p) << 7) | ((a << (7 - p)) & 0x7Fu);
  return (unsigned short)(bits | (d < 0 ? 0x8000u : 0u));
}

// the six balanced base-256 digits of X (d_0 most significant): d_1..d_5 in
// [-128, 127], d_0 in [-128, 128] since |X| <= 2^47; written as BF16 to
// out + t * stride
__device__ __forceinline__ void slice_store(long long X, __nv_bfloat16* out, size_t stride) {
#pragma unroll
  for (int t = CS_S - 1; t >= 1; --t) {
    int lo = (int)(X & 255);
    lo = lo >= 128 ? lo - 256 : lo;
    X = (X - lo) >> 8;
    out[(size_t)t * stride] = __ushort_as_bfloat16(bf16_bits_of_int(lo));
  }
  out[0] = __ushort_as_bfloat16(bf16_bits_of_int((int)X));
}

// slices of the panel rows r0..r1-1 (columns k0..k0+kb-1 of the workspace);
// rows up to the padded count are written (zeros past r1)
__global__ void k_chol_slice(const OutMap W, int64_t k0, int kb, int64_t r0, int64_t nrows, int64_t nrows_pad,
                             __nv_bfloat16* slices, int* rexp) {
  int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (r >= nrows_pad) return;
  double x0 = 0.0, x1 = 0.0;
  if (r < nrows) {
    const double* row = W.at(r0 + r, k0);
    if (lane < kb) x0 = row[lane];
    if (lane + 32 < kb) x1 = row[lane + 32];
  }
  double mx = fmax(fabs(x0), fabs(x1));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);
  const size_t stride = (size_t)nrows_pad * CS_K;
  __nv_bfloat16* out = slices + (size_t)r * CS_K;
  slice_store(slice_int(x0, e), out + lane, stride);
  slice_store(slice_int(x1, e), out + lane + 32, stride);
  if (lane == 0) rexp[r] = e;
}

__device__ __forceinline__ uint32_t cs_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t cs_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(cs_smem_u32(bar)), "r"(parity)
      : "memory");
  return ok;
}

__device__ __forceinline__ bool cs_wait(uint64_t* bar, uint32_t parity, int* status) {
  for (uint32_t i = 0; i < CS_SPIN; ++i)
    if (cs_try(bar, parity)) return true;
  atomicExch(status, 1);
  return false;
}

__device__ __forceinline__ uint64_t cs_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;  // 8 rows x 128 B
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;  // SWIZZLE_128B
  return d;
}

// 32 lanes x 8 columns of TMEM into registers; the caller issues
// tcgen05.wait::ld before using them
__device__ __forceinline__ void cs_tmem_ld8_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

// 32 lanes x 16 columns of TMEM into registers; the caller issues
// tcgen05.wait::ld before using them
__device__ __forceinline__ void cs_tmem_ld16_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// The integer held exactly by an FP32 value of magnitude below 2^24 (its
// bits b), by integer operations: the conversion instruction goes through a
// narrow unit on this part and dominated the epilogue.
__device__ __forceinline__ int exact_f2i(uint32_t b) {
  const int e = (int)((b >> 23) & 0xFFu);
  const uint32_t m = (b & 0x7FFFFFu) | 0x800000u;
  const int v = e < 127 ? 0 : (int)(m >> (150 - e));
  return (b >> 31) ? -v : v;
}

// RN(a) 2^ex as an FP64 value, for |a| < 2^63, by integer operations: the
// leading bit sets the exponent, the 53 leading bits (rounded to nearest,
// ties to even, as the FP64 conversion rounds) the significand.  Results
// outside the normal range take the FP64 path.
__device__ __forceinline__ double scaled_to_double(long long a, int ex) {
  if (a == 0) return 0.0;
  unsigned long long sign = a < 0 ? (1ull << 63) : 0ull;
  unsigned long long u = a < 0 ? (unsigned long long)(-a) : (unsigned long long)a;
  int msb = 63 - __clzll((long long)u);
  unsigned long long m;
  if (msb <= 52) {
    m = u << (52 - msb);
  } else {
    int sh = msb - 52;
    m = u >> sh;
    unsigned long long rem = u & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) ++m;
    if (m >> 53) {
      m >>= 1;
      ++msb;
    }
  }
  int e = msb + ex + 1023;
  if (e <= 0 || e >= 2047) return ldexp((double)a, ex);
  return __longlong_as_double((long long)(sign | ((unsigned long long)e << 52) | (m & ((1ull << 52) - 1))));
}

// RN(a) 2^ex as an FP64 value for 0 < |a| < 2^63, without branches on the
// value: normalise |a| so that its leading bit is bit 63, keep the 53 leading
// bits rounded to nearest (ties to even), and add the rounded significand
// (2^52 <= r <= 2^53) to the biased exponent field, which carries a rounding
// overflow into the exponent by itself.  Results outside the normal range take
// the FP64 path.
__device__ __forceinline__ double scaled_to_double_rn(long long a, int ex) {
  if (a == 0) return 0.0;
  const unsigned long long sign = (unsigned long long)a & (1ull << 63);
  const unsigned long long u = a < 0 ? 0ull - (unsigned long long)a : (unsigned long long)a;
  const int lz = __clzll((long long)u);
  const unsigned long long mn = u << lz;
  const unsigned long long r0 = mn >> 11;
  const unsigned long long rb = (mn >> 10) & 1ull;
  const unsigned long long sticky = ((mn & 0x3FFull) != 0ull) | (r0 & 1ull);
  const unsigned long long r = r0 + (rb & sticky);
  const int e = (63 - lz) + ex + 1023;
  if (e <= 0 || e >= 2046) return ldexp((double)a, ex);
  return __longlong_as_double((long long)(sign | (((unsigned long long)(e - 1) << 52) + r)));
}

// Lower tiles of one update launch, row by row: tile row ti (128 rows, from
// ti0 = tj0 * 64 / 128) holds the column tiles tj0 .. min(tj0 + ntj - 1,
// 2 ti + 1) (64 columns each).  cum(ti) counts the tiles of rows ti0 .. ti-1.
struct TileRows {
  int tj0, ntj, ti0, nti;
  __host__ __device__ int64_t cnt(int64_t i) const {
    int64_t c = 2 * i + 2 - tj0;
    return c < ntj ? c : ntj;
  }
  __host__ __device__ int64_t cum(int64_t ti) const {
    // rows below i_star = ceil((ntj + tj0 - 2) / 2) grow by two tiles per row; the rest hold ntj
    int64_t istar = (ntj + tj0 - 2 + 1) / 2;
    if (istar < ti0) istar = ti0;
    int64_t b = ti < istar ? ti : istar, a = ti0;
    int64_t tri = b > a ? (b - a) * (2 - tj0) + (b * (b - 1) - a * (a - 1)) : 0;
    int64_t rect = ti > istar ? (ti - istar) * (int64_t)ntj : 0;
    return tri + rect;
  }
};

__global__ void __launch_bounds__(128, 1)
    k_chol_update(const __grid_constant__ CUtensorMap map_i, const __grid_constant__ CUtensorMap map_j,
                  int64_t nrows, int64_t nrows_pad, const int* __restrict__ rexp, OutMap W, int64_t r0, int* status,
                  TileRows tr) {
  // the launch holds only lower tiles: find the row of this block by bisection
  const int64_t id = blockIdx.x;
  int64_t lo = tr.ti0, hi = tr.ti0 + tr.nti;  // cum(lo) <= id < cum(hi)
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) >> 1;
    if (tr.cum(mid) <= id) lo = mid; else hi = mid;
  }
  const int ti = (int)lo;
  const int tj = tr.tj0 + (int)(id - tr.cum(lo));
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar;
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t tmem_sh;
  __shared__ int rexp_sh[CS_BI];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int row_i = ti * CS_BI, row_j = tj * CS_BJ;
  rexp_sh[threadIdx.x] = (row_i + (int)threadIdx.x < nrows) ? rexp[row_i + threadIdx.x] : 0;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cs_smem_u32(&full_bar)), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cs_smem_u32(&acc_bar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(cs_smem_u32(&tmem_sh)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  uint32_t tmem = tmem_sh;
  bool loaded = false;
  double* ctile = (double*)(smem + CS_STAGE);  // [128][64] FP64 copy of the trailing tile
  if (warp >= 2) {
    // warps 2-3 stream the FP64 tile into shared memory while the slices load
    // and the MMAs run: thread t copies column t down the 128 rows (8-byte
    // cp.async, coalesced across the threads), stepping its source address
    // by the row stride and recomputing it only where a new tile row begins
    const int t = threadIdx.x - 64;
    const int64_t gc = (int64_t)row_j + t, ac = r0 + gc;
    const int64_t stride = W.tiled ? 256 : W.ldc;
    const double* src = nullptr;
    for (int rr = 0; rr < CS_BI; ++rr) {
      const int64_t gr = (int64_t)row_i + rr, ar = r0 + gr;
      if (gr < nrows && gc < nrows && gc <= gr) {
        if (!src || (W.tiled && (ar & 255) == 0)) src = W.at(ar, ac);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(cs_smem_u32(ctile + rr * CS_BJ + t)), "l"(src)
                     : "memory");
      }
      if (src) src += stride;
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  } else if (warp == 0 && lane == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cs_smem_u32(&full_bar)),
                 "r"(CS_STAGE)
                 : "memory");
    for (int t = 0; t < CS_S; ++t) {
      int yi = (int)(t * nrows_pad + row_i), yj = (int)(t * nrows_pad + row_j);
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
          "[%2];" ::"r"(cs_smem_u32(smem + t * CS_IBYTES)),
          "l"((uint64_t)&map_i), "r"(cs_smem_u32(&full_bar)), "r"(0), "r"(yi)
          : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
          "[%2];" ::"r"(cs_smem_u32(smem + CS_S * CS_IBYTES + t * CS_JBYTES)),
          "l"((uint64_t)&map_j), "r"(cs_smem_u32(&full_bar)), "r"(0), "r"(yj)
          : "memory");
    }
  } else if (warp == 1 && lane == 0) {
    loaded = cs_wait(&full_bar, 0u, status);
    if (loaded) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // kind::f16, BF16 x BF16 -> FP32, K-major, M = 128, N = 64
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CS_BJ >> 3) << 17) |
                             ((uint32_t)(CS_BI >> 4) << 24);
      uint32_t base_i = cs_smem_u32(smem), base_j = cs_smem_u32(smem + CS_S * CS_IBYTES);
      // consecutive MMAs go to different accumulators (round r pairs slice
      // t = r with u = g - r for g = r .. 5), so no MMA waits on the one
      // before it; the first round of the first K step initialises all six
#pragma unroll 1
      for (int k = 0; k < CS_K / 16; ++k)
#pragma unroll
        for (int r = 0; r < CS_S; ++r)
#pragma unroll
          for (int g = r; g < CS_S; ++g) {
            uint32_t dt = tmem + (uint32_t)(g * CS_BJ);
            uint64_t ad = cs_desc_sw128(base_i + r * CS_IBYTES + k * 32);
            uint64_t bd = cs_desc_sw128(base_j + (g - r) * CS_JBYTES + k * 32);
            uint32_t acc = (k == 0 && r == 0) ? 0u : 1u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, "
                "p;\n}\n" ::"r"(dt),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
          }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     cs_smem_u32(&acc_bar))
                 : "memory");
  }
  __syncwarp();
  bool have = cs_wait(&acc_bar, 0u, status);
  if (warp == 0 && lane == 0) {
    // the copies must have landed before the CTA exits (bounded)
    for (uint32_t i = 0; i < CS_SPIN && !cs_try(&full_bar, 0u); ++i) {
    }
  }
  if (warp >= 2) asm volatile("cp.async.wait_all;" ::: "memory");
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (have && *(volatile int*)status == 0) {
    // 16 columns at a time: each thread first owns one row (TMEM lane) and
    // combines the six exact group sums a_g (|a_g| < 2^23) into
    // v = sum_g a_g 2^(8 (5 - g)) = ((p0 2^16) + p1) 2^16 + p2 with the int32
    // pairs p = a_(2k) 2^8 + a_(2k+1) (|p| < 2^31); the values are then
    // staged so that each thread owns one column and 16 consecutive rows for
    // the coalesced read-modify-write of the FP64 tile.
    long long* stg = (long long*)smem + warp * (32 * 17);
    const int jc = lane & 15, rh = lane >> 4;
    const int64_t stride = W.tiled ? 256 : W.ldc;
#pragma unroll 1
    for (int c = 0; c < CS_BJ / 16; ++c) {
      // all six TMEM loads in flight before one wait: the load latency is paid
      // once per chunk instead of once per group
      uint32_t r[CS_S][16];
#pragma unroll
      for (int g = 0; g < CS_S; ++g)
        cs_tmem_ld16_nowait(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * CS_BJ + c * 16), r[g]);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int g = 0; g < CS_S; ++g)
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) asm volatile("" : "+r"(r[g][jj]));  // uses stay after the wait
      long long acc[16];
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        long long a = 0;
#pragma unroll
        for (int k = 0; k < CS_S; k += 2)
          a = a * 65536 + (long long)(exact_f2i(r[k][jj]) * 256 + exact_f2i(r[k + 1][jj]));
        acc[jj] = a;
      }
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) stg[lane * 17 + jj] = acc[jj];
      __syncwarp();
      // value = acc 2^(e_i + e_j - 14 - 8 (S - 1)); this thread: column jc,
      // rows 16 rh .. 16 rh + 15 of the warp's 32.  The 16 rows never cross a
      // 256-row tile row, so one base address serves them all, and the 16
      // values are independent (all in flight before the stores).
      const int64_t gj = (int64_t)row_j + c * 16 + jc, aj = r0 + gj;
      const int ej = (gj < nrows) ? rexp[gj] : 0;
      const int lr0 = warp * 32 + rh * 16;
      const int64_t gr0 = (int64_t)row_i + lr0, ar0 = r0 + gr0;
      if (gj < nrows && gr0 + 15 >= gj && (!W.tiled || (aj >> 8) <= (ar0 >> 8))) {
        double* base = W.at(ar0, aj);
        double nv[16];
#pragma unroll
        for (int k = 0; k < 16; ++k)
          nv[k] = ctile[(lr0 + k) * CS_BJ + c * 16 + jc] -
                  scaled_to_double(stg[(rh * 16 + k) * 17 + jc], rexp_sh[lr0 + k] + ej - 54);
#pragma unroll
        for (int k = 0; k < 16; ++k)
          if (gr0 + k < nrows && gj <= gr0 + k) base[k * stride] = nv[k];
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------------- persistent update
// The same exact-slicing update as k_chol_update, restructured so that the
// tensor cores, the exact recombination and the FP64 read-modify-write of
// different tiles overlap:
//
//  * tiles are 128 x 32, aligned to absolute multiples of 128 rows and 32
//    columns of the workspace, so every tile lies inside one 256 x 256 storage
//    tile of the lower-packed layout (or inside the dense rows): its FP64
//    values move by TMA, in as two 128 x 16 boxes with the 128-byte swizzle
//    (a thread then reads and writes its own row without bank conflicts), and
//    back out by TMA stores.  The slices of the panel rows are stored from the
//    128-aligned row sbase <= r0, with zero slices for rows outside [r0, r1),
//    so rows and columns outside the trailing matrix get a zero update;
//    elements above the diagonal are computed and stored into storage no
//    kernel reads (the upper part of diagonal storage tiles, or of the dense
//    rows);
//  * one persistent CTA per SM takes a contiguous range of the launch's tiles
//    (row block by row block, columns left to right), so the six 128 x 64
//    slices of a row block (96 KB) load once per row block;
//  * warp 0 / lane 0 loads (row-block slices, per tile the six 32 x 64 column
//    slices and the FP64 tile, each double-buffered); warp 1 / lane 0 issues
//    the 84 MMAs of a tile (M = 128, N = 32) into one of two TMEM accumulator
//    sets (6 x 32 columns each); warps 2-5 recombine a finished set exactly,
//    subtract from the FP64 tile in shared memory and store it, while the
//    MMAs of the next tile run in the other set.
// Every product is exact and so is every FP32 group sum, so the result is
// bit for bit that of k_chol_update.
#define PU_BJ 32                                   // tile columns
#define PU_IBYTES (CS_BI * CS_K * 2)               // 16 KB: one 128 x 64 row-block slice
#define PU_JBYTES (PU_BJ * CS_K * 2)               // 4 KB: one 32 x 64 column slice
#define PU_CBOX (CS_BI * 16 * 8)                   // 16 KB: 128 rows x 16 FP64
#define PU_OFF_J (CS_S * PU_IBYTES)                // 96 KB
#define PU_OFF_C (PU_OFF_J + 2 * CS_S * PU_JBYTES) // 144 KB
#define PU_SMEM (PU_OFF_C + 2 * 2 * PU_CBOX + 1024)
#define PU_EPI 16         // epilogue warps: four per TMEM lane quarter, 8 columns each
#define PU_THREADS (64 + 32 * PU_EPI)

struct UpdRange {
  int64_t sbase;       // first row of the slice buffer (a multiple of 128)
  int64_t r0, r1;      // trailing rows [r0, r1) (r0 a multiple of 64)
  int64_t ib0, ib1;    // row blocks [ib0, ib1) (absolute, 128 rows)
  int64_t jc0, jc1;    // column tiles [jc0, jc1) (absolute, 32 columns)
  int64_t padS;        // rows per slice in the slice buffer
  int64_t ntiles;      // tiles of the launch
  int64_t tile0;       // first storage tile of W (lower-packed layout)
  int tiled;           // W layout: lower-packed 256 x 256 tiles (1) or dense rows (0)
};

// column tiles of row block ib: [jc0, min(jc1, last column tile at or below the
// block's last row, last column tile of the trailing matrix) ]
__device__ __forceinline__ int64_t pu_jhi(const UpdRange& u, int64_t ib) {
  int64_t j = 4 * ib + 3;
  const int64_t jr = (u.r1 - 1) >> 5;
  if (j > jr) j = jr;
  if (j > u.jc1 - 1) j = u.jc1 - 1;
  return j;
}

__device__ __forceinline__ void pu_tma_load(const CUtensorMap* map, uint64_t* bar, void* dst, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          cs_smem_u32(dst)),
      "l"((uint64_t)map), "r"(cs_smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void pu_tma_store(const CUtensorMap* map, const void* src, int c0, int c1) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"((uint64_t)map),
               "r"(cs_smem_u32(src)), "r"(c0), "r"(c1)
               : "memory");
}
__device__ __forceinline__ void pu_init(uint64_t* bar, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cs_smem_u32(bar)), "r"(n) : "memory");
}
__device__ __forceinline__ void pu_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cs_smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void pu_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(cs_smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void pu_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(cs_smem_u32(bar))
               : "memory");
}
// bounded wait that also gives up once any CTA has raised the status word
__device__ __forceinline__ bool pu_wait(uint64_t* bar, uint32_t parity, int* status) {
  for (uint32_t i = 0; i < CS_SPIN; ++i) {
    if (cs_try(bar, parity)) return true;
    if ((i & 1023u) == 1023u && *(volatile int*)status) return false;
  }
  atomicExch(status, 1);
  return false;
}

// storage coordinates of FP64 element (r, c) for the tile maps: x = column
// inside the storage row, y = storage row
__device__ __forceinline__ void pu_coord(const UpdRange& u, int64_t r, int64_t c, int* x, int* y) {
  if (u.tiled) {
    const int64_t ti = r >> 8, tj = c >> 8;
    *x = (int)(c & 255);
    *y = (int)(((ti * (ti + 1) / 2 + tj - u.tile0) << 8) + (r & 255));
  } else {
    *x = (int)c;
    *y = (int)r;
  }
}

__global__ void __launch_bounds__(PU_THREADS, 1)
    k_chol_upd(const __grid_constant__ CUtensorMap map_i, const __grid_constant__ CUtensorMap map_j,
               const __grid_constant__ CUtensorMap map_c, const int* __restrict__ rexp, UpdRange u, int* status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t i_full, i_empty, j_full[2], j_empty[2], c_full[2], c_empty[2], t_full[2],
      t_empty[2], e_done[2], mma_done;
  __shared__ uint32_t tmem_sh;
  __shared__ int64_t start_ib, start_jb;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // this CTA's tiles [x0, x1) of the launch, in row-block order
  const int64_t x0 = u.ntiles * blockIdx.x / gridDim.x, x1 = u.ntiles * (blockIdx.x + 1) / gridDim.x;
  if (threadIdx.x == 0) {
    int64_t ib = u.ib0, x = 0;
    for (;; ++ib) {
      const int64_t n = pu_jhi(u, ib) - u.jc0 + 1;
      if (n > 0 && x + n > x0) break;
      if (n > 0) x += n;
    }
    start_ib = ib;
    start_jb = u.jc0 + (x0 - x);
    pu_init(&i_full, 1);
    pu_init(&i_empty, 1);
    for (int b = 0; b < 2; ++b) {
      pu_init(&j_full[b], 1);
      pu_init(&j_empty[b], 1);
      pu_init(&c_full[b], 1);
      pu_init(&c_empty[b], 1);
      pu_init(&t_full[b], 1);
      pu_init(&t_empty[b], PU_EPI);  // one arrival per epilogue warp
      pu_init(&e_done[b], PU_EPI);   // one arrival per epilogue warp: the tile's values are in shared memory
    }
    pu_init(&mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(cs_smem_u32(&tmem_sh)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_sh;
  const int64_t n_my = x1 - x0;

  if (warp == 0 && lane == 0) {
    // ---------------- producer
    int64_t ib = start_ib, jb = start_jb, jh = pu_jhi(u, ib);
    int64_t nib = 0;  // row blocks loaded so far
    bool ok = true;
    for (int64_t t = 0; t < n_my && ok; ++t) {
      if (t == 0 || jb == u.jc0) {  // a new row block: its six slices
        if (!pu_wait(&i_empty, (uint32_t)(nib & 1) ^ 1u, status)) break;
        pu_expect(&i_full, CS_S * PU_IBYTES);
        const int yi = (int)(ib * CS_BI - u.sbase);
        for (int k = 0; k < CS_S; ++k)
          pu_tma_load(&map_i, &i_full, smem + k * PU_IBYTES, 0, (int)(k * u.padS) + yi);
        ++nib;
      }
      const int b = (int)(t & 1);
      const uint32_t ph = (uint32_t)((t >> 1) & 1);
      if (!pu_wait(&j_empty[b], ph ^ 1u, status)) break;
      pu_expect(&j_full[b], CS_S * PU_JBYTES);
      const int yj = (int)(jb * PU_BJ - u.sbase);
      for (int k = 0; k < CS_S; ++k)
        pu_tma_load(&map_j, &j_full[b], smem + PU_OFF_J + (b * CS_S + k) * PU_JBYTES, 0, (int)(k * u.padS) + yj);
      if (!pu_wait(&c_empty[b], ph ^ 1u, status)) break;
      pu_expect(&c_full[b], 2 * PU_CBOX);
      for (int h = 0; h < 2; ++h) {
        int x, y;
        pu_coord(u, ib * CS_BI, jb * PU_BJ + 16 * h, &x, &y);
        pu_tma_load(&map_c, &c_full[b], smem + PU_OFF_C + (2 * b + h) * PU_CBOX, x, y);
      }
      if (++jb > jh) {
        ++ib;
        jh = pu_jhi(u, ib);
        jb = u.jc0;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issue
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(PU_BJ >> 3) << 17) |
                           ((uint32_t)(CS_BI >> 4) << 24);
    const uint32_t base_i = cs_smem_u32(smem);
    int64_t ib = start_ib, jb = start_jb, jh = pu_jhi(u, ib), nib = 0;
    for (int64_t t = 0; t < n_my; ++t) {
      if (t == 0 || jb == u.jc0) {
        if (t > 0) pu_commit(&i_empty);  // the previous row block's slices are free once its MMAs finish
        if (!pu_wait(&i_full, (uint32_t)(nib & 1), status)) break;
        ++nib;
      }
      const int b = (int)(t & 1);
      const uint32_t ph = (uint32_t)((t >> 1) & 1);
      if (!pu_wait(&j_full[b], ph, status)) break;
      if (!pu_wait(&t_empty[b], ph ^ 1u, status)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base_j = cs_smem_u32(smem + PU_OFF_J + b * CS_S * PU_JBYTES);
      const uint32_t tset = tmem + (uint32_t)(b * CS_S * PU_BJ);
#pragma unroll 1
      for (int k = 0; k < CS_K / 16; ++k)
#pragma unroll
        for (int r = 0; r < CS_S; ++r)
#pragma unroll
          for (int g = r; g < CS_S; ++g) {
            const uint32_t dt = tset + (uint32_t)(g * PU_BJ);
            const uint64_t ad = cs_desc_sw128(base_i + r * PU_IBYTES + k * 32);
            const uint64_t bd = cs_desc_sw128(base_j + (g - r) * PU_JBYTES + k * 32);
            const uint32_t acc = (k == 0 && r == 0) ? 0u : 1u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, "
                "p;\n}\n" ::"r"(dt),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
          }
      pu_commit(&j_empty[b]);
      pu_commit(&t_full[b]);
      if (++jb > jh) {
        ++ib;
        jh = pu_jhi(u, ib);
        jb = u.jc0;
      }
    }
    // every MMA of this CTA has completed before its TMEM is released
    pu_commit(&mma_done);
    for (uint32_t i = 0; i < CS_SPIN && !cs_try(&mma_done, 0u); ++i) {
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: warp w owns TMEM lanes / tile rows 32 (w % 4) ..
    // and the 8-column quarter cq = (w - 2) / 4 of the tile.  Every wait is
    // taken by lane 0 and its outcome shared with the warp, so a warp leaves
    // its loop as a whole (the TMEM loads are warp-collective) and no wait is
    // unbounded.
    const int q = warp & 3, cq = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    int64_t ib = start_ib, jb = start_jb, jh = pu_jhi(u, ib);
    for (int64_t t = 0; t < n_my; ++t) {
      const int b = (int)(t & 1);
      const uint32_t ph = (uint32_t)((t >> 1) & 1);
      int ok = 1;
      if (lane == 0) ok = pu_wait(&t_full[b], ph, status) && pu_wait(&c_full[b], ph, status);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      __syncwarp();
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t rr[CS_S][8];
#pragma unroll
      for (int g = 0; g < CS_S; ++g)
        cs_tmem_ld8_nowait(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * CS_S * PU_BJ + g * PU_BJ + cq * 8),
                           rr[g]);
      const int64_t gr = ib * CS_BI + row;  // absolute row of this thread
      const int ei = (gr >= u.r0 && gr < u.r1) ? rexp[gr - u.sbase] : 0;
      const int64_t gj0 = jb * PU_BJ + 8 * cq;
      // the 8 column exponents of this quarter, one per lane, shared by shuffles
      const int64_t gcl = gj0 + (lane & 7);
      const int ejl = (gcl >= u.r0 && gcl < u.r1) ? __ldg(rexp + (gcl - u.sbase)) : 0;
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int g = 0; g < CS_S; ++g)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) asm volatile("" : "+r"(rr[g][jj]));
      double* cb = (double*)(smem + PU_OFF_C + (2 * b + (cq >> 1)) * PU_CBOX);
#pragma unroll
      for (int jq = 0; jq < 4; ++jq) {
        double v[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int jj = 2 * jq + e;
          // the group sums are exact FP32 integers (|A_g| < 2^23): A_0 2^40 + ... + A_5
          const int p0 = __float2int_rz(__uint_as_float(rr[0][jj])) * 256 + __float2int_rz(__uint_as_float(rr[1][jj]));
          const int p1 = __float2int_rz(__uint_as_float(rr[2][jj])) * 256 + __float2int_rz(__uint_as_float(rr[3][jj]));
          const int p2 = __float2int_rz(__uint_as_float(rr[4][jj])) * 256 + __float2int_rz(__uint_as_float(rr[5][jj]));
          const long long a = ((long long)p0 << 32) + ((long long)p1 << 16) + (long long)p2;
          const int ej = __shfl_sync(0xffffffffu, ejl, jj);
          v[e] = scaled_to_double_rn(a, ei + ej - 54);
        }
        // 128-byte swizzle: 16-byte chunk jp of row `row` sits at chunk jp ^ (row & 7)
        const int jp = 4 * (cq & 1) + jq;
        double2* p = (double2*)(cb + row * 16) + (jp ^ (row & 7));
        double2 c2 = *p;
        c2.x -= v[0];
        c2.y -= v[1];
        *p = c2;
      }
      // the accumulator set is free for the MMAs of tile t + 2, and this
      // warp's values are in shared memory, visible to the bulk copy
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        pu_arrive(&t_empty[b]);
        pu_arrive(&e_done[b]);
      }
      if (warp == 2) {
        // warp 2 stores the tile once every epilogue warp has written its values
        int ok2 = 1;
        if (lane == 0) ok2 = pu_wait(&e_done[b], ph, status);
        ok2 = __shfl_sync(0xffffffffu, ok2, 0);
        __syncwarp();
        if (!ok2) break;
        if (lane == 0) {
          for (int hh = 0; hh < 2; ++hh) {
            int x, y;
            pu_coord(u, ib * CS_BI, jb * PU_BJ + 16 * hh, &x, &y);
            if (u.tiled || x < u.r1) pu_tma_store(&map_c, smem + PU_OFF_C + (2 * b + hh) * PU_CBOX, x, y);
          }
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // the buffer may be refilled now
          pu_arrive(&c_empty[b]);
        }
        __syncwarp();
      }
      if (++jb > jh) {
        ++ib;
        jh = pu_jhi(u, ib);
        jb = u.jc0;
      }
    }
    if (warp == 2 && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // stores complete
  }
  __syncwarp();
  // after an expired wait some copies may still be in flight: a bounded
  // pause (~1 ms) lets them land before the CTA's shared memory is released
  if (warp == 0 && lane == 0 && *(volatile int*)status != 0)
    for (int i = 0; i < 1000; ++i) __nanosleep(1000);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

static PFN_cuTensorMapEncodeTiled_v12000 cs_encode() { return wl_encode_tiled(); }

static int cs_map(cov_handle* h, CUtensorMap* map, void* base, int64_t total_rows, int box_rows) {
  auto fn = cs_encode();
  if (!fn) return wl_fail(h, COV_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[2] = {(cuuint64_t)CS_K, (cuuint64_t)total_rows};
  cuuint64_t strides[1] = {(cuuint64_t)CS_K * 2};
  cuuint32_t box[2] = {(cuuint32_t)CS_K, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return wl_fail(h, COV_ERR_CUDA, "cuTensorMapEncodeTiled failed (Cholesky slices)");
  return COV_OK;
}

// bytes of one slice buffer for up to n trailing rows (either kernel's layout:
// the persistent kernel's rows start up to 64 rows before the trailing matrix)
size_t wl_chol_tc_bytes(int64_t n) {
  int64_t pad = (n + 64 + CS_BI - 1) / CS_BI * CS_BI;
  return (size_t)CS_S * pad * CS_K * 2 + (size_t)pad * sizeof(int);
}

// The panel solve and the slicing in one pass, in the persistent update's
// 128-aligned slice layout: each row sbase + i (i < pad) inside [r0, r1)
// solves x L11^T = a by forward substitution, is written back, and is cut into
// slices from the same registers; rows outside [r0, r1) get zero slices.
// Eight lanes per row, lane q owning the entries j = q mod 8: at column l the
// owner scales its entry by 1 / L11[l][l] and passes it to the row's other
// lanes by a shuffle, and each lane subtracts x_l L11[j][l] from its entries
// j > l, so every entry receives the FMAs and the scaling of the plain forward
// substitution in its order.  On this part one warp issues at most one FP64
// instruction per 64 cycles and an SM needs four warps to fill its FP64 pipe,
// so rows are spread thin: 16 rows per block of four warps, one block per
// ~16 rows of the panel.  The slice digits are integer work (slice_int).
#define TS_THREADS 128
#define TS_LANES 8
__global__ void __launch_bounds__(TS_THREADS) k_trsm_slice(OutMap W, int64_t k0, int kb, int64_t sbase, int64_t r0,
                                                           int64_t r1, int64_t pad, __nv_bfloat16* slices,
                                                           int* rexp) {
  __shared__ double L[CS_K][CS_K + 1];
  __shared__ double invd[CS_K];
  for (int e = threadIdx.x; e < CS_K * CS_K; e += blockDim.x) {
    const int i = e >> 6, l = e & 63;
    L[i][l] = (i < kb && l <= i) ? *W.at(k0 + i, k0 + l) : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kb; i += blockDim.x) invd[i] = 1.0 / L[i][i];
  __syncthreads();
  constexpr int NE = CS_K / TS_LANES;  // entries per lane
  const int lane = threadIdx.x & 31, q = lane & (TS_LANES - 1), g = lane & ~(TS_LANES - 1);
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TS_LANES;
  const int64_t r = sbase + i;
  const bool in = i < pad;
  const bool valid = in && r >= r0 && r < r1;
  double* row = valid ? W.at(r, k0) : nullptr;
  double a[NE];
#pragma unroll
  for (int m = 0; m < NE; ++m) a[m] = (valid && q + TS_LANES * m < kb) ? row[q + TS_LANES * m] : 0.0;
#pragma unroll
  for (int l = 0; l < CS_K; ++l) {
    if (l >= kb) break;
    if (q == (l % TS_LANES)) a[l / TS_LANES] *= invd[l];
    const double xl = __shfl_sync(0xffffffffu, a[l / TS_LANES], g + (l % TS_LANES));
#pragma unroll
    for (int m = (l + 1) / TS_LANES; m < NE; ++m) {
      const int j = q + TS_LANES * m;
      if (j > l) a[m] = fma(-xl, L[j][l], a[m]);
    }
  }
  if (valid) {
#pragma unroll
    for (int m = 0; m < NE; ++m)
      if (q + TS_LANES * m < kb) row[q + TS_LANES * m] = a[m];
  }
  // slicing: the row's largest magnitude over its eight lanes, then six slices
#pragma unroll
  for (int m = 0; m < NE; ++m)
    if (q + TS_LANES * m >= kb) a[m] = 0.0;
  double mx = 0.0;
#pragma unroll
  for (int m = 0; m < NE; ++m) mx = fmax(mx, fabs(a[m]));
#pragma unroll
  for (int o = 1; o < TS_LANES; o <<= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);
  if (!in) return;
  const size_t stride = (size_t)pad * CS_K;
  __nv_bfloat16* out = slices + (size_t)i * CS_K + q;
#pragma unroll
  for (int m = 0; m < NE; ++m) slice_store(slice_int(a[m], e), out + TS_LANES * m, stride);
  if (q == 0) rexp[i] = e;
}

// whether the persistent kernel serves this workspace: it addresses the FP64
// tiles by TMA from the start of the workspace (rows from 0, 16-byte rows)
static bool pu_usable(const cov_handle* h, const OutMap& W) {
  if (h->chol_kernel == 1) return false;
  if (W.row0 != 0 || W.tile0 != 0) return false;
  return W.tiled || (W.ldc % 2 == 0);
}

static int pu_num_sms() {
  static std::once_flag once[WL_MAX_DEVICES];
  static int n[WL_MAX_DEVICES];
  int d = 0;
  cudaGetDevice(&d);
  if (d < 0 || d >= WL_MAX_DEVICES) return 1;
  std::call_once(once[d], [&] {
    n[d] = 1;
    cudaDeviceGetAttribute(&n[d], cudaDevAttrMultiProcessorCount, d);
    if (n[d] < 1) n[d] = 1;
  });
  return n[d];
}

// slices of the panel rows r0..r1-1, columns k0..k0+kb-1 of the workspace
int wl_chol_slice(cov_handle* h, OutMap W, int64_t k0, int kb, int64_t r0, int64_t r1, void* buf, cudaStream_t s) {
  int64_t n = r1 - r0;
  if (n <= 0) return COV_OK;
  // (where the persistent kernel serves the workspace, wl_chol_trsm_slice cuts the slices)
  int64_t pad = (n + CS_BI - 1) / CS_BI * CS_BI;
  __nv_bfloat16* slices = (__nv_bfloat16*)buf;
  int* rexp = (int*)((uint8_t*)buf + (size_t)CS_S * pad * CS_K * 2);
  k_chol_slice<<<(unsigned)((pad + 7) / 8), 256, 0, s>>>(W, k0, kb, r0, n, pad, slices, rexp);
  WL_LAUNCH(h, "k_chol_slice");
  return COV_OK;
}

bool wl_chol_fused_panel(const cov_handle* h, const OutMap& W) { return pu_usable(h, W); }

// the panel solve of rows r0..r1-1 against the factored diagonal block at k0,
// fused with their slicing (only where wl_chol_fused_panel holds)
int wl_chol_trsm_slice(cov_handle* h, OutMap W, int64_t k0, int kb, int64_t r0, int64_t r1, void* buf,
                       cudaStream_t s) {
  if (r1 <= r0) return COV_OK;
  const int64_t sbase = r0 / CS_BI * CS_BI, pad = (r1 - sbase + CS_BI - 1) / CS_BI * CS_BI;
  __nv_bfloat16* slices = (__nv_bfloat16*)buf;
  int* rexp = (int*)((uint8_t*)buf + (size_t)CS_S * pad * CS_K * 2);
  // eight threads per row: pad / 16 blocks of 128 threads cover the pad rows exactly
  k_trsm_slice<<<(unsigned)(pad * TS_LANES / TS_THREADS), TS_THREADS, 0, s>>>(W, k0, kb, sbase, r0, r1, pad, slices,
                                                                              rexp);
  WL_LAUNCH(h, "k_trsm_slice");
  return COV_OK;
}

// Csub (rows/cols r0..r1-1 of the workspace) -= L21 L21^T over the column
// tiles tj0 .. tj0+ntj-1 (64 columns each; ntj < 0: all remaining), lower
// triangle only, from the slices in buf
// The persistent update over the column tiles [jc0, jc1) (32 columns each,
// absolute) of the trailing rows [r0, r1).
static int pu_update(cov_handle* h, OutMap W, int64_t r0, int64_t r1, const void* buf, int64_t jc0, int64_t jc1,
                     int* status, cudaStream_t s) {
  UpdRange u;
  u.sbase = r0 / CS_BI * CS_BI;
  u.r0 = r0;
  u.r1 = r1;
  u.padS = (r1 - u.sbase + CS_BI - 1) / CS_BI * CS_BI;
  u.ib0 = u.sbase / CS_BI;
  u.ib1 = (r1 - 1) / CS_BI + 1;
  u.jc0 = jc0;
  u.jc1 = jc1;
  u.tile0 = 0;
  u.tiled = W.tiled;
  int64_t nt = 0;
  for (int64_t ib = u.ib0; ib < u.ib1; ++ib) {
    int64_t j = std::min<int64_t>(std::min<int64_t>(4 * ib + 3, (r1 - 1) >> 5), jc1 - 1);
    if (j >= jc0) nt += j - jc0 + 1;
  }
  u.ntiles = nt;
  if (nt == 0) return COV_OK;
  auto fn = cs_encode();
  if (!fn) return wl_fail(h, COV_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  const int* rexp = (const int*)((const uint8_t*)buf + (size_t)CS_S * u.padS * CS_K * 2);
  CUtensorMap mi, mj, mc;
  int rc;
  if ((rc = cs_map(h, &mi, (void*)buf, CS_S * u.padS, CS_BI))) return rc;
  if ((rc = cs_map(h, &mj, (void*)buf, CS_S * u.padS, PU_BJ))) return rc;
  {
    cuuint64_t dims[2], strides[1];
    if (W.tiled) {
      const int64_t T = (r1 + 255) / 256;
      dims[0] = 256;
      dims[1] = (cuuint64_t)(T * (T + 1) / 2) * 256;
      strides[0] = 256 * 8;
    } else {
      dims[0] = (cuuint64_t)r1;
      dims[1] = (cuuint64_t)r1;
      strides[0] = (cuuint64_t)W.ldc * 8;
    }
    cuuint32_t box[2] = {16, (cuuint32_t)CS_BI};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(&mc, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, W.C, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return wl_fail(h, COV_ERR_CUDA, "cuTensorMapEncodeTiled failed (Cholesky FP64 tiles)");
  }
  static std::once_flag attr_once[WL_MAX_DEVICES];
  static int attr_rc[WL_MAX_DEVICES];
  if (wl_once_per_device(attr_once, attr_rc, [] {
        return (int)cudaFuncSetAttribute(k_chol_upd, cudaFuncAttributeMaxDynamicSharedMemorySize, PU_SMEM);
      }) != 0)
    return wl_fail(h, COV_ERR_CUDA, "cudaFuncSetAttribute(k_chol_upd) failed");
  const int64_t grid = std::min<int64_t>(pu_num_sms(), nt);
  k_chol_upd<<<(unsigned)grid, PU_THREADS, PU_SMEM, s>>>(mi, mj, mc, rexp, u, status);
  WL_LAUNCH(h, "k_chol_upd");
  return COV_OK;
}

int wl_chol_update(cov_handle* h, OutMap W, int64_t r0, int64_t r1, const void* buf, int tj0, int ntj, int* status,
                   cudaStream_t s) {
  int64_t n = r1 - r0;
  if (n <= 0) return COV_OK;
  if (pu_usable(h, W)) {
    // the 64-column tiles tj0 .. tj0 + ntj - 1 of the trailing matrix are the
    // 32-column tiles from r0 / 32 + 2 tj0
    const int64_t jc0 = r0 / PU_BJ + 2 * (int64_t)tj0;
    const int64_t jc1 = ntj < 0 ? ((int64_t)1 << 40) : jc0 + 2 * (int64_t)ntj;
    return pu_update(h, W, r0, r1, buf, jc0, jc1, status, s);
  }
  int64_t pad = (n + CS_BI - 1) / CS_BI * CS_BI;
  int total_tj = (int)((n + CS_BJ - 1) / CS_BJ);
  if (ntj < 0 || tj0 + ntj > total_tj) ntj = total_tj - tj0;
  if (ntj <= 0) return COV_OK;
  void* slices = (void*)buf;
  const int* rexp = (const int*)((const uint8_t*)buf + (size_t)CS_S * pad * CS_K * 2);
  CUtensorMap mi, mj;
  int rc;
  if ((rc = cs_map(h, &mi, slices, CS_S * pad, CS_BI))) return rc;
  if ((rc = cs_map(h, &mj, slices, CS_S * pad, CS_BJ))) return rc;
  static std::once_flag attr_once[WL_MAX_DEVICES];
  static int attr_rc[WL_MAX_DEVICES];
  if (wl_once_per_device(attr_once, attr_rc, [] {
        return (int)cudaFuncSetAttribute(k_chol_update, cudaFuncAttributeMaxDynamicSharedMemorySize, CS_SMEM);
      }) != 0)
    return wl_fail(h, COV_ERR_CUDA, "cudaFuncSetAttribute(k_chol_update) failed");
  // only the lower tiles of the tile rows that reach the requested columns
  TileRows tr;
  tr.tj0 = tj0;
  tr.ntj = ntj;
  tr.ti0 = (int)(((int64_t)tj0 * CS_BJ) / CS_BI);
  tr.nti = (int)(pad / CS_BI) - tr.ti0;
  if (tr.nti <= 0) return COV_OK;
  int64_t nblk = tr.cum(tr.ti0 + tr.nti);
  k_chol_update<<<(unsigned)nblk, 128, CS_SMEM, s>>>(mi, mj, n, pad, rexp, W, r0, status, tr);
  WL_LAUNCH(h, "k_chol_update");
  return COV_OK;
}
