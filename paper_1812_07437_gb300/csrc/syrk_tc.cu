// Tensor-core form of the 1-halo (chi, M) contraction (paper Eqs. CovPPNG,
// Ins5P, Ins6P recast as C_1h = A A^T with A the factor rows):
//
//   * k_rows_split builds each factor row in FP64, scales it by an exact power
//     of two s_a so that its largest entry lies in [0.5, 1), and splits it into
//     two BF16 rows, hi = bf16(a / s_a), lo = bf16(a / s_a - hi).
//   * k_syrk_tc256 computes, per 256 x 256 lower-triangle tile, the FP32 sum
//     hi_i hi_j + hi_i lo_j + lo_i hi_j over K on the tcgen05 tensor cores
//     (kind::f16, BF16 operands, FP32 accumulators in TMEM) and stores
//     acc * s_i * s_j into the FP64 lower triangle (first writer of C).
//
// The split rows are stored tile-blocked (256 rows x 32 K contiguous) so that
// every TMA box is one contiguous 16 KB block of HBM.  Per CTA (128 threads):
// warp 0 / lane 0 issues the TMA loads of a K block (hi/lo of the 256 I rows
// and of the 256 J rows, 64-byte swizzle) into a 3-stage shared-memory ring;
// warp 1 / lane 0 issues the 12 MMAs of 128 x 256 x 16 per K block into two
// TMEM accumulators (row halves) and releases each stage with tcgen05.commit;
// after the last block all four warps read the accumulators (tcgen05.ld
// 32x32b) and write the tile.  Every wait on an mbarrier is bounded: on expiry
// the kernel raises a status word, stops issuing work, waits (bounded) for its
// own copies, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"

#define TC_SPIN_LIMIT (1u << 22)
#define TW_BM 256
#define TW_BK 32

// Tile-blocked operand layout: entry (r, k) of a split row array lives at
// ((r / 256) * nk + k / 32) * 8192 + (r % 256) * 32 + k % 32, with nk = Kp / 32,
// so that each 256 x 32 TMA box is one contiguous 16 KB block in HBM.
__device__ __forceinline__ int64_t blk_off(int64_t r, int k, int nk) {
  return (((r >> 8) * nk + (k >> 5)) << 13) + ((r & 255) << 5) + (k & 31);
}

// ---------------------------------------------------------------- row split
// Per-(n, q) and per-n factors of the 1-halo rows, so that the row builder
// needs only products: g_mu[n][q] = sqrt(w_n omega_q f_nq / Omega) (m_q/rho)^mu
// and c_mu[n] = chi_n^(1 - 2 mu), for mu = 2 (P rows) and 3 (B rows).
__global__ void k_rows_prep(int nchi, int nm, double inv_omega, const cov_cosmology* __restrict__ cosmo_p,
                            const double* chi, const double* wchi,
                            const double* m, const double* om, const double* f, double* g2, double* g3, double* c2,
                            double* c3) {
  const double rho = WL_RHO_CRIT0 * cosmo_p->Om;
  int kk = blockIdx.x * blockDim.x + threadIdx.x;
  if (kk >= nchi * nm) return;
  int n = kk / nm, q = kk % nm;
  double mr = m[q] / rho;
  double base = sqrt(wchi[n] * om[q] * f[kk] * inv_omega);
  g2[kk] = base * mr * mr;
  g3[kk] = base * mr * mr * mr;
  if (q == 0) {
    double ch = chi[n];
    c2[n] = 1.0 / (ch * ch * ch);
    c3[n] = 1.0 / (ch * ch * ch * ch * ch);
  }
}

// Rows that share their ell bins share the (n, q) part of the 1-halo factor:
// a P row of bin b has F_b[n][q] = g2[n][q] c2[n] U_b[n][q]^2, a B row of
// triangle (a, b, c) has F_abc[n][q] = g3[n][q] c3[n] U_a U_b U_c, and the row
// itself is F[n][q] times the product of its lensing kernels W_i(chi_n).  One
// block per (signature s, node n) stores F[s][n][.] / 2^E[s][n] in FP32 (its
// largest magnitude in [0.5, 1)), E[s][n] and the FP64 maximum.
// pairs: signatures are the bin pairs b1 <= b2 (trispectrum rows, mu = 2)
// instead of the P bins and B triangles.
__global__ void k_rows_sig(int nl, int ntri, int nchi, int nm, const int32_t* tris, const double* U, const double* g2,
                           const double* g3, const double* c2, const double* c3, float* F, int* E, double* Mx,
                           int pairs) {
  __shared__ double red[32];
  int s = blockIdx.x, n = blockIdx.y;
  bool isP = pairs || s < nl;
  int a, b, c;
  if (pairs) {
    a = 0;
    int base = 0;
    while (base + (nl - a) <= s) {
      base += nl - a;
      ++a;
    }
    b = a + (s - base);
    c = b;
  } else if (isP) {
    a = b = c = s;
  } else {
    a = tris[3 * (s - nl)];
    b = tris[3 * (s - nl) + 1];
    c = tris[3 * (s - nl) + 2];
  }
  const size_t K = (size_t)nchi * nm;
  const double* Ua = U + a * K + (size_t)n * nm;
  const double* Ub = U + b * K + (size_t)n * nm;
  const double* Uc = U + c * K + (size_t)n * nm;
  const double* g = (isP ? g2 : g3) + (size_t)n * nm;
  double cn = isP ? c2[n] : c3[n];
  auto value = [&](int q) { return isP ? g[q] * cn * Ua[q] * Ub[q] : g[q] * cn * Ua[q] * Ub[q] * Uc[q]; };
  double mx = 0.0;
  for (int q = threadIdx.x; q < nm; q += blockDim.x) mx = fmax(mx, fabs(value(q)));
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    t = warp_max(t);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  mx = red[0];
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);
  float* Fo = F + (size_t)s * K + (size_t)n * nm;
  for (int q = threadIdx.x; q < nm; q += blockDim.x) Fo[q] = (float)ldexp(value(q), -e);
  if (threadIdx.x == 0) {
    E[(size_t)s * nchi + n] = e;
    Mx[(size_t)s * nchi + n] = mx;
  }
}

// One block per row a: entries 0..K-1 are the 1-halo factor row; when
// nssc > 0, entries K..K+nssc-1 are the super-sample row S[a][n] (so that one
// contraction gives A A^T + S S^T); the rest of Kp is zero.  The row is scaled
// by an exact power of two s_a (largest entry in [0.5, 1)) and split into
// BF16 hi/lo.  FP64 work is per node (kernel products, row maximum, the
// super-sample entries); each factor entry is one FP32 product of the
// signature table and a per-node FP32 weight, exact to a few 2^-24, well
// inside the 2^-17 of the hi/lo split.
__global__ void k_rows_split(int64_t M, int nl, int nchi, int nm, int Kp, int nssc, const int32_t* rd,
                             const double* W, const float* F, const int* E, const double* Mx, const double* wchi,
                             const double* sigw2, const double* chi, const double* RP3, const double* RB3,
                             __nv_bfloat16* hi, __nv_bfloat16* lo, double* rscale) {
  extern __shared__ double rs_sh[];  // [nchi] node weights, [nchi] super-sample entries
  __shared__ double red[32];
  int64_t a = blockIdx.x;
  if (a >= M) return;
  const int32_t* r = rd + 8 * a;
  const int K = nchi * nm;
  const bool isP = (r[0] == 0);
  const int sg = isP ? r[1] : nl + r[7];
  const double* W1 = W + r[4] * nchi;
  const double* W2 = W + r[5] * nchi;
  const double* W3 = W + (isP ? r[4] : r[6]) * nchi;
  const int* Es = E + (size_t)sg * nchi;
  const double* Ms = Mx + (size_t)sg * nchi;
  double* wsh = rs_sh;
  double* ssh = rs_sh + nchi;
  // pass 1 (per node): kernel products, super-sample entries, row maximum
  double mx = 0.0;
  for (int n = threadIdx.x; n < nchi; n += blockDim.x) {
    double w = W1[n] * W2[n];
    if (!isP) w *= W3[n];
    wsh[n] = w;
    mx = fmax(mx, fabs(w) * Ms[n]);
    double v = 0.0;
    if (n < nssc) {
      double ch = chi[n], c2_ = ch * ch;
      v = sqrt(wchi[n] * sigw2[n]) * w;
      v = isP ? v / c2_ * RP3[r[1] * nchi + n] : v / (c2_ * c2_) * RB3[r[7] * nchi + n];
      mx = fmax(mx, fabs(v));
    }
    ssh[n] = v;
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    t = warp_max(t);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  mx = red[0];
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);
  // pass 2 (per node): FP32 weights relative to the row scale 2^ex
  float* wf = (float*)(rs_sh + 2 * nchi);
  float* sf = wf + nchi;
  for (int n = threadIdx.x; n < nchi; n += blockDim.x) {
    wf[n] = (float)ldexp(wsh[n], Es[n] - ex);
    sf[n] = (float)ldexp(ssh[n], -ex);
  }
  __syncthreads();
  // pass 3 (per entry pair): one FP32 product, BF16 hi/lo split, paired stores
  const float* Fs = F + (size_t)sg * K;
  const int Kt = K + nssc;
  const int nk = Kp / TW_BK;
  auto value = [&](int kk) -> float {
    if (kk < K) return Fs[kk] * wf[(unsigned)kk / (unsigned)nm];
    return kk < Kt ? sf[kk - K] : 0.0f;
  };
  for (int kk = 2 * threadIdx.x; kk < Kp; kk += 2 * blockDim.x) {
    float x0 = value(kk), x1 = value(kk + 1);
    __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
    __nv_bfloat162 l2 = __floats2bfloat162_rn(x0 - __low2float(h2), x1 - __high2float(h2));
    int64_t o = blk_off(a, kk, nk);
    *(__nv_bfloat162*)(hi + o) = h2;
    *(__nv_bfloat162*)(lo + o) = l2;
  }
  if (threadIdx.x == 0) rscale[a] = ldexp(1.0, ex);
}

// Trispectrum rows of the PT term, one block per leg pair (L1 <= L2),
// L = bin * n_t + tomo: T[(n, q)] = sqrt(w_n omega_q f_nq) (m_q/rho)^2
// chi_n^-3 W_t1 W_t2 U_b1 U_b2, i.e. the pair signature (b1, b2) times the
// node weight sqrt(Omega) W_t1(chi_n) W_t2(chi_n); scaled and split as
// k_rows_split does.
__global__ void k_trows_split(int64_t ntrow, int nleg, int nt, int nl, int nchi, int nm, int Kp, double sqrt_omega,
                              const double* W, const float* F, const int* E, const double* Mx, __nv_bfloat16* hi,
                              __nv_bfloat16* lo, double* rscale) {
  extern __shared__ double ts_sh[];  // [nchi] node weights (FP64), then [nchi] FP32
  __shared__ double red[32];
  int64_t r = blockIdx.x;
  if (r >= ntrow) return;
  int L1 = 0;
  int64_t base = 0;
  while (base + (nleg - L1) <= r) {
    base += nleg - L1;
    ++L1;
  }
  int L2 = L1 + (int)(r - base);
  int b1 = L1 / nt, t1 = L1 % nt, b2 = L2 / nt, t2 = L2 % nt;
  int lo_b = b1 < b2 ? b1 : b2, hi_b = b1 < b2 ? b2 : b1;
  int sg = lo_b * nl - lo_b * (lo_b - 1) / 2 + (hi_b - lo_b);
  const int K = nchi * nm;
  const double* W1 = W + t1 * nchi;
  const double* W2 = W + t2 * nchi;
  const int* Es = E + (size_t)sg * nchi;
  const double* Ms = Mx + (size_t)sg * nchi;
  double* wsh = ts_sh;
  double mx = 0.0;
  for (int n = threadIdx.x; n < nchi; n += blockDim.x) {
    double w = W1[n] * W2[n] * sqrt_omega;
    wsh[n] = w;
    mx = fmax(mx, fabs(w) * Ms[n]);
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    t = warp_max(t);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  mx = red[0];
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);
  float* wf = (float*)(ts_sh + nchi);
  for (int n = threadIdx.x; n < nchi; n += blockDim.x) wf[n] = (float)ldexp(wsh[n], Es[n] - ex);
  __syncthreads();
  const float* Fs = F + (size_t)sg * K;
  const int nk = Kp / TW_BK;
  for (int kk = 2 * threadIdx.x; kk < Kp; kk += 2 * blockDim.x) {
    float x0 = kk < K ? Fs[kk] * wf[(unsigned)kk / (unsigned)nm] : 0.0f;
    float x1 = kk + 1 < K ? Fs[kk + 1] * wf[(unsigned)(kk + 1) / (unsigned)nm] : 0.0f;
    __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
    __nv_bfloat162 l2 = __floats2bfloat162_rn(x0 - __low2float(h2), x1 - __high2float(h2));
    int64_t o = blk_off(r, kk, nk);
    *(__nv_bfloat162*)(hi + o) = h2;
    *(__nv_bfloat162*)(lo + o) = l2;
  }
  if (threadIdx.x == 0) rscale[r] = ldexp(1.0, ex);
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

// bounded wait; false when the limit expired, another role of this CTA gave
// up, or any CTA of the launch raised the status word (so that one expired
// wait ends the whole launch quickly)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status) {
  for (uint32_t i = 0; i < TC_SPIN_LIMIT; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 1023u) == 1023u && (*abort_flag || *(volatile int*)status)) {
      *abort_flag = 1;
      return false;
    }
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

__device__ __forceinline__ void tri_tile_tc(int64_t id, int64_t* ti, int64_t* tj) {
  int64_t i = (int64_t)((sqrt(8.0 * (double)id + 1.0) - 1.0) * 0.5);
  while (i * (i + 1) / 2 > id) --i;
  while ((i + 1) * (i + 2) / 2 <= id) ++i;
  *ti = i;
  *tj = id - i * (i + 1) / 2;
}

// ---------------------------------------------------------------- 256 x 256 tiles
// One CTA per 256 x 256 lower tile: rows I0..I0+255 against rows J0..J0+255.
// Two TMEM accumulators of 128 x 256 FP32 (all 512 columns), D_h for the row
// half h.  K blocks of 32 BF16 (64-byte rows, SWIZZLE_64B); a stage holds
// hi/lo of the 256 I rows and hi/lo of the 256 J rows (4 x 16 KB) and feeds
// 12 MMAs of 128 x 256 x 16 (2 halves x 2 K steps x 3 products).
#define TW_STAGES 3
#define TW_OP_BYTES (TW_BM * TW_BK * 2)              // 16 KB per operand panel
#define TW_STAGE_BYTES (4 * TW_OP_BYTES)             // 64 KB
#define TW_SMEM (TW_STAGES * TW_STAGE_BYTES + 1024)

#define TW_PREFETCH 4

// TMA prefetch of one box into L2 (no shared memory, no completion signal)
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int c0, int c1) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"((uint64_t)map), "r"(c0),
               "r"(c1)
               : "memory");
}

__device__ __forceinline__ uint64_t umma_desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);        // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;               // stride byte offset: 8 rows x 64 B
  d |= (uint64_t)1 << 46;                        // descriptor version (sm_100 family)
  d |= (uint64_t)4 << 61;                        // SWIZZLE_64B
  return d;
}

// kind::f16, BF16 x BF16 -> FP32, K-major, M = 128, N = 256
__device__ __forceinline__ uint32_t idesc_bf16_128x256() {
  uint32_t d = 0;
  d |= 1u << 4;
  d |= 1u << 7;
  d |= 1u << 10;
  d |= (uint32_t)(256 >> 3) << 17;
  d |= (uint32_t)(128 >> 4) << 24;
  return d;
}

// v 2^s as FP64 for the bits b of an FP32 value: FP32 to FP64 is exact and
// the row scales are exact powers of two, so the product is an exponent sum,
// done with integer operations (the FP64 pipe is narrow on this part).  Zero,
// FP32 subnormals and results outside the FP64 normal range take the FP64
// path; the value is the same either way.
__device__ __forceinline__ double f32_scaled(uint32_t b, int s) {
  const int e = (int)((b >> 23) & 0xFFu);
  const int E = e - 127 + 1023 + s;
  if (e == 0 || e == 255 || E <= 0 || E >= 2047) return ldexp((double)__uint_as_float(b), s);
  return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) | ((unsigned long long)E << 52) |
                                          ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

// exponent of an exact power of two (a row scale); rows past M have scale 0
__device__ __forceinline__ int pow2_exp(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF) - 1023;
}

// Epilogue of one 256 x 256 tile: C = s_i s_j acc, plain stores (the
// contraction is the first writer of the tile).  Each warp stages a 32 x 32
// block of FP32 bits through the idle shared-memory ring (transpose) so that
// every store instruction writes 32 consecutive doubles of one row.
__device__ __forceinline__ void tile_epilogue(uint8_t* smem, uint32_t tmem, int warp, int lane, int row_i, int row_j,
                                              int64_t M, const double* __restrict__ rscale, const OutMap& out) {
  uint32_t* stg = (uint32_t*)smem + warp * (32 * 33 + 32);
  int* erow = (int*)(stg + 32 * 33);
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    const int64_t r0 = (int64_t)row_i + 128 * h + warp * 32;
    const int64_t gi = r0 + lane;
    erow[lane] = (gi < M) ? pow2_exp(rscale[gi]) : 0;
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(256 * h + c * 32), v);
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) stg[lane * 33 + jj] = __float_as_uint(v[jj]);
      __syncwarp();
      const int64_t gj = (int64_t)row_j + c * 32 + lane;
      const int ej = (gj < M) ? pow2_exp(rscale[gj]) : 0;
#pragma unroll 4
      for (int rr = 0; rr < 32; ++rr) {
        const int64_t gr = r0 + rr;
        if (gr < M && gj < M && gj <= gr) *out.at(gr, gj) = f32_scaled(stg[rr * 33 + lane], erow[rr] + ej);
      }
      __syncwarp();
    }
  }
}

__global__ void __launch_bounds__(128, 1)
    k_syrk_tc256(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo, int64_t M,
                 int nk, const double* __restrict__ rscale, OutMap out, int* status, const int2* __restrict__ tiles) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[TW_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[TW_STAGES];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;

  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t ti, tj;
  {
    int2 t = tiles[blockIdx.x];  // grouped order: about one wave shares a 12 x 12 block of tiles
    ti = t.x;
    tj = t.y;
  }
  if (tj < 0 || tj > ti || ti * TW_BM >= M) {  // outside the lower triangle: reported, skipped
    if (threadIdx.x == 0) atomicExch(status, 2);
    return;
  }
  int row_i = (int)(ti * TW_BM), row_j = (int)(tj * TW_BM);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < TW_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&acc_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  uint32_t tmem = tmem_base_sh;

  // All CTAs sweep K in the same order so that the ~M/256 CTAs sharing an
  // operand panel read it from L2 at about the same time; the producer also
  // prefetches the K block TW_PREFETCH steps ahead into L2, so the HBM latency
  // is hidden in L2 instead of in the shared-memory ring.
  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int kb = 0; kb < TW_PREFETCH && kb < nk; ++kb) {
      tma_prefetch_2d(&map_hi, 0, (int)((ti * nk + kb) * TW_BM));
      tma_prefetch_2d(&map_lo, 0, (int)((ti * nk + kb) * TW_BM));
      tma_prefetch_2d(&map_hi, 0, (int)((tj * nk + kb) * TW_BM));
      tma_prefetch_2d(&map_lo, 0, (int)((tj * nk + kb) * TW_BM));
    }
    for (int kb = 0; kb < nk; ++kb) {
      int s = kb % TW_STAGES;
      uint32_t ph = (uint32_t)(kb / TW_STAGES) & 1u;
      if (!mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag, status)) break;
      issued = kb + 1;
      uint8_t* st = smem + (size_t)s * TW_STAGE_BYTES;
      mbar_expect_tx(&full_bar[s], TW_STAGE_BYTES);
      int yi = (int)((ti * nk + kb) * TW_BM), yj = (int)((tj * nk + kb) * TW_BM);
      if (kb + TW_PREFETCH < nk) {
        int pi = yi + TW_PREFETCH * TW_BM, pj = yj + TW_PREFETCH * TW_BM;
        tma_prefetch_2d(&map_hi, 0, pi);
        tma_prefetch_2d(&map_lo, 0, pi);
        tma_prefetch_2d(&map_hi, 0, pj);
        tma_prefetch_2d(&map_lo, 0, pj);
      }
      tma_load_2d(&map_hi, &full_bar[s], st + 0 * TW_OP_BYTES, 0, yi);
      tma_load_2d(&map_lo, &full_bar[s], st + 1 * TW_OP_BYTES, 0, yi);
      tma_load_2d(&map_hi, &full_bar[s], st + 2 * TW_OP_BYTES, 0, yj);
      tma_load_2d(&map_lo, &full_bar[s], st + 3 * TW_OP_BYTES, 0, yj);
    }
    if (abort_flag) {
      for (int kb = issued - TW_STAGES < 0 ? 0 : issued - TW_STAGES; kb < issued; ++kb) {
        uint32_t ph = (uint32_t)(kb / TW_STAGES) & 1u;
        for (uint32_t i = 0; i < TC_SPIN_LIMIT && !mbar_try(&full_bar[kb % TW_STAGES], ph); ++i) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16_128x256();
    for (int kb = 0; kb < nk; ++kb) {
      int s = kb % TW_STAGES;
      uint32_t ph = (uint32_t)(kb / TW_STAGES) & 1u;
      if (!mbar_wait(&full_bar[s], ph, &abort_flag, status)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t st = smem_u32(smem + (size_t)s * TW_STAGE_BYTES);
      uint32_t a_hi = st, a_lo = st + TW_OP_BYTES, b_hi = st + 2 * TW_OP_BYTES, b_lo = st + 3 * TW_OP_BYTES;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t dt = tmem + (uint32_t)(256 * h);
        uint32_t aoff = (uint32_t)(h * 128 * 64);  // 128 rows x 64 B into the A panel
#pragma unroll
        for (int k = 0; k < TW_BK / 16; ++k) {
          uint32_t off = k * 32;
          uint32_t first = (kb == 0 && k == 0) ? 0u : 1u;
          umma_bf16(dt, umma_desc_sw64(a_hi + aoff + off), umma_desc_sw64(b_hi + off), idesc, first);
          umma_bf16(dt, umma_desc_sw64(a_hi + aoff + off), umma_desc_sw64(b_lo + off), idesc, 1u);
          umma_bf16(dt, umma_desc_sw64(a_lo + aoff + off), umma_desc_sw64(b_hi + off), idesc, 1u);
        }
      }
      umma_commit(&empty_bar[s]);
    }
    umma_commit(&acc_bar);
  }
  __syncwarp();
  bool have = mbar_wait(&acc_bar, 0u, &abort_flag, status);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (have && !abort_flag) {
    // Epilogue: C = s_i s_j acc (plain stores; this contraction is the first
    // writer of the tile).  Each warp stages a 32 x 32 block through the idle
    // shared-memory ring (transpose) so that every store instruction writes 32
    // consecutive doubles of one row.
    tile_epilogue(smem, tmem, warp, lane, row_i, row_j, M, rscale, out);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// ---------------------------------------------------------------- CTA pairs
// Two CTAs of a 2-CTA cluster compute one 256 x 512 pair tile, the 256 x 256
// lower tiles (I, J) and (I, J + 1), with tcgen05.mma.cta_group::2: M = 256
// rows split over the pair (128 per CTA), N = 256 columns per MMA, of which
// each CTA holds 128 in its own shared memory.  CTA p (p = 0, 1) loads rows
// 128 p .. 128 p + 127 of the row panel I and of the column panels J and
// J + 1 (hi and lo: 48 KB per K block), so a pair reads 96 KB from L2 per K
// block for two tiles where two one-CTA tiles read 128 KB.  CTA p accumulates
// rows 128 p .. 128 p + 127 of both tiles in its TMEM (128 x 512 FP32).  The
// even CTA waits for the copies of both CTAs (they complete on its full
// barrier), issues the MMAs and commits to the empty and accumulator barriers
// of both CTAs.  Pair tiles whose second tile lies above the diagonal load and
// multiply the first tile only.
#define PR_STAGES 4
#define PR_HALF (128 * TW_BK * 2)         // 8 KB: 128 rows x 32 BF16
#define PR_STAGE_BYTES (6 * PR_HALF)      // A hi/lo, B0 hi/lo, B1 hi/lo
#define PR_SMEM (PR_STAGES * PR_STAGE_BYTES + 1024)
#define PR_GROUP 8  // tile rows per launch-order group

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
// TMA load into this CTA's shared memory, completing on a barrier of either
// CTA of the pair
__device__ __forceinline__ void tma_load_2d_pair(const CUtensorMap* map, uint32_t bar, void* dst, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void umma_bf16_pair(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                               uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
// arrive on one barrier (of either CTA) when the pair MMAs issued so far complete
__device__ __forceinline__ void umma_commit_pair(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// kind::f16, BF16 x BF16 -> FP32, K-major, M = 256 (a CTA pair), N = 256
__device__ __forceinline__ uint32_t idesc_bf16_256x256() {
  uint32_t d = 0;
  d |= 1u << 4;
  d |= 1u << 7;
  d |= 1u << 10;
  d |= (uint32_t)(256 >> 3) << 17;
  d |= (uint32_t)(256 >> 4) << 24;
  return d;
}

// Epilogue of this CTA's 128 rows of a pair tile: C = s_i s_j acc for rows
// r_base .. r_base + 127 and the nh column halves of 256 from col0, staged
// through shared memory (transpose) as in tile_epilogue.
__device__ __forceinline__ void pair_epilogue(uint8_t* smem, uint32_t tmem, int warp, int lane, int64_t r_base,
                                              int64_t col0, int nh, int64_t M, const double* __restrict__ rscale,
                                              const OutMap& out) {
  uint32_t* stg = (uint32_t*)smem + warp * (32 * 33 + 32);
  int* erow = (int*)(stg + 32 * 33);
  const int64_t r0 = r_base + warp * 32;
  const int64_t gi = r0 + lane;
  erow[lane] = (gi < M) ? pow2_exp(rscale[gi]) : 0;
#pragma unroll 1
  for (int h = 0; h < nh; ++h) {
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(256 * h + c * 32), v);
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) stg[lane * 33 + jj] = __float_as_uint(v[jj]);
      __syncwarp();
      const int64_t gj = col0 + 256 * h + c * 32 + lane;
      const int ej = (gj < M) ? pow2_exp(rscale[gj]) : 0;
#pragma unroll 4
      for (int rr = 0; rr < 32; ++rr) {
        const int64_t gr = r0 + rr;
        if (gr < M && gj < M && gj <= gr) *out.at(gr, gj) = f32_scaled(stg[rr * 33 + lane], erow[rr] + ej);
      }
      __syncwarp();
    }
  }
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(128, 1)
    k_syrk_pair(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo, int64_t M,
                int nk, const double* __restrict__ rscale, OutMap out, int* status, const int2* __restrict__ pairs) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[PR_STAGES];   // used in the even CTA
  __shared__ __align__(8) uint64_t empty_bar[PR_STAGES];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;
  __shared__ volatile int issued_sh[2];  // even CTA: K blocks issued by itself [0] and by the odd CTA [1]

  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t p = cluster_rank() & 1u;  // 0: the CTA that issues the MMAs
  const int2 pt = pairs[blockIdx.x >> 1];
  const int64_t ti = pt.x, tj = pt.y;
  // an entry of the launch order outside the lower triangle is reported
  // (status 2) and skipped before any barrier, copy or allocation; both CTAs
  // of the pair read the same entry and leave together
  if (tj < 0 || tj > ti || ti * TW_BM >= M) {
    if (threadIdx.x == 0) atomicExch(status, 2);
    return;
  }
  const bool two = tj + 1 <= ti;  // the second tile (ti, tj + 1) is a lower tile
  const int row_i = (int)(ti * TW_BM), row_j = (int)(tj * TW_BM);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    issued_sh[0] = 0;
    issued_sh[1] = 0;
    for (int st = 0; st < PR_STAGES; ++st) {
      mbar_init(&full_bar[st], 1);
      mbar_init(&empty_bar[st], 1);
    }
    mbar_init(&acc_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync_all();  // both CTAs' barriers are initialised before any copy or commit reaches them
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0 && lane == 0) {
    const uint32_t bytes = (uint32_t)((two ? 6 : 4) * PR_HALF * 2);  // both CTAs' copies of one K block
    const int64_t pi = ti * nk, pj0 = tj * nk, pj1 = (tj + 1) * nk;
    const int off = (int)p * 128;
    for (int kb = 0; kb < TW_PREFETCH && kb < nk; ++kb) {
      tma_prefetch_2d(&map_hi, 0, (int)((pi + kb) * TW_BM) + off);
      tma_prefetch_2d(&map_lo, 0, (int)((pi + kb) * TW_BM) + off);
      tma_prefetch_2d(&map_hi, 0, (int)((pj0 + kb) * TW_BM) + off);
      tma_prefetch_2d(&map_lo, 0, (int)((pj0 + kb) * TW_BM) + off);
      if (two) {
        tma_prefetch_2d(&map_hi, 0, (int)((pj1 + kb) * TW_BM) + off);
        tma_prefetch_2d(&map_lo, 0, (int)((pj1 + kb) * TW_BM) + off);
      }
    }
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int st = kb % PR_STAGES;
      const uint32_t ph = (uint32_t)(kb / PR_STAGES) & 1u;
      if (!mbar_wait(&empty_bar[st], ph ^ 1u, &abort_flag, status)) break;
      issued = kb + 1;
      if (p == 0) mbar_expect_tx(&full_bar[st], bytes);
      const uint32_t fb = cluster_addr(&full_bar[st], 0);
      uint8_t* sp = smem + (size_t)st * PR_STAGE_BYTES;
      const int yi = (int)((pi + kb) * TW_BM) + off, yj0 = (int)((pj0 + kb) * TW_BM) + off,
                yj1 = (int)((pj1 + kb) * TW_BM) + off;
      if (kb + TW_PREFETCH < nk) {
        tma_prefetch_2d(&map_hi, 0, yi + TW_PREFETCH * TW_BM);
        tma_prefetch_2d(&map_lo, 0, yi + TW_PREFETCH * TW_BM);
        tma_prefetch_2d(&map_hi, 0, yj0 + TW_PREFETCH * TW_BM);
        tma_prefetch_2d(&map_lo, 0, yj0 + TW_PREFETCH * TW_BM);
        if (two) {
          tma_prefetch_2d(&map_hi, 0, yj1 + TW_PREFETCH * TW_BM);
          tma_prefetch_2d(&map_lo, 0, yj1 + TW_PREFETCH * TW_BM);
        }
      }
      tma_load_2d_pair(&map_hi, fb, sp + 0 * PR_HALF, 0, yi);
      tma_load_2d_pair(&map_lo, fb, sp + 1 * PR_HALF, 0, yi);
      tma_load_2d_pair(&map_hi, fb, sp + 2 * PR_HALF, 0, yj0);
      tma_load_2d_pair(&map_lo, fb, sp + 3 * PR_HALF, 0, yj0);
      if (two) {
        tma_load_2d_pair(&map_hi, fb, sp + 4 * PR_HALF, 0, yj1);
        tma_load_2d_pair(&map_lo, fb, sp + 5 * PR_HALF, 0, yj1);
      }
    }
    // the even CTA learns how many K blocks each CTA issued (for the drain)
    if (p == 0) {
      issued_sh[0] = issued;
    } else {
      asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr((const void*)&issued_sh[1], 0)),
                   "r"(issued)
                   : "memory");
    }
    // wait until the MMAs have released the last use of every stage: no
    // commit of the even CTA reaches this CTA's barriers after that
    for (int kb = issued; kb < issued + PR_STAGES && !abort_flag; ++kb) {
      if (kb < PR_STAGES) continue;  // stage never used
      const int st = kb % PR_STAGES;
      const uint32_t ph = (uint32_t)(kb / PR_STAGES) & 1u;
      if (!mbar_wait(&empty_bar[st], ph ^ 1u, &abort_flag, status)) break;
    }
  } else if (warp == 1 && lane == 0 && p == 0) {
    const uint32_t idesc = idesc_bf16_256x256();
    const uint32_t empty_peer0 = cluster_addr(&empty_bar[0], 1), acc_peer = cluster_addr(&acc_bar, 1);
    for (int kb = 0; kb < nk; ++kb) {
      const int st = kb % PR_STAGES;
      const uint32_t ph = (uint32_t)(kb / PR_STAGES) & 1u;
      if (!mbar_wait(&full_bar[st], ph, &abort_flag, status)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(smem + (size_t)st * PR_STAGE_BYTES);
      const uint32_t a_hi = sa, a_lo = sa + PR_HALF;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !two) break;
        const uint32_t dt = tmem + (uint32_t)(256 * h);
        const uint32_t b_hi = sa + (2 + 2 * h) * PR_HALF, b_lo = b_hi + PR_HALF;
#pragma unroll
        for (int k = 0; k < TW_BK / 16; ++k) {
          const uint32_t o = k * 32;
          const uint32_t first = (kb == 0 && k == 0) ? 0u : 1u;
          umma_bf16_pair(dt, umma_desc_sw64(a_hi + o), umma_desc_sw64(b_hi + o), idesc, first);
          umma_bf16_pair(dt, umma_desc_sw64(a_hi + o), umma_desc_sw64(b_lo + o), idesc, 1u);
          umma_bf16_pair(dt, umma_desc_sw64(a_lo + o), umma_desc_sw64(b_hi + o), idesc, 1u);
        }
      }
      umma_commit_pair(smem_u32(&empty_bar[st]));
      umma_commit_pair(empty_peer0 + 8u * (uint32_t)st);
    }
    umma_commit_pair(smem_u32(&acc_bar));
    umma_commit_pair(acc_peer);
  }
  __syncwarp();
  const bool have = mbar_wait(&acc_bar, 0u, &abort_flag, status);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (have && !abort_flag && *(volatile int*)status == 0)
    pair_epilogue(smem, tmem, warp, lane, (int64_t)row_i + 128 * p, row_j, two ? 2 : 1, M, rscale, out);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync_all();  // both CTAs are past their MMAs, copies and epilogues
  if (p == 0 && threadIdx.x == 0 && *(volatile int*)status != 0) {
    // bounded drain of copies that may still be in flight after an expired wait
    const int n = issued_sh[0] > issued_sh[1] ? issued_sh[0] : issued_sh[1];
    for (int kb = n - PR_STAGES < 0 ? 0 : n - PR_STAGES; kb < n; ++kb) {
      const uint32_t ph = (uint32_t)(kb / PR_STAGES) & 1u;
      for (uint32_t i = 0; i < (1u << 16) && !mbar_try(&full_bar[kb % PR_STAGES], ph); ++i) {
      }
    }
  }
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  cluster_sync_all();  // no CTA leaves while its peer may still reach it
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 wl_encode_tiled() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (PFN_cuTensorMapEncodeTiled_v12000)p;
    return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
  }();
  return fn;
}
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() { return wl_encode_tiled(); }

// 2D view of the blocked array: inner dimension 32 (64 B rows), outer
// dimension ntiles * nk * 256 block rows; box 32 x 256 = one 16 KB block
static int make_map(cov_handle* h, CUtensorMap* map, void* base, int64_t rows, int64_t kp, int box_rows = TW_BM) {
  auto fn = encode_fn();
  if (!fn) return wl_fail(h, COV_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  int64_t ntiles = (rows + TW_BM - 1) / TW_BM;
  cuuint64_t dims[2] = {(cuuint64_t)TW_BK, (cuuint64_t)(ntiles * (kp / TW_BK) * TW_BM)};
  cuuint64_t strides[1] = {(cuuint64_t)TW_BK * 2};
  cuuint32_t box[2] = {(cuuint32_t)TW_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return wl_fail(h, COV_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return COV_OK;
}

static inline int kpad(int K) { return (K + 63) / 64 * 64; }
int wl_kpad(int K) { return kpad(K); }

// bytes of one split array: rows padded to whole 256-row tiles (zero rows)
int wl_split_bytes(int64_t M, int K, size_t* bytes) {
  *bytes = (size_t)((M + TW_BM - 1) / TW_BM) * TW_BM * kpad(K) * 2;
  return COV_OK;
}

// the rows past M in the last 256-row tile must read as zero
static int zero_last_tile(cov_handle* h, void* base, int64_t rows, int K, cudaStream_t s) {
  if (rows % TW_BM == 0) return COV_OK;
  int64_t nk = kpad(K) / TW_BK;
  int64_t first = ((rows / TW_BM) * nk) * (int64_t)TW_BM * TW_BK;
  WL_CHECK(h, cudaMemsetAsync((uint16_t*)base + first, 0, (size_t)nk * TW_BM * TW_BK * 2, s));
  return COV_OK;
}

int wl_rows_split(cov_handle* h, int nssc, cudaStream_t s) {
  int Kt = h->K + nssc;
  int nsig = h->nl + h->ntri;
  int rc;
  if ((rc = wl_ensure(h, (void**)&h->Fsig, sizeof(float) * (size_t)nsig * h->K, "row signature table"))) return rc;
  if ((rc = wl_ensure(h, (void**)&h->Esig, sizeof(int) * (size_t)nsig * h->nchi, "row signature exponents")))
    return rc;
  if ((rc = wl_ensure(h, (void**)&h->Msig, sizeof(double) * (size_t)nsig * h->nchi, "row signature maxima")))
    return rc;
  if ((rc = zero_last_tile(h, h->Ahi, h->M, Kt, s))) return rc;
  if ((rc = zero_last_tile(h, h->Alo, h->M, Kt, s))) return rc;
  k_rows_prep<<<(h->K + 255) / 256, 256, 0, s>>>(h->nchi, h->nm, 1.0 / h->omega, h->cosmo_d, h->chi, h->wchi,
                                                 h->m, h->om, h->f, h->G2, h->G3, h->C2, h->C3);
  WL_LAUNCH(h, "k_rows_prep");
  k_rows_sig<<<dim3((unsigned)nsig, (unsigned)h->nchi), 128, 0, s>>>(h->nl, h->ntri, h->nchi, h->nm, h->tris_d, h->U,
                                                                     h->G2, h->G3, h->C2, h->C3, h->Fsig, h->Esig,
                                                                     h->Msig, 0);
  WL_LAUNCH(h, "k_rows_sig");
  size_t smem = (size_t)h->nchi * (2 * sizeof(double) + 2 * sizeof(float));  // <= 96 KB for N_chi <= 4096
  static std::once_flag attr_once[WL_MAX_DEVICES];
  static int attr_rc[WL_MAX_DEVICES];
  if (wl_once_per_device(attr_once, attr_rc, [] {
        return (int)cudaFuncSetAttribute(k_rows_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         4096 * (2 * sizeof(double) + 2 * sizeof(float)));
      }) != 0)
    return wl_fail(h, COV_ERR_CUDA, "cudaFuncSetAttribute(k_rows_split) failed");
  k_rows_split<<<(unsigned)h->M, 256, smem, s>>>(h->M, h->nl, h->nchi, h->nm, kpad(Kt), nssc, h->rowdesc_d, h->W,
                                                  h->Fsig, h->Esig, h->Msig, h->wchi, h->sigw2, h->chi, h->RP3,
                                                  h->RB3, (__nv_bfloat16*)h->Ahi, (__nv_bfloat16*)h->Alo,
                                                  (double*)h->Ascale);
  WL_LAUNCH(h, "k_rows_split");
  return COV_OK;
}

// BF16 hi/lo trispectrum rows straight from the pair signatures (no FP64
// row array): the PT term's table T = rows rows^T in the split form.
int wl_trows_split(cov_handle* h, cudaStream_t s) {
  int npair = h->nl * (h->nl + 1) / 2;
  int rc;
  if ((rc = wl_ensure(h, (void**)&h->FsigT, sizeof(float) * (size_t)npair * h->K, "pair signature table")))
    return rc;
  if ((rc = wl_ensure(h, (void**)&h->EsigT, sizeof(int) * (size_t)npair * h->nchi, "pair signature exponents")))
    return rc;
  if ((rc = wl_ensure(h, (void**)&h->MsigT, sizeof(double) * (size_t)npair * h->nchi, "pair signature maxima")))
    return rc;
  if ((rc = wl_ensure(h, (void**)&h->G2, sizeof(double) * h->K, "row factor table"))) return rc;
  if ((rc = wl_ensure(h, (void**)&h->G3, sizeof(double) * h->K, "row factor table"))) return rc;
  if ((rc = wl_ensure(h, (void**)&h->C2, sizeof(double) * h->nchi, "row factor table"))) return rc;
  if ((rc = wl_ensure(h, (void**)&h->C3, sizeof(double) * h->nchi, "row factor table"))) return rc;
  if ((rc = zero_last_tile(h, h->Thi, h->ntrow, h->K, s))) return rc;
  if ((rc = zero_last_tile(h, h->Tlo, h->ntrow, h->K, s))) return rc;
  k_rows_prep<<<(h->K + 255) / 256, 256, 0, s>>>(h->nchi, h->nm, 1.0 / h->omega, h->cosmo_d, h->chi, h->wchi,
                                                 h->m, h->om, h->f, h->G2, h->G3, h->C2, h->C3);
  WL_LAUNCH(h, "k_rows_prep");
  k_rows_sig<<<dim3((unsigned)npair, (unsigned)h->nchi), 128, 0, s>>>(h->nl, h->ntri, h->nchi, h->nm, h->tris_d, h->U,
                                                                      h->G2, h->G3, h->C2, h->C3, h->FsigT, h->EsigT,
                                                                      h->MsigT, 1);
  WL_LAUNCH(h, "k_rows_sig");
  size_t smem = (size_t)h->nchi * (sizeof(double) + sizeof(float));
  k_trows_split<<<(unsigned)h->ntrow, 256, smem, s>>>(h->ntrow, h->nleg, h->nt, h->nl, h->nchi, h->nm, kpad(h->K),
                                                       sqrt(h->omega), h->W, h->FsigT, h->EsigT, h->MsigT,
                                                       (__nv_bfloat16*)h->Thi, (__nv_bfloat16*)h->Tlo, h->Tscale);
  WL_LAUNCH(h, "k_trows_split");
  return COV_OK;
}

// C (lower, FP64) = (hi + lo)(hi + lo)^T scaled, without the lo lo^T term
// Launch orders, cached per (tile-row range, kind).  kind 0: the lower tiles
// (ti, tj), tj <= ti, of tile rows [t0, t1), row by row.  kind 1: the pair
// tiles (ti, tj), tj even, each covering the lower tiles (ti, tj) and
// (ti, tj + 1) (the second only when tj + 1 <= ti).
int wl_tile_order(cov_handle* h, int kind, int64_t t0, int64_t t1, const int2** tiles, int64_t* n, cudaStream_t s) {
  const int group = kind == 1 ? h->pr_group : 0;
  for (auto& c : h->tile_cache)
    if (c.p && c.kind == kind && c.group == group && c.t0 == t0 && c.t1 == t1) {
      *tiles = c.p;
      *n = c.n;
      return COV_OK;
    }
  std::vector<int2> v;
  if (kind == 0) {
    for (int64_t ti = t0; ti < t1; ++ti)
      for (int64_t tj = 0; tj <= ti; ++tj) v.push_back(make_int2((int)ti, (int)tj));
  } else {
    // groups of `group` tile rows (PR_GROUP unless tuned); inside a group,
    // column pair by column pair, so the ~76 pairs of one wave share a few row
    // and column panels in L2
    for (int64_t g0 = t0; g0 < t1; g0 += group) {
      int64_t g1 = std::min<int64_t>(g0 + group, t1);
      for (int64_t j0 = 0; j0 < g1; j0 += 2)
        for (int64_t i = g0; i < g1; ++i)
          if (j0 <= i) v.push_back(make_int2((int)i, (int)j0));
    }
  }
  // One allocation for the whole ring, sized for the largest matrix of the
  // handle, so that no entry is ever freed: launches of one band call use
  // fewer than WL_TILE_CACHE entries and may still be in flight when the next
  // entry is written; band calls end with a stream synchronisation.
  if (!h->tile_ring) {
    int64_t t = (std::max<int64_t>(h->M, h->ntrow) + 255) / 256 + 1;
    h->tile_ring_cap = (size_t)(t * (t + 1) / 2);
    size_t bytes = sizeof(int2) * h->tile_ring_cap * WL_TILE_CACHE;
    WL_CHECK(h, cudaMalloc(&h->tile_ring, bytes));
    h->allocated += bytes;
    for (int k = 0; k < WL_TILE_CACHE; ++k) h->tile_cache[k].p = nullptr;
  }
  if (v.size() > h->tile_ring_cap) return wl_fail(h, COV_ERR_INVALID, "launch order larger than its ring slot");
  // a captured step reuses the orders of its eager first run: a copy from
  // host memory cannot become part of a graph
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  WL_CHECK(h, cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return wl_fail(h, COV_ERR_INVALID, "contraction launch order not built before stream capture");
  int slot = h->tile_cache_next;
  h->tile_cache_next = (h->tile_cache_next + 1) % WL_TILE_CACHE;
  auto& c = h->tile_cache[slot];
  c.p = h->tile_ring + (size_t)slot * h->tile_ring_cap;
  // On the stream of the launches that read it: ordered after the earlier
  // readers of this slot and before the next ones.  (A synchronous copy goes
  // through the legacy default stream, which a non-blocking stream does not
  // wait for: a kernel could read the slot before the copy lands.)  The copy
  // from pageable memory is staged before the call returns, so v may go.
  WL_CHECK(h, cudaMemcpyAsync(c.p, v.data(), sizeof(int2) * v.size(), cudaMemcpyHostToDevice, s));
  c.kind = kind;
  c.group = group;
  c.t0 = t0;
  c.t1 = t1;
  c.n = (int64_t)v.size();
  *tiles = c.p;
  *n = c.n;
  return COV_OK;
}

// Whether CTA pairs of the pair kernel can be resident on this device.
static int pair_clusters_ok() {
  static std::once_flag once[WL_MAX_DEVICES];
  static int ok[WL_MAX_DEVICES];
  int d = 0;
  cudaGetDevice(&d);
  if (d < 0 || d >= WL_MAX_DEVICES) return 0;
  std::call_once(once[d], [&] {
    ok[d] = 0;
    if (cudaFuncSetAttribute(k_syrk_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, PR_SMEM) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = PR_SMEM;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (void*)k_syrk_pair, &cfg) == cudaSuccess && n > 0) ok[d] = n;
    cudaGetLastError();
  });
  return ok[d];
}

// Launch the contraction over tile rows [r0, row1) of out's band (no status
// handling): CTA pairs when 2-CTA clusters can be placed, else one CTA per
// tile.
static int launch_tc(cov_handle* h, const void* hi, const void* lo, const double* rscale, int64_t rows, int Kp,
                     OutMap out, int64_t r0, int64_t row1, cudaStream_t s) {
  int rc;
  if (row1 < 0 || row1 > rows) row1 = rows;
  int64_t t0 = r0 / TW_BM, t1 = (row1 + TW_BM - 1) / TW_BM;
  if (t1 <= t0) return COV_OK;
  const int2* tiles = nullptr;
  int64_t nblk = 0;
  if (h->tc_kernel != 0 && pair_clusters_ok()) {
    CUtensorMap mhi, mlo;
    if ((rc = make_map(h, &mhi, (void*)hi, rows, Kp, 128))) return rc;
    if ((rc = make_map(h, &mlo, (void*)lo, rows, Kp, 128))) return rc;
    if ((rc = wl_tile_order(h, 1, t0, t1, &tiles, &nblk, s))) return rc;
    k_syrk_pair<<<(unsigned)(2 * nblk), 128, PR_SMEM, s>>>(mhi, mlo, rows, Kp / TW_BK, rscale, out, h->tc_status,
                                                           tiles);
    WL_LAUNCH(h, "k_syrk_pair");
  } else {
    CUtensorMap mhi, mlo;
    if ((rc = make_map(h, &mhi, (void*)hi, rows, Kp))) return rc;
    if ((rc = make_map(h, &mlo, (void*)lo, rows, Kp))) return rc;
    static std::once_flag attr_once[WL_MAX_DEVICES];
    static int attr_rc[WL_MAX_DEVICES];
    if (wl_once_per_device(attr_once, attr_rc, [] {
          return (int)cudaFuncSetAttribute(k_syrk_tc256, cudaFuncAttributeMaxDynamicSharedMemorySize, TW_SMEM);
        }) != 0)
      return wl_fail(h, COV_ERR_CUDA, "cudaFuncSetAttribute(k_syrk_tc256) failed");
    if ((rc = wl_tile_order(h, 0, t0, t1, &tiles, &nblk, s))) return rc;
    k_syrk_tc256<<<(unsigned)nblk, 128, TW_SMEM, s>>>(mhi, mlo, rows, Kp / TW_BK, rscale, out, h->tc_status, tiles);
    WL_LAUNCH(h, "k_syrk_tc256");
  }
  return COV_OK;
}

// The contraction kernels raise a device status word when a bounded wait
// expires; it is cleared before a group of launches and read after them.
int wl_tc_status_reset(cov_handle* h, cudaStream_t s) {
  if (h->deferred) return COV_OK;  // inside a captured batch step the word accumulates over replays
  if (!h->tc_status) {
    WL_CHECK(h, cudaMalloc(&h->tc_status, sizeof(int)));
    h->allocated += sizeof(int);
  }
  WL_CHECK(h, cudaMemsetAsync(h->tc_status, 0, sizeof(int), s));
  return COV_OK;
}

int wl_tc_status_check(cov_handle* h, cudaStream_t s) {
  if (h->deferred) return COV_OK;  // read by the batch driver after the replays
  int st = 0;
  WL_CHECK(h, cudaMemcpyAsync(&st, h->tc_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  WL_CHECK(h, cudaStreamSynchronize(s));
  if (st == 2) return wl_fail(h, COV_ERR_CUDA, "tensor-core contraction: launch order entry out of range");
  if (st) return wl_fail(h, COV_ERR_TIMEOUT, "tensor-core contraction: a bounded mbarrier wait expired");
  return COV_OK;
}

int wl_syrk_tc_rows(cov_handle* h, const void* hi, const void* lo, const double* rscale, int64_t rows, int Kp,
                    OutMap out, cudaStream_t s, int64_t row1) {
  int rc;
  if ((rc = wl_tc_status_reset(h, s))) return rc;
  if ((rc = launch_tc(h, hi, lo, rscale, rows, Kp, out, out.row0, row1, s))) return rc;
  return wl_tc_status_check(h, s);
}

int wl_syrk_tc(cov_handle* h, int nssc, OutMap out, cudaStream_t s, int64_t row1) {
  return wl_syrk_tc_rows(h, h->Ahi, h->Alo, h->Ascale, h->M, kpad(h->K + nssc), out, s, row1);
}

// 1-halo (+ SSC) contraction of rows [r0, r1) into out, launch only
int wl_syrk_tc_part(cov_handle* h, int nssc, OutMap out, int64_t r0, int64_t r1, cudaStream_t s) {
  return launch_tc(h, h->Ahi, h->Alo, h->Ascale, h->M, kpad(h->K + nssc), out, r0, r1, s);
}

