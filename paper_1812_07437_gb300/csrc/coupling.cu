// Exact bin-averaged couplings of the BB+PT terms (App. B: the binned
// bispectrum estimator; Eq. CovBB), built once per binning.
//
// A BB or PT Wick term joins leg x of triangle bin tau to leg y of tau' in the
// same ell bin A.  With the polyspectra constant over the bins its exact
// coupling is kappa = sum_{q in A} n_{tau,x}(q) n_{tau',y}(q) / (N_tau N_tau'),
// n_{tau,x}(q) = #{p in Y : q + p in Z} the lattice triangles of tau whose leg
// x is the mode q, {Y, Z} the bins of the two other legs.  n depends on
// (A; {Y, Z}) only, so bin A has one column per such pair.
//
//  * k_leg_counts  n_c(q) for every column c of bin A and every q of A's
//                  fundamental domain 0 <= y <= x (the eight symmetries of
//                  the square map the lattice and the annuli onto
//                  themselves, so n is constant on an orbit; orbit weight 4
//                  on the axis and the diagonal, else 8).  One thread per
//                  (q, c): for each row of p the admissible x of p form at
//                  most 2 x 2 integer intervals, intersected exactly (the row
//                  tables of counts.cu).  Column-major int32 matrix Nm[c][q],
//                  with the weighted column sums (= N_tri, checked).
//  * k_gram        G[c][c'] = sum_q w_q Nm[c][q] Nm[c'][q], exact in unsigned
//                  64-bit, lower half: 32 x 32 output tiles per block over
//                  chunks of orbits, partial sums added atomically (all terms
//                  >= 0), with an FP64 shadow of each sum.  The entries come
//                  close to 2^63 at l_max = 5000 (cfg2_5bin: 2^62.7).
//  * k_kappa       kappa[c][c'] = G / (N_tri(c) N_tri(c')) in FP64, both
//                  halves; an entry at or beyond 2^63 (by its shadow) is an
//                  error.
#include <algorithm>

#include "common.cuh"

namespace {

struct ColDesc {  // one column of a bin: the other two legs' bins and radii
  int Y, Z, rY, rZ;
};

constexpr int LC_THREADS = 128;
constexpr int64_t GRAM_CHUNK = 4096;  // orbits per k_gram block

int64_t isqrt_host(int64_t v) {
  if (v <= 0) return 0;
  int64_t r = (int64_t)sqrt((double)v);
  while (r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

__device__ __forceinline__ int intervals_of(int2 row, int* lo, int* hi) {
  const int xo = row.x, xi = row.y;
  if (xo < 0 || xi > xo) return 0;
  if (xi == 0) {
    lo[0] = -xo;
    hi[0] = xo;
    return 1;
  }
  lo[0] = -xo;
  hi[0] = -xi;
  lo[1] = xi;
  hi[1] = xo;
  return 2;
}

__global__ void __launch_bounds__(LC_THREADS) k_leg_counts(int rmax, const int32_t* __restrict__ tab,
                                                           const int2* __restrict__ orb, int64_t norb,
                                                           const ColDesc* __restrict__ cols, int32_t* Nm,
                                                           unsigned long long* colsum) {
  extern __shared__ int2 rows_sh[];  // [2][rmax + 1]: rows (x_outer, x_inner) of Y and Z
  __shared__ unsigned long long wsh[LC_THREADS / 32];
  const int c = blockIdx.y;
  const ColDesc cd = cols[c];
  const size_t stride = (size_t)rmax + 1;
  for (int y = threadIdx.x; y <= rmax; y += blockDim.x) {
    rows_sh[y] = make_int2(tab[((size_t)cd.Y * 2 + 0) * stride + y], tab[((size_t)cd.Y * 2 + 1) * stride + y]);
    rows_sh[stride + y] =
        make_int2(tab[((size_t)cd.Z * 2 + 0) * stride + y], tab[((size_t)cd.Z * 2 + 1) * stride + y]);
  }
  __syncthreads();
  const int2* ry = rows_sh;
  const int2* rz = rows_sh + stride;
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long ws = 0;
  if (o < norb) {
    const int2 q = orb[o];
    const int x1 = q.x, y1 = q.y;
    // rows y2 of p with |y2| <= rY and |y1 + y2| <= rZ
    const int ylo = max(-cd.rY, -y1 - cd.rZ), yhi = min(cd.rY, -y1 + cd.rZ);
    int64_t n = 0;
    for (int y2 = ylo; y2 <= yhi; ++y2) {
      int plo[2], phi[2], zlo[2], zhi[2];
      const int np = intervals_of(ry[y2 < 0 ? -y2 : y2], plo, phi);
      if (np == 0) continue;
      const int yz = y1 + y2;
      const int nz = intervals_of(rz[yz < 0 ? -yz : yz], zlo, zhi);
      for (int i = 0; i < np; ++i)
        for (int j = 0; j < nz; ++j) {
          const int lo = max(plo[i], zlo[j] - x1), hi = min(phi[i], zhi[j] - x1);
          if (hi >= lo) n += hi - lo + 1;
        }
    }
    Nm[(size_t)c * norb + o] = (int32_t)n;  // n <= N(Y) < 2^31 (checked on the host)
    ws = (unsigned long long)n * ((y1 == 0 || y1 == x1) ? 4ull : 8ull);
  }
  ws = warp_sum(ws);
  if ((threadIdx.x & 31) == 0) wsh[threadIdx.x >> 5] = ws;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int k = 0; k < LC_THREADS / 32; ++k) t += wsh[k];
    if (t) atomicAdd(&colsum[c], t);
  }
}

__global__ void __launch_bounds__(256) k_gram(const int32_t* __restrict__ Nm, const int2* __restrict__ orb,
                                              int64_t norb, int ncol, unsigned long long* G, double* Gf) {
  __shared__ int32_t sa[32][33], sb[32][33];
  __shared__ int ssh[32];
  // lower tile (ti, tj), ti >= tj, of the ncol x ncol output
  const int64_t id = blockIdx.x;
  int64_t ti = (int64_t)((sqrt(8.0 * (double)id + 1.0) - 1.0) * 0.5);
  while (ti * (ti + 1) / 2 > id) --ti;
  while ((ti + 1) * (ti + 2) / 2 <= id) ++ti;
  const int64_t tj = id - ti * (ti + 1) / 2;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  unsigned long long acc[4] = {0, 0, 0, 0};
  double accf[4] = {0.0, 0.0, 0.0, 0.0};  // FP64 shadow of the same sums: detects an entry beyond 2^63
  const int64_t o0 = (int64_t)blockIdx.y * GRAM_CHUNK, o1 = min(norb, o0 + GRAM_CHUNK);
  for (int64_t ob = o0; ob < o1; ob += 32) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      const int i = e >> 5, j = e & 31;
      const int64_t o = ob + j;
      const int64_t r = ti * 32 + i, c = tj * 32 + i;
      sa[i][j] = (r < ncol && o < o1) ? Nm[(size_t)r * norb + o] : 0;
      sb[i][j] = (c < ncol && o < o1) ? Nm[(size_t)c * norb + o] : 0;
    }
    if (threadIdx.x < 32) {
      const int64_t o = ob + threadIdx.x;
      int sh = 0;
      if (o < o1) {
        const int2 q = orb[o];
        sh = (q.y == 0 || q.y == q.x) ? 2 : 3;  // orbit weight 4 or 8
      }
      ssh[threadIdx.x] = sh;
    }
    __syncthreads();
#pragma unroll 4
    for (int j = 0; j < 32; ++j) {
      const unsigned long long b = (unsigned)sb[tx][j];
      const int sh = ssh[j];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const unsigned long long p = ((unsigned long long)(unsigned)sa[ty + 8 * k][j] * b) << sh;
        acc[k] += p;
        accf[k] += (double)p;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t r = ti * 32 + ty + 8 * k, c = tj * 32 + tx;
    if (r < ncol && c < ncol && r >= c && acc[k] != 0) {
      atomicAdd(&G[(size_t)r * ncol + c], acc[k]);
      atomicAdd(&Gf[(size_t)r * ncol + c], accf[k]);
    }
  }
}

// kappa = G / (N_tri N_tri'); an entry whose 64-bit sum wrapped or reached
// 2^63 (its FP64 shadow disagrees, or is that large) raises *bad
__global__ void k_kappa(int ncol, const unsigned long long* __restrict__ G, const double* __restrict__ Gf,
                        const int32_t* __restrict__ ctri, const int64_t* __restrict__ Ntri, double* kap, int* bad) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)ncol * ncol) return;
  const int r = (int)(idx / ncol), c = (int)(idx % ncol);
  const size_t l = r >= c ? (size_t)r * ncol + c : (size_t)c * ncol + r;
  const unsigned long long g = G[l];
  const double gf = Gf[l];
  if (gf >= 9.2e18 || g >= (1ull << 63) || fabs(__ull2double_rn(g) - gf) > 1e-9 * gf) atomicExch(bad, 1);
  kap[idx] = __ll2double_rn((long long)g) / (__ll2double_rn(Ntri[ctri[r]]) * __ll2double_rn(Ntri[ctri[c]]));
}

struct DevTmp {  // transient device buffer, freed on scope exit
  void* p = nullptr;
  ~DevTmp() {
    if (p) cudaFree(p);
  }
};

}  // namespace

void wl_coupling_plan(cov_handle* h) {
  const int nl = h->nl, ntri = h->ntri;
  std::vector<std::vector<std::pair<int, int>>> cols(nl);
  std::vector<std::vector<int>> ctri(nl);
  h->kcol_h.assign((size_t)3 * ntri, 0);
  for (int t = 0; t < ntri; ++t) {
    const int32_t* tr = &h->tris[3 * (size_t)t];
    for (int x = 0; x < 3; ++x) {
      const int A = tr[x];
      int Y = tr[(x + 1) % 3], Z = tr[(x + 2) % 3];
      if (Y > Z) std::swap(Y, Z);
      auto& v = cols[A];
      int k = (int)(std::find(v.begin(), v.end(), std::make_pair(Y, Z)) - v.begin());
      if (k == (int)v.size()) {
        v.emplace_back(Y, Z);
        ctri[A].push_back(t);
      }
      h->kcol_h[3 * (size_t)t + x] = k;
    }
  }
  h->kn_h.assign(nl, 0);
  h->koff_h.assign(nl + 1, 0);
  h->kcoff_h.assign(nl + 1, 0);
  h->kyz_h.clear();
  h->ktri_h.clear();
  for (int A = 0; A < nl; ++A) {
    const int n = (int)cols[A].size();
    h->kn_h[A] = n;
    h->koff_h[A + 1] = h->koff_h[A] + (int64_t)n * n;
    h->kcoff_h[A + 1] = h->kcoff_h[A] + n;
    for (int k = 0; k < n; ++k) {
      h->kyz_h.push_back(cols[A][k].first);
      h->kyz_h.push_back(cols[A][k].second);
      h->ktri_h.push_back(ctri[A][k]);
    }
  }
}

size_t wl_coupling_bytes(const cov_handle* h) {
  if (h->coupling != COV_COUPLING_EXACT || h->koff_h.empty()) return 0;
  const size_t sq = (size_t)h->koff_h.back();
  return sq * (sizeof(double) + sizeof(unsigned long long)) + 4 * 3 * (size_t)h->ntri + 4 * (size_t)h->nl +
         8 * (size_t)(h->nl + 1);
}

int wl_couplings(cov_handle* h, cudaStream_t s) {
  if (h->coupling != COV_COUPLING_EXACT || h->kap) return COV_OK;
  if (h->ntri == 0) return COV_OK;
  wl_coupling_plan(h);
  const int nl = h->nl;
  // fundamental-domain orbits of every bin: 0 <= y <= x, s_lo <= x^2 + y^2 < s_hi
  std::vector<int2> orb;
  std::vector<int64_t> ooff(nl + 1, 0);
  for (int A = 0; A < nl; ++A) {
    const int64_t lo = h->s_lo[A], hi = h->s_hi[A];
    const int64_t R = isqrt_host(hi - 1);
    for (int64_t x = 0; x <= R; ++x) {
      const int64_t x2 = x * x;
      if (x2 >= hi || 2 * x2 < lo) continue;
      int64_t y0 = lo - x2 <= 0 ? 0 : isqrt_host(lo - x2 - 1) + 1;  // smallest y with x^2 + y^2 >= lo
      int64_t y1 = std::min<int64_t>(x, isqrt_host(hi - 1 - x2));  // largest y <= x with x^2 + y^2 < hi
      for (int64_t y = y0; y <= y1; ++y) orb.push_back(make_int2((int)x, (int)y));
    }
    ooff[A + 1] = (int64_t)orb.size();
  }
  const int64_t ncol_all = h->kcoff_h[nl], sq = h->koff_h[nl];
  // a leg count is at most the lattice points of one annulus, < 3.2 (rmax + 1)^2
  if (3.2 * ((double)h->rmax + 1.0) * ((double)h->rmax + 1.0) >= 2147483647.0)
    return wl_fail(h, COV_ERR_INVALID, "exact couplings: l_max / l_f too large for 32-bit leg counts");
  std::vector<ColDesc> cd((size_t)ncol_all);
  for (int64_t k = 0; k < ncol_all; ++k) {
    const int Y = h->kyz_h[2 * k], Z = h->kyz_h[2 * k + 1];
    cd[k] = ColDesc{Y, Z, (int)isqrt_host(h->s_hi[Y] - 1), (int)isqrt_host(h->s_hi[Z] - 1)};
  }
  size_t nm_bytes = 4;
  for (int A = 0; A < nl; ++A)
    nm_bytes = std::max(nm_bytes, (size_t)4 * (size_t)(ooff[A + 1] - ooff[A]) * (size_t)h->kn_h[A]);
  const size_t resident = wl_coupling_bytes(h);
  const size_t transient = nm_bytes + sizeof(int2) * orb.size() + sizeof(ColDesc) * cd.size() +
                           (8 + 4) * (size_t)ncol_all + 8 * (size_t)sq;
  if (h->budget && h->allocated + resident + transient > h->budget)
    return wl_fail(h, COV_ERR_NOMEM, "hbm_budget exceeded by the exact couplings");
  DevTmp d_orb, d_cd, d_nm, d_sum, d_ctri, d_gf, d_bad;
  WL_CHECK(h, cudaMalloc(&d_orb.p, sizeof(int2) * std::max<size_t>(orb.size(), 1)));
  WL_CHECK(h, cudaMalloc(&d_cd.p, sizeof(ColDesc) * (size_t)ncol_all));
  WL_CHECK(h, cudaMalloc(&d_nm.p, nm_bytes));
  WL_CHECK(h, cudaMalloc(&d_sum.p, 8 * (size_t)ncol_all));
  WL_CHECK(h, cudaMalloc(&d_ctri.p, 4 * (size_t)ncol_all));
  WL_CHECK(h, cudaMalloc(&d_gf.p, 8 * (size_t)sq));
  WL_CHECK(h, cudaMalloc(&d_bad.p, sizeof(int)));
  WL_CHECK(h, cudaMalloc(&h->kgram, 8 * (size_t)sq));
  WL_CHECK(h, cudaMalloc(&h->kap, 8 * (size_t)sq));
  WL_CHECK(h, cudaMalloc(&h->kcol, 4 * h->kcol_h.size()));
  WL_CHECK(h, cudaMalloc(&h->kn, 4 * (size_t)nl));
  WL_CHECK(h, cudaMalloc(&h->koff, 8 * (size_t)(nl + 1)));
  h->allocated += resident;
  if (!orb.empty())
    WL_CHECK(h, cudaMemcpyAsync(d_orb.p, orb.data(), sizeof(int2) * orb.size(), cudaMemcpyHostToDevice, s));
  WL_CHECK(h, cudaMemcpyAsync(d_cd.p, cd.data(), sizeof(ColDesc) * cd.size(), cudaMemcpyHostToDevice, s));
  WL_CHECK(h, cudaMemcpyAsync(d_ctri.p, h->ktri_h.data(), 4 * (size_t)ncol_all, cudaMemcpyHostToDevice, s));
  WL_CHECK(h, cudaMemcpyAsync(h->kcol, h->kcol_h.data(), 4 * h->kcol_h.size(), cudaMemcpyHostToDevice, s));
  WL_CHECK(h, cudaMemcpyAsync(h->kn, h->kn_h.data(), 4 * (size_t)nl, cudaMemcpyHostToDevice, s));
  WL_CHECK(h, cudaMemcpyAsync(h->koff, h->koff_h.data(), 8 * (size_t)(nl + 1), cudaMemcpyHostToDevice, s));
  WL_CHECK(h, cudaMemsetAsync(d_sum.p, 0, 8 * (size_t)ncol_all, s));
  WL_CHECK(h, cudaMemsetAsync(h->kgram, 0, 8 * (size_t)sq, s));
  WL_CHECK(h, cudaMemsetAsync(d_gf.p, 0, 8 * (size_t)sq, s));
  WL_CHECK(h, cudaMemsetAsync(d_bad.p, 0, sizeof(int), s));
  const size_t shb = sizeof(int2) * 2 * ((size_t)h->rmax + 1);
  if (shb > 48 * 1024)
    WL_CHECK(h, cudaFuncSetAttribute(k_leg_counts, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb));
  for (int A = 0; A < nl; ++A) {
    const int64_t norb = ooff[A + 1] - ooff[A];
    const int ncol = h->kn_h[A];
    if (norb == 0 || ncol == 0) continue;
    const int2* o = (const int2*)d_orb.p + ooff[A];
    const ColDesc* c = (const ColDesc*)d_cd.p + h->kcoff_h[A];
    unsigned long long* csum = (unsigned long long*)d_sum.p + h->kcoff_h[A];
    dim3 g1((unsigned)((norb + LC_THREADS - 1) / LC_THREADS), (unsigned)ncol);
    k_leg_counts<<<g1, LC_THREADS, shb, s>>>(h->rmax, h->rowtab, o, norb, c, (int32_t*)d_nm.p, csum);
    const int64_t nt = (ncol + 31) / 32;
    dim3 g2((unsigned)(nt * (nt + 1) / 2), (unsigned)((norb + GRAM_CHUNK - 1) / GRAM_CHUNK));
    k_gram<<<g2, 256, 0, s>>>((const int32_t*)d_nm.p, o, norb, ncol, h->kgram + h->koff_h[A],
                              (double*)d_gf.p + h->koff_h[A]);
    const int64_t nn = (int64_t)ncol * ncol;
    k_kappa<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(ncol, h->kgram + h->koff_h[A], (double*)d_gf.p + h->koff_h[A],
                                                         (const int32_t*)d_ctri.p + h->kcoff_h[A], h->Ntri,
                                                         h->kap + h->koff_h[A], (int*)d_bad.p);
    WL_LAUNCH(h, "exact coupling kernels");
  }
  // checks: every column sums to the N_tri of its triangle (the counting
  // kernel's own result); no Gram entry left int64 (the FP64 shadow sums)
  std::vector<unsigned long long> csum((size_t)ncol_all);
  std::vector<int64_t> ntri_h((size_t)h->ntri);
  int bad = 0;
  WL_CHECK(h, cudaMemcpyAsync(csum.data(), d_sum.p, 8 * (size_t)ncol_all, cudaMemcpyDeviceToHost, s));
  WL_CHECK(h, cudaMemcpyAsync(ntri_h.data(), h->Ntri, 8 * (size_t)h->ntri, cudaMemcpyDeviceToHost, s));
  WL_CHECK(h, cudaMemcpyAsync(&bad, d_bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  WL_CHECK(h, cudaStreamSynchronize(s));
  for (int64_t k = 0; k < ncol_all; ++k)
    if ((int64_t)csum[k] != ntri_h[h->ktri_h[k]])
      return wl_fail(h, COV_ERR_CUDA, "exact couplings: a leg-count column does not sum to its N_tri");
  if (bad) return wl_fail(h, COV_ERR_INVALID, "exact couplings: a Gram entry exceeds int64 for this binning");
  return COV_OK;
}

extern "C" int cov_coupling_gram(cov_handle* h, int ell_bin, int* ncol, int32_t* cols, int64_t* gram, void* stream) {
  if (!h || !ncol) return COV_ERR_INVALID;
  if (h->coupling != COV_COUPLING_EXACT || ell_bin < 0 || ell_bin >= h->nl)
    return wl_fail(h, COV_ERR_INVALID, "cov_coupling_gram: handle without exact couplings, or bad ell bin");
  const int n = h->kn_h.empty() ? 0 : h->kn_h[ell_bin];
  const int cap = *ncol;
  *ncol = n;
  if (!cols || !gram || cap < n || n == 0) return COV_OK;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<unsigned long long> g((size_t)n * n);
  WL_CHECK(h, cudaMemcpyAsync(g.data(), h->kgram + h->koff_h[ell_bin], 8 * g.size(), cudaMemcpyDeviceToHost, s));
  WL_CHECK(h, cudaStreamSynchronize(s));
  for (int r = 0; r < n; ++r) {
    cols[2 * r] = h->kyz_h[2 * (h->kcoff_h[ell_bin] + r)];
    cols[2 * r + 1] = h->kyz_h[2 * (h->kcoff_h[ell_bin] + r) + 1];
    for (int c = 0; c < n; ++c)
      gram[(size_t)r * n + c] = (int64_t)(r >= c ? g[(size_t)r * n + c] : g[(size_t)c * n + r]);
  }
  return COV_OK;
}
