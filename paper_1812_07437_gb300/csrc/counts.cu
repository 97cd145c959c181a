// Exact integer mode and triangle counts on the l_f Z^2 lattice (Sec. 3.2.2,
// Eq. PSest; Appendix B, first equality of the N_tri definition).
//
// A bin b is the set of lattice vectors n with s_lo[b] <= |n|^2 < s_hi[b].
// Row tables hold, for every bin and every row y >= 0, the outer and inner
// x bounds of that annulus: xo = max{x >= 0 : x^2 + y^2 < s_hi} (-1 if none)
// and xi = min{x >= 0 : x^2 + y^2 >= s_lo}, so the row holds |x| in [xi, xo].
//
// N_tri(a,b,c) = #{(n1, n2) : n1 in A_a, n2 in A_b, n1 + n2 in A_c}.  The
// dihedral group of the square maps the three annuli onto themselves, so n1 is
// taken from the fundamental domain 0 <= y1 <= x1 with orbit weights (8, or 4
// on the axes and the diagonal); for each n1 and each row y2 the admissible x2
// form at most 2 x 2 integer intervals, intersected exactly.  Everything is
// integer arithmetic; the sums are int64.
#include "common.cuh"

__device__ __forceinline__ int64_t isqrt64(int64_t v) {
  if (v <= 0) return 0;
  int64_t r = (int64_t)sqrt((double)v);
  while (r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

__global__ void k_rowtab(int nl, int rmax, const int64_t* slo, const int64_t* shi, int32_t* tab) {
  int b = blockIdx.y;
  int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nl || y > rmax) return;
  int64_t y2 = (int64_t)y * y;
  int32_t xo = -1, xi = 0;
  if (y2 < shi[b]) xo = (int32_t)isqrt64(shi[b] - 1 - y2);
  if (y2 < slo[b]) {
    int64_t need = slo[b] - y2;  // x^2 >= need
    int64_t r = isqrt64(need);
    if (r * r < need) ++r;
    xi = (int32_t)r;
  }
  tab[((size_t)b * 2 + 0) * (rmax + 1) + y] = xo;
  tab[((size_t)b * 2 + 1) * (rmax + 1) + y] = xi;
}

__device__ __forceinline__ int row_intervals_from(int xo, int xi, int* lo, int* hi) {
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

__device__ __forceinline__ int row_intervals(const int32_t* tab, int rmax, int b, int y, int* lo, int* hi) {
  int ay = y < 0 ? -y : y;
  if (ay > rmax) return 0;
  int xo = tab[((size_t)b * 2 + 0) * (rmax + 1) + ay];
  int xi = tab[((size_t)b * 2 + 1) * (rmax + 1) + ay];
  return row_intervals_from(xo, xi, lo, hi);
}

__global__ void k_nmodes(int rmax, const int32_t* tab, int64_t* N) {
  __shared__ unsigned long long sh[32];
  int b = blockIdx.x;
  unsigned long long cnt = 0;
  for (int y = -rmax + (int)threadIdx.x; y <= rmax; y += blockDim.x) {
    int lo[2], hi[2];
    int k = row_intervals(tab, rmax, b, y, lo, hi);
    for (int i = 0; i < k; ++i) cnt += (unsigned long long)(hi[i] - lo[i] + 1);
  }
  cnt = warp_sum(cnt);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    N[b] = (int64_t)t;
  }
}

// grid: x = x1 (row of the fundamental domain), y = triangle
__global__ void k_ntri(int rmax, const int32_t* tris, const int64_t* slo, const int64_t* shi, const int32_t* tab,
                       unsigned long long* out) {
  __shared__ unsigned long long sh[32];
  extern __shared__ int2 rows_sh[];  // [2][rmax+1]: (x_outer, x_inner) of bins b and c
  int t = blockIdx.y;
  int x1 = blockIdx.x;
  int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
  unsigned long long cnt = 0;
  int64_t x1s = (int64_t)x1 * x1;
  bool any = (x1s < shi[a]) && (2 * x1s >= slo[a]);  // the row can hold a point with y1 <= x1
  if (!any) return;
  for (int y = threadIdx.x; y <= rmax; y += blockDim.x) {
    rows_sh[y] = make_int2(tab[((size_t)b * 2 + 0) * (rmax + 1) + y], tab[((size_t)b * 2 + 1) * (rmax + 1) + y]);
    rows_sh[rmax + 1 + y] =
        make_int2(tab[((size_t)c * 2 + 0) * (rmax + 1) + y], tab[((size_t)c * 2 + 1) * (rmax + 1) + y]);
  }
  __syncthreads();
  const int2* rb_sh = rows_sh;
  const int2* rc_sh = rows_sh + rmax + 1;
  {
    for (int y1 = threadIdx.x; y1 <= x1; y1 += blockDim.x) {
      int64_t s1 = x1s + (int64_t)y1 * y1;
      if (s1 < slo[a] || s1 >= shi[a]) continue;
      unsigned long long wgt = (y1 == 0 || y1 == x1) ? 4ull : 8ull;
      unsigned long long local = 0;
      int rb = (int)isqrt64(shi[b] - 1), rc = (int)isqrt64(shi[c] - 1);
      int ylo = max(-rb, -y1 - rc), yhi = min(rb, -y1 + rc);
      for (int y2 = ylo; y2 <= yhi; ++y2) {
        int blo[2], bhi[2], clo[2], chi_[2];
        int2 pb = rb_sh[y2 < 0 ? -y2 : y2];
        int nb = row_intervals_from(pb.x, pb.y, blo, bhi);
        if (nb == 0) continue;
        int yc = y1 + y2;
        int ayc = yc < 0 ? -yc : yc;
        if (ayc > rmax) continue;
        int2 pc = rc_sh[ayc];
        int nc = row_intervals_from(pc.x, pc.y, clo, chi_);
        for (int i = 0; i < nb; ++i)
          for (int j = 0; j < nc; ++j) {
            int lo = max(blo[i], clo[j] - x1);
            int hi = min(bhi[i], chi_[j] - x1);
            if (hi >= lo) local += (unsigned long long)(hi - lo + 1);
          }
      }
      cnt += wgt * local;
    }
  }
  cnt = warp_sum(cnt);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    if (s) atomicAdd(&out[t], s);
  }
}

int wl_counts(cov_handle* h, cudaStream_t s) {
  int rmax = h->rmax;
  dim3 g1((rmax + 1 + 127) / 128, h->nl);
  k_rowtab<<<g1, 128, 0, s>>>(h->nl, rmax, h->slo_d, h->shi_d, h->rowtab);
  k_nmodes<<<h->nl, 256, 0, s>>>(rmax, h->rowtab, h->Nmodes);
  WL_CHECK(h, cudaMemsetAsync(h->Ntri, 0, sizeof(int64_t) * h->ntri, s));
  if (h->ntri > 0) {
    dim3 g2(rmax + 1, h->ntri);
    size_t shb = sizeof(int2) * 2 * (size_t)(rmax + 1);
    if (shb > 48 * 1024)
      WL_CHECK(h, cudaFuncSetAttribute(k_ntri, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb));
    k_ntri<<<g2, 128, shb, s>>>(rmax, h->tris_d, h->slo_d, h->shi_d, h->rowtab, (unsigned long long*)h->Ntri);
  }
  WL_LAUNCH(h, "count kernels");
  return COV_OK;
}
