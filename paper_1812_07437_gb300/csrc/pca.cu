// Principal components of the joint covariance (paper Sec. 6, Eqs. SNPCA,
// NewObs, SNperEign, CumulSN) on the GPU, in FP64.
//
// The eigen-pairs of C come from one-sided Jacobi on its Cholesky factor
// (Demmel & Veselic 1992), which keeps high relative accuracy on every
// eigenvalue of a graded positive definite matrix, however small (the paper's
// covariances span ~23 decades):
//
//  * the FP64-accurate Cholesky of the S/N (cov_snr, joint selection) gives,
//    on the Jacobi-scaled matrix C' = d^-1/2 C d^-1/2, the factor L' and the
//    solved data row y = L'^-1 d^-1/2 D = L^-1 D with L = d^1/2 L';
//  * G = L^T: column j of G is row j of L, i.e. sqrt(C_jj) times row j of L'
//    (k_pca_build stores it as row j of a row-major array, so every column of
//    G is one contiguous row);
//  * sweeps of plane rotations of column pairs make the columns of G
//    orthogonal: G J = U diag(sigma), C = G^T G = J diag(sigma^2) J^T, so the
//    eigenvalues are lambda_a = |g_a|^2.  Each sweep visits every pair once in
//    the round-robin order (n/2 disjoint pairs per step, one CTA per pair,
//    position 0 fixed, the others rotating), with the rotation and the skip
//    test |c| <= tol sqrt(a b) of the sequential algorithm;
//  * (S/N)^2 of mode a, (v_a . D)^2 / lambda_a, is (u_a . y)^2 with
//    u_a = g_a / sigma_a, since y = G^-T D = U diag(sigma)^-1 J^T D: no
//    eigenvector needs to be accumulated;
//  * eigenvalues sorted ascending by rank, the cumulative (S/N)^2 in both of
//    the paper's orders and the mode counts for 90/95/99% of the total S/N
//    computed on the device.
#include <chrono>
#include <vector>

#include "common.cuh"

#define PCA_TOL 1e-15
#define PCA_MAX_SWEEPS 60

// G row j = sqrt(C_{p_j p_j}) x factor row j (entries k <= j, zero beyond); y
// = the solved data row (row Ms of the workspace)
__global__ void k_pca_build(int64_t Ms, const double* __restrict__ W, int64_t ldw, const int* __restrict__ perm,
                            const double* __restrict__ C, int64_t ldc, double* G, double* y) {
  const int64_t j = blockIdx.x;
  if (j == Ms) {
    for (int64_t k = threadIdx.x; k < Ms; k += blockDim.x) y[k] = W[Ms * ldw + k];
    return;
  }
  const int64_t pj = perm[j];
  const double s = sqrt(C[pj * ldc + pj]);
  for (int64_t k = threadIdx.x; k < Ms; k += blockDim.x) G[j * Ms + k] = (k <= j) ? s * W[j * ldw + k] : 0.0;
}

__device__ __forceinline__ void pca_block_sum3(double& a, double& b, double& c, double* sh) {
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    sh[w] = a;
    sh[32 + w] = b;
    sh[64 + w] = c;
  }
  __syncthreads();
  if (w == 0) {
    a = lane < nw ? sh[lane] : 0.0;
    b = lane < nw ? sh[32 + lane] : 0.0;
    c = lane < nw ? sh[64 + lane] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    if (lane == 0) {
      sh[0] = a;
      sh[32] = b;
      sh[64] = c;
    }
  }
  __syncthreads();
  a = sh[0];
  b = sh[32];
  c = sh[64];
}

// One step of a round-robin sweep: pair k of the arrangement of `step`
// (positions k and npad-1-k; position 0 fixed, positions 1..npad-1 hold the
// columns 1 + (i - 1 + step) mod (npad - 1)); column n is a dummy when n is odd.
__global__ void __launch_bounds__(256) k_pca_rotate(double* G, int n, int npad, int step, double tol,
                                                    int* rotated) {
  __shared__ double sh[96];
  const int k = blockIdx.x;
  auto col = [&](int i) { return i == 0 ? 0 : 1 + (i - 1 + step) % (npad - 1); };
  int p = col(k), q = col(npad - 1 - k);
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
  if (q >= n) return;
  double* gp = G + (int64_t)p * n;
  double* gq = G + (int64_t)q * n;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = gp[i], z = gq[i];
    a = fma(x, x, a);
    b = fma(z, z, b);
    c = fma(x, z, c);
  }
  pca_block_sum3(a, b, c, sh);
  if (!(fabs(c) > tol * sqrt(a * b))) return;  // uniform across the block
  const double zeta = (b - a) / (2.0 * c);
  const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = gp[i], z = gq[i];
    gp[i] = cs * x - sn * z;
    gq[i] = sn * x + cs * z;
  }
  if (threadIdx.x == 0) atomicAdd(rotated, 1);
}

// per mode a: lambda_a = |g_a|^2, (S/N)^2_a = (g_a . y)^2 / |g_a|^2
__global__ void __launch_bounds__(256) k_pca_modes(const double* G, int n, const double* y, double* lam,
                                                   double* snr2) {
  __shared__ double sh[96];
  const int a = blockIdx.x;
  const double* g = G + (int64_t)a * n;
  double s = 0.0, d = 0.0, u = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = g[i];
    s = fma(x, x, s);
    d = fma(x, y[i], d);
  }
  pca_block_sum3(s, d, u, sh);
  if (threadIdx.x == 0) {
    lam[a] = s;
    snr2[a] = d * d / s;
  }
}

// ascending rank of key[i] (ties by index); with desc, descending
__global__ void k_pca_rank(int n, const double* key, int desc, int* pos) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double ki = key[i];
  int r = 0;
  for (int j = 0; j < n; ++j) {
    const double kj = key[j];
    const bool before = desc ? (kj > ki) : (kj < ki);
    r += (before || (kj == ki && j < i)) ? 1 : 0;
  }
  pos[i] = r;
}

// sorted copies (by the ranks), cumulative (S/N)^2 in both orders (Eq. CumulSN,
// sequential sums as written) and the mode counts for 90/95/99% of the total S/N
__global__ void k_pca_cumulative(int n, const double* lam, const double* snr2, const int* pos_var,
                                 const int* pos_info, double* lam_s, double* snr2_s, double* info_s, double* cum_var,
                                 double* cum_info, int* modes) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    lam_s[pos_var[i]] = lam[i];
    snr2_s[pos_var[i]] = snr2[i];
    info_s[pos_info[i]] = snr2[i];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double sv = 0.0, si = 0.0;
  for (int a = 0; a < n; ++a) {
    sv += snr2_s[a];
    si += info_s[a];
    cum_var[a] = sv;
    cum_info[a] = si;
  }
  const double fr[3] = {0.90, 0.95, 0.99};
  for (int f = 0; f < 3; ++f) {
    const double target = fr[f] * sqrt(cum_info[n - 1]);
    int m = n;
    for (int a = 0; a < n; ++a)
      if (sqrt(cum_info[a]) >= target) {
        m = a + 1;
        break;
      }
    modes[f] = m;
  }
}

extern "C" int cov_pca(cov_handle* h, const double* d_C, int64_t ldc, const double* d_D, double* h_lam,
                       double* h_snr2, double* h_cum_var, double* h_cum_info, cov_pca_info* info, void* stream) {
  if (!h) return COV_ERR_INVALID;
  if (!d_C || !d_D || ldc < h->M) return wl_fail(h, COV_ERR_INVALID, "cov_pca: null input or ldc < M");
  if (h->M > (1 << 20)) return wl_fail(h, COV_ERR_INVALID, "cov_pca: M above 2^20");
  cudaStream_t s = (cudaStream_t)stream;
  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point t) { return std::chrono::duration<double, std::milli>(clk::now() - t).count(); };
  // 1. the FP64-accurate Cholesky of the joint selection, with y = L^-1 D
  auto t0 = clk::now();
  std::vector<double> snr_cum(h->nl);
  int rc;
  if ((rc = wl_snr(h, d_C, ldc, d_D, COV_WHICH_JOINT, snr_cum.data(), s))) return rc;
  const double ms_chol = ms_since(t0);
  const auto& z = h->sel[COV_WHICH_JOINT];
  const int64_t n64 = z.Ms;
  if (n64 < 1) return wl_fail(h, COV_ERR_INVALID, "cov_pca: empty selection");
  const int n = (int)n64;
  // 2. G and y; the per-mode, sorted and cumulative arrays
  const size_t gbytes = sizeof(double) * (size_t)n * n;
  const size_t vbytes = sizeof(double) * (size_t)n * 9 + sizeof(int) * ((size_t)n * 2 + 4);
  if (gbytes + vbytes > h->pca_bytes) {
    if (h->pca_buf) {
      cudaFree(h->pca_buf);
      h->allocated -= h->pca_bytes;
      h->pca_buf = nullptr;
      h->pca_bytes = 0;
    }
    if (h->budget && h->allocated + gbytes + vbytes > h->budget)
      return wl_fail(h, COV_ERR_NOMEM, "hbm_budget exceeded allocating the PCA workspace");
    WL_CHECK(h, cudaMalloc(&h->pca_buf, gbytes + vbytes));
    h->pca_bytes = gbytes + vbytes;
    h->allocated += h->pca_bytes;
  }
  double* G = (double*)h->pca_buf;
  double* y = G + (size_t)n * n;
  double *lam = y + n, *snr2 = lam + n, *lam_s = snr2 + n, *snr2_s = lam_s + n, *info_s = snr2_s + n;
  double *cum_var = info_s + n, *cum_info = cum_var + n, *spare = cum_info + n;
  int* pos_var = (int*)(spare + n);
  int* pos_info = pos_var + n;
  int* rotated = pos_info + n;
  int* modes = rotated + 1;
  k_pca_build<<<(unsigned)(n64 + 1), 256, 0, s>>>(n64, h->work, h->work_ld, z.perm, d_C, ldc, G, y);
  WL_LAUNCH(h, "k_pca_build");
  // 3. Jacobi sweeps until a sweep rotates no pair
  auto t1 = clk::now();
  const int npad = n + (n & 1);
  int sweeps = 0, converged = 0;
  if (n > 1) {
    for (sweeps = 1; sweeps <= PCA_MAX_SWEEPS; ++sweeps) {
      WL_CHECK(h, cudaMemsetAsync(rotated, 0, sizeof(int), s));
      for (int step = 0; step < npad - 1; ++step)
        k_pca_rotate<<<(unsigned)(npad / 2), 256, 0, s>>>(G, n, npad, step, PCA_TOL, rotated);
      WL_LAUNCH(h, "k_pca_rotate");
      int r = 0;
      WL_CHECK(h, cudaMemcpyAsync(&r, rotated, sizeof(int), cudaMemcpyDeviceToHost, s));
      WL_CHECK(h, cudaStreamSynchronize(s));
      if (r == 0) {
        converged = 1;
        break;
      }
    }
    if (sweeps > PCA_MAX_SWEEPS) sweeps = PCA_MAX_SWEEPS;
  } else {
    converged = 1;
  }
  // 4. modes, order, cumulative forms
  k_pca_modes<<<(unsigned)n, 256, 0, s>>>(G, n, y, lam, snr2);
  k_pca_rank<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, lam, 0, pos_var);
  k_pca_rank<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, snr2, 1, pos_info);
  k_pca_cumulative<<<1, 256, 0, s>>>(n, lam, snr2, pos_var, pos_info, lam_s, snr2_s, info_s, cum_var, cum_info,
                                     modes);
  WL_LAUNCH(h, "PCA mode kernels");
  int hm[3] = {0, 0, 0};
  double tot = 0.0;
  if (h_lam) WL_CHECK(h, cudaMemcpyAsync(h_lam, lam_s, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  if (h_snr2) WL_CHECK(h, cudaMemcpyAsync(h_snr2, snr2_s, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  if (h_cum_var) WL_CHECK(h, cudaMemcpyAsync(h_cum_var, cum_var, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  if (h_cum_info) WL_CHECK(h, cudaMemcpyAsync(h_cum_info, cum_info, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  WL_CHECK(h, cudaMemcpyAsync(hm, modes, sizeof(hm), cudaMemcpyDeviceToHost, s));
  WL_CHECK(h, cudaMemcpyAsync(&tot, cum_info + (n - 1), sizeof(double), cudaMemcpyDeviceToHost, s));
  WL_CHECK(h, cudaStreamSynchronize(s));
  const double ms_jac = ms_since(t1);
  if (info) {
    info->M = n64;
    info->sweeps = sweeps;
    info->converged = converged;
    info->total_snr2 = tot;
    info->modes_90 = hm[0];
    info->modes_95 = hm[1];
    info->modes_99 = hm[2];
    info->ms_cholesky = ms_chol;
    info->ms_jacobi = ms_jac;
  }
  if (!converged) return wl_fail(h, COV_ERR_TIMEOUT, "cov_pca: Jacobi did not converge within the sweep limit");
  return COV_OK;
}
