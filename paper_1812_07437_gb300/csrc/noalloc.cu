// Allocation-free variant of the cumulative S/N solve.
//
// Some callers cannot allocate device memory at all: a host application that
// owns every byte of the GPU through its own pool and forbids further
// cudaMalloc calls (a plugin inside a larger framework, an embedded serving
// runtime with a fixed memory budget), or a latency-critical loop where an
// allocation would stall the device.  cov_snr_noalloc serves them: it runs
// the same Jacobi-scaled FP64 Cholesky as cov_snr, but its workspace is a
// file-scope device array of fixed size instead of memory allocated per call,
// and it takes no handle.  The caller passes every input and output.
//
// The array (g_snr_scratch) is part of this library's device image: every GPU
// that loads the library holds it (COV_NOALLOC_MAX_M + 1)^2 doubles, 32 MiB,
// until the process exits.  In host code its name is only a host-side
// stand-in, so the device address is looked up through cudaGetSymbolAddress,
// with the device current, on the first call made in each CUDA context (the
// device's primary context, normally); that first call should come before any
// stream capture.  A device reset ends the context: the next call finds a new
// context and looks the address up again instead of using a stale one.  All calls
// share the one array and it keeps the last call's contents: calls whose work
// overlaps on the GPU (different streams, or several host threads) race on
// it and must be serialised by the caller.  Every workspace entry a call reads
// is written by that call first; the status word is cleared by each call.
#include <mutex>
#include <string>

#include "common.cuh"

// kernels of the handle-based path, reused unchanged
__global__ void k_potrf_diag(OutMap W, int64_t k0, int kb, int* status);
__global__ void k_trsm_rows(OutMap W, int64_t k0, int kb, int64_t r0, int64_t r1);
__global__ void k_gemm_lower(const double* __restrict__ A, int64_t lda, const double* __restrict__ B, int64_t ldb,
                             OutMap out, int64_t n, int64_t k, double alpha, double beta, int lower_only,
                             int64_t ntiles_1d, int64_t tile_off);

#define NA_NB 64
#define NA_MAX_PREFIX 64

static __device__ __align__(256) double g_snr_scratch[(COV_NOALLOC_MAX_M + 1) * (COV_NOALLOC_MAX_M + 1)];

struct PrefixCounts {
  int64_t cnt[NA_MAX_PREFIX];
};

// workspace rows 0..M-1: scaled lower triangle of C; row M: scaled D
__global__ void k_na_pack(int64_t M, const double* C, int64_t ldc, const double* D, double* Wk, int64_t ldw) {
  int64_t i = blockIdx.x;
  int64_t j = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (i > M || j > i) return;
  if (i == M) {
    Wk[i * ldw + j] = (j < M) ? D[j] / sqrt(C[j * ldc + j]) : 0.0;
    return;
  }
  Wk[i * ldw + j] = C[i * ldc + j] / sqrt(C[i * ldc + i] * C[j * ldc + j]);
}

__global__ void k_na_prefix(int64_t M, const double* Wk, int64_t ldw, PrefixCounts pc, double* out) {
  __shared__ double sh[32];
  int c = blockIdx.x;
  int64_t n = pc.cnt[c];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double y = Wk[M * ldw + i];
    s += y * y;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[c] = (n > 0) ? sqrt(s) : nan("");
}

void wl_set_global_error(const std::string& msg);  // api.cu: read by cov_last_error(NULL)
static std::mutex g_na_mutex;
// the array's device address per device, with the context it was looked up in
static double* g_na_ptr[128] = {nullptr};
static CUcontext g_na_ctx[128] = {nullptr};

// the calling thread's current CUDA context (the driver entry point, looked up
// once; cudart makes the device's primary context current first)
static CUcontext na_current_context(int dev) {
  typedef CUresult (*PFN_ctx)(CUcontext*);
  static PFN_ctx fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (PFN_ctx)p;
    return (PFN_ctx) nullptr;
  }();
  CUcontext c = nullptr;
  cudaSetDevice(dev);  // makes the device's primary context current (allocates nothing)
  if (fn) fn(&c);
  return c;
}

static int na_fail(int code, const std::string& msg) {
  wl_set_global_error(msg);
  return code;
}

extern "C" int cov_snr_noalloc(const double* d_C, int64_t ldc, const double* d_D, int64_t M, const int64_t* prefix,
                               int n_prefix, double* d_snr, int* d_status, void* stream) {
  if (!d_C || !d_D || !d_snr || !d_status || !prefix) return na_fail(COV_ERR_INVALID, "cov_snr_noalloc: null argument");
  if (M < 1 || M > COV_NOALLOC_MAX_M)
    return na_fail(COV_ERR_INVALID, "cov_snr_noalloc: M = " + std::to_string(M) + " is outside [1, " +
                                        std::to_string(COV_NOALLOC_MAX_M) + "], the size of the static workspace");
  if (ldc < M) return na_fail(COV_ERR_INVALID, "cov_snr_noalloc: ldc < M");
  if (n_prefix < 1 || n_prefix > NA_MAX_PREFIX)
    return na_fail(COV_ERR_INVALID, "cov_snr_noalloc: n_prefix outside [1, 64]");
  PrefixCounts pc{};
  for (int c = 0; c < n_prefix; ++c) {
    if (prefix[c] < 0 || prefix[c] > M || (c > 0 && prefix[c] < prefix[c - 1]))
      return na_fail(COV_ERR_INVALID, "cov_snr_noalloc: prefix counts must be non-decreasing within [0, M]");
    pc.cnt[c] = prefix[c];
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 128) return na_fail(COV_ERR_CUDA, "cov_snr_noalloc: cudaGetDevice failed");
  double* work = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mutex);
    const CUcontext ctx = na_current_context(dev);
    if (!g_na_ptr[dev] || g_na_ctx[dev] != ctx) {
      g_na_ctx[dev] = ctx;
      e = cudaGetSymbolAddress((void**)&g_na_ptr[dev], g_snr_scratch);
      if (e != cudaSuccess) {
        g_na_ptr[dev] = nullptr;
        cudaGetLastError();
        return na_fail(COV_ERR_CUDA, std::string("cov_snr_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
    }
    work = g_na_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  int64_t ldw = M + 1;
  e = cudaMemsetAsync(d_status, 0, sizeof(int), s);
  if (e != cudaSuccess) return na_fail(COV_ERR_CUDA, std::string("cov_snr_noalloc: ") + cudaGetErrorString(e));
  dim3 gp((unsigned)(M + 1), (unsigned)((M + 1 + 255) / 256));
  k_na_pack<<<gp, 256, 0, s>>>(M, d_C, ldc, d_D, work, ldw);
  for (int64_t k0 = 0; k0 < M; k0 += NA_NB) {
    int kb = (int)((M - k0) < NA_NB ? (M - k0) : NA_NB);
    k_potrf_diag<<<1, 256, 0, s>>>(out_rows(work, ldw), k0, kb, d_status);
    int64_t r0 = k0 + kb, r1 = M + 1;
    if (r1 > r0) {
      k_trsm_rows<<<(unsigned)((r1 - r0 + 31) / 32), 32, 0, s>>>(out_rows(work, ldw), k0, kb, r0, r1);
      int64_t n = r1 - r0;
      int64_t nt1 = (n + 63) / 64;
      double* P = work + r0 * ldw + k0;
      double* Cs = work + r0 * ldw + r0;
      k_gemm_lower<<<(unsigned)(nt1 * (nt1 + 1) / 2), 256, 0, s>>>(P, ldw, P, ldw, out_rows(Cs, ldw), n, kb, -1.0,
                                                                    1.0, 1, nt1, 0);
    }
  }
  k_na_prefix<<<n_prefix, 256, 0, s>>>(M, work, ldw, pc, d_snr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(COV_ERR_CUDA, std::string("cov_snr_noalloc: ") + cudaGetErrorString(e));
  return COV_OK;
}
