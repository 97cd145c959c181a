// Batched covariance + cumulative S/N over many cosmologies of one survey
// set-up (host code): the Fisher pattern (finite-difference steps around a
// fiducial cosmology) and emulator training sets.
//
// The first cosmology runs eagerly: it allocates every workspace, builds the
// S/N selections and launch orders and, when asked, times the candidate
// launch configurations and keeps the fastest.  The step that depends on the
// cosmology (tables, spectra, the dense covariance, the three S/N
// factorisations) is then captured once, into the body of a graph "while"
// node: every kernel reads the cosmology from device memory, host
// synchronisation and status reads are deferred to the end of the batch, a
// first kernel of the body loads the next cosmology and a last one stores the
// results and sets the loop condition, so the remaining cosmologies run as one
// graph launch (fallback: the step captured alone and replayed per
// cosmology).  The exact integer counts do not depend on the cosmology and are
// computed once.
#include <chrono>

#include "common.cuh"

namespace {

// one eager step for the handle's current cosmology (tables already built)
int eager_step(cov_handle* h, unsigned terms, int precision, double* C, double* D, double* snr3, cudaStream_t s) {
  int rc;
  if ((rc = wl_spectra(h, D, s))) return rc;
  if ((rc = wl_assemble(h, C, h->M, terms, precision, s))) return rc;
  for (int w = 0; w < 3; ++w)
    if ((rc = wl_snr(h, C, h->M, D, w, snr3 + (size_t)w * h->nl, s))) return rc;
  return COV_OK;
}

struct Pinned {
  void* p = nullptr;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

// Loop body, first kernel: the cosmology of iteration *idx into the copy the
// kernels of the step read.
__global__ void k_batch_in(const cov_cosmology* __restrict__ cosmos, const int* __restrict__ idx,
                           cov_cosmology* cosmo_d) {
  if (threadIdx.x == 0) *cosmo_d = cosmos[*idx];
}

// Loop body, last kernel: the three cumulative S/N (and D) of iteration *idx
// into its slot, then the next iteration, or the end of the loop.
__global__ void k_batch_out(int* idx, int n, int nl, int64_t M, const double* s0, const double* s1,
                            const double* s2, const double* D, double* out, int64_t per,
                            cudaGraphConditionalHandle loop) {
  __shared__ int k_sh;
  if (threadIdx.x == 0) k_sh = *idx;
  __syncthreads();
  const int k = k_sh;
  double* o = out + per * k;
  for (int i = threadIdx.x; i < 3 * nl; i += blockDim.x) {
    const int w = i / nl, c = i % nl;
    o[i] = (w == 0 ? s0 : (w == 1 ? s1 : s2))[c];
  }
  if (D)
    for (int64_t i = threadIdx.x; i < M; i += blockDim.x) o[3 * nl + i] = D[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    *idx = k + 1;
    cudaGraphSetConditional(loop, k + 1 < n ? 1u : 0u);
  }
}

// The step of cosmologies 1..n-1 as one graph launch: a "while" node whose
// body is k_batch_in, the captured step and k_batch_out.  *built is false when
// the graph could not be built (the caller then replays the step per cosmology).
int single_launch(cov_handle* h, const cov_cosmology* cosmos, int n, unsigned terms, int precision, bool with_D,
                  double* out_host, size_t per, cudaStream_t s, double* cap_ms, double* run_ms, bool* built) {
  *built = false;
  const int64_t M = h->M;
  DevBuf dc, dout, didx;
  const size_t bytes = sizeof(cov_cosmology) * n + sizeof(double) * per * n + sizeof(int);
  if (h->budget && h->allocated + bytes > h->budget) return COV_OK;  // no room: replay instead
  if (cudaMalloc(&dc.p, sizeof(cov_cosmology) * n) != cudaSuccess ||
      cudaMalloc(&dout.p, sizeof(double) * per * n) != cudaSuccess || cudaMalloc(&didx.p, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return COV_OK;
  }
  const int one = 1;
  WL_CHECK(h, cudaMemcpyAsync(dc.p, cosmos, sizeof(cov_cosmology) * n, cudaMemcpyHostToDevice, s));
  WL_CHECK(h, cudaMemcpyAsync(didx.p, &one, sizeof(int), cudaMemcpyHostToDevice, s));
  WL_CHECK(h, cudaStreamSynchronize(s));
  auto t0 = std::chrono::steady_clock::now();
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle loop;
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t node;
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) {
    cudaGetLastError();
    return COV_OK;
  }
  bool ok = cudaGraphConditionalHandleCreate(&loop, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  if (ok) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    ok = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) == cudaSuccess;
  }
  int rc = COV_OK;
  if (ok) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
         cudaSuccess;
    if (ok) {
      const bool prof = h->prof;
      h->prof = false;
      h->deferred = true;
      k_batch_in<<<1, 32, 0, s>>>((const cov_cosmology*)dc.p, (const int*)didx.p, h->cosmo_d);
      rc = wl_tables(h, s);
      if (!rc) rc = wl_spectra(h, h->batch_D, s);
      if (!rc) rc = wl_assemble(h, h->batch_C, M, terms, precision, s);
      for (int w = 0; w < 3 && !rc; ++w) rc = wl_snr(h, h->batch_C, M, h->batch_D, w, nullptr, s);
      k_batch_out<<<1, 256, 0, s>>>((int*)didx.p, n, h->nl, M, h->sel[0].out, h->sel[1].out, h->sel[2].out,
                                    with_D ? h->batch_D : nullptr, (double*)dout.p, (int64_t)per, loop);
      cudaGraph_t captured = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(s, &captured);
      h->deferred = false;
      h->prof = prof;
      ok = ce == cudaSuccess && rc == COV_OK;
    }
  }
  if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  cudaGraphDestroy(graph);
  if (!ok) {
    cudaGetLastError();
    return rc;  // a failure of the step itself is reported; one of the graph API falls back
  }
  *cap_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *built = true;
  auto t1 = std::chrono::steady_clock::now();
  cudaError_t ce = cudaGraphLaunch(exec, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(out_host, dout.p, sizeof(double) * per * n, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  *run_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
  cudaGraphExecDestroy(exec);
  if (ce != cudaSuccess) return wl_cuda(h, ce, "batch graph launch");
  return COV_OK;
}

}  // namespace

extern "C" int cov_batch_snr(cov_handle* h, const cov_cosmology* cosmos, int n, unsigned terms, int precision,
                             double* h_D, double* h_snr, unsigned flags, cov_batch_info* info, void* stream) {
  if (!h) return COV_ERR_INVALID;
  if (!cosmos || n < 1 || !h_snr || (terms & ~COV_TERMS_ALL) ||
      (precision != COV_FP64 && precision != COV_SPLIT_BF16) || (flags & ~COV_BATCH_TUNE))
    return wl_fail(h, COV_ERR_INVALID, "cov_batch_snr: bad cosmologies, outputs, terms, precision or flags");
  if ((terms & COV_TERM_SSC) && !(terms & COV_TERM_1H) && precision != COV_FP64)
    return wl_fail(h, COV_ERR_INVALID, "cov_batch_snr: COV_TERM_SSC needs COV_TERM_1H in the split form");
  // The batch runs on a stream of its own (a capture cannot record the legacy
  // default stream), ordered after the caller's stream; it returns when done.
  if (!h->batch_stream) {
    WL_CHECK(h, cudaStreamCreateWithFlags(&h->batch_stream, cudaStreamNonBlocking));
    WL_CHECK(h, cudaEventCreateWithFlags(&h->batch_ev, cudaEventDisableTiming));
  }
  WL_CHECK(h, cudaEventRecord(h->batch_ev, (cudaStream_t)stream));
  WL_CHECK(h, cudaStreamWaitEvent(h->batch_stream, h->batch_ev, 0));
  cudaStream_t s = h->batch_stream;
  const int64_t M = h->M;
  const int nl = h->nl;
  int rc;
  if ((rc = wl_ensure(h, (void**)&h->batch_C, sizeof(double) * (size_t)M * (size_t)M, "batch covariance"))) return rc;
  if ((rc = wl_ensure(h, (void**)&h->batch_D, sizeof(double) * (size_t)M, "batch data vector"))) return rc;
  cov_batch_info inf{};
  const bool prof = h->prof;
  auto ms_since = [](std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
  };

  // 1. the first cosmology, eagerly (optionally once per candidate configuration)
  auto t0 = std::chrono::steady_clock::now();
  if ((rc = cov_update(h, &cosmos[0], s))) return rc;
  if (flags & COV_BATCH_TUNE) {
    // candidate launch configurations, one factor at a time away from the
    // default: contraction kernel and its launch-order grouping, Cholesky
    // look-ahead and trailing-update kernel; the fastest eager step wins
    struct Cand {
      int tc, group;
      bool look;
      int chol;
    };
    const Cand cands[COV_BATCH_CANDIDATES] = {{1, 8, true, 0},  {1, 4, true, 0}, {1, 16, true, 0},
                                              {0, 8, true, 0},  {1, 8, false, 0}, {1, 8, true, 1}};
    double best = 1e300;
    int bi = 0;
    for (int a = 0; a < COV_BATCH_CANDIDATES; ++a) {
      h->tc_kernel = cands[a].tc;
      h->pr_group = cands[a].group;
      h->chol_lookahead = cands[a].look;
      h->chol_kernel = cands[a].chol;
      WL_CHECK(h, cudaStreamSynchronize(s));
      auto t = std::chrono::steady_clock::now();
      if ((rc = eager_step(h, terms, precision, h->batch_C, h->batch_D, h_snr, s))) return rc;
      WL_CHECK(h, cudaStreamSynchronize(s));
      const double ms = ms_since(t);
      inf.candidate_ms[a] = ms;
      if (ms < best) {
        best = ms;
        bi = a;
      }
    }
    h->tc_kernel = cands[bi].tc;
    h->pr_group = cands[bi].group;
    h->chol_lookahead = cands[bi].look;
    h->chol_kernel = cands[bi].chol;
    inf.tuned = bi;
  }
  if ((rc = eager_step(h, terms, precision, h->batch_C, h->batch_D, h_snr, s))) return rc;
  if (h_D) WL_CHECK(h, cudaMemcpyAsync(h_D, h->batch_D, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
  WL_CHECK(h, cudaStreamSynchronize(s));
  inf.first_ms = ms_since(t0);
  inf.tc_kernel = h->tc_kernel;
  inf.chol_lookahead = h->chol_lookahead ? 1 : 0;
  inf.pr_group = h->pr_group;
  inf.chol_kernel = h->chol_kernel;

  if (n > 1) {
    const size_t per = (size_t)3 * nl + (h_D ? (size_t)M : 0);
    Pinned po;
    cudaError_t ce = cudaHostAlloc(&po.p, sizeof(double) * per * n, cudaHostAllocDefault);
    if (ce != cudaSuccess) return wl_cuda(h, ce, "cudaHostAlloc (batch staging)");
    double* out = (double*)po.p;
    int* words[3] = {h->tc_status, h->chol_status, h->piv_status};  // the first is unused by the FP64 form
    for (int* w : words)
      if (w) WL_CHECK(h, cudaMemsetAsync(w, 0, sizeof(int), s));
    // 2. cosmologies 1..n-1 as one graph launch (a device-side loop)
    bool built = false;
    double cap_ms = 0.0, run_ms = 0.0;
    if ((rc = single_launch(h, cosmos, n, terms, precision, h_D != nullptr, out, per, s, &cap_ms, &run_ms, &built)))
      return rc;
    if (built) {
      inf.single_launch = 1;
      inf.capture_ms = cap_ms;
      inf.replay_ms = run_ms / (n - 1);
    } else {
      // 2'. or the step captured alone and replayed once per cosmology
      auto t1 = std::chrono::steady_clock::now();
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      h->prof = false;
      h->deferred = true;
      WL_CHECK(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      rc = wl_tables(h, s);
      if (!rc) rc = wl_spectra(h, h->batch_D, s);
      if (!rc) rc = wl_assemble(h, h->batch_C, M, terms, precision, s);
      for (int w = 0; w < 3 && !rc; ++w) rc = wl_snr(h, h->batch_C, M, h->batch_D, w, nullptr, s);
      ce = cudaStreamEndCapture(s, &graph);
      h->deferred = false;
      h->prof = prof;
      if (rc) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc;
      }
      if (ce != cudaSuccess) return wl_cuda(h, ce, "cudaStreamEndCapture (batch step)");
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) return wl_cuda(h, ce, "cudaGraphInstantiate (batch step)");
      inf.capture_ms = ms_since(t1);
      Pinned pc;
      ce = cudaHostAlloc(&pc.p, sizeof(cov_cosmology) * n, cudaHostAllocDefault);
      if (ce != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return wl_cuda(h, ce, "cudaHostAlloc (batch staging)");
      }
      std::copy(cosmos, cosmos + n, (cov_cosmology*)pc.p);
      WL_CHECK(h, cudaStreamSynchronize(s));
      auto t2 = std::chrono::steady_clock::now();
      for (int k = 1; k < n; ++k) {
        WL_CHECK(h, cudaMemcpyAsync(h->cosmo_d, (cov_cosmology*)pc.p + k, sizeof(cov_cosmology),
                                    cudaMemcpyHostToDevice, s));
        WL_CHECK(h, cudaGraphLaunch(exec, s));
        double* o = out + per * k;
        for (int w = 0; w < 3; ++w)
          WL_CHECK(h, cudaMemcpyAsync(o + (size_t)w * nl, h->sel[w].out, sizeof(double) * nl,
                                      cudaMemcpyDeviceToHost, s));
        if (h_D) WL_CHECK(h, cudaMemcpyAsync(o + 3 * nl, h->batch_D, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
      }
      ce = cudaStreamSynchronize(s);
      inf.replay_ms = ms_since(t2) / (n - 1);
      cudaGraphExecDestroy(exec);
      if (ce != cudaSuccess) return wl_cuda(h, ce, "batch replays");
    }
    int st[3] = {0, 0, 0};
    for (int w = 0; w < 3; ++w)
      if (words[w]) WL_CHECK(h, cudaMemcpyAsync(&st[w], words[w], sizeof(int), cudaMemcpyDeviceToHost, s));
    WL_CHECK(h, cudaStreamSynchronize(s));
    if (st[0] || st[1]) return wl_fail(h, COV_ERR_TIMEOUT, "batch: a bounded mbarrier wait expired");
    if (st[2]) return wl_fail(h, COV_ERR_NOT_PD, "batch: a Cholesky met a non-positive pivot");
    // S/N of a selection with no rows stays NaN (the eager step wrote the host copy)
    for (int k = 1; k < n; ++k) {
      double* o = out + per * k;
      for (int w = 0; w < 3; ++w)
        for (int c = 0; c < nl; ++c)
          h_snr[((size_t)k * 3 + w) * nl + c] = h->sel[w].Ms ? o[(size_t)w * nl + c] : h_snr[(size_t)w * nl + c];
      if (h_D) std::copy(o + 3 * nl, o + 3 * nl + M, h_D + (size_t)k * M);
    }
    h->cosmo = cosmos[n - 1];
  }
  h->ops_terms = -1;  // the band-assembly operands were overwritten
  h->spectra_ready = true;
  if (info) *info = inf;
  return COV_OK;
}
