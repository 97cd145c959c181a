// Batched covariance + cumulative S/N over many cosmologies of one survey
// set-up (host code): the Fisher pattern (finite-difference steps around a
// fiducial cosmology) and emulator training sets.
//
// The first cosmology runs eagerly: it allocates every workspace, builds the
// S/N selections and launch orders and, when asked, times the candidate
// launch configurations (tensor-core contraction in CTA pairs or one CTA
// per tile; Cholesky with or without panel look-ahead) and keeps the fastest.
// The step that depends on the cosmology (tables, spectra, the dense
// covariance, the three S/N factorisations) is then captured once into a CUDA
// graph: every kernel reads the cosmology from device memory, host
// synchronisation and status reads are deferred to the end of the batch, and
// each remaining cosmology costs one parameter copy, one graph launch and the
// copies of its results.  The exact integer counts do not depend on the
// cosmology and are computed once.
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
    const int kernels[2] = {1, 0};
    const bool look[2] = {true, false};
    double best = 1e300;
    int bk = 1;
    bool bl = true;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        h->tc_kernel = kernels[a];
        h->chol_lookahead = look[b];
        WL_CHECK(h, cudaStreamSynchronize(s));
        auto t = std::chrono::steady_clock::now();
        if ((rc = eager_step(h, terms, precision, h->batch_C, h->batch_D, h_snr, s))) return rc;
        WL_CHECK(h, cudaStreamSynchronize(s));
        double ms = ms_since(t);
        inf.candidate_ms[2 * a + b] = ms;
        if (ms < best) {
          best = ms;
          bk = kernels[a];
          bl = look[b];
        }
      }
    h->tc_kernel = bk;
    h->chol_lookahead = bl;
  }
  if ((rc = eager_step(h, terms, precision, h->batch_C, h->batch_D, h_snr, s))) return rc;
  if (h_D) WL_CHECK(h, cudaMemcpyAsync(h_D, h->batch_D, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
  WL_CHECK(h, cudaStreamSynchronize(s));
  inf.first_ms = ms_since(t0);
  inf.tc_kernel = h->tc_kernel;
  inf.chol_lookahead = h->chol_lookahead ? 1 : 0;

  if (n > 1) {
    // 2. capture the cosmology-dependent step
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
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
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

    // 3. replays: parameters in, S/N (and D) out, all stream-ordered
    const size_t per = (size_t)3 * nl + (h_D ? (size_t)M : 0);
    Pinned pc, po;
    ce = cudaHostAlloc(&pc.p, sizeof(cov_cosmology) * n, cudaHostAllocDefault);
    if (ce == cudaSuccess) ce = cudaHostAlloc(&po.p, sizeof(double) * per * n, cudaHostAllocDefault);
    if (ce != cudaSuccess) {
      cudaGraphExecDestroy(exec);
      return wl_cuda(h, ce, "cudaHostAlloc (batch staging)");
    }
    std::copy(cosmos, cosmos + n, (cov_cosmology*)pc.p);
    double* out = (double*)po.p;
    int* words[3] = {h->tc_status, h->chol_status, h->piv_status};  // the first is unused by the FP64 form
    for (int* w : words)
      if (w) WL_CHECK(h, cudaMemsetAsync(w, 0, sizeof(int), s));
    WL_CHECK(h, cudaStreamSynchronize(s));
    auto t2 = std::chrono::steady_clock::now();
    for (int k = 1; k < n; ++k) {
      WL_CHECK(h, cudaMemcpyAsync(h->cosmo_d, (cov_cosmology*)pc.p + k, sizeof(cov_cosmology),
                                  cudaMemcpyHostToDevice, s));
      WL_CHECK(h, cudaGraphLaunch(exec, s));
      double* o = out + per * k;
      for (int w = 0; w < 3; ++w)
        WL_CHECK(h, cudaMemcpyAsync(o + (size_t)w * nl, h->sel[w].out, sizeof(double) * nl, cudaMemcpyDeviceToHost,
                                    s));
      if (h_D) WL_CHECK(h, cudaMemcpyAsync(o + 3 * nl, h->batch_D, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
    }
    int st[3] = {0, 0, 0};
    for (int w = 0; w < 3; ++w)
      if (words[w]) WL_CHECK(h, cudaMemcpyAsync(&st[w], words[w], sizeof(int), cudaMemcpyDeviceToHost, s));
    ce = cudaStreamSynchronize(s);
    inf.replay_ms = ms_since(t2) / (n - 1);
    cudaGraphExecDestroy(exec);
    if (ce != cudaSuccess) return wl_cuda(h, ce, "batch replays");
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
