// Serving loop: continuous batching of covariance + S/N requests (host code).
//
// n_slots worker threads, each with its own non-blocking CUDA stream, take
// requests from one arrival-ordered queue.  A request starts when a worker is
// free and its footprint fits in the HBM budget next to what running requests
// and resident state hold (first fit, with a bound on how often an earlier
// request may be passed over).  The device state of a finished request stays
// resident, keyed by n(z) and binning, and is reused through cov_update by the
// next request with the same key; idle resident state is freed, least recently
// used first, when an admission needs the room.  Every step of a request runs
// in the same library calls as a single covariance (cov_init / cov_update,
// cov_spectra, cov_assemble, cov_snr), so a request's result does not depend on
// what else runs.
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>

#include "common.cuh"

namespace {

struct Resident {  // device state of one n(z) + binning
  std::string key;
  cov_handle* h = nullptr;
  double* C = nullptr;
  double* D = nullptr;
  int64_t M = 0;
  size_t reserved = 0;  // bytes counted against the budget
  bool busy = false;
  bool ready = false;  // a request has completed on it
  uint64_t last_use = 0;
};

struct Rec {
  cov_request r{};
  cov_request_info info{};
  std::vector<double> snr;
  std::string key, err;
  int bypassed = 0;
};

std::string key_of(const cov_request& r) {
  char buf[512];
  const cov_nz& z = r.nz;
  const cov_bins& b = r.bins;
  snprintf(buf, sizeof buf, "%d|%a|%a|%a|%a|%a|%a|%a|%d|%a|%a|%a|%d|%d|%a|%a|%a|%d|%a|%d", z.n_tomo, z.z0,
           z.alpha, z.zmin, z.zmax, z.photoz_sigma0, z.n_gal_arcmin2, z.sigma_e, b.n_ell, b.ell_min, b.ell_max,
           b.f_sky, b.n_chi, b.n_mass, b.m_min, b.m_max, b.k_max, b.n_conc > 1 ? b.n_conc : 1,
           b.n_conc > 1 ? b.sigma_lnc : 0.0, b.conc_model);
  return buf;
}

void free_resident(Resident* r) {
  if (r->h) cov_free(r->h);
  if (r->C) cudaFree(r->C);
  if (r->D) cudaFree(r->D);
  r->h = nullptr;
  r->C = r->D = nullptr;
}

}  // namespace

struct cov_server {
  cov_server_opts o{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, Rec> recs;
  std::vector<std::unique_ptr<Resident>> res;
  size_t reserved = 0;      // running + resident + evicted-but-not-yet-freed
  size_t pending_free = 0;  // evicted bytes whose free has not finished
  int running = 0;
  int64_t next_id = 0;
  uint64_t tick = 0;
  bool stop = false;
  cov_server_stats st{};
  std::vector<std::thread> workers;
  std::chrono::steady_clock::time_point t0;

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
  void note_peak() {
    size_t committed = reserved - pending_free;
    if (committed > st.peak_reserved) st.peak_reserved = committed;
  }
};

// Pick the next request to start (lock held).  On success the request has
// left the queue, *slot_res is a busy resident (new or reused) and *evicted
// holds idle residents that the caller must free before allocating.
static bool admit(cov_server* s, int64_t* rid, Resident** slot_res,
                  std::vector<std::unique_ptr<Resident>>* evicted) {
  const size_t budget = s->o.hbm_budget;
  size_t idx = 0;
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it, ++idx) {
    Rec& q = s->recs[*it];
    Resident* hit = nullptr;
    for (auto& r : s->res)
      if (!r->busy && r->key == q.key) {
        hit = r.get();
        break;
      }
    bool ok = false;
    if (hit) {
      hit->busy = true;
      *slot_res = hit;
      ok = true;
    } else {
      size_t need = q.info.footprint;
      size_t idle = 0;
      for (auto& r : s->res)
        if (!r->busy) idle += r->reserved;
      if (s->reserved - idle + need <= budget) {
        // evict idle residents, least recently used first, until it fits;
        // their bytes stay reserved until the caller has freed them
        size_t freed = 0;
        while (s->reserved - freed + need > budget) {
          size_t lru = SIZE_MAX;
          for (size_t k = 0; k < s->res.size(); ++k)
            if (!s->res[k]->busy && (lru == SIZE_MAX || s->res[k]->last_use < s->res[lru]->last_use)) lru = k;
          freed += s->res[lru]->reserved;
          evicted->push_back(std::move(s->res[lru]));
          s->res.erase(s->res.begin() + (long)lru);
        }
        s->pending_free += freed;
        auto r = std::make_unique<Resident>();
        r->key = q.key;
        r->M = q.info.M;
        r->reserved = need;
        r->busy = true;
        s->reserved += need;
        *slot_res = r.get();
        s->res.push_back(std::move(r));
        ok = true;
      }
    }
    if (ok) {
      for (auto jt = s->queue.begin(); jt != it; ++jt) s->recs[*jt].bypassed++;
      *rid = *it;
      s->queue.erase(it);
      s->note_peak();
      return true;
    }
    // a request passed over max_bypass times blocks everything behind it
    if (q.bypassed >= s->o.max_bypass) return false;
  }
  return false;
}

static int run_request(cov_server* s, Rec& q, Resident* res, cudaStream_t stream, bool* reused) {
  const int nl = q.r.bins.n_ell;
  q.snr.assign((size_t)3 * nl, 0.0);
  *reused = res->ready;
  if (s->o.dry_run_us > 0) {
    std::this_thread::sleep_for(std::chrono::microseconds(s->o.dry_run_us));
    return COV_OK;
  }
  int rc;
  if (!res->h) {
    cov_opts op{s->o.device, 0};
    if ((rc = cov_init(&q.r.cosmo, &q.r.nz, &q.r.bins, &op, &res->h)) != COV_OK) {
      q.err = cov_last_error(nullptr);
      return rc;
    }
    const size_t M = (size_t)res->h->M;
    if (cudaMalloc(&res->C, sizeof(double) * M * M) != cudaSuccess ||
        cudaMalloc(&res->D, sizeof(double) * M) != cudaSuccess) {
      cudaGetLastError();
      q.err = "cudaMalloc of the covariance failed";
      return COV_ERR_NOMEM;
    }
  } else {
    if ((rc = cov_update(res->h, &q.r.cosmo, stream)) != COV_OK) {
      q.err = cov_last_error(res->h);
      return rc;
    }
  }
  cov_handle* h = res->h;
  const int64_t M = h->M;
  if ((rc = cov_spectra(h, res->D, stream)) != COV_OK ||
      (rc = cov_assemble(h, res->C, M, s->o.terms, s->o.precision, stream)) != COV_OK) {
    q.err = cov_last_error(h);
    return rc;
  }
  for (int w = 0; w < 3; ++w)
    if ((rc = cov_snr(h, res->C, M, res->D, w, q.snr.data() + (size_t)w * nl, stream)) != COV_OK) {
      q.err = cov_last_error(h);
      return rc;
    }
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    q.err = cudaGetErrorString(e);
    return COV_ERR_CUDA;
  }
  return COV_OK;
}

static void worker(cov_server* s, int slot) {
  cudaStream_t stream = nullptr;
  if (s->o.dry_run_us <= 0) {
    cudaSetDevice(s->o.device);
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  }
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    int64_t rid = -1;
    Resident* res = nullptr;
    std::vector<std::unique_ptr<Resident>> evicted;
    s->cv_work.wait(lk, [&] { return s->stop || admit(s, &rid, &res, &evicted); });
    if (rid < 0) break;  // stopping
    Rec& q = s->recs[rid];
    q.info.state = COV_REQ_RUNNING;
    q.info.slot = slot;
    q.info.t_start = s->now();
    s->running++;
    if (s->running > s->st.max_running) s->st.max_running = s->running;
    lk.unlock();

    size_t freed = 0;
    for (auto& r : evicted) {
      freed += r->reserved;
      if (s->o.dry_run_us <= 0) free_resident(r.get());
    }
    if (freed) {
      lk.lock();
      s->reserved -= freed;
      s->pending_free -= freed;
      s->note_peak();
      lk.unlock();
    }
    bool reused = false;
    int rc = run_request(s, q, res, stream, &reused);

    lk.lock();
    q.info.rc = rc;
    q.info.reused = reused ? 1 : 0;
    q.info.footprint = res->reserved;
    q.info.t_done = s->now();
    q.info.state = rc == COV_OK ? COV_REQ_DONE : COV_REQ_FAILED;
    rc == COV_OK ? s->st.done++ : s->st.failed++;
    s->running--;
    if (rc == COV_OK && res->h) {
      // keep the accounting honest if the handle grew past its estimate
      size_t actual = wl_handle_bytes(res->h) + sizeof(double) * (size_t)res->M * (size_t)(res->M + 1);
      if (actual > res->reserved) {
        s->reserved += actual - res->reserved;
        res->reserved = actual;
        s->note_peak();
      }
    }
    res->busy = false;
    res->ready = rc == COV_OK;
    res->last_use = ++s->tick;
    if (rc != COV_OK) {  // do not keep state of a failed request
      for (size_t k = 0; k < s->res.size(); ++k)
        if (s->res[k].get() == res) {
          std::unique_ptr<Resident> dead = std::move(s->res[k]);
          s->res.erase(s->res.begin() + (long)k);
          size_t b = dead->reserved;
          lk.unlock();
          if (s->o.dry_run_us <= 0) free_resident(dead.get());
          lk.lock();
          s->reserved -= b;
          break;
        }
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  lk.unlock();
  if (stream) cudaStreamDestroy(stream);
}

extern "C" int cov_request_footprint(const cov_request* r, int precision, unsigned terms, int64_t* M,
                                     size_t* bytes) {
  if (!r || !M || !bytes) return COV_ERR_INVALID;
  return wl_request_bytes(&r->nz, &r->bins, precision, terms, M, bytes);
}

extern "C" int cov_server_create(const cov_server_opts* opts, cov_server** out) {
  if (!opts || !out) return COV_ERR_INVALID;
  *out = nullptr;
  cov_server_opts o = *opts;
  if (o.n_slots < 1 || o.n_slots > 64 || (o.precision != COV_FP64 && o.precision != COV_SPLIT_BF16) ||
      (o.terms & ~COV_TERMS_ALL) || !(o.terms & COV_TERMS_ALL)) {
    wl_set_global_error("cov_server_create: bad n_slots, precision or terms");
    return COV_ERR_INVALID;
  }
  if (o.max_bypass <= 0) o.max_bypass = 4;
  if (o.hbm_budget == 0) {
    if (o.dry_run_us > 0) {
      wl_set_global_error("cov_server_create: a dry run needs an explicit hbm_budget");
      return COV_ERR_INVALID;
    }
    size_t fr = 0, tot = 0;
    if (cudaSetDevice(o.device) != cudaSuccess || cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      wl_set_global_error("cov_server_create: cannot query device memory");
      return COV_ERR_CUDA;
    }
    o.hbm_budget = fr / 10 * 9;
  }
  cov_server* s = new cov_server();
  s->o = o;
  s->st.budget = o.hbm_budget;
  s->t0 = std::chrono::steady_clock::now();
  for (int k = 0; k < o.n_slots; ++k) s->workers.emplace_back(worker, s, k);
  *out = s;
  return COV_OK;
}

extern "C" int cov_server_submit(cov_server* s, const cov_request* r, int64_t* id) {
  if (!s || !r || !id) return COV_ERR_INVALID;
  Rec q;
  q.r = *r;
  q.key = key_of(*r);
  q.info.slot = -1;
  q.info.n_ell = r->bins.n_ell;
  int rc = wl_request_bytes(&r->nz, &r->bins, s->o.precision, s->o.terms, &q.info.M, &q.info.footprint);
  cov_cosmology c = r->cosmo;
  if (rc == COV_OK && !(c.Om > 0 && c.Om <= 1 && c.Ob > 0 && c.Ob < c.Om && c.h > 0 && c.sigma8 > 0 && c.Tcmb > 0))
    rc = COV_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return COV_ERR_INVALID;
  *id = s->next_id++;
  q.info.t_submit = s->now();
  s->st.submitted++;
  if (rc != COV_OK) {
    q.info.state = COV_REQ_FAILED;
    q.info.rc = rc;
    q.err = "invalid request parameters";
    s->st.failed++;
    s->recs.emplace(*id, std::move(q));
    s->cv_done.notify_all();
    return COV_OK;
  }
  if (q.info.footprint > s->o.hbm_budget) {
    q.info.state = COV_REQ_REJECTED;
    q.info.rc = COV_ERR_NOMEM;
    q.info.t_done = q.info.t_submit;
    s->st.rejected++;
    s->recs.emplace(*id, std::move(q));
    s->cv_done.notify_all();
    return COV_OK;
  }
  q.info.state = COV_REQ_QUEUED;
  s->recs.emplace(*id, std::move(q));
  s->queue.push_back(*id);
  s->cv_work.notify_all();
  return COV_OK;
}

extern "C" int cov_server_wait(cov_server* s, int64_t id, double timeout_s, cov_request_info* info, double* snr) {
  if (!s) return COV_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->recs.find(id);
  if (it == s->recs.end()) return COV_ERR_INVALID;
  auto finished = [&] { return it->second.info.state >= COV_REQ_DONE; };
  if (timeout_s < 0)
    s->cv_done.wait(lk, finished);
  else if (timeout_s > 0)
    s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), finished);
  if (info) *info = it->second.info;
  if (!finished()) return COV_ERR_TIMEOUT;
  if (snr && it->second.info.state == COV_REQ_DONE)
    std::copy(it->second.snr.begin(), it->second.snr.end(), snr);
  return COV_OK;
}

extern "C" const char* cov_server_error(cov_server* s, int64_t id) {
  if (!s) return "";
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->recs.find(id);
  return it == s->recs.end() ? "" : it->second.err.c_str();
}

extern "C" int cov_server_stats_get(cov_server* s, cov_server_stats* st) {
  if (!s || !st) return COV_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  *st = s->st;
  st->reserved = s->reserved - s->pending_free;
  return COV_OK;
}

extern "C" double cov_server_clock(cov_server* s) { return s ? s->now() : 0.0; }

extern "C" void cov_server_free(cov_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  if (s->o.dry_run_us <= 0)
    for (auto& r : s->res) free_resident(r.get());
  delete s;
}
