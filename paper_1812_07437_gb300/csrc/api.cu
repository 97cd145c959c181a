// C ABI of libwlcov: host-side planning (binning, data-vector layout of the
// paper's Sec. 5, lattice thresholds), device allocation and stage dispatch.
// All arithmetic of the method runs in the device kernels of the other
// translation units.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>

#include "common.cuh"

int wl_fail(cov_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int wl_cuda(cov_handle* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) return wl_fail(h, COV_ERR_NOMEM, m);
  return wl_fail(h, COV_ERR_CUDA, m);
}

static thread_local std::string g_init_err;

void wl_set_global_error(const std::string& msg) { g_init_err = msg; }

static const char* kStageNames[ST_COUNT] = {"tables", "counts", "spectra", "rows_T", "syrk_T", "gather",
                                            "rows_A", "syrk_1h", "rows_S", "syrk_ssc", "snr_pack",
                                            "snr_cholesky", "snr_prefix"};

static cudaEvent_t ev_get(cov_handle* h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// The handle's side stream (and the two events that order it against the
// caller's stream), created once.  Its work is the short critical chain beside
// a long tensor-core launch on the caller's stream (the per-element products
// of the previous sub-band; the next Cholesky panel), so it runs at the
// greatest priority: the block scheduler then places its blocks before the
// long launch's pending ones as SM room frees up.
int wl_side_stream(cov_handle* h) {
  if (h->side) return COV_OK;
  int least = 0, greatest = 0;
  WL_CHECK(h, cudaDeviceGetStreamPriorityRange(&least, &greatest));
  WL_CHECK(h, cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, greatest));
  WL_CHECK(h, cudaEventCreateWithFlags(&h->ev_cols, cudaEventDisableTiming));
  WL_CHECK(h, cudaEventCreateWithFlags(&h->ev_panel, cudaEventDisableTiming));
  return COV_OK;
}

int wl_stage_begin(cov_handle* h, int stage, cudaStream_t s) {
  if (!h->prof) return -1;
  StageEvent se{stage, ev_get(h), ev_get(h)};
  cudaEventRecord(se.a, s);
  h->pending.push_back(se);
  return (int)h->pending.size() - 1;
}

void wl_stage_end(cov_handle* h, int token, cudaStream_t s) {
  if (token < 0 || token >= (int)h->pending.size()) return;
  cudaEventRecord(h->pending[token].b, s);
}

static int dalloc(cov_handle* h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 8;
  if (h->budget && h->allocated + bytes > h->budget) return wl_fail(h, COV_ERR_NOMEM, "hbm_budget exceeded");
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return wl_cuda(h, e, "cudaMalloc");
  }
  h->allocated += bytes;
  return COV_OK;
}

static void tomo_triples(int a, int b, int c, int nt, std::vector<int>& out) {
  out.clear();
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j < nt; ++j)
      for (int k = 0; k < nt; ++k) {
        bool ok;
        if (a == b && b == c)
          ok = i <= j && j <= k;
        else if (a == b)
          ok = i <= j;
        else if (b == c)
          ok = j <= k;
        else
          ok = true;
        if (ok) {
          out.push_back(i);
          out.push_back(j);
          out.push_back(k);
        }
      }
}

static int plan(cov_handle* h) {
  const cov_bins& b = h->bins;
  const cov_nz& nz = h->nz;
  h->nl = b.n_ell;
  h->nt = nz.n_tomo;
  h->nchi = b.n_chi;
  h->nmb = b.n_mass;
  h->nc = b.n_conc > 1 ? b.n_conc : 1;  // concentration nodes (Eq. LogNormC); 1 without scatter
  h->nm = b.n_mass * h->nc;
  h->K = b.n_chi * h->nm;
  // ell bins: log-spaced edges, centre = (lo + hi)/2, width = hi - lo
  double r = b.ell_max / b.ell_min;
  h->ell_edges.resize(h->nl + 1);
  for (int i = 0; i <= h->nl; ++i) h->ell_edges[i] = b.ell_min * pow(r, (double)i / h->nl);
  h->ell.resize(h->nl);
  h->dell.resize(h->nl);
  for (int i = 0; i < h->nl; ++i) {
    h->ell[i] = 0.5 * (h->ell_edges[i] + h->ell_edges[i + 1]);
    h->dell[i] = h->ell_edges[i + 1] - h->ell_edges[i];
  }
  // closed triples, l_c <= l_a + l_b on bin centres; c slowest, b fastest
  h->tris.clear();
  for (int c = 0; c < h->nl; ++c)
    for (int a = 0; a <= c; ++a)
      for (int bb = a; bb <= c; ++bb)
        if (h->ell[c] <= h->ell[a] + h->ell[bb]) {
          h->tris.push_back(a);
          h->tris.push_back(bb);
          h->tris.push_back(c);
        }
  h->ntri = (int)(h->tris.size() / 3);
  // data-vector rows: P rows of bin b (i <= j), B rows of triangle t (the
  // tomographic triples of its bins); natural order P then B, or cumulative
  // order by largest ell bin (P rows of bin c, then the B rows of the
  // triangles whose largest bin is c: those are contiguous, c being slowest)
  h->rowdesc.clear();
  const bool wantP = h->row_set != COV_ROWS_B, wantB = h->row_set != COV_ROWS_P;
  std::vector<int> tt;
  auto emitP = [&](int bb) {
    for (int i = 0; i < h->nt; ++i)
      for (int j = i; j < h->nt; ++j) {
        int32_t d[8] = {0, bb, bb, bb, i, j, -1, bb};
        h->rowdesc.insert(h->rowdesc.end(), d, d + 8);
      }
  };
  auto emitB = [&](int t) {
    int a = h->tris[3 * t], bb = h->tris[3 * t + 1], c = h->tris[3 * t + 2];
    tomo_triples(a, bb, c, h->nt, tt);
    for (size_t k = 0; k < tt.size(); k += 3) {
      int32_t d[8] = {1, a, bb, c, tt[k], tt[k + 1], tt[k + 2], t};
      h->rowdesc.insert(h->rowdesc.end(), d, d + 8);
    }
  };
  h->nP = 0;
  if (h->row_order == COV_ORDER_CUMULATIVE) {
    for (int c = 0; c < h->nl; ++c) {
      if (wantP) {
        size_t before = h->rowdesc.size();
        emitP(c);
        h->nP += (int64_t)(h->rowdesc.size() - before) / 8;
      }
      if (wantB)
        for (int t = 0; t < h->ntri; ++t)
          if (h->tris[3 * t + 2] == c) emitB(t);
    }
  } else {
    if (wantP)
      for (int bb = 0; bb < h->nl; ++bb) emitP(bb);
    h->nP = (int64_t)h->rowdesc.size() / 8;
    if (wantB)
      for (int t = 0; t < h->ntri; ++t) emitB(t);
  }
  h->M = (int64_t)h->rowdesc.size() / 8;
  h->nB = h->M - h->nP;
  // sky and lattice: l_f = 2 pi / sqrt(Omega), Omega = 4 pi f_sky
  h->omega = 4.0 * WL_PI * b.f_sky;
  h->theta = acos(1.0 - 2.0 * b.f_sky);
  h->ell_f = 2.0 * WL_PI / sqrt(h->omega);
  h->s_lo.resize(h->nl);
  h->s_hi.resize(h->nl);
  for (int i = 0; i < h->nl; ++i) {
    double x = h->ell_edges[i] / h->ell_f;
    h->s_lo[i] = (int64_t)ceil(x * x);
  }
  double xt = h->ell_edges[h->nl] / h->ell_f;
  for (int i = 0; i + 1 < h->nl; ++i) h->s_hi[i] = h->s_lo[i + 1];
  h->s_hi[h->nl - 1] = (int64_t)floor(xt * xt) + 1;
  int64_t smax = *std::max_element(h->s_hi.begin(), h->s_hi.end()) - 1;
  int64_t rm = (int64_t)sqrt((double)smax);
  while (rm * rm > smax) --rm;
  while ((rm + 1) * (rm + 1) <= smax) ++rm;
  h->rmax = (int)rm;
  h->nleg = h->nl * h->nt;
  h->ntrow = (int64_t)h->nleg * (h->nleg + 1) / 2;
  return COV_OK;
}

static int validate(const cov_cosmology* c, const cov_nz* nz, const cov_bins* b) {
  if (!c || !nz || !b) return COV_ERR_INVALID;
  if (nz->n_tomo < 1 || nz->n_tomo > 32) return COV_ERR_INVALID;
  if (nz->alpha != 1.5 || !(nz->z0 > 0) || !(nz->zmin >= 0) || !(nz->zmax > nz->zmin)) return COV_ERR_INVALID;
  if (!(nz->photoz_sigma0 >= 0) || !(nz->n_gal_arcmin2 > 0) || !(nz->sigma_e >= 0)) return COV_ERR_INVALID;
  if (b->n_ell < 1 || b->n_ell > 64 || !(b->ell_min > 0) || !(b->ell_max > b->ell_min)) return COV_ERR_INVALID;
  if (!(b->f_sky > 0 && b->f_sky < 1)) return COV_ERR_INVALID;
  if (b->n_chi < 2 || b->n_chi > 4096 || b->n_mass < 2 || b->n_mass > 4096) return COV_ERR_INVALID;
  if (!(b->m_min > 0) || !(b->m_max > b->m_min) || !(b->k_max > 0)) return COV_ERR_INVALID;
  if (b->n_conc < 0 || b->n_conc > 32 || !(b->sigma_lnc >= 0 && b->sigma_lnc <= 2) ||
      b->n_mass * std::max(b->n_conc, 1) > 4096 || (b->conc_model != COV_CONC_DUFFY && b->conc_model != COV_CONC_BULLOCK))
    return COV_ERR_INVALID;
  if (!(c->Om > 0 && c->Om <= 1) || !(c->Ob > 0 && c->Ob < c->Om) || !(c->h > 0) || !(c->sigma8 > 0) ||
      !(c->Tcmb > 0))
    return COV_ERR_INVALID;
  return COV_OK;
}

static void free_all(cov_handle* h) {
  for (auto& se : h->pending) {
    cudaEventDestroy(se.a);
    cudaEventDestroy(se.b);
  }
  for (auto e : h->pool) cudaEventDestroy(e);
  if (h->ev_cols) cudaEventDestroy(h->ev_cols);
  if (h->ev_panel) cudaEventDestroy(h->ev_panel);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->batch_stream) cudaStreamDestroy(h->batch_stream);
  if (h->batch_ev) cudaEventDestroy(h->batch_ev);
  h->pending.clear();
  h->pool.clear();
  void* ptrs[] = {h->gl64x, h->gl64w, h->gl16x,   h->gl16w,   h->glkx,    h->glkw,    h->glcx,   h->glcw,   h->scal,      h->chi,
                  h->wchi,  h->z,     h->D,       h->ell_d,   h->m,      h->om,     h->sig0,      h->dlns,
                  h->f,     h->b1,    h->b2,      h->U,       h->Pl,     h->dPl,    h->Psh,       h->zedges,
                  h->norms, h->W,     h->sigw2,   h->slo_d,   h->shi_d,  h->Nmodes, h->Ntri,      h->rowtab,
                  h->tris_d, h->rowdesc_d, h->P3, h->RP3,     h->B3,     h->RB3,    h->B1h3,      h->Ps,
                  h->B1hp,  h->Bp,    h->A,       h->Ahi,     h->Alo,    h->Ascale, h->G2,        h->G3,
                  h->C2,    h->C3,    h->tc_status, h->Thi,   h->Tlo,    h->Tscale, h->Trows,     h->Tmat,
                  h->Srows, h->cosmo_d, h->Fsig,  h->Esig,    h->Msig,   h->FsigT,  h->EsigT,     h->MsigT,
                  h->invN,  h->omN,   h->work,    h->chol_scratch, h->chol_status, h->mb, h->omb, h->cs,
                  h->cw,    h->sigF,  h->ac,      h->bmask,   h->gblk,   h->wait_flag, h->pca_buf,
                  h->kap,   h->kgram, h->kcol,    h->kn,      h->koff,      h->plist};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->tile_ring) cudaFree(h->tile_ring);
  for (auto& z : h->sel) {
    if (z.perm) cudaFree(z.perm);
    if (z.cnt) cudaFree(z.cnt);
    if (z.out) cudaFree(z.out);
  }
  if (h->piv_status) cudaFree(h->piv_status);
  if (h->batch_C) cudaFree(h->batch_C);
  if (h->batch_D) cudaFree(h->batch_D);
}

// Device tables that cov_init allocates for a planned handle (pointer, bytes).
static void init_allocs(cov_handle* h, std::vector<std::pair<void**, size_t>>& al) {
  const size_t d = sizeof(double);
  size_t nl = h->nl, nt = h->nt, nchi = h->nchi, nm = h->nm, nmb = h->nmb, nc = h->nc;
  size_t ntri = std::max(h->ntri, 1);
  al = {
      {(void**)&h->gl64x, d * WL_N_GL_CHI}, {(void**)&h->gl64w, d * WL_N_GL_CHI},
      {(void**)&h->glkx, d * WL_N_K},       {(void**)&h->glkw, d * WL_N_K},
      {(void**)&h->glcx, d * nchi},         {(void**)&h->glcw, d * nchi},
      {(void**)&h->gl16x, d * 16},          {(void**)&h->gl16w, d * 16},
      {(void**)&h->scal, d * SC_N},         {(void**)&h->chi, d * nchi},
      {(void**)&h->wchi, d * nchi},         {(void**)&h->z, d * nchi},
      {(void**)&h->D, d * nchi},            {(void**)&h->ell_d, d * nl},
      {(void**)&h->m, d * nm},              {(void**)&h->om, d * nm},
      {(void**)&h->sig0, d * nmb},          {(void**)&h->dlns, d * nmb},
      {(void**)&h->mb, d * nmb},            {(void**)&h->omb, d * nmb},
      {(void**)&h->cs, d * nc},             {(void**)&h->cw, d * nc},
      {(void**)&h->sigF, d * nmb},          {(void**)&h->ac, d * nmb},
      {(void**)&h->f, d * nchi * nm},       {(void**)&h->b1, d * nchi * nm},
      {(void**)&h->b2, d * nchi * nm},      {(void**)&h->U, d * nl * nchi * nm},
      {(void**)&h->Pl, d * nl * nchi},      {(void**)&h->dPl, d * nl * nchi},
      {(void**)&h->Psh, d * 4 * nl * nchi},
      {(void**)&h->zedges, d * (nt + 1)},   {(void**)&h->norms, d * nt},
      {(void**)&h->W, d * nt * nchi},       {(void**)&h->sigw2, d * nchi},
      {(void**)&h->slo_d, 8 * nl},          {(void**)&h->shi_d, 8 * nl},
      {(void**)&h->Nmodes, 8 * nl},         {(void**)&h->Ntri, 8 * ntri},
      {(void**)&h->rowtab, 4 * nl * 2 * (size_t)(h->rmax + 1)},
      {(void**)&h->tris_d, 4 * 3 * ntri},
      {(void**)&h->rowdesc_d, 4 * 8 * (size_t)h->M},
      {(void**)&h->P3, d * nl * nchi},      {(void**)&h->RP3, d * nl * nchi},
      {(void**)&h->B3, d * ntri * nchi},    {(void**)&h->RB3, d * ntri * nchi},
      {(void**)&h->B1h3, d * ntri * nchi},  {(void**)&h->Ps, d * nl * nt * nt},
      {(void**)&h->B1hp, d * ntri * nt * nt * nt},
      {(void**)&h->cosmo_d, sizeof(cov_cosmology)},
  };
}

// Host-only upper estimate of the device bytes one request holds at its peak:
// the handle's tables, the dense covariance and data vector, the contraction
// operands of the chosen precision, the trispectrum table, the Cholesky
// workspace of the joint vector and the launch-order tables.  No CUDA call.
int wl_request_bytes(const cov_nz* nz, const cov_bins* bins, int precision, unsigned terms, int64_t* M_out,
                     size_t* bytes) {
  cov_cosmology c0{0.31, 0.049, 0.68, 0.96, 0.83, -1.0, 2.7255};
  if (validate(&c0, nz, bins) != COV_OK) return COV_ERR_INVALID;
  cov_handle h;
  h.nz = *nz;
  h.bins = *bins;
  plan(&h);
  std::vector<std::pair<void**, size_t>> al;
  init_allocs(&h, al);
  size_t b = 0;
  for (auto& a : al) b += a.second;
  const size_t M = (size_t)h.M, K = (size_t)h.K, nchi = (size_t)h.nchi, nt = (size_t)h.ntrow;
  auto pad256 = [](size_t x) { return (x + 255) / 256 * 256; };
  auto kpad = [](size_t x) { return (x + 63) / 64 * 64; };
  b += M * M * 8 + M * 8;                                        // covariance, data vector
  if (terms & COV_TERM_1H) {
    if (precision == COV_FP64)
      b += M * K * 8 + M * nchi * 8;                             // FP64 factor and SSC rows
    else
      b += 2 * pad256(M) * kpad(K + nchi) * 2 + M * 8 + 16 * (K + nchi) +
           ((size_t)h.nl + (size_t)h.ntri) * (K * 4 + nchi * 12);  // BF16 hi/lo rows, signature tables
  }
  if (terms & COV_TERM_BBPT) {
    b += nt * nt * 8;                                            // trispectrum table
    if (precision == COV_FP64)
      b += nt * K * 8;                                           // FP64 trispectrum rows
    else
      b += 2 * pad256(nt) * kpad(K) * 2 + nt * 8 +
           (size_t)h.nl * (h.nl + 1) / 2 * (K * 4 + nchi * 12);   // BF16 rows, pair signatures
  }
  b += (M + 8) * (M + 1) * 8 + 2 * ((wl_chol_tc_bytes((int64_t)M + 1) + 255) / 256 * 256) + M * 4;
  size_t t = (std::max(M, nt) + 255) / 256 + 1;
  b += WL_TILE_CACHE * (t * (t + 1) / 2) * 8;                    // launch-order ring
  const size_t nb32 = (M + 31) / 32;
  if (terms & (COV_TERM_BBPT | COV_TERM_PB)) b += nb32 * (nb32 + 1) / 2 * 4;  // product-term block list (bound)
  b += (size_t)64 << 20;                                         // small buffers, allocation granularity
  *M_out = h.M;
  *bytes = b;
  return COV_OK;
}

size_t wl_handle_bytes(const cov_handle* h) { return h->allocated; }

extern "C" int cov_init(const cov_cosmology* cosmo, const cov_nz* nz, const cov_bins* bins, const cov_opts* opts,
                        cov_handle** out) {
  if (!out) return COV_ERR_INVALID;
  *out = nullptr;
  if (validate(cosmo, nz, bins) != COV_OK) {
    g_init_err = "invalid cosmology, n(z) or binning parameters";
    return COV_ERR_INVALID;
  }
  cov_handle* h = new cov_handle();
  h->cosmo = *cosmo;
  h->nz = *nz;
  h->bins = *bins;
  h->device = opts ? opts->device : 0;
  h->budget = opts ? opts->hbm_budget : 0;
  h->row_set = opts ? opts->rows : COV_ROWS_JOINT;
  h->row_order = opts ? opts->order : COV_ORDER_NATURAL;
  h->tc_kernel = (opts && opts->tc_kernel == COV_TC_SINGLE) ? 0 : -1;
  h->chol_kernel = (opts && opts->chol_kernel == COV_CHOL_TILE) ? 1 : 0;
  h->coupling = opts ? opts->coupling : COV_COUPLING_MODES;
  if (h->row_set < 0 || h->row_set > 2 || h->row_order < 0 || h->row_order > 1 ||
      (h->coupling != COV_COUPLING_MODES && h->coupling != COV_COUPLING_EXACT)) {
    g_init_err = "invalid row set, row order or coupling";
    delete h;
    return COV_ERR_INVALID;
  }
  int rc;
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) {
    g_init_err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
    delete h;
    return COV_ERR_CUDA;
  }
  plan(h);
  std::vector<std::pair<void**, size_t>> al;
  init_allocs(h, al);
  for (auto& a : al) {
    if ((rc = dalloc(h, a.first, a.second)) != COV_OK) {
      g_init_err = h->err;
      free_all(h);
      delete h;
      return rc;
    }
  }
  const size_t d = sizeof(double);
  int nl = h->nl;
  // a private non-blocking stream: the set-up neither waits for nor holds up
  // work that other threads have on the legacy default stream
  cudaStream_t s = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->ell_d, h->ell.data(), d * nl, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->slo_d, h->s_lo.data(), 8 * nl, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->shi_d, h->s_hi.data(), 8 * nl, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && h->ntri)
    e = cudaMemcpyAsync(h->tris_d, h->tris.data(), 4 * h->tris.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->rowdesc_d, h->rowdesc.data(), 4 * h->rowdesc.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->scal, 0, d * SC_N, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->cosmo_d, &h->cosmo, sizeof(cov_cosmology), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    g_init_err = std::string("upload: ") + cudaGetErrorString(e);
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
    free_all(h);
    delete h;
    return COV_ERR_CUDA;
  }
  if ((rc = wl_quadrature(h, s)) == COV_OK && (rc = wl_tables(h, s)) == COV_OK && (rc = wl_counts(h, s)) == COV_OK)
    rc = wl_couplings(h, s);  // the exact BB+PT couplings, when asked for (binning only: once)
  e = cudaStreamSynchronize(s);
  if (rc == COV_OK && e != cudaSuccess) rc = wl_cuda(h, e, "cov_init tables");
  cudaStreamDestroy(s);
  if (rc != COV_OK) {
    g_init_err = h->err;
    free_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return COV_OK;
}

extern "C" int cov_update(cov_handle* h, const cov_cosmology* cosmo, void* stream) {
  if (!h || !cosmo) return COV_ERR_INVALID;
  if (validate(cosmo, &h->nz, &h->bins) != COV_OK) return wl_fail(h, COV_ERR_INVALID, "invalid cosmology");
  h->cosmo = *cosmo;
  h->spectra_ready = false;
  h->ops_terms = -1;
  cudaStream_t s = (cudaStream_t)stream;
  // the kernels read the cosmology from device memory; a captured batch step
  // leaves this copy to its driver, which writes each cosmology before a replay
  if (!h->deferred)
    WL_CHECK(h, cudaMemcpyAsync(h->cosmo_d, &h->cosmo, sizeof(cov_cosmology), cudaMemcpyHostToDevice, s));
  int tk = wl_stage_begin(h, ST_TABLES, s);
  int rc = wl_tables(h, s);
  wl_stage_end(h, tk, s);
  // the integer counts (and the exact couplings) depend on the binning only:
  // cov_init computed them once
  return rc;
}

extern "C" int cov_layout(const cov_handle* h, int64_t* M, int64_t* n_P, int64_t* n_B, int64_t* n_tri,
                          int32_t* row_desc) {
  if (!h) return COV_ERR_INVALID;
  if (M) *M = h->M;
  if (n_P) *n_P = h->nP;
  if (n_B) *n_B = h->nB;
  if (n_tri) *n_tri = h->ntri;
  if (row_desc) memcpy(row_desc, h->rowdesc.data(), sizeof(int32_t) * h->rowdesc.size());
  return COV_OK;
}

extern "C" int cov_counts(cov_handle* h, int64_t* N_ell, int64_t* N_tri, void* stream) {
  if (!h) return COV_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (N_ell) WL_CHECK(h, cudaMemcpyAsync(N_ell, h->Nmodes, 8 * h->nl, cudaMemcpyDeviceToHost, s));
  if (N_tri && h->ntri) WL_CHECK(h, cudaMemcpyAsync(N_tri, h->Ntri, 8 * (size_t)h->ntri, cudaMemcpyDeviceToHost, s));
  WL_CHECK(h, cudaStreamSynchronize(s));
  return COV_OK;
}

extern "C" int cov_spectra(cov_handle* h, double* d_D, void* stream) {
  if (!h) return COV_ERR_INVALID;
  h->ops_terms = -1;
  int tk = wl_stage_begin(h, ST_SPECTRA, (cudaStream_t)stream);
  int rc = wl_spectra(h, d_D, (cudaStream_t)stream);
  wl_stage_end(h, tk, (cudaStream_t)stream);
  return rc;
}

extern "C" int cov_assemble(cov_handle* h, double* d_C, int64_t ldc, unsigned terms, int precision, void* stream) {
  if (!h || !d_C || ldc < h->M || (terms & ~COV_TERMS_ALL)) return wl_fail(h, COV_ERR_INVALID, "bad cov_assemble args");
  if (precision != COV_FP64 && precision != COV_SPLIT_BF16) return wl_fail(h, COV_ERR_INVALID, "bad precision");
  if (!h->spectra_ready) return wl_fail(h, COV_ERR_INVALID, "cov_spectra must run before cov_assemble");
  h->ops_terms = -1;  // the full assembly rebuilds (and may resize) the operands
  return wl_assemble(h, d_C, ldc, terms, precision, (cudaStream_t)stream);
}

extern "C" int cov_assemble_band(cov_handle* h, int64_t row0, int64_t nrows, double* d_C, int64_t ldc,
                                 int layout, unsigned terms, int precision, void* stream) {
  if (!h) return COV_ERR_INVALID;
  if (!d_C || (terms & ~COV_TERMS_ALL) || (precision != COV_FP64 && precision != COV_SPLIT_BF16) ||
      (layout != COV_LAYOUT_ROWS && layout != COV_LAYOUT_TILES))
    return wl_fail(h, COV_ERR_INVALID, "cov_assemble_band: bad buffer, terms, precision or layout");
  if ((terms & COV_TERM_SSC) && !(terms & COV_TERM_1H))
    return wl_fail(h, COV_ERR_INVALID, "cov_assemble_band: COV_TERM_SSC needs COV_TERM_1H");
  if (row0 < 0 || nrows <= 0 || row0 % 256 != 0 || row0 + nrows > h->M ||
      (row0 + nrows != h->M && (row0 + nrows) % 256 != 0))
    return wl_fail(h, COV_ERR_INVALID,
                   "cov_assemble_band: the band must start on a multiple of 256 and end on one or at M");
  if (layout == COV_LAYOUT_ROWS && ldc < row0 + nrows)
    return wl_fail(h, COV_ERR_INVALID, "cov_assemble_band: ldc below row0 + nrows");
  if (!h->spectra_ready) return wl_fail(h, COV_ERR_INVALID, "cov_spectra must run before cov_assemble_band");
  OutMap out = layout == COV_LAYOUT_TILES ? out_tiles(d_C, row0) : out_rows(d_C, ldc, row0);
  return wl_assemble_band(h, row0, nrows, out, terms, precision, (cudaStream_t)stream);
}

extern "C" int cov_snr_tiles(cov_handle* h, double* d_Ct, const double* d_D, double* h_snr, void* stream) {
  if (!h) return COV_ERR_INVALID;
  if (!d_Ct || !d_D || !h_snr) return wl_fail(h, COV_ERR_INVALID, "cov_snr_tiles: null buffer");
  if (h->row_order != COV_ORDER_CUMULATIVE)
    return wl_fail(h, COV_ERR_INVALID, "cov_snr_tiles needs a handle created with COV_ORDER_CUMULATIVE");
  return wl_snr_tiles(h, d_Ct, d_D, h_snr, (cudaStream_t)stream);
}

extern "C" int cov_snr(cov_handle* h, const double* d_C, int64_t ldc, const double* d_D, int which, double* h_snr,
                       void* stream) {
  if (!h || !d_C || !d_D || !h_snr || ldc < h->M) return wl_fail(h, COV_ERR_INVALID, "bad cov_snr args");
  if (which < COV_WHICH_P || which > COV_WHICH_JOINT) return wl_fail(h, COV_ERR_INVALID, "bad selection");
  return wl_snr(h, d_C, ldc, d_D, which, h_snr, (cudaStream_t)stream);
}

extern "C" int cov_table(cov_handle* h, const char* name, double* host, int64_t* count, void* stream) {
  if (!h || !name || !count) return COV_ERR_INVALID;
  struct {
    const char* n;
    const double* p;
    int64_t c;
  } tab[] = {
      {"chi", h->chi, h->nchi},
      {"wchi", h->wchi, h->nchi},
      {"z", h->z, h->nchi},
      {"growth", h->D, h->nchi},
      {"mass", h->m, h->nm},
      {"conc_offsets", h->cs, h->nc},
      {"conc_weights", h->cw, h->nc},
      {"collapse_a", h->ac, h->bins.conc_model == COV_CONC_BULLOCK ? h->nmb : 0},
      {"f", h->f, (int64_t)h->nchi * h->nm},
      {"b1", h->b1, (int64_t)h->nchi * h->nm},
      {"b2", h->b2, (int64_t)h->nchi * h->nm},
      {"U", h->U, (int64_t)h->nl * h->nchi * h->nm},
      {"Plin", h->Pl, (int64_t)h->nl * h->nchi},
      {"dPlin", h->dPl, (int64_t)h->nl * h->nchi},
      {"W", h->W, (int64_t)h->nt * h->nchi},
      {"sigw2", h->sigw2, h->nchi},
      {"P3", h->P3, (int64_t)h->nl * h->nchi},
      {"RP3", h->RP3, (int64_t)h->nl * h->nchi},
      {"B3", h->B3, (int64_t)h->ntri * h->nchi},
      {"RB3", h->RB3, (int64_t)h->ntri * h->nchi},
      {"B1h3", h->B1h3, (int64_t)h->ntri * h->nchi},
      {"Ps", h->Ps, (int64_t)h->nl * h->nt * h->nt},
      {"B1h", h->B1hp, (int64_t)h->ntri * h->nt * h->nt * h->nt},
      {"zedges", h->zedges, h->nt + 1},
  };
  for (auto& t : tab) {
    if (strcmp(t.n, name) == 0) {
      *count = t.c;
      if (host && t.c > 0) {
        cudaStream_t s = (cudaStream_t)stream;
        WL_CHECK(h, cudaMemcpyAsync(host, t.p, sizeof(double) * t.c, cudaMemcpyDeviceToHost, s));
        WL_CHECK(h, cudaStreamSynchronize(s));
      }
      return COV_OK;
    }
  }
  return wl_fail(h, COV_ERR_INVALID, std::string("unknown table ") + name);
}

// One lane polls a device flag up to `spins` times with the bounded-wait
// protocol of the tensor-core kernels: on expiry it raises the status word
// and returns.  Nothing asynchronous (bulk copy, MMA) is in flight meanwhile.
__global__ void k_wait_flag(const volatile int* flag, unsigned spins, int* status) {
  if (threadIdx.x != 0) return;
  for (unsigned i = 0; i < spins; ++i) {
    if (*flag) return;
    __nanosleep(100);
  }
  atomicExch(status, 1);
}

extern "C" int cov_wait_selftest(cov_handle* h, unsigned spins, int flag_preset, void* stream) {
  if (!h) return COV_ERR_INVALID;
  if (spins == 0 || spins > (1u << 24))
    return wl_fail(h, COV_ERR_INVALID, "cov_wait_selftest: spins must be in [1, 2^24]");
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  if ((rc = wl_ensure(h, (void**)&h->wait_flag, sizeof(int), "self-test flag"))) return rc;
  WL_CHECK(h, cudaMemsetAsync(h->wait_flag, flag_preset ? 1 : 0, sizeof(int), s));  // nonzero word when set
  const bool deferred = h->deferred;
  h->deferred = false;
  rc = wl_tc_status_reset(h, s);
  if (rc == COV_OK) {
    k_wait_flag<<<1, 32, 0, s>>>(h->wait_flag, spins, h->tc_status);
    cudaError_t e = cudaGetLastError();
    rc = e != cudaSuccess ? wl_cuda(h, e, "k_wait_flag") : wl_tc_status_check(h, s);
  }
  h->deferred = deferred;
  return rc;
}

extern "C" int cov_profile(cov_handle* h, int enable) {
  if (!h) return COV_ERR_INVALID;
  h->prof = enable != 0;
  return COV_OK;
}

extern "C" int cov_stage_times(cov_handle* h, double* ms, int64_t* calls, int n_stages) {
  if (!h || n_stages < 0) return COV_ERR_INVALID;
  for (auto& se : h->pending) {
    cudaError_t e = cudaEventSynchronize(se.b);
    if (e != cudaSuccess) return wl_cuda(h, e, "cudaEventSynchronize");
    float t = 0.f;
    cudaEventElapsedTime(&t, se.a, se.b);
    h->stage_ms[se.stage] += t;
    h->stage_calls[se.stage] += 1;
    h->pool.push_back(se.a);
    h->pool.push_back(se.b);
  }
  h->pending.clear();
  for (int i = 0; i < n_stages && i < ST_COUNT; ++i) {
    if (ms) ms[i] = h->stage_ms[i];
    if (calls) calls[i] = h->stage_calls[i];
    h->stage_ms[i] = 0.0;
    h->stage_calls[i] = 0;
  }
  return COV_OK;
}

extern "C" const char* cov_stage_name(int stage) {
  return (stage >= 0 && stage < ST_COUNT) ? kStageNames[stage] : nullptr;
}

extern "C" const char* cov_last_error(const cov_handle* h) {
  return h ? h->err.c_str() : g_init_err.c_str();
}

extern "C" void cov_free(cov_handle* h) {
  if (!h) return;
  free_all(h);
  delete h;
}
