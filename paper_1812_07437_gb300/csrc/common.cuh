// Internal declarations shared by the translation units of libwlcov.
// Device helpers are header-inline (no relocatable device code).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/wlcov.h"

#define WL_PI 3.14159265358979323846
#define WL_EULER_GAMMA 0.57721566490153286061
#define WL_C_OVER_H0 2997.92458      // Mpc/h
#define WL_RHO_CRIT0 2.77536627e11   // (Msun/h)/(Mpc/h)^3
#define WL_DELTA_C 1.686
#define WL_ST_Q 0.707
#define WL_ST_P 0.3
#define WL_DUFFY_A 10.14
#define WL_DUFFY_B (-0.081)
#define WL_DUFFY_C (-1.01)
#define WL_DUFFY_MPIVOT 2.0e12
#define WL_DELTA_VIR 200.0
#define WL_N_GL_CHI 64     // nodes of the chi(z) rule on [0, z]
#define WL_N_ZS 64         // nodes per source-redshift piece of W_i
#define WL_N_RK4 1024      // RK4 steps of the growth ODE
#define WL_A_INIT 1.0e-3
#define WL_BULLOCK_F 0.01        // Bullock et al. median: nu(F m, a_c) = 1, c = K a / a_c
#define WL_BULLOCK_K 4.0
#define WL_NFW_C_INTEGRAL 1.0    // below this concentration u is the quadrature of its defining integral
#define WL_A_COLLAPSE_MAX 100.0  // a_c where F m has not collapsed by then
#define WL_N_K 4096        // nodes of the sigma(R) and sigma_W^2 rules
#define WL_LNK_MIN (-11.512925464970229)  // ln 1e-5
#define WL_LNK_MAX (6.907755278982137)    // ln 1e3
#define WL_FD_H 1.0e-3     // ln k step of the 4th-order differences

// scalars kept on the device (index into h->scal)
enum { SC_CHIMAX = 0, SC_AMP = 1, SC_NOISE = 2, SC_D1 = 3, SC_STATUS = 7, SC_N = 8 };

struct DevCosmo {
  double Om, Ob, h, ns, sigma8, w0, Tcmb;
};

// timed stages (cov_stage_times)
enum {
  ST_TABLES = 0, ST_COUNTS, ST_SPECTRA, ST_ROWS_T, ST_SYRK_T, ST_GATHER, ST_ROWS_A, ST_SYRK_1H, ST_ROWS_S,
  ST_SYRK_SSC, ST_SNR_PACK, ST_SNR_CHOL, ST_SNR_PREFIX, ST_COUNT
};

struct StageEvent {
  int stage;
  cudaEvent_t a, b;
};

// Where a kernel stores element (r, c) of the lower triangle (c <= r).
//  rows : C[(r - row0) * ldc + c]                     (dense row-major band)
//  tiles: 256 x 256 lower tiles, tile (ti, tj) (tj <= ti) stored row-major
//         at tile index ti (ti + 1) / 2 + tj - tile0, 65536 doubles apart
// cuTensorMapEncodeTiled from the driver, looked up once per process
// (thread-safe: the serving scheduler runs requests on several host threads).
PFN_cuTensorMapEncodeTiled_v12000 wl_encode_tiled();
#define WL_TILE_CACHE 16
int wl_ensure(struct cov_handle* h, void** p, size_t bytes, const char* what);  // assemble.cu: allocate once
// Run f once per CUDA device for the calling thread's current device.
#define WL_MAX_DEVICES 64
template <typename F>
inline int wl_once_per_device(std::once_flag (&flags)[WL_MAX_DEVICES], int (&rc)[WL_MAX_DEVICES], F f) {
  int d = 0;
  cudaGetDevice(&d);
  if (d < 0 || d >= WL_MAX_DEVICES) return COV_ERR_INVALID;
  std::call_once(flags[d], [&] { rc[d] = f(); });
  return rc[d];
}

struct OutMap {
  double* C;
  int64_t ldc, row0, tile0;
  int tiled;
  __device__ __forceinline__ double* at(int64_t r, int64_t c) const {
    if (tiled) {
      int64_t ti = r >> 8, tj = c >> 8;
      return C + ((ti * (ti + 1) / 2 + tj - tile0) << 16) + ((r & 255) << 8) + (c & 255);
    }
    return C + (r - row0) * ldc + c;
  }
};
static inline OutMap out_rows(double* C, int64_t ldc, int64_t row0 = 0) { return OutMap{C, ldc, row0, 0, 0}; }
static inline OutMap out_tiles(double* C, int64_t row0) {
  int64_t t0 = row0 >> 8;
  return OutMap{C, 0, row0, t0 * (t0 + 1) / 2, 1};
}

struct cov_handle {
  int device = 0;
  size_t budget = 0, allocated = 0;
  cov_cosmology cosmo{};
  cov_nz nz{};
  cov_bins bins{};
  // plan (host)
  // nm counts the halo-integral nodes: n_mass mass nodes (nmb) times nc
  // concentration nodes, the concentration index fastest (nc = 1 without scatter)
  int nl = 0, nt = 0, nchi = 0, nm = 0, ntri = 0, K = 0, nmb = 0, nc = 1;
  int64_t M = 0, nP = 0, nB = 0;
  int nleg = 0;            // n_ell * n_tomo
  int64_t ntrow = 0;       // rows of the 1-halo trispectrum factor
  int rmax = 0;            // largest lattice radius
  double omega = 0, theta = 0, ell_f = 0;
  std::vector<double> ell_edges, ell, dell;
  std::vector<int64_t> s_lo, s_hi;
  std::vector<int32_t> tris;      // 3 per triple
  std::vector<int32_t> rowdesc;   // 8 per row
  // device: quadrature nodes on [-1, 1]
  double *gl64x = nullptr, *gl64w = nullptr, *glkx = nullptr, *glkw = nullptr, *glcx = nullptr, *glcw = nullptr;
  double *gl16x = nullptr, *gl16w = nullptr;  // 16-point rule of the small-concentration profiles
  // device: tables
  double* scal = nullptr;
  double *chi = nullptr, *wchi = nullptr, *z = nullptr, *D = nullptr;
  double *ell_d = nullptr, *m = nullptr, *om = nullptr, *sig0 = nullptr, *dlns = nullptr;
  double *mb = nullptr, *omb = nullptr;  // [nmb] mass nodes and weights; m, om: [nm] per (mass, c) node
  double *cs = nullptr, *cw = nullptr;   // [nc] ln c offsets from the median and their weights
  double *sigF = nullptr, *ac = nullptr; // [nmb] sigma(F m, 0) and collapse epoch a_c (Bullock median)
  double *f = nullptr, *b1 = nullptr, *b2 = nullptr, *U = nullptr, *Pl = nullptr, *dPl = nullptr;
  double* Psh = nullptr;  // [n_ell][n_chi][4] P_lin at the shifted k of the ln k differences
  double *zedges = nullptr, *norms = nullptr, *W = nullptr, *sigw2 = nullptr;
  int64_t *slo_d = nullptr, *shi_d = nullptr, *Nmodes = nullptr, *Ntri = nullptr;
  int32_t* rowtab = nullptr;  // [nl][2][rmax+1]: x_outer, x_inner per row
  int32_t *tris_d = nullptr, *rowdesc_d = nullptr;
  // device: spectra
  double *P3 = nullptr, *RP3 = nullptr, *B3 = nullptr, *RB3 = nullptr, *B1h3 = nullptr;
  double *Ps = nullptr, *B1hp = nullptr, *Bp = nullptr;
  // device: contraction operands and workspaces
  double* A = nullptr;      // [M][K] FP64 1-halo factor rows
  uint16_t *Ahi = nullptr, *Alo = nullptr;  // [M][K] BF16 split rows (tensor-core form)
  double* Ascale = nullptr; // per-row power-of-two scales of the split rows
  double *G2 = nullptr, *G3 = nullptr, *C2 = nullptr, *C3 = nullptr;  // row-builder factor tables
  // per leg-bin signature s (P: ell bin; B: nl + triangle): F[s][n][q] / 2^E[s][n] in FP32,
  // E[s][n], and the FP64 row-block maximum max_q |F[s][n][q]|
  double *invN = nullptr, *omN = nullptr;  // 1 / N(l^b), Omega / N_tri(t)
  // exact BB+PT couplings (COV_COUPLING_EXACT): per ell bin A one column per
  // pair (Y, Z) of other-leg bins, the int64 Gram matrix of their leg counts
  // (lower half) and kappa = G / (N_tri N_tri') (both halves, FP64)
  int coupling = 0;                 // COV_COUPLING_*
  std::vector<int32_t> kcol_h;      // [ntri][3] column of each leg in its bin
  std::vector<int32_t> kn_h;        // [nl] columns of each bin
  std::vector<int64_t> koff_h;      // [nl + 1] offset of each bin's ncol x ncol block
  std::vector<int32_t> kyz_h;       // per bin, per column: Y, Z
  std::vector<int32_t> ktri_h;      // per bin, per column: its triangle
  std::vector<int64_t> kcoff_h;     // [nl + 1] first column of each bin
  double* kap = nullptr;
  unsigned long long* kgram = nullptr;
  int32_t *kcol = nullptr, *kn = nullptr;
  int64_t* koff = nullptr;
  uint64_t* bmask = nullptr;  // ell bins present in each 32-row block (the product terms skip the rest)
  bool bmask_ready = false;
  int4* gblk = nullptr;       // 32 x 32 sub-blocks of the Gaussian-term diagonal blocks, by first row
  uint32_t* plist = nullptr;  // 32 x 32 lower blocks whose row blocks share an ell bin, (ti << 16) | tj
  std::vector<int64_t> plist_start;  // (host) index of row block ti's first listed block; nb + 1 entries
  bool plist_off = false;     // the list does not serve this layout (more than 64 ell bins or 65536 row blocks)
  std::vector<int64_t> gblk_row;  // (host) first row of each sub-block, ascending
  // launch orders of the tensor-core contraction, by tile-row range
  struct TileOrder {
    int kind = -1, group = 0;
    int64_t t0 = -1, t1 = -1, n = 0;
    int2* p = nullptr;  // a slot of tile_ring
  } tile_cache[WL_TILE_CACHE];
  int2* tile_ring = nullptr;
  size_t tile_ring_cap = 0;  // entries per slot
  int tile_cache_next = 0;
  float* Fsig = nullptr;
  float* FsigT = nullptr;  // the same for the bin pairs of the trispectrum rows
  int* EsigT = nullptr;
  double* MsigT = nullptr;
  int* Esig = nullptr;
  double* Msig = nullptr;
  int* tc_status = nullptr; // status word of the tensor-core contraction
  int* wait_flag = nullptr; // flag of the bounded-wait self-test
  double* Trows = nullptr;  // [ntrow][K]
  double* Tmat = nullptr;   // [ntrow][ntrow] lower
  uint16_t *Thi = nullptr, *Tlo = nullptr;  // split trispectrum rows (tensor-core form)
  double* Tscale = nullptr;
  double* Srows = nullptr;  // [M][nchi]
  double* work = nullptr;   // Cholesky workspace (M+1) rows
  int64_t work_n = 0;
  int64_t work_ld = 0;      // its row length (the last dense cov_snr)
  void* pca_buf = nullptr;  // PCA: G, y and the per-mode arrays
  size_t pca_bytes = 0;
  void* chol_scratch = nullptr;  // two slice buffers of the tensor-core trailing update
  size_t chol_scratch_n = 0;
  cudaStream_t side = nullptr;   // look-ahead stream of the Cholesky panel kernels
  cudaEvent_t ev_cols = nullptr, ev_panel = nullptr;
  int* chol_status = nullptr;
  bool spectra_ready = false;
  int row_set = 0, row_order = 0;  // COV_ROWS_*, COV_ORDER_*
  cov_cosmology* cosmo_d = nullptr;  // the cosmology the kernels read (device copy of cosmo)
  bool deferred = false;  // inside a captured batch step: no host synchronisation, no host-side copies
  bool chol_lookahead = true;  // Cholesky panel look-ahead on the side stream
  int chol_kernel = 0;         // Cholesky trailing update: 0 persistent (k_chol_upd), 1 one CTA per tile
  int tc_kernel = -1;          // contraction kernel: -1 automatic, 0 one CTA per tile, 1 CTA pairs
  int pr_group = 8;            // tile rows per group of the pair-tile launch order
  struct Selection {           // cumulative S/N selections (P, B, joint; all rows in place)
    bool ready = false;
    int64_t Ms = 0;
    int* perm = nullptr;
    int64_t* cnt = nullptr;
    double* out = nullptr;
  } sel[4];
  int* piv_status = nullptr;  // non-positive pivot seen (sticky inside a batch)
  double *batch_C = nullptr, *batch_D = nullptr;  // covariance and data vector of cov_batch_snr
  cudaStream_t batch_stream = nullptr;             // cov_batch_snr runs (and captures) on this stream
  cudaEvent_t batch_ev = nullptr;
  int ops_terms = -1, ops_precision = -1;  // operands prepared for the band assembly (-1: none)
  bool prof = false;
  std::vector<StageEvent> pending;
  std::vector<cudaEvent_t> pool;
  double stage_ms[ST_COUNT] = {0};
  int64_t stage_calls[ST_COUNT] = {0};
  std::string err;
};

// ---- host helpers (api.cu) -------------------------------------------------
int wl_fail(cov_handle* h, int code, const std::string& msg);
int wl_cuda(cov_handle* h, cudaError_t e, const char* what);
#define WL_CHECK(h, call)                                 \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return wl_cuda((h), e_, #call); \
  } while (0)
#define WL_LAUNCH(h, what)                                 \
  do {                                                     \
    cudaError_t e_ = cudaGetLastError();                   \
    if (e_ != cudaSuccess) return wl_cuda((h), e_, (what)); \
  } while (0)

// stage timing: the returned index pairs a begin with its end (-1 = off)
int wl_stage_begin(cov_handle* h, int stage, cudaStream_t s);
void wl_stage_end(cov_handle* h, int token, cudaStream_t s);

// ---- stage entry points (one per translation unit) -------------------------
int wl_quadrature(cov_handle* h, cudaStream_t s);  // tables.cu
int wl_tables(cov_handle* h, cudaStream_t s);   // tables.cu
int wl_counts(cov_handle* h, cudaStream_t s);   // counts.cu
int wl_couplings(cov_handle* h, cudaStream_t s);  // coupling.cu: exact BB+PT couplings (synchronises s)
void wl_coupling_plan(cov_handle* h);             // coupling.cu: columns per bin (host)
size_t wl_coupling_bytes(const cov_handle* h);    // coupling.cu: resident bytes of the exact couplings
int wl_spectra(cov_handle* h, double* d_D, cudaStream_t s);  // spectra.cu
int wl_assemble(cov_handle* h, double* d_C, int64_t ldc, unsigned terms, int precision, cudaStream_t s);
int wl_snr_tiles(cov_handle* h, double* Ct, const double* D, double* h_snr, cudaStream_t s);  // chol.cu
int wl_assemble_band(cov_handle* h, int64_t row0, int64_t nrows, OutMap out, unsigned terms, int precision,
                     cudaStream_t s);
int wl_snr(cov_handle* h, const double* d_C, int64_t ldc, const double* d_D, int which, double* h_snr,
           cudaStream_t s);  // chol.cu
int wl_gemm_lower_fp64(cov_handle* h, const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                       int64_t ldc, int64_t n, int64_t k, double alpha, double beta, bool lower_only,
                       cudaStream_t s);  // assemble.cu
int wl_syrk_tc(cov_handle* h, int nssc, OutMap out, cudaStream_t s, int64_t row1 = -1);  // syrk_tc.cu
int wl_syrk_tc_part(cov_handle* h, int nssc, OutMap out, int64_t r0, int64_t r1, cudaStream_t s);
int wl_tc_status_reset(cov_handle* h, cudaStream_t s);
int wl_tc_status_check(cov_handle* h, cudaStream_t s);
int wl_split_bytes(int64_t M, int K, size_t* bytes);                      // syrk_tc.cu
int wl_kpad(int K);  // K padded to the contraction's K granularity
int wl_request_bytes(const cov_nz* nz, const cov_bins* bins, int precision, unsigned terms, int64_t* M,
                     size_t* bytes);  // api.cu: host-only footprint estimate of one request
size_t wl_handle_bytes(const cov_handle* h);
void wl_set_global_error(const std::string& msg);  // api.cu: read by cov_last_error(NULL)
size_t wl_chol_tc_bytes(int64_t n);  // chol_tc.cu
int wl_chol_slice(cov_handle* h, OutMap W, int64_t k0, int kb, int64_t r0, int64_t r1, void* buf, cudaStream_t s);
bool wl_chol_fused_panel(const cov_handle* h, const OutMap& W);  // chol_tc.cu
int wl_side_stream(cov_handle* h);  // api.cu: the handle's high-priority side stream
int wl_chol_trsm_slice(cov_handle* h, OutMap W, int64_t k0, int kb, int64_t r0, int64_t r1, void* buf,
                       cudaStream_t s);
int wl_chol_update(cov_handle* h, OutMap W, int64_t r0, int64_t r1, const void* buf, int tj0, int ntj, int* status,
                   cudaStream_t s);
int wl_syrk_tc_rows(cov_handle* h, const void* hi, const void* lo, const double* rscale, int64_t rows, int Kp,
                    OutMap out, cudaStream_t s, int64_t row1 = -1);
// ---- device helpers ------------------------------------------------------------
__device__ __forceinline__ DevCosmo dev_cosmo(const cov_cosmology& c) {
  return DevCosmo{c.Om, c.Ob, c.h, c.ns, c.sigma8, c.w0, c.Tcmb};
}

// E(z) = H(z)/H0 for flat w0-CDM
__device__ __forceinline__ double dev_E(double z, const cov_cosmology& c) {
  double zp1 = 1.0 + z;
  return sqrt(c.Om * zp1 * zp1 * zp1 + (1.0 - c.Om) * pow(zp1, 3.0 * (1.0 + c.w0)));
}

// chi(z) with the 64-node Gauss-Legendre rule on [0, z]
__device__ __forceinline__ double dev_chi_of_z(double z, const cov_cosmology& c, const double* glx,
                                               const double* glw) {
  double s = 0.0;
  for (int i = 0; i < WL_N_GL_CHI; ++i) {
    double zz = 0.5 * z * (glx[i] + 1.0);
    s += glw[i] / dev_E(zz, c);
  }
  return WL_C_OVER_H0 * 0.5 * z * s;
}

// Eisenstein & Hu (1998) no-wiggle transfer function, k in h/Mpc
__device__ __forceinline__ double dev_eh_T(double k, const cov_cosmology& c) {
  double omh2 = c.Om * c.h * c.h, obh2 = c.Ob * c.h * c.h, fb = c.Ob / c.Om;
  double th = c.Tcmb / 2.7;
  double s = 44.5 * log(9.83 / omh2) / sqrt(1.0 + 10.0 * pow(obh2, 0.75));
  double al = 1.0 - 0.328 * log(431.0 * omh2) * fb + 0.38 * log(22.3 * omh2) * fb * fb;
  double ks = 0.43 * k * c.h * s;
  double ks2 = ks * ks;
  double geff = c.Om * c.h * (al + (1.0 - al) / (1.0 + ks2 * ks2));
  double q = k * th * th / geff;
  double L0 = log(2.0 * 2.718281828459045 + 1.8 * q);
  double C0 = 14.2 + 731.0 / (1.0 + 62.5 * q);
  return L0 / (L0 + C0 * q * q);
}

__device__ __forceinline__ double dev_plin(double k, double Dg, double amp, const cov_cosmology& c) {
  double T = dev_eh_T(k, c);
  return amp * pow(k, c.ns) * T * T * Dg * Dg;
}

__device__ __forceinline__ double dev_dplin(double k, double Dg, double amp, const cov_cosmology& c) {
  const double h = WL_FD_H;
  double f2 = dev_plin(k * exp(2 * h), Dg, amp, c), f1 = dev_plin(k * exp(h), Dg, amp, c);
  double m1 = dev_plin(k * exp(-h), Dg, amp, c), m2 = dev_plin(k * exp(-2 * h), Dg, amp, c);
  return (-f2 + 8.0 * f1 - 8.0 * m1 + m2) / (12.0 * h);
}

// spherical top-hat window and its derivative (Taylor series below x = 0.5)
__device__ __forceinline__ double dev_tophat(double x) {
  if (x < 0.5) {
    // coefficients 3 (-1)^n (2n+2)/(2n+3)!, n = 0..6
    const double c[7] = {1.0, -0.1, 1.0 / 280.0, -1.0 / 15120.0, 1.0 / 1330560.0, -1.0 / 172972800.0,
                         1.0 / 31135104000.0};
    double x2 = x * x, acc = 0.0;
    for (int n = 6; n >= 0; --n) acc = acc * x2 + c[n];
    return acc;
  }
  double sx, cx;
  sincos(x, &sx, &cx);
  return 3.0 * (sx - x * cx) / (x * x * x);
}

__device__ __forceinline__ double dev_dtophat(double x) {
  if (x < 0.5) {
    // 2n c_n for n = 1..7
    const double c[8] = {0.0, -0.1, 1.0 / 280.0, -1.0 / 15120.0, 1.0 / 1330560.0, -1.0 / 172972800.0,
                         1.0 / 31135104000.0, -1.0 / 7410154752000.0};
    double x2 = x * x, acc = 0.0;
    for (int n = 7; n >= 1; --n) acc = acc * x2 + 2.0 * n * c[n];
    return acc * x;
  }
  double sx, cx;
  sincos(x, &sx, &cx);
  return 3.0 * ((x * x - 3.0) * sx + 3.0 * x * cx) / (x * x * x * x);
}

// Sine and cosine integrals Si(x), Ci(x) for x > 0.
// x <= 4: the power series Si = sum (-1)^k x^(2k+1)/((2k+1)(2k+1)!),
//         Ci = gamma + ln x + sum_{k>=1} (-1)^k x^(2k)/(2k (2k)!).
// x > 4:  E1(ix) = -Ci(x) + i (Si(x) - pi/2) from the continued fraction
//         E1(z) = e^-z / (z + 1 - 1^2/(z + 3 - 2^2/(z + 5 - ...))) evaluated by
//         the modified Lentz method (Lentz 1976; Thompson & Barnett 1986).
__device__ __forceinline__ void dev_sici(double x, double* si, double* ci) {
  if (x <= 4.0) {
    double x2 = x * x;
    double ts = x, ssum = x;  // (-1)^k x^(2k+1)/(2k+1)!
    double tc = 1.0, csum = 0.0;  // (-1)^k x^(2k)/(2k)!
    for (int k = 1; k < 60; ++k) {
      double tk = 2.0 * k;
      tc *= -x2 / ((tk - 1.0) * tk);
      csum += tc / tk;
      ts *= -x2 / (tk * (tk + 1.0));
      ssum += ts / (tk + 1.0);
      if (fabs(ts) < 1e-18 * fabs(ssum) && fabs(tc) < 1e-18) break;
    }
    *si = ssum;
    *ci = WL_EULER_GAMMA + log(x) + csum;
    return;
  }
  const double tiny = 1e-300;
  // complex arithmetic on (re, im)
  double br = 1.0, bi = x;              // b = 1 + i x
  double cr = 1.0 / tiny, ci_ = 0.0;    // c
  double den = br * br + bi * bi;
  double dr = br / den, di = -bi / den; // d = 1/b
  double hr = dr, hi = di;              // h = d
  for (int i = 2; i < 400; ++i) {
    double a = -(double)(i - 1) * (i - 1);
    br += 2.0;
    // d = 1/(a d + b)
    double tr = a * dr + br, ti = a * di + bi;
    den = tr * tr + ti * ti;
    dr = tr / den;
    di = -ti / den;
    // c = b + a/c
    den = cr * cr + ci_ * ci_;
    double acr = a * cr / den, aci = -a * ci_ / den;
    cr = br + acr;
    ci_ = bi + aci;
    // del = c d ; h *= del
    double er = cr * dr - ci_ * di, ei = cr * di + ci_ * dr;
    double nr = hr * er - hi * ei, ni = hr * ei + hi * er;
    hr = nr;
    hi = ni;
    if (fabs(er - 1.0) + fabs(ei) < 1e-16) break;
  }
  double sx, cx;
  sincos(x, &sx, &cx);
  // E1(ix) = (cos x - i sin x) h
  double er = cx * hr + sx * hi, ei = cx * hi - sx * hr;
  *ci = -er;
  *si = 0.5 * WL_PI + ei;
}

// Normalised truncated-NFW Fourier profile u(k|m) with the mean-density
// (200 x rho_com) mass definition and the Duffy et al. (2008) concentration.
// median concentration c(m, z) (Duffy et al. 2008, 200 x mean density)
__device__ __forceinline__ double dev_conc(double m, double z) {
  return WL_DUFFY_A * pow(m / WL_DUFFY_MPIVOT, WL_DUFFY_B) * pow(1.0 + z, WL_DUFFY_C);
}

// u(k | m, c) for c < 1 from its defining integral in t = r / r_vir:
// int_0^1 w(t) sinc(K t) dt / int_0^1 w(t) dt, w(t) = t / (1 + c t)^2,
// K = k r_vir, both on one composite 16-point Gauss-Legendre rule (x16, w16
// on [-1, 1]) of ceil(K / (2 pi)) panels: no term cancels, so the result is
// good to rounding where the closed form loses ~1/c^2 of its digits.
__device__ __forceinline__ double dev_nfw_u_integral(double K, double c, const double* x16, const double* w16) {
  const int P = K > 2.0 * WL_PI ? (int)ceil(K / (2.0 * WL_PI)) : 1;
  const double hp = 1.0 / P;
  double num = 0.0, den = 0.0;
  for (int p = 0; p < P; ++p)
    for (int i = 0; i < 16; ++i) {
      const double t = (p + 0.5 * (x16[i] + 1.0)) * hp;
      const double ct = 1.0 + c * t;
      const double wt = w16[i] * t / (ct * ct);
      const double Kt = K * t;
      num += wt * sin(Kt) / Kt;
      den += wt;
    }
  return num / den;
}

// normalised Fourier transform u(k | m, c) of the truncated NFW profile: the
// closed form in sine/cosine integrals for c >= 1, the defining integral below
__device__ __forceinline__ double dev_nfw_u(double k, double m, double c, double rho, const double* x16,
                                           const double* w16) {
  double rv = cbrt(3.0 * m / (4.0 * WL_PI * WL_DELTA_VIR * rho));
  if (c < WL_NFW_C_INTEGRAL) return dev_nfw_u_integral(k * rv, c, x16, w16);
  double x = k * rv / c;
  double s1, c1, s2, c2;
  dev_sici(x, &s1, &c1);
  dev_sici((1.0 + c) * x, &s2, &c2);
  double sx, cx;
  sincos(x, &sx, &cx);
  double num = sx * (s2 - s1) - sin(c * x) / ((1.0 + c) * x) + cx * (c2 - c1);
  return num / (log(1.0 + c) - c / (1.0 + c));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// block-wide sum for blockDim.x a multiple of 32 (<= 1024); result on all threads
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}
