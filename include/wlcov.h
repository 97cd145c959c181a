/*
 * wlcov.h -- C ABI of the GB300 library for the joint tomographic weak-lensing
 * power spectrum + bispectrum covariance (Rizzato, Benabed, Bernardeau &
 * Lacasa, arXiv:1812.07437).
 *
 * One handle holds every device-resident table for one survey set-up
 * (cosmology, source distribution, binning).  All device pointers passed in
 * are caller-owned CUDA device memory; the handle owns its internal tables
 * and workspaces.  Calls taking a stream are ordered on that stream
 * (``stream`` is a cudaStream_t passed as void*, NULL = legacy default
 * stream).  A handle is not thread-safe: use one handle per host thread /
 * stream.
 *
 * Every call returns COV_OK (0) or a negative COV_ERR_* code; the message of
 * the last failure is available from cov_last_error().  No call aborts the
 * process; device-side failures (a non-positive pivot) are reported through a
 * device status word read back by the call that needs it.
 *
 * Matrix layout: covariance matrices are dense FP64, row-major, M x M with a
 * leading dimension ldc >= M; only the lower triangle (row >= column) is
 * written by cov_assemble and read by cov_snr.
 */
#ifndef WLCOV_H
#define WLCOV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define COV_OK 0
#define COV_ERR_INVALID (-1) /* bad argument or size                        */
#define COV_ERR_NOMEM (-2)   /* device allocation failed / over hbm_budget   */
#define COV_ERR_NOT_PD (-3)  /* Cholesky met a non-positive pivot            */
#define COV_ERR_TIMEOUT (-4) /* a bounded device wait gave up                */
#define COV_ERR_CUDA (-5)    /* any other CUDA runtime error                 */

/* covariance terms (bitmask), Sec. 3.2 and Appendix B of the paper */
#define COV_TERM_G 1u    /* Gaussian PP (Eq. CovPPG) and BB (App. B)          */
#define COV_TERM_1H 2u   /* 1-halo 4/5/6-point (Eqs. CovPPNG, Ins5P, Ins6P)   */
#define COV_TERM_BBPT 4u /* BB and PT products (Eq. CovBB)                    */
#define COV_TERM_PB 8u   /* PB products (Eq. Covpb)                           */
#define COV_TERM_SSC 16u /* super-sample term (Eq. WLSSCflatskyLimber)        */
#define COV_TERMS_ALL 31u

/* arithmetic of the (chi, M) contractions.  The split form's elements carry
 * an error of ~1e-5 sqrt(C_aa C_bb); a covariance whose unit-diagonal scaling
 * has eigenvalues near that (strongly overlapping tomographic kernels, e.g. no
 * photo-z scatter and several bins) can then lose positive definiteness and
 * the S/N returns COV_ERR_NOT_PD: assemble such covariances in COV_FP64. */
#define COV_FP64 0       /* plain FP64 on CUDA cores                          */
#define COV_SPLIT_BF16 1 /* tcgen05 tensor cores, A = hi + lo in BF16, FP32 acc */

/* selection for the signal-to-noise (Sec. 5, Eq. eq:SN2) */
#define COV_WHICH_P 0
#define COV_WHICH_B 1
#define COV_WHICH_JOINT 2

/* flat w0-CDM cosmology, c = 1, lengths in Mpc/h (Sec. 1) */
typedef struct {
  double Om, Ob, h, ns, sigma8, w0, Tcmb;
} cov_cosmology;

/* source distribution n(z) ~ z^2 exp(-(z/z0)^alpha) split into n_tomo
 * equipopulated bins with Gaussian photo-z scatter photoz_sigma0 (1+z)
 * (Sec. 2, Appendix A); shape noise sigma_e with n_gal_arcmin2 sources per
 * arcmin^2 in total (Eq. ShotNoise).  alpha must be 1.5. */
typedef struct {
  int n_tomo;
  double z0, alpha, zmin, zmax, photoz_sigma0, n_gal_arcmin2, sigma_e;
} cov_nz;

/* Median concentration c(m, z) of the NFW profiles (Sec. 4.1, Sec. 5.4). */
#define COV_CONC_DUFFY 0   /* Duffy et al. (2008), 200 x mean density: 10.14 (m/2e12)^-0.081 (1+z)^-1.01 */
#define COV_CONC_BULLOCK 1 /* Bullock et al. (2001), the paper's choice: K a(z)/a_c with nu(F m, a_c) = 1, */
                           /* F = 0.01, K = 4 (a_c capped at a = 100 where F m never collapses); c < 1   */
                           /* (late-collapsing masses) is allowed: u is then the quadrature of its      */
                           /* defining integral                                                          */

/* n_ell log-spaced ell bins on [ell_min, ell_max] (Sec. 3.2.1, App. A), sky
 * fraction f_sky, n_chi Gauss-Legendre line-of-sight nodes, n_mass log mass
 * nodes on [m_min, m_max] Msun/h, 3D cut k_max h/Mpc (Sec. 4.5), median
 * concentration conc_model (COV_CONC_*; zero-initialised: Duffy).
 *
 * Concentration scatter (Eq. LogNormC; the paper's "model A" of Sec. 5.4):
 * with n_conc >= 2 every halo integral of Eq. ImunuHalos also averages the
 * NFW profiles over a lognormal concentration of width sigma_lnc (0.18 in the
 * paper) about the median c(m, z), on an n_conc-point Gauss-Hermite rule in
 * ln c.  n_conc = 0 or 1 is the delta-function p(c) ("model B", the
 * default).  The 1-halo contraction then runs over n_chi * n_mass * n_conc
 * nodes: its work and its operand memory grow by n_conc.  n_conc <= 32,
 * 0 <= sigma_lnc <= 2, n_mass * max(n_conc, 1) <= 4096. */
typedef struct {
  int n_ell;
  double ell_min, ell_max, f_sky;
  int n_chi, n_mass;
  double m_min, m_max, k_max;
  int n_conc;
  double sigma_lnc;
  int conc_model;
} cov_bins;

/* Row set and row order of the data vector (Sec. 5). */
#define COV_ROWS_JOINT 0      /* P rows and B rows                                    */
#define COV_ROWS_P 1          /* power-spectrum rows only                             */
#define COV_ROWS_B 2          /* bispectrum rows only                                 */
#define COV_ORDER_NATURAL 0   /* P rows (ell bin slowest, i <= j), then B rows         */
                              /* (triangle: c slowest, then a, b; tomography fastest)  */
#define COV_ORDER_CUMULATIVE 1 /* by largest ell bin c: the P rows of bin c, then the */
                               /* B rows whose largest bin is c, for c = 0, 1, ...    */

typedef struct {
  int device;        /* CUDA device ordinal                                  */
  size_t hbm_budget; /* bytes the handle may allocate; 0 = no limit          */
  int rows;          /* COV_ROWS_*                                           */
  int order;         /* COV_ORDER_*: the cumulative order makes every        */
                     /* cumulative S/N selection a leading block (cov_snr_tiles) */
  int tc_kernel;     /* split-form contraction kernel: COV_TC_AUTO (CTA pairs */
                     /* where 2-CTA clusters fit) or COV_TC_SINGLE (one CTA   */
                     /* per 256 x 256 tile); both give the same sums          */
  int chol_kernel;   /* Cholesky trailing update (cov_snr, cov_snr_tiles):    */
                     /* COV_CHOL_AUTO (persistent, 128 x 32 tiles, epilogue   */
                     /* overlapping the next tile's MMAs) or COV_CHOL_TILE    */
                     /* (one CTA per 128 x 64 tile); bit-identical results    */
  int coupling;      /* coupling of the BB+PT terms (Eq. CovBB):             */
                     /* COV_COUPLING_MODES: 1/N(l^b) with the exact mode     */
                     /* count, the paper's prefactor 2 pi/(Omega l Delta l)  */
                     /* at its continuum value; COV_COUPLING_EXACT: the      */
                     /* exact lattice sum over the shared leg, see           */
                     /* cov_coupling_gram (built once, at cov_init)          */
} cov_opts;
#define COV_TC_AUTO 0
#define COV_TC_SINGLE 1
#define COV_CHOL_AUTO 0
#define COV_CHOL_TILE 1
#define COV_COUPLING_MODES 0
#define COV_COUPLING_EXACT 1

typedef struct cov_handle cov_handle;

/* Plan the data vector (layout of Sec. 5), allocate the device tables and
 * build every table of the path for this cosmology: background, growth,
 * P_lin, halo mass function, biases and regularisation (Sec. 4), NFW
 * profiles on the Limber grid k = l/chi, lensing kernels (Eqs.
 * KernelLensing1, LensEff), sigma_W^2 (App. B) and the exact integer mode and
 * triangle counts.  Synchronous.  *out receives the handle (NULL on error). */
int cov_init(const cov_cosmology* cosmo, const cov_nz* nz, const cov_bins* bins,
             const cov_opts* opts, cov_handle** out);

/* Rebuild every cosmology-dependent table (and the counts) for a new
 * cosmology without reallocation; stream-ordered. */
int cov_update(cov_handle* h, const cov_cosmology* cosmo, void* stream);

/* Sizes of the joint data vector D = {P, B} (Eq. eq:SN2): M = n_P + n_B,
 * and the number of closed bin triples.  row_desc, if not NULL, receives
 * M x 8 int32 host values: type (0 = P, 1 = B), three ell bins, three
 * tomographic bins (the P rows repeat the first bin and leave the third
 * tomographic slot -1), triple index (or the ell bin for P rows). */
int cov_layout(const cov_handle* h, int64_t* M, int64_t* n_P, int64_t* n_B, int64_t* n_tri,
               int32_t* row_desc);

/* Copy the exact integer counts to host memory: N(l^b) for the n_ell bins
 * (Eq. PSest) and N_tri for the n_tri closed triples (App. B, first
 * equality of the N_tri definition).  Synchronises the stream. */
int cov_counts(cov_handle* h, int64_t* N_ell, int64_t* N_tri, void* stream);

/* Exact bin-averaged coupling of the BB+PT terms (App. B: the binned
 * bispectrum estimator and Eq. CovBB).  A BB or PT Wick term joins leg x of
 * triangle bin tau to leg y of tau', both in ell bin A; with the polyspectra
 * constant over the bins its exact coupling is
 *   kappa = sum_{q in A} n_{tau,x}(q) n_{tau',y}(q) / (N_tri(tau) N_tri(tau')),
 * n_{tau,x}(q) = #{p in Y : q + p in Z} the number of lattice triangles of tau
 * whose leg x is the mode q ({Y, Z} the bins of the other two legs).  n
 * depends on A and the unordered pair {Y, Z} only: bin A has one column per
 * pair (Y <= Z) such that sorted (A, Y, Z) is a closed triple, in order of
 * first appearance over the triples and their legs.  With
 * opts->coupling == COV_COUPLING_EXACT, cov_init computes for every bin the
 * integer Gram matrix G_A[c][c'] = sum_q n_c(q) n_c'(q) (int64, exact) and
 * cov_assemble uses kappa = G / (N_tri N_tri') in place of 1/N(l^b).
 *
 * cov_coupling_gram copies bin `ell_bin`'s columns and Gram matrix to host
 * memory: on entry *ncol is the capacity of cols (2 * capacity int32: Y, Z)
 * and gram (capacity^2 int64, row-major, both halves); on return *ncol is the
 * number of columns, and nothing is copied if the capacity was too small (or
 * cols or gram is NULL).  COV_ERR_INVALID if the handle was created without
 * COV_COUPLING_EXACT or ell_bin is out of range.  Synchronises the stream. */
int cov_coupling_gram(cov_handle* h, int ell_bin, int* ncol, int32_t* cols, int64_t* gram, void* stream);

/* Predict the data vector: d_D[M] (device) receives P_ij(l) (Eqs.
 * nProjection, PspHMtot2) and B_ijk(l1,l2,l3) (Eq. BspHMtot) in the layout
 * order, without shot noise.  Also prepares the projected spectra the
 * covariance needs. */
int cov_spectra(cov_handle* h, double* d_D, void* stream);

/* Assemble the lower triangle of the joint covariance into d_C (device,
 * M x M, leading dimension ldc) as the sum of the selected terms.
 * precision selects the arithmetic of the 1-halo (chi, M) contraction
 * (COV_FP64 or COV_SPLIT_BF16); every other term is FP64.  Requires a
 * preceding cov_spectra on the same handle. */
int cov_assemble(cov_handle* h, double* d_C, int64_t ldc, unsigned terms, int precision, void* stream);

/* Output layouts of cov_assemble_band. */
#define COV_LAYOUT_ROWS 0  /* dense rows: element (r, c) at d_C[(r - row0) * ldc + c]                */
#define COV_LAYOUT_TILES 1 /* lower-packed 256 x 256 tiles: tile (ti, tj), tj <= ti, row-major, at  */
                           /* d_C + (ti (ti + 1) / 2 + tj - t0 (t0 + 1) / 2) * 65536, t0 = row0 / 256 */

/* Streaming assembly of one band of rows (Eqs. CovPPG, CovPPNG, Ins5P, Ins6P,
 * CovBB, Covpb, WLSSCflatskyLimber summed as in cov_assemble), for
 * covariances too large to hold as a dense square: the 10-bin, 20-ell-bin
 * data vector has M = 181350, 263 GB dense, 132 GB as lower tiles.
 * Writes the lower part (columns 0 .. r) of rows r in [row0, row0 + nrows)
 * into d_C (device, caller-owned) in the given layout:
 *   COV_LAYOUT_ROWS : ldc >= row0 + nrows, nrows * ldc doubles;
 *   COV_LAYOUT_TILES: ldc ignored; the band's tiles, 65536 doubles each.
 *   With row0 = 0 and nrows = M this is the whole lower-packed matrix.
 * Tile entries above the diagonal and below row M are not written.
 * row0 must be a multiple of 256 and row0 + nrows a multiple of 256 or M.
 * precision: COV_SPLIT_BF16 or COV_FP64 as in cov_assemble; COV_TERM_SSC
 * requires COV_TERM_1H.  The operands (factor rows, trispectrum table) are
 * built by the first band after cov_spectra (or a change of terms or
 * precision) and reused by the following bands; a band computes exactly what
 * cov_assemble computes for its rows.  Requires a preceding cov_spectra. */
int cov_assemble_band(cov_handle* h, int64_t row0, int64_t nrows, double* d_C, int64_t ldc, int layout,
                      unsigned terms, int precision, void* stream);

/* Cumulative signal-to-noise of the handle's whole row set (Eqs. SNprim,
 * eq:SN) in place on its lower-packed covariance: the form for data vectors
 * whose dense square (and a scaled copy of it) does not fit.  Requires a
 * handle created with order COV_ORDER_CUMULATIVE (the rows of every
 * cumulative selection then form a leading block) and d_Ct (device) holding
 * the lower-packed 256 x 256 tiles of rows 0..M, i.e. the tiles of M + 1 rows
 * ((t (t + 1) / 2) * 65536 doubles, t = M / 256 + 1), as written by
 * cov_assemble_band(h, 0, M, d_Ct, 0, COV_LAYOUT_TILES, ...).  d_Ct is
 * overwritten: Jacobi scaling, D' = d^-1/2 D (d_D: device, M) as row M, and
 * the same blocked FP64-accurate Cholesky as cov_snr; h_snr (host, n_ell)
 * receives S/N for ell_max = bin 0 .. n_ell - 1 of the handle's rows (P, B or
 * joint by the handle's row set).  COV_ERR_NOT_PD / COV_ERR_TIMEOUT as for
 * cov_snr; COV_ERR_INVALID for a handle not in cumulative order. */
int cov_snr_tiles(cov_handle* h, double* d_Ct, const double* d_D, double* h_snr, void* stream);

/* Cumulative signal-to-noise (Eqs. SNprim, eq:SN): h_snr[c] (host, n_ell
 * values) = sqrt(D^T C^-1 D) over the selected entries whose largest ell bin
 * is <= c, via a Jacobi-scaled FP64 Cholesky of a workspace copy (d_C is not
 * modified).  Returns COV_ERR_NOT_PD on a non-positive pivot.  Synchronises
 * the stream. */
int cov_snr(cov_handle* h, const double* d_C, int64_t ldc, const double* d_D, int which,
            double* h_snr, void* stream);

/* Copy an internal FP64 table to host memory for inspection (tests).  name is
 * one of "chi", "wchi", "z", "growth", "mass", "conc_offsets", "conc_weights",
 * "collapse_a" (Bullock median only; empty otherwise), "f", "b1", "b2", "U",
 * "Plin", "dPlin", "W", "sigw2", "P3", "RP3", "B3", "RB3", "B1h3", "Ps",
 * "B1h"; *count receives the number of doubles (pass
 * host = NULL to query).  "mass", "f", "b1", "b2" and "U" run over the
 * (mass, concentration) nodes, the concentration index fastest. */
int cov_table(cov_handle* h, const char* name, double* host, int64_t* count, void* stream);

/* Stage timing with CUDA events recorded on the caller's stream around each
 * stage (tables, counts, spectra, row builders, each contraction, the
 * gather pass, the S/N factorisation).  cov_profile(h, 1) starts recording;
 * cov_stage_times synchronises on the recorded events, writes the summed
 * milliseconds and the number of timed calls per stage into the first
 * n_stages entries of ms / calls (host arrays, either may be NULL) and
 * clears the record.  cov_stage_name(i) names stage i (NULL past the end). */
/* Self-test of failure detection (the paper has no counterpart).  Every wait
 * of the library's tensor-core kernels on an mbarrier is bounded: when it
 * expires, the kernel raises a status word, stops issuing work and returns,
 * and the call returns COV_ERR_TIMEOUT.  This call runs that protocol on a
 * wait that nothing asynchronous depends on: one kernel polls a device flag
 * up to `spins` times (1 <= spins <= 2^24, ~0.1 us apart).  With
 * flag_preset != 0 the flag is set before the kernel starts and the call
 * returns COV_OK; with flag_preset == 0 nothing sets it, the wait expires and
 * the call returns COV_ERR_TIMEOUT (message in cov_last_error(h)).  The
 * handle stays usable either way.  Synchronous on `stream`. */
int cov_wait_selftest(cov_handle* h, unsigned spins, int flag_preset, void* stream);

int cov_profile(cov_handle* h, int enable);
int cov_stage_times(cov_handle* h, double* ms, int64_t* calls, int n_stages);
const char* cov_stage_name(int stage);

/* Allocation-free cumulative S/N, for callers that cannot allocate device
 * memory: a host application that owns all device memory through its own
 * pool and forbids further cudaMalloc calls (a plugin inside a larger
 * framework, an embedded serving runtime with a fixed budget), or a loop that
 * must never stall on an allocation.  The paper has no counterpart; this is a
 * deployment variant of cov_snr.
 *
 * It runs the same Jacobi-scaled FP64 Cholesky as cov_snr on d_C (device,
 * M x M lower triangle, row-major, leading dimension ldc >= M) and d_D
 * (device, M values), both already in cumulative order, and writes
 * d_snr[c] = sqrt(D^T C^-1 D) over the first prefix[c] entries, for
 * c < n_prefix (1 <= n_prefix <= 64; prefix: host array, non-decreasing,
 * each <= M; an empty prefix gives NaN).  *d_status (device int) is set to 0,
 * or to 1 when a pivot was not positive.  Nothing is allocated and nothing
 * is synchronised: the call is ordered on stream and the caller reads
 * d_snr / d_status after it.  Because nothing is synchronised, a covariance
 * that is not positive definite is reported only through *d_status: the call
 * itself still returns COV_OK (its return code covers the arguments and the
 * launches), and d_snr then holds meaningless values.
 *
 * The workspace is one static device array of (COV_NOALLOC_MAX_M + 1)^2
 * doubles (32 MiB) that every GPU loading the library holds until the process
 * exits; M > COV_NOALLOC_MAX_M is rejected with COV_ERR_INVALID (message in
 * cov_last_error(NULL)).  The first call in each CUDA context (each device's
 * primary context, normally) looks up the array's device address with that
 * context current; make that first call before any stream capture.  After a
 * device reset the next call runs in a new context and looks the address up
 * again.  All calls share the array and it keeps the last call's
 * contents, so calls that overlap on the GPU race and must be serialised by
 * the caller. */
#define COV_NOALLOC_MAX_M 2047
int cov_snr_noalloc(const double* d_C, int64_t ldc, const double* d_D, int64_t M, const int64_t* prefix,
                    int n_prefix, double* d_snr, int* d_status, void* stream);

/* ---- Principal components of the joint covariance (Sec. 6) ---------------
 *
 * Eigen-pairs of the handle's covariance C (Eq. SNPCA: C = sum_a lambda_a v_a
 * v_a^T), the signal-to-noise of each uncorrelated mode (Eqs. NewObs,
 * SNperEign: (S/N)^2_a = (v_a . D)^2 / lambda_a) and its cumulative forms
 * (Eq. CumulSN).  The eigenvalues of these covariances span ~23 decades, so
 * they come from one-sided Jacobi on the Cholesky factor, which keeps every
 * eigenvalue to high relative accuracy (in FP64, on the GPU): the factor of
 * cov_snr (FP64-accurate), then sweeps of plane rotations of column pairs of
 * L^T in round-robin order until a sweep rotates no pair (at most 60 sweeps).
 *
 * d_C: device, M x M FP64 with the lower triangle (the upper is not read),
 * leading dimension ldc >= M, rows in the handle's order; d_D: device, M.
 * Host outputs of M values, each optional (NULL): h_lam the eigenvalues in
 * ascending order; h_snr2 the (S/N)^2 of the mode of each eigenvalue, same
 * order; h_cum_var the cumulative (S/N)^2 with modes by increasing variance
 * lambda; h_cum_info the cumulative (S/N)^2 with modes by decreasing (S/N)_a.
 * *info: M, sweeps, convergence, the total (S/N)^2 (= D^T C^-1 D), the fewest
 * modes, by decreasing (S/N)_a, whose cumulative S/N reaches 90/95/99% of the
 * total S/N, and host-clock timings.  The eigenvectors are not returned: the
 * per-mode S/N comes from the rotated factor and the solved data vector.
 * Allocates the handle's Cholesky workspace (as cov_snr) and M^2 + 9 M
 * doubles.  Synchronous.  COV_ERR_NOT_PD as cov_snr; COV_ERR_TIMEOUT if the
 * sweeps did not converge; COV_ERR_NOMEM beyond hbm_budget. */
typedef struct {
  int64_t M;
  int sweeps, converged;
  double total_snr2;
  int modes_90, modes_95, modes_99;
  double ms_cholesky, ms_jacobi;
} cov_pca_info;
int cov_pca(cov_handle* h, const double* d_C, int64_t ldc, const double* d_D, double* h_lam, double* h_snr2,
            double* h_cum_var, double* h_cum_info, cov_pca_info* info, void* stream);

/* ---- Batched cosmologies: one survey set-up, many cosmologies -------------
 *
 * For each of n cosmologies (cosmos, host array), the data vector (Eq.
 * nProjection; into h_D + k M when h_D is not NULL, host) and the three
 * cumulative S/N curves (Eqs. SNprim, eq:SN; h_snr + 3 k n_ell, host, in the
 * order P, B, joint) of the handle's survey set-up, with the covariance terms
 * `terms` in `precision`: the Fisher pattern (finite-difference steps around a
 * fiducial cosmology) and emulator training sets.  The first cosmology runs
 * eagerly and prepares everything; with COV_BATCH_TUNE it first runs once per
 * candidate launch configuration (tensor-core contraction in CTA pairs with
 * three launch-order groupings, or one CTA per tile; Cholesky with or without
 * panel look-ahead, persistent or one-tile trailing update), keeps the fastest
 * for this handle and reports the candidate times in *info.  The
 * cosmology-dependent step (tables, spectra, dense covariance, three S/N) is
 * then captured once into the body of a CUDA graph "while" node, between a
 * kernel that loads cosmology k from a device copy of the list and one that
 * stores its S/N (and D) and advances k: the other cosmologies run as one
 * graph launch, a loop on the device.  Where the driver cannot build that
 * graph, the step is captured alone and replayed once per cosmology
 * (info->single_launch tells which).  The exact counts are computed once.  Results equal those of cov_update + cov_spectra +
 * cov_assemble + cov_snr for each cosmology.  The handle keeps a dense M x M
 * covariance and the (M + 1)^2 Cholesky workspace.  A non-positive pivot or an
 * expired wait in any cosmology fails the whole batch (COV_ERR_NOT_PD /
 * COV_ERR_TIMEOUT).  Afterwards the handle holds the last cosmology. */
#define COV_BATCH_TUNE 1u

#define COV_BATCH_CANDIDATES 6
typedef struct {
  int tc_kernel;          /* contraction kernel used: 1 = CTA pairs, 0 = one CTA per tile, -1 = automatic       */
  int chol_lookahead;     /* 1: Cholesky panel look-ahead on a side stream                                    */
  double candidate_ms[COV_BATCH_CANDIDATES]; /* tuning, eager step per candidate: (pairs, group 8, look-ahead,
                             persistent update) = the default, then group 4, group 16, one CTA per tile, no
                             look-ahead, one-tile Cholesky update                                              */
  int tuned;              /* index of the candidate kept (0 without tuning)                                   */
  int pr_group;           /* tile rows per group of the pair-tile launch order                                */
  int chol_kernel;        /* Cholesky trailing update: 0 persistent, 1 one CTA per tile                       */
  int single_launch;      /* 1: the other cosmologies ran as one graph launch (a device-side loop)            */
  double first_ms;        /* the first cosmology, tuning included                                             */
  double capture_ms;      /* capture and instantiation of the step                                            */
  double replay_ms;       /* per further cosmology (host clock, copies included)                              */
} cov_batch_info;

int cov_batch_snr(cov_handle* h, const cov_cosmology* cosmos, int n, unsigned terms, int precision, double* h_D,
                  double* h_snr, unsigned flags, cov_batch_info* info, void* stream);

/* ---- Serving: continuous batching of covariance + S/N requests ----------
 *
 * A request is one covariance with every term and the three cumulative S/N
 * curves (Eqs. SNprim, eq:SN) for one survey set-up: its own cosmology,
 * tomographic bins and ell binning.  Requests arrive at any time and differ
 * in size by orders of magnitude.  The server runs n_slots host workers, each
 * with its own non-blocking CUDA stream, so the kernels of several requests
 * overlap on the GPU.  Admission is by HBM footprint: a request starts when a
 * worker is free and its footprint (a host-side upper estimate: tables,
 * dense covariance, contraction operands, Cholesky workspace) fits in
 * hbm_budget next to what running requests and resident state hold.  Requests
 * are taken in arrival order, except that a later request that fits may start
 * before an earlier one that does not yet fit (first fit); an earlier
 * request is passed over at most max_bypass times, after which nothing starts
 * before it.  A request whose footprint exceeds hbm_budget is rejected at
 * submission (state COV_REQ_REJECTED).  The device state of a finished
 * request (tables, counts, operands, covariance and Cholesky workspaces) stays
 * resident, keyed by its n(z) and binning, and a later request with the same
 * key reuses it through cov_update (new cosmology, no reallocation); idle
 * resident state is freed, least recently used first, when a new request
 * needs the room.  Every result equals that of the same request run alone.
 * All calls are thread-safe.  The paper has no counterpart: this is the
 * serving loop around cov_init/cov_update, cov_spectra, cov_assemble and
 * cov_snr. */
typedef struct cov_server cov_server;

typedef struct {
  int device;
  int n_slots;          /* requests in flight at once, 1..64                        */
  size_t hbm_budget;    /* bytes the server may hold; 0: 90% of free device memory  */
  int precision;        /* COV_SPLIT_BF16 or COV_FP64 (the 1-halo contraction)      */
  unsigned terms;       /* covariance terms, e.g. COV_TERMS_ALL                     */
  int max_bypass;       /* <= 0: 4                                                  */
  int dry_run_us;       /* > 0: no device work at all (scheduling only): each request
                           holds its slot and footprint for dry_run_us microseconds
                           and returns zero S/N; for testing the scheduler without
                           a GPU                                                   */
} cov_server_opts;

typedef struct {
  cov_cosmology cosmo;
  cov_nz nz;
  cov_bins bins;
} cov_request;

#define COV_REQ_QUEUED 0
#define COV_REQ_RUNNING 1
#define COV_REQ_DONE 2
#define COV_REQ_FAILED 3   /* rc holds the COV_ERR_* code; message in cov_server_error */
#define COV_REQ_REJECTED 4 /* footprint above hbm_budget */

typedef struct {
  int state, rc;
  int64_t M;          /* data-vector length                                  */
  int n_ell;
  int slot;           /* worker that ran it (-1 before)                      */
  int reused;         /* 1: ran on resident state of an earlier request      */
  size_t footprint;   /* bytes reserved for it while it ran                  */
  double t_submit, t_start, t_done; /* seconds on the server clock           */
} cov_request_info;

typedef struct {
  int64_t submitted, done, failed, rejected;
  size_t reserved;      /* bytes currently reserved (running + resident)    */
  size_t peak_reserved; /* maximum of reserved since creation               */
  size_t budget;
  int max_running;      /* most requests that ran at the same time          */
} cov_server_stats;

/* Create a server (starts its workers).  COV_ERR_INVALID for bad options. */
int cov_server_create(const cov_server_opts* opts, cov_server** out);
/* Queue a request; returns at once with its id (>= 0).  A request that can
 * never fit is recorded as COV_REQ_REJECTED (still COV_OK here). */
int cov_server_submit(cov_server* s, const cov_request* r, int64_t* id);
/* Wait up to timeout_s seconds (< 0: no limit, 0: poll) for request id to
 * finish.  Fills *info (may be NULL) and, when done, copies its S/N into
 * snr (host, 3 * n_ell doubles: P, B, joint; may be NULL).  Returns COV_OK
 * when the request has finished (done, failed or rejected: see info->state),
 * COV_ERR_TIMEOUT when it has not, COV_ERR_INVALID for an unknown id. */
int cov_server_wait(cov_server* s, int64_t id, double timeout_s, cov_request_info* info, double* snr);
/* Message of a failed request (empty otherwise). */
const char* cov_server_error(cov_server* s, int64_t id);
int cov_server_stats_get(cov_server* s, cov_server_stats* st);
/* Seconds since creation (the clock of t_submit / t_start / t_done). */
double cov_server_clock(cov_server* s);
/* Host-only footprint estimate that admission uses, and the data-vector length. */
int cov_request_footprint(const cov_request* r, int precision, unsigned terms, int64_t* M, size_t* bytes);
/* Wait for running requests, drop queued ones, free everything. */
void cov_server_free(cov_server* s);

const char* cov_last_error(const cov_handle* h);
void cov_free(cov_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* WLCOV_H */
