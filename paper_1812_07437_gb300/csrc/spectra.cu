// Halo-model 3D polyspectra, responses and their Limber projections (paper
// Sec. 4, Eqs. ImunuHalos, PspHMtot2, B1halo, B2halos, B3halos, PowerHMResp,
// BispHMResp, RespP, RespB; Eq. nProjection), and the row builders of the
// (chi, M) contractions: the 1-halo factor rows A (Eqs. CovPPNG, Ins5P,
// Ins6P), the 1-halo trispectrum rows of the PT term (Eq. CovBB) and the
// super-sample rows (Eq. WLSSCflatskyLimber).
//
// Layout: per-node spectra are [entry][n_chi] (node contiguous); factor rows
// are [row][n_chi * nm] with the halo-integral node index q contiguous,
// matching the chi-major halo tables U[b][n][q], f[n][q].  q runs over the
// mass nodes, or over (mass, concentration) pairs with the concentration
// fastest when the lognormal scatter of Eq. LogNormC is on: every sum over q
// here is then the mass and the concentration integral at once.
#include "common.cuh"

// One warp per (ell bin, node): I_2^0(k,k), I_1^1(k), I_2^1(k,k) -> P^HM and
// its response; the k_max rule zeroes everything beyond k_max.
__global__ void k_pspec(const cov_cosmology* __restrict__ cosmo_p, int nl, int nchi, int nm, double kmax,
                        const double* ell, const double* chi,
                        const double* m, const double* om, const double* f, const double* b1, const double* U,
                        const double* Pl, const double* dPl, double* P3, double* RP3) {
  const cov_cosmology c = *cosmo_p;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nl * nchi) return;
  int b = warp / nchi, n = warp % nchi;
  double rho = WL_RHO_CRIT0 * c.Om;
  double i20 = 0, i11 = 0, i21 = 0;
  const double* u = U + ((size_t)b * nchi + n) * nm;
  for (int q = lane; q < nm; q += 32) {
    double mr = m[q] / rho, g1 = om[q] * f[n * nm + q] * mr, uq = u[q];
    i20 += g1 * mr * uq * uq;
    i11 += g1 * b1[n * nm + q] * uq;
    i21 += g1 * mr * b1[n * nm + q] * uq * uq;
  }
  i20 = warp_sum(i20);
  i11 = warp_sum(i11);
  i21 = warp_sum(i21);
  if (lane == 0) {
    int bn = b * nchi + n;
    bool valid = ell[b] / chi[n] <= kmax;
    double pl = Pl[bn], rlin = 47.0 / 21.0 * pl - dPl[bn] / 3.0;
    P3[bn] = valid ? i20 + i11 * i11 * pl : 0.0;
    RP3[bn] = valid ? i11 * i11 * rlin + i21 : 0.0;
  }
}

__device__ __forceinline__ double f2k(double ka, double kb, double mu) {
  return 5.0 / 7.0 + 0.5 * mu * (ka / kb + kb / ka) + 2.0 / 7.0 * mu * mu;
}

__device__ __forceinline__ void mus3(double k1, double k2, double k3, double* m12, double* m23, double* m31) {
  *m12 = (k3 * k3 - k1 * k1 - k2 * k2) / (2.0 * k1 * k2);
  *m23 = (k1 * k1 - k2 * k2 - k3 * k3) / (2.0 * k2 * k3);
  *m31 = (k2 * k2 - k3 * k3 - k1 * k1) / (2.0 * k3 * k1);
}

__device__ __forceinline__ double bpt3(double k1, double k2, double k3, double P1, double P2, double P3) {
  double m12, m23, m31;
  mus3(k1, k2, k3, &m12, &m23, &m31);
  return 2.0 * f2k(k1, k2, m12) * P1 * P2 + 2.0 * f2k(k2, k3, m23) * P2 * P3 + 2.0 * f2k(k3, k1, m31) * P3 * P1;
}

// B^PT with side i scaled by exp(s) (the other two fixed); Pi_s is P_lin at
// the shifted side, read from the table of shifted linear spectra
__device__ __forceinline__ double bpt_shift(const double* k, const double* P, int i, double s, double Pi_s) {
  double kk[3] = {k[0], k[1], k[2]};
  double pp[3] = {P[0], P[1], P[2]};
  kk[i] *= exp(s);
  pp[i] = Pi_s;
  return bpt3(kk[0], kk[1], kk[2], pp[0], pp[1], pp[2]);
}

// One warp per (triple, node): B^HM, its response and the 1-halo B.
__global__ void k_bspec(const cov_cosmology* __restrict__ cosmo_p, int ntri, int nchi, int nm, double kmax,
                        const int32_t* tris,
                        const double* ell, const double* chi, const double* D, const double* m, const double* om,
                        const double* f, const double* b1, const double* b2, const double* U, const double* Pl,
                        const double* dPl, const double* Psh, const double* scal, double* B3, double* RB3,
                        double* B1h3) {
  const cov_cosmology c = *cosmo_p;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= ntri * nchi) return;
  int t = warp / nchi, n = warp % nchi;
  int l[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
  double rho = WL_RHO_CRIT0 * c.Om;
  // accumulators: I30, I31, I11[3], I12[3], I21[3] (pairs opposite leg x), I22[3]
  double i30 = 0, i31 = 0, i11[3] = {0, 0, 0}, i12[3] = {0, 0, 0}, i21[3] = {0, 0, 0}, i22[3] = {0, 0, 0};
  const double* u0 = U + ((size_t)l[0] * nchi + n) * nm;
  const double* u1 = U + ((size_t)l[1] * nchi + n) * nm;
  const double* u2 = U + ((size_t)l[2] * nchi + n) * nm;
  for (int q = lane; q < nm; q += 32) {
    double mr = m[q] / rho, g1 = om[q] * f[n * nm + q] * mr;
    double bb1 = b1[n * nm + q], bb2 = b2[n * nm + q];
    double u[3] = {u0[q], u1[q], u2[q]};
    double g3 = g1 * mr * mr * u[0] * u[1] * u[2];
    i30 += g3;
    i31 += g3 * bb1;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      i11[x] += g1 * bb1 * u[x];
      i12[x] += g1 * bb2 * u[x];
      double pu = g1 * mr * u[(x + 1) % 3] * u[(x + 2) % 3];
      i21[x] += pu * bb1;
      i22[x] += pu * bb2;
    }
  }
  i30 = warp_sum(i30);
  i31 = warp_sum(i31);
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    i11[x] = warp_sum(i11[x]);
    i12[x] = warp_sum(i12[x]);
    i21[x] = warp_sum(i21[x]);
    i22[x] = warp_sum(i22[x]);
  }
  if (lane != 0) return;
  int tn = t * nchi + n;
  double k[3], P[3], rl[3];
  bool valid = true;
  for (int x = 0; x < 3; ++x) {
    k[x] = ell[l[x]] / chi[n];
    valid = valid && (k[x] <= kmax);
    P[x] = Pl[l[x] * nchi + n];
    rl[x] = 47.0 / 21.0 * P[x] - dPl[l[x] * nchi + n] / 3.0;
  }
  if (!valid) {
    B3[tn] = 0.0;
    RB3[tn] = 0.0;
    B1h3[tn] = 0.0;
    return;
  }
  double m12, m23, m31;
  mus3(k[0], k[1], k[2], &m12, &m23, &m31);
  double mus[3] = {m12, m23, m31};  // cyclic pairs (0,1;2), (1,2;0), (2,0;1)
  double bpt = bpt3(k[0], k[1], k[2], P[0], P[1], P[2]);
  // B^2h: I_1^1(k_x) I_2^1(other two) P(k_x)
  double b2h = 0.0;
  for (int x = 0; x < 3; ++x) b2h += i11[x] * i21[x] * P[x];
  double b3h = i11[0] * i11[1] * i11[2] * bpt;
  for (int cyc = 0; cyc < 3; ++cyc) {
    int a = cyc, bq = (cyc + 1) % 3, cc = (cyc + 2) % 3;
    double s2 = mus[cyc] * mus[cyc] - 1.0 / 3.0;
    b3h += i11[a] * i11[bq] * i12[cc] * P[a] * P[bq];
    b3h += 4.0 / 7.0 * i11[a] * i11[bq] * s2 * P[a] * P[bq] * (1.0 - i11[cc]);
  }
  B3[tn] = i30 + b2h + b3h;
  B1h3[tn] = i30;
  // response (Eqs. BispHMResp, RespB)
  double bg2 = 2.0 * ((m12 * m12 - 1.0) * P[0] * P[1] + (m23 * m23 - 1.0) * P[1] * P[2] +
                      (m31 * m31 - 1.0) * P[2] * P[0]);
  const double h = WL_FD_H;
  double dsum = 0.0;
  for (int i = 0; i < 3; ++i) {
    const double* ps = Psh + ((size_t)l[i] * nchi + n) * 4;  // s = -2h, -h, +h, +2h
    dsum += (-bpt_shift(k, P, i, 2 * h, ps[3]) + 8.0 * bpt_shift(k, P, i, h, ps[2]) -
             8.0 * bpt_shift(k, P, i, -h, ps[1]) + bpt_shift(k, P, i, -2 * h, ps[0])) /
            (12.0 * h);
  }
  double rbpt = 433.0 / 126.0 * bpt + 5.0 / 126.0 * bg2 - dsum / 3.0;
  double r = i11[0] * i11[1] * i11[2] * rbpt;
  for (int x = 0; x < 3; ++x) r += i11[x] * i22[x] * P[x] + i11[x] * i21[x] * rl[x];
  RB3[tn] = r + i31;
}

// projected power spectra with noise: Ps[b][i][j]
__global__ void k_proj_p(int nl, int nt, int nchi, const double* chi, const double* wchi, const double* W,
                         const double* P3, const double* scal, double* Ps) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nl * nt * nt) return;
  int b = id / (nt * nt), i = (id / nt) % nt, j = id % nt;
  double s = 0.0;
  for (int n = 0; n < nchi; ++n)
    s += wchi[n] / (chi[n] * chi[n]) * W[i * nchi + n] * W[j * nchi + n] * P3[b * nchi + n];
  Ps[id] = s + (i == j ? scal[SC_NOISE] : 0.0);
}

// projected 1-halo bispectra for every tomographic triple: B1hp[t][i][j][k]
__global__ void k_proj_b(int ntri, int nt, int nchi, const double* chi, const double* wchi, const double* W,
                         const double* B1h3, double* B1hp) {
  int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int nt3 = nt * nt * nt;
  if (id >= (int64_t)ntri * nt3) return;
  int t = (int)(id / nt3), r = (int)(id % nt3);
  int i = r / (nt * nt), j = (r / nt) % nt, k = r % nt;
  double s = 0.0;
  for (int n = 0; n < nchi; ++n) {
    double c2 = chi[n] * chi[n];
    s += wchi[n] / (c2 * c2) * W[i * nchi + n] * W[j * nchi + n] * W[k * nchi + n] * B1h3[t * nchi + n];
  }
  B1hp[id] = s;
}

// data vector D (no noise): one thread per row
__global__ void k_datavec(int64_t M, int nchi, const int32_t* rd, const double* chi, const double* wchi,
                          const double* W, const double* P3, const double* B3, double* Dv) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= M) return;
  const int32_t* r = rd + 8 * a;
  double s = 0.0;
  if (r[0] == 0) {
    int b = r[1], i = r[4], j = r[5];
    for (int n = 0; n < nchi; ++n)
      s += wchi[n] / (chi[n] * chi[n]) * W[i * nchi + n] * W[j * nchi + n] * P3[b * nchi + n];
  } else {
    int t = r[7], i = r[4], j = r[5], k = r[6];
    for (int n = 0; n < nchi; ++n) {
      double c2 = chi[n] * chi[n];
      s += wchi[n] / (c2 * c2) * W[i * nchi + n] * W[j * nchi + n] * W[k * nchi + n] * B3[t * nchi + n];
    }
  }
  Dv[a] = s;
}

// 1-halo factor rows A[a][(n,q)] = sqrt(w_n omega_q f_nq / Omega) chi^(1-2mu)
// prod W (m_q/rho)^mu prod U; grid (row blocks of K), coalesced along K.
__global__ void k_rows_a(int64_t M, int nchi, int nm, double inv_omega, const cov_cosmology* __restrict__ cosmo_p,
                         const int32_t* rd,
                         const double* chi, const double* wchi, const double* W, const double* m, const double* om,
                         const double* f, const double* U, double* A) {
  const double rho = WL_RHO_CRIT0 * cosmo_p->Om;
  int64_t a = blockIdx.x;
  int K = nchi * nm;
  int kk = blockIdx.y * blockDim.x + threadIdx.x;
  if (a >= M || kk >= K) return;
  int n = kk / nm, q = kk % nm;
  const int32_t* r = rd + 8 * a;
  int mu = (r[0] == 0) ? 2 : 3;
  double mr = m[q] / rho;
  double v = sqrt(wchi[n] * om[q] * f[kk] * inv_omega);
  double ch = chi[n];
  v *= (mu == 2) ? 1.0 / (ch * ch * ch) : 1.0 / (ch * ch * ch * ch * ch);
  v *= (mu == 2) ? mr * mr : mr * mr * mr;
  v *= W[r[4] * nchi + n] * W[r[5] * nchi + n];
  v *= U[((size_t)r[1] * nchi + n) * nm + q] * U[((size_t)r[2] * nchi + n) * nm + q];
  if (mu == 3) v *= W[r[6] * nchi + n] * U[((size_t)r[3] * nchi + n) * nm + q];
  A[a * K + kk] = v;
}

// trispectrum rows for leg pairs (L1 <= L2), L = bin * nt + tomo
__global__ void k_rows_t(int nleg, int nt, int nchi, int nm, const cov_cosmology* __restrict__ cosmo_p,
                         const double* chi, const double* wchi,
                         const double* W, const double* m, const double* om, const double* f, const double* U,
                         double* Tr) {
  const double rho = WL_RHO_CRIT0 * cosmo_p->Om;
  int64_t r = blockIdx.x;
  int K = nchi * nm;
  int kk = blockIdx.y * blockDim.x + threadIdx.x;
  if (kk >= K) return;
  // invert the pair index r = L1 * (2 nleg - L1 + 1)/2 + (L2 - L1)
  int L1 = 0;
  int64_t base = 0;
  while (base + (nleg - L1) <= r) {
    base += nleg - L1;
    ++L1;
  }
  int L2 = L1 + (int)(r - base);
  int b1 = L1 / nt, t1 = L1 % nt, b2 = L2 / nt, t2 = L2 % nt;
  int n = kk / nm, q = kk % nm;
  double mr = m[q] / rho, ch = chi[n];
  double v = sqrt(wchi[n] * om[q] * f[kk]) / (ch * ch * ch) * mr * mr;
  v *= W[t1 * nchi + n] * W[t2 * nchi + n];
  v *= U[((size_t)b1 * nchi + n) * nm + q] * U[((size_t)b2 * nchi + n) * nm + q];
  Tr[r * K + kk] = v;
}

// super-sample rows S[a][n] = sqrt(w_n sigma_W^2) chi^(2-2mu) prod W R_a
__global__ void k_rows_s(int64_t M, int nchi, const int32_t* rd, const double* chi, const double* wchi,
                         const double* W, const double* sigw2, const double* RP3, const double* RB3, double* S) {
  int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= M * nchi) return;
  int64_t a = id / nchi;
  int n = (int)(id % nchi);
  const int32_t* r = rd + 8 * a;
  double ch = chi[n], v = sqrt(wchi[n] * sigw2[n]);
  if (r[0] == 0) {
    v *= W[r[4] * nchi + n] * W[r[5] * nchi + n] / (ch * ch) * RP3[r[1] * nchi + n];
  } else {
    double c2 = ch * ch;
    v *= W[r[4] * nchi + n] * W[r[5] * nchi + n] * W[r[6] * nchi + n] / (c2 * c2) * RB3[r[7] * nchi + n];
  }
  S[id] = v;
}

int wl_spectra(cov_handle* h, double* d_D, cudaStream_t s) {
  const cov_cosmology* c = h->cosmo_d;
  int nl = h->nl, nchi = h->nchi, nm = h->nm, nt = h->nt;
  double kmax = h->bins.k_max;
  int warps = nl * nchi;
  k_pspec<<<(warps * 32 + 255) / 256, 256, 0, s>>>(c, nl, nchi, nm, kmax, h->ell_d, h->chi, h->m, h->om, h->f,
                                                   h->b1, h->U, h->Pl, h->dPl, h->P3, h->RP3);
  if (h->ntri > 0) {
    warps = h->ntri * nchi;
    k_bspec<<<(warps * 32 + 255) / 256, 256, 0, s>>>(c, h->ntri, nchi, nm, kmax, h->tris_d, h->ell_d, h->chi, h->D,
                                                     h->m, h->om, h->f, h->b1, h->b2, h->U, h->Pl, h->dPl, h->Psh,
                                                     h->scal, h->B3, h->RB3, h->B1h3);
    int64_t nb = (int64_t)h->ntri * nt * nt * nt;
    k_proj_b<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(h->ntri, nt, nchi, h->chi, h->wchi, h->W, h->B1h3,
                                                          h->B1hp);
  }
  k_proj_p<<<(nl * nt * nt + 255) / 256, 256, 0, s>>>(nl, nt, nchi, h->chi, h->wchi, h->W, h->P3, h->scal, h->Ps);
  if (d_D)
    k_datavec<<<(unsigned)((h->M + 255) / 256), 256, 0, s>>>(h->M, nchi, h->rowdesc_d, h->chi, h->wchi, h->W,
                                                             h->P3, h->B3, d_D);
  WL_LAUNCH(h, "spectra kernels");
  h->spectra_ready = true;
  return COV_OK;
}

int wl_rows_a(cov_handle* h, cudaStream_t s) {
  dim3 g((unsigned)h->M, (h->K + 255) / 256);
  k_rows_a<<<g, 256, 0, s>>>(h->M, h->nchi, h->nm, 1.0 / h->omega, h->cosmo_d, h->rowdesc_d, h->chi, h->wchi, h->W,
                             h->m,
                             h->om, h->f, h->U, h->A);
  WL_LAUNCH(h, "k_rows_a");
  return COV_OK;
}

int wl_rows_t(cov_handle* h, cudaStream_t s) {
  dim3 g((unsigned)h->ntrow, (h->K + 255) / 256);
  k_rows_t<<<g, 256, 0, s>>>(h->nleg, h->nt, h->nchi, h->nm, h->cosmo_d, h->chi, h->wchi, h->W, h->m, h->om, h->f, h->U,
                             h->Trows);
  WL_LAUNCH(h, "k_rows_t");
  return COV_OK;
}

int wl_rows_s(cov_handle* h, cudaStream_t s) {
  int64_t n = h->M * h->nchi;
  k_rows_s<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(h->M, h->nchi, h->rowdesc_d, h->chi, h->wchi, h->W, h->sigw2,
                                                       h->RP3, h->RB3, h->Srows);
  WL_LAUNCH(h, "k_rows_s");
  return COV_OK;
}
