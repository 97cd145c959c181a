// Table builder: background, growth, linear power, halo model, profiles,
// lensing kernels and sigma_W^2 on the device (paper Secs. 2 and 4,
// Appendices A and B).  Every kernel writes FP64 tables laid out chi-major
// (node index outermost, mass index contiguous) so that the row builders read
// them coalesced.
#include "common.cuh"

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n with the
// three-term recurrence; nodes ascending.
__global__ void k_gauss_legendre(int n, double* x, double* w) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double zz = cos(WL_PI * (i + 0.75) / (n + 0.5));
  double pp = 1.0;
  // Newton from the cosine guess: quadratic convergence reaches double
  // precision in a handful of steps; stop at 5e-16 or after 10 steps
  for (int it = 0; it < 10; ++it) {
    double p1 = 1.0, p2 = 0.0;
    for (int j = 1; j <= n; ++j) {
      double p3 = p2;
      p2 = p1;
      p1 = ((2.0 * j - 1.0) * zz * p2 - (j - 1.0) * p3) / j;
    }
    pp = n * (zz * p1 - p2) / (zz * zz - 1.0);
    double z1 = zz;
    zz = z1 - p1 / pp;
    if (fabs(zz - z1) <= 5e-16) break;
  }
  double p1 = 1.0, p2 = 0.0;
  for (int j = 1; j <= n; ++j) {
    double p3 = p2;
    p2 = p1;
    p1 = ((2.0 * j - 1.0) * zz * p2 - (j - 1.0) * p3) / j;
  }
  pp = n * (zz * p1 - p2) / (zz * zz - 1.0);
  x[i] = -zz;
  w[i] = 2.0 / ((1.0 - zz * zz) * pp * pp);
}

__global__ void k_chimax(const cov_cosmology* __restrict__ cosmo_p, double zmax, const double* glx,
                         const double* glw, double* scal);

// Normalised probabilists' Hermite polynomials h_k = He_k / sqrt(k!) by the
// three-term recurrence h_{k+1} = (x h_k - sqrt(k) h_{k-1}) / sqrt(k+1),
// h_0 = 1, h_1 = x.  Returns h_n(x) and h_{n-1}(x) in *prev (n >= 1).
__device__ double dev_hermite_h(int n, double x, double* prev) {
  double p0 = 1.0, p1 = x;
  for (int k = 1; k < n; ++k) {
    double p2 = (x * p1 - sqrt((double)k) * p0) / sqrt(k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *prev = p0;
  return p1;
}

#define WL_GH_GRID 1023
// Concentration rule of Eq. LogNormC (one block of 256 threads): Gauss-Hermite
// nodes x_j and weights w_j of the standard normal density (sum w_j = 1),
// written as ln c offsets cs[j] = sigma x_j and weights cw[j].  The roots of
// He_n lie in |x| < sqrt(4n + 2); the grid of WL_GH_GRID intervals on that
// range is finer than their spacing for n <= 32, so each interval holds at
// most one root.  Each root is bisected to the last bit and weighted by
// w = 1 / (n h_{n-1}(x)^2).  n <= 1: one node, offset 0, weight 1.  A rule
// that does not find n roots is written with NaN weights.
__global__ void k_gauss_hermite(int n, double sigma, double* cs, double* cw) {
  __shared__ double root[WL_GH_GRID];
  if (n <= 1) {
    if (threadIdx.x == 0) {
      cs[0] = 0.0;
      cw[0] = 1.0;
    }
    return;
  }
  const double L = sqrt(4.0 * n + 2.0) + 0.5, dx = 2.0 * L / WL_GH_GRID;
  double pr;
  for (int i = threadIdx.x; i < WL_GH_GRID; i += blockDim.x) {
    double xa = -L + i * dx, xb = -L + (i + 1) * dx;
    double va = dev_hermite_h(n, xa, &pr), vb = dev_hermite_h(n, xb, &pr);
    double r = nan("");
    if (va == 0.0) {
      r = xa;  // a root on the left end; one on the right end belongs to the next interval
    } else if (vb != 0.0 && (va < 0.0) != (vb < 0.0)) {
      double lo = xa, hi = xb;
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double vm = dev_hermite_h(n, mid, &pr);
        if (vm == 0.0) {
          lo = hi = mid;
          break;
        }
        if ((vm < 0.0) == (va < 0.0))
          lo = mid;
        else
          hi = mid;
      }
      r = 0.5 * (lo + hi);
    }
    root[i] = r;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int found = 0;
    for (int i = 0; i < WL_GH_GRID; ++i) {
      if (root[i] != root[i]) continue;
      if (found < n) {
        double hprev;
        dev_hermite_h(n, root[i], &hprev);
        cs[found] = sigma * root[i];
        cw[found] = 1.0 / (n * hprev * hprev);
      }
      ++found;
    }
    if (found != n)
      for (int j = 0; j < n; ++j) cw[j] = nan("");
  }
}

// RK4 integration of the linear growth ODE in ln a from a = 1e-3 to a_t
__device__ double dev_growth_raw(double at, const cov_cosmology& c) {
  double x = log(WL_A_INIT), x1 = log(at);
  double h = (x1 - x) / WL_N_RK4;
  double d = WL_A_INIT, dp = WL_A_INIT;
  double om = c.Om, ode = 1.0 - c.Om, w = c.w0;
  // a^-3 and a^(-3(1+w)) at the RK4 stage points x, x + h/2, x + h advance
  // by constant factors, so the loop needs no transcendental per stage
  const double qm = exp(-1.5 * h), qd = exp(-1.5 * (1.0 + w) * h);
  double am = exp(-3.0 * x), ad = exp(-3.0 * (1.0 + w) * x);
  auto rhs = [&](double em_a, double ed_a, double yd, double yp, double* fd, double* fp) {
    double em = om * em_a;
    double ed = ode * ed_a;
    double e2 = em + ed;
    double dlnh = 0.5 * (-3.0 * em - 3.0 * (1.0 + w) * ed) / e2;
    *fd = yp;
    *fp = -(2.0 + dlnh) * yp + 1.5 * (em / e2) * yd;
  };
  for (int s = 0; s < WL_N_RK4; ++s) {
    double k1d, k1p, k2d, k2p, k3d, k3p, k4d, k4p;
    double am_h = am * qm, ad_h = ad * qd, am_1 = am_h * qm, ad_1 = ad_h * qd;
    rhs(am, ad, d, dp, &k1d, &k1p);
    rhs(am_h, ad_h, d + 0.5 * h * k1d, dp + 0.5 * h * k1p, &k2d, &k2p);
    rhs(am_h, ad_h, d + 0.5 * h * k2d, dp + 0.5 * h * k2p, &k3d, &k3p);
    rhs(am_1, ad_1, d + h * k3d, dp + h * k3p, &k4d, &k4p);
    am = am_1;
    ad = ad_1;
    d = d + (h / 6.0) * (k1d + 2.0 * k2d + 2.0 * k3d + k4d);
    dp = dp + (h / 6.0) * (k1p + 2.0 * k2p + 2.0 * k3p + k4p);
    x = x + h;
  }
  return d;
}

// chi(z_max)
__global__ void k_chimax(const cov_cosmology* __restrict__ cosmo_p, double zmax, const double* glx,
                         const double* glw, double* scal) {
  const cov_cosmology c = *cosmo_p;
  if (threadIdx.x == 0 && blockIdx.x == 0) scal[SC_CHIMAX] = dev_chi_of_z(zmax, c, glx, glw);
}

// D(z_n) = D_raw(a_n) / D_raw(1)
__global__ void k_growth_norm(int nchi, const double* scal, double* D) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < nchi) D[n] /= scal[SC_D1];
}

// line-of-sight nodes: chi_n (GL on [0, chi_max]), weights, z(chi_n), D(z_n);
// one node per block so that the sequential RK4 runs spread over the SMs
__global__ void k_los(const cov_cosmology* __restrict__ cosmo_p, int nchi, const double* glcx, const double* glcw,
                      const double* gl64x,
                      const double* gl64w, const double* scal, double* chi, double* wchi, double* z, double* D) {
  const cov_cosmology c = *cosmo_p;
  int n = blockIdx.x;
  if (threadIdx.x != 0 || n > nchi) return;
  if (n == nchi) {  // one extra block: the growth integration carried to a = 1
    double* sc = (double*)scal;
    sc[SC_D1] = dev_growth_raw(1.0, c);
    return;
  }
  double cm = scal[SC_CHIMAX];
  double ch = 0.5 * cm * (glcx[n] + 1.0);
  chi[n] = ch;
  wchi[n] = 0.5 * cm * glcw[n];
  double zz = ch / WL_C_OVER_H0;
  for (int it = 0; it < 40; ++it) {
    double f = dev_chi_of_z(zz, c, gl64x, gl64w) - ch;
    double step = f / WL_C_OVER_H0 * dev_E(zz, c);
    zz -= step;
    if (fabs(step) < 1e-15 * (1.0 + zz)) break;
  }
  z[n] = zz;
  D[n] = dev_growth_raw(1.0 / (1.0 + zz), c);  // normalised by k_growth_norm
}

// sigma_8 normalisation: amplitude A of P_lin(k,0) = A k^ns T^2
__global__ void k_amplitude(const cov_cosmology* __restrict__ cosmo_p, const double* glkx, const double* glkw,
                            double* scal) {
  const cov_cosmology c = *cosmo_p;
  __shared__ double sh[32];
  double half = 0.5 * (WL_LNK_MAX - WL_LNK_MIN), s = 0.0;
  for (int i = threadIdx.x; i < WL_N_K; i += blockDim.x) {
    double lk = WL_LNK_MIN + half * (glkx[i] + 1.0);
    double k = exp(lk), T = dev_eh_T(k, c), Wt = dev_tophat(8.0 * k);
    s += half * glkw[i] * k * k * k * pow(k, c.ns) * T * T / (2.0 * WL_PI * WL_PI) * Wt * Wt;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) scal[SC_AMP] = c.sigma8 * c.sigma8 / s;
}

// mass nodes, sigma(m, 0) and d ln sigma / d ln m (one block per mass node);
// m, om are also written per (mass, concentration) node: om times the c weight.
// For the Bullock median also sigma(F m, 0), the variance of the collapsing mass.
__global__ void k_sigma(const cov_cosmology* __restrict__ cosmo_p, cov_bins b, const double* glkx,
                        const double* glkw, const double* scal, int nc, const double* cw,
                        double* mb, double* omb, double* sig0, double* dlns, double* m, double* om, double* sigF) {
  const cov_cosmology c = *cosmo_p;
  __shared__ double sh[32];
  int q = blockIdx.x;
  double dl = log(b.m_max / b.m_min) / (b.n_mass - 1);
  double mq = b.m_min * exp(dl * q);
  double rho = WL_RHO_CRIT0 * c.Om;
  double R = cbrt(3.0 * mq / (4.0 * WL_PI * rho));
  const bool bullock = b.conc_model == COV_CONC_BULLOCK;
  double RF = cbrt(3.0 * (WL_BULLOCK_F * mq) / (4.0 * WL_PI * rho));
  double amp = scal[SC_AMP];
  double half = 0.5 * (WL_LNK_MAX - WL_LNK_MIN), s2 = 0.0, ds2 = 0.0, s2F = 0.0;
  for (int i = threadIdx.x; i < WL_N_K; i += blockDim.x) {
    double lk = WL_LNK_MIN + half * (glkx[i] + 1.0);
    double k = exp(lk), T = dev_eh_T(k, c);
    double d2 = amp * k * k * k * pow(k, c.ns) * T * T / (2.0 * WL_PI * WL_PI);
    double x = k * R, Wx = dev_tophat(x);
    s2 += half * glkw[i] * d2 * Wx * Wx;
    ds2 += half * glkw[i] * d2 * 2.0 * Wx * dev_dtophat(x) * k;
    if (bullock) {
      double WF = dev_tophat(k * RF);
      s2F += half * glkw[i] * d2 * WF * WF;
    }
  }
  s2 = block_sum(s2, sh);
  ds2 = block_sum(ds2, sh);
  if (bullock) s2F = block_sum(s2F, sh);
  if (threadIdx.x == 0) {
    mb[q] = mq;
    double w = dl * mq;
    if (q == 0 || q == b.n_mass - 1) w *= 0.5;
    omb[q] = w;
    sig0[q] = sqrt(s2);
    dlns[q] = (R / 6.0) * ds2 / s2;
    if (bullock) sigF[q] = sqrt(s2F);
    for (int j = 0; j < nc; ++j) {
      m[q * nc + j] = mq;
      om[q * nc + j] = w * cw[j];
    }
  }
}

// Collapse epoch of the Bullock et al. median (Sec. 5.4), one warp per mass
// node: a_c with D(a_c) sigma(F m, 0) = delta_c, D(1) = 1, D the growth ODE's
// solution (dev_growth_raw).  Each round the 32 lanes evaluate D at 32
// interior points of the bracket in ln a and keep the sub-interval where D
// crosses the target, 33 times narrower, until the bracket stops shrinking
// (about 11 rounds; at most 40).  a_c = WL_A_COLLAPSE_MAX where D stays below
// the target up to there; the start of the growth rule where D starts above it.
__global__ void k_collapse(const cov_cosmology* __restrict__ cosmo_p, const double* scal, const double* sigF,
                           double* ac) {
  const cov_cosmology c = *cosmo_p;
  const int q = blockIdx.x, lane = threadIdx.x;
  const double d1 = scal[SC_D1], target = WL_DELTA_C / sigF[q];
  double out;
  if (dev_growth_raw(WL_A_COLLAPSE_MAX, c) / d1 <= target) {
    out = WL_A_COLLAPSE_MAX;
  } else if (dev_growth_raw(WL_A_INIT, c) / d1 >= target) {
    out = WL_A_INIT;
  } else {
    double lo = log(WL_A_INIT), hi = log(WL_A_COLLAPSE_MAX);
    for (int it = 0; it < 40; ++it) {
      double w = (hi - lo) / 33.0;
      bool above = dev_growth_raw(exp(lo + (lane + 1) * w), c) / d1 >= target;
      unsigned mask = __ballot_sync(0xffffffffu, above);
      double nlo = lo + 32 * w, nhi = hi;
      if (mask) {
        int f = __ffs(mask) - 1;
        nlo = f ? lo + f * w : lo;
        nhi = lo + (f + 1) * w;
      }
      if (!(nlo > lo || nhi < hi) || !(nlo < nhi)) break;  // converged to the last bit
      lo = nlo;
      hi = nhi;
    }
    out = exp(0.5 * (lo + hi));
  }
  if (lane == 0) ac[q] = out;
}

__device__ __forceinline__ double st_amp() {
  return 1.0 / (1.0 + pow(2.0, -WL_ST_P) * tgamma(0.5 - WL_ST_P) / sqrt(WL_PI));
}

// Sheth-Tormen f_m, PBS biases and the m_min regularisation on the mass rule;
// one block per line-of-sight node.  The values are written for every
// concentration node of each mass node ([n][q * nc + j]), so the regularised
// halos at m_min carry the same concentration scatter as the others.
__global__ void k_halo(const cov_cosmology* __restrict__ cosmo_p, int nm, int nc, const double* D, const double* m,
                       const double* om,
                       const double* sig0, const double* dlns, double* f, double* b1, double* b2) {
  const cov_cosmology c = *cosmo_p;
  __shared__ double sh[32];
  int n = blockIdx.x;
  double rho = WL_RHO_CRIT0 * c.Om, A = st_amp();
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int q = threadIdx.x; q < nm; q += blockDim.x) {
    double sg = D[n] * sig0[q];
    double nu = (WL_DELTA_C / sg) * (WL_DELTA_C / sg);
    double qn = WL_ST_Q * nu, qp = pow(qn, WL_ST_P);
    double G = A * sqrt(qn / (2.0 * WL_PI)) * (1.0 + 1.0 / qp) * exp(-0.5 * qn);
    double fm = rho / (m[q] * m[q]) * G * (-2.0 * dlns[q]);
    double a = 0.5 / nu - WL_ST_P / (nu * (1.0 + qp)) - 0.5 * WL_ST_Q;
    double ap = -0.5 / (nu * nu) + WL_ST_P * (1.0 + (WL_ST_P + 1.0) * qp) / (nu * nu * (1.0 + qp) * (1.0 + qp));
    double b1L = -2.0 * nu * a / WL_DELTA_C;
    double b2L = (a * a + ap) * 4.0 * nu * nu / (WL_DELTA_C * WL_DELTA_C) + a * 2.0 * nu / (WL_DELTA_C * WL_DELTA_C);
    double bb1 = 1.0 + b1L, bb2 = (8.0 / 21.0) * b1L + b2L;
    for (int j = 0; j < nc; ++j) {
      size_t idx = ((size_t)n * nm + q) * nc + j;
      f[idx] = fm;
      b1[idx] = bb1;
      b2[idx] = bb2;
    }
    double wq = om[q] * m[q] / rho * fm;
    s0 += wq;
    if (q > 0) {
      s1 += wq * bb1;
      s2 += wq * bb2;
    }
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  s2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    size_t i0 = (size_t)n * nm * nc;
    double mr0 = m[0] / rho;
    double alpha0 = (1.0 - s0) / mr0;
    double ft = f[i0] + alpha0 / om[0];
    double den = om[0] * mr0 * ft;
    double a1 = (1.0 - s1) / den, a2 = (0.0 - s2) / den;
    for (int j = 0; j < nc; ++j) {
      f[i0 + j] = ft;
      b1[i0 + j] = a1;
      b2[i0 + j] = a2;
    }
  }
}

// NFW profiles on the Limber grid and P_lin, dP_lin/dln k at k = l_b/chi_n
// at every (mass, concentration) node: u(k | m_q, c_bar(m_q, z_n) exp(cs[j])),
// c_bar the Duffy fit or the Bullock median K / ((1 + z) a_c(m_q))
__global__ void k_profiles(const cov_cosmology* __restrict__ cosmo_p, cov_bins b, int nm, int nc, const double* cs,
                           const double* ac, const double* ell, const double* chi, const double* z,
                           const double* D, const double* m, const double* scal, const double* gl16x,
                           const double* gl16w, double* U, double* Pl, double* dPl, double* Psh) {
  __shared__ double x16[16], w16[16];
  if (threadIdx.x < 16) {
    x16[threadIdx.x] = gl16x[threadIdx.x];
    w16[threadIdx.x] = gl16w[threadIdx.x];
  }
  __syncthreads();
  const cov_cosmology c = *cosmo_p;
  int bn = blockIdx.x;  // b * nchi + n
  int nchi = b.n_chi;
  int bb = bn / nchi, n = bn % nchi;
  double k = ell[bb] / chi[n];
  bool valid = k <= b.k_max;
  double rho = WL_RHO_CRIT0 * c.Om;
  for (int q = threadIdx.x; q < nm; q += blockDim.x) {
    double cq = b.conc_model == COV_CONC_BULLOCK ? WL_BULLOCK_K / ((1.0 + z[n]) * ac[q / nc]) : dev_conc(m[q], z[n]);
    if (nc > 1) cq *= exp(cs[q % nc]);
    U[(size_t)bn * nm + q] = valid ? dev_nfw_u(k, m[q], cq, rho, x16, w16) : 0.0;
  }
  if (threadIdx.x < 4) {
    // P_lin at k exp(s), s = -2h, -h, +h, +2h (the 4th-order differences in ln k)
    const double sh[4] = {-2.0 * WL_FD_H, -WL_FD_H, WL_FD_H, 2.0 * WL_FD_H};
    double amp = scal[SC_AMP];
    Psh[(size_t)bn * 4 + threadIdx.x] = valid ? dev_plin(k * exp(sh[threadIdx.x]), D[n], amp, c) : 0.0;
  }
  if (threadIdx.x == 0) {
    double amp = scal[SC_AMP];
    Pl[bn] = valid ? dev_plin(k, D[n], amp, c) : 0.0;
    dPl[bn] = valid ? dev_dplin(k, D[n], amp, c) : 0.0;
  }
}

// ---- survey: equipopulated edges, bin normalisations, lensing kernels ----
__device__ __forceinline__ double cdf15(double z, double z0) {
  double x = pow(z / z0, 1.5);
  return 1.0 - (1.0 + x) * exp(-x);
}

__device__ __forceinline__ double nz_shape(double z, const cov_nz& nz) {
  return z * z * exp(-pow(z / nz.z0, nz.alpha));
}

__device__ __forceinline__ double bin_sel(double z, int i, const double* e, int nt, double s0) {
  double lo = e[i], hi = e[i + 1];
  if (s0 == 0.0) {
    bool last = (i == nt - 1);
    return (z >= lo && (last ? z <= hi : z < hi)) ? 1.0 : 0.0;
  }
  double s = sqrt(2.0) * s0 * (1.0 + z);
  return 0.5 * (erf((hi - z) / s) - erf((lo - z) / s));
}

__global__ void k_edges(cov_nz nz, double* e, double* scal) {
  int t = threadIdx.x;
  int nt = nz.n_tomo;
  if (t > nt) return;
  if (t == 0) {
    e[0] = nz.zmin;
    double nbar = nz.n_gal_arcmin2 * (10800.0 / WL_PI) * (10800.0 / WL_PI) / nt;
    scal[SC_NOISE] = nz.sigma_e * nz.sigma_e / nbar;
    return;
  }
  if (t == nt) {
    e[nt] = nz.zmax;
    return;
  }
  double g0 = cdf15(nz.zmin, nz.z0), g1 = cdf15(nz.zmax, nz.z0);
  double target = (double)t / nt, lo = nz.zmin, hi = nz.zmax;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if ((cdf15(mid, nz.z0) - g0) / (g1 - g0) < target)
      lo = mid;
    else
      hi = mid;
  }
  e[t] = 0.5 * (lo + hi);
}

// pieces of [a, b] split at the edges strictly inside it; returns the count
__device__ __forceinline__ int make_pieces(double a, double b, const double* e, int nt, double* pts) {
  int np = 0;
  pts[np++] = a;
  for (int i = 0; i <= nt; ++i)
    if (e[i] > a && e[i] < b) pts[np++] = e[i];
  pts[np++] = b;
  return np - 1;
}

__global__ void k_norms(cov_nz nz, const double* e, const double* gx, const double* gw, double* norms) {
  __shared__ double sh[32];
  int i = blockIdx.x, nt = nz.n_tomo;
  double pts[40];
  int np = make_pieces(nz.zmin, nz.zmax, e, nt, pts);
  double s = 0.0;
  for (int p = 0; p < np; ++p) {
    double a = pts[p], b = pts[p + 1], half = 0.5 * (b - a);
    for (int j = threadIdx.x; j < WL_N_ZS; j += blockDim.x) {
      double zz = a + half * (gx[j] + 1.0);
      s += half * gw[j] * nz_shape(zz, nz) * bin_sel(zz, i, e, nt, nz.photoz_sigma0);
    }
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) norms[i] = s;
}

// W_i(chi_n): one block per node, threads over the source-redshift nodes
__global__ void k_kernels(const cov_cosmology* __restrict__ cosmo_p, cov_nz nz, int nchi, const double* chi,
                          const double* z,
                          const double* e, const double* norms, const double* gx, const double* gw, double* W) {
  const cov_cosmology c = *cosmo_p;
  __shared__ double sh[32];
  int n = blockIdx.x, nt = nz.n_tomo;
  double ch = chi[n], zn = z[n];
  double pref = 1.5 * c.Om / (WL_C_OVER_H0 * WL_C_OVER_H0) * (1.0 + zn) * ch;
  double pts[40];
  int np = (zn < nz.zmax) ? make_pieces(zn, nz.zmax, e, nt, pts) : 0;
  // each thread owns one source node per piece: chi(z_s) and the geometric
  // weight are computed once and reused for every tomographic bin
  double acc[32];
  for (int i = 0; i < nt; ++i) acc[i] = 0.0;
  for (int p = 0; p < np; ++p) {
    double a = pts[p], b = pts[p + 1], half = 0.5 * (b - a);
    for (int j = threadIdx.x; j < WL_N_ZS; j += blockDim.x) {
      double zs = a + half * (gx[j] + 1.0);
      double cs = dev_chi_of_z(zs, c, gx, gw);
      double geo = half * gw[j] * nz_shape(zs, nz) * (cs - ch) / cs;
      for (int i = 0; i < nt; ++i) acc[i] += geo * bin_sel(zs, i, e, nt, nz.photoz_sigma0);
    }
  }
  for (int i = 0; i < nt; ++i) {
    double s = block_sum(acc[i], sh);
    if (threadIdx.x == 0) W[i * nchi + n] = (np > 0) ? pref * s / norms[i] : 0.0;
  }
}

// sigma_W^2(chi_n) of a disk of angular radius Theta (Appendix B)
__global__ void k_sigw2(const cov_cosmology* __restrict__ cosmo_p, double theta, const double* chi, const double* D,
                        const double* glkx,
                        const double* glkw, const double* scal, double* out) {
  const cov_cosmology c = *cosmo_p;
  __shared__ double sh[32];
  int n = blockIdx.x;
  double amp = scal[SC_AMP], half = 0.5 * (WL_LNK_MAX - WL_LNK_MIN), s = 0.0;
  for (int i = threadIdx.x; i < WL_N_K; i += blockDim.x) {
    double le = WL_LNK_MIN + half * (glkx[i] + 1.0);
    double eps = exp(le), x = eps * chi[n] * theta;
    double win = j1(x) / x;
    s += half * glkw[i] * eps * eps * win * win * dev_plin(eps, 1.0, amp, c);
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[n] = 4.0 / (2.0 * WL_PI) * s * D[n] * D[n];
}

// quadrature nodes depend on no cosmology: built once per handle
int wl_quadrature(cov_handle* h, cudaStream_t s) {
  k_gauss_legendre<<<1, 64, 0, s>>>(WL_N_GL_CHI, h->gl64x, h->gl64w);
  k_gauss_legendre<<<1, 32, 0, s>>>(16, h->gl16x, h->gl16w);
  k_gauss_legendre<<<(WL_N_K + 127) / 128, 128, 0, s>>>(WL_N_K, h->glkx, h->glkw);
  k_gauss_legendre<<<(h->nchi + 127) / 128, 128, 0, s>>>(h->nchi, h->glcx, h->glcw);
  k_gauss_hermite<<<1, 256, 0, s>>>(h->nc, h->bins.sigma_lnc, h->cs, h->cw);
  WL_LAUNCH(h, "quadrature kernels");
  return COV_OK;
}

int wl_tables(cov_handle* h, cudaStream_t s) {
  const cov_cosmology* c = h->cosmo_d;  // read by the kernels: a captured graph replays with new values
  const cov_bins b = h->bins;
  const cov_nz nz = h->nz;
  k_chimax<<<1, 1, 0, s>>>(c, nz.zmax, h->gl64x, h->gl64w, h->scal);
  k_los<<<h->nchi + 1, 32, 0, s>>>(c, h->nchi, h->glcx, h->glcw, h->gl64x, h->gl64w, h->scal, h->chi,
                                            h->wchi, h->z, h->D);
  k_growth_norm<<<(h->nchi + 127) / 128, 128, 0, s>>>(h->nchi, h->scal, h->D);
  k_amplitude<<<1, 256, 0, s>>>(c, h->glkx, h->glkw, h->scal);
  k_sigma<<<h->nmb, 256, 0, s>>>(c, b, h->glkx, h->glkw, h->scal, h->nc, h->cw, h->mb, h->omb, h->sig0, h->dlns,
                                 h->m, h->om, h->sigF);
  if (b.conc_model == COV_CONC_BULLOCK) k_collapse<<<h->nmb, 32, 0, s>>>(c, h->scal, h->sigF, h->ac);
  k_halo<<<h->nchi, 128, 0, s>>>(c, h->nmb, h->nc, h->D, h->mb, h->omb, h->sig0, h->dlns, h->f, h->b1, h->b2);
  k_profiles<<<h->nl * h->nchi, 128, 0, s>>>(c, b, h->nm, h->nc, h->cs, h->ac, h->ell_d, h->chi, h->z, h->D, h->m,
                                             h->scal, h->gl16x, h->gl16w, h->U, h->Pl, h->dPl, h->Psh);
  k_edges<<<1, 64, 0, s>>>(nz, h->zedges, h->scal);
  k_norms<<<h->nt, 64, 0, s>>>(nz, h->zedges, h->gl64x, h->gl64w, h->norms);
  k_kernels<<<h->nchi, 64, 0, s>>>(c, nz, h->nchi, h->chi, h->z, h->zedges, h->norms, h->gl64x, h->gl64w, h->W);
  k_sigw2<<<h->nchi, 256, 0, s>>>(c, h->theta, h->chi, h->D, h->glkx, h->glkw, h->scal, h->sigw2);
  WL_LAUNCH(h, "table kernels");
  return COV_OK;
}
