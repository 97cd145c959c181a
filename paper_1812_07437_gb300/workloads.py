"""Synthetic Euclid-like workloads (parameters only; no arithmetic of the method).

Both the CUDA path and the CPU oracle are driven from these dictionaries.
They stand in for the Euclid-like survey of the paper's Appendix A with the
cosmology and binning of the benchmark configurations:

* ``cfg1_1bin``  1 tomographic bin, 8 log ell bins in [20, 3000], N_chi = 64,
  N_M = 64, Gaussian + 1-halo terms only.
* ``cfg2_5bin``  5 equipopulated bins with photo-z scatter 0.05 (1+z), 12 log
  ell bins in [10, 5000], N_chi = 128, N_M = 96, every covariance term.
* ``cfg3_10bin`` 10 equipopulated bins (same n(z) and photo-z), 20 log ell
  bins in [10, 5000], N_chi = 256, N_M = 128, every term.
* ``cfg3_5bin`` / ``cfg3_4bin`` the 10-bin binning and quadrature (20 ell
  bins, N_chi = 256, N_M = 128, K = 32768) with 5 (M = 24400) or 4
  (M = 12944) tomographic bins: the reduced 10-bin configuration whose dense
  square fits (S/N of the split form against the FP64 form), and the
  few-GB case on which the 10-bin contraction is profiled.
* ``tiny_*`` / ``mid_*`` small cases that the oracle finishes in seconds but
  that still span several kernel tiles and a ragged tail.

Fixed choices where the configurations are silent: Omega_b = 0.049,
T_CMB = 2.7255 K, w0 = -1, k_max = 50 h/Mpc, m in [1e10, 1e16] Msun/h.
"""
import copy
import math

TERM_G = 1
TERM_1H = 2
TERM_BBPT = 4
TERM_PB = 8
TERM_SSC = 16
TERMS_ALL = 31

FIDUCIAL = dict(Om=0.31, Ob=0.049, h=0.68, ns=0.96, sigma8=0.83, w0=-1.0, Tcmb=2.7255)
# width of the lognormal concentration scatter of "model A" (Eq. LogNormC, Sec. 4.2.2; Sec. 5.4)
SIGMA_LNC = 0.18


def _nz(n_tomo, photoz):
    return dict(n_tomo=n_tomo, z0=0.636, alpha=1.5, zmin=0.0, zmax=3.0,
                photoz_sigma0=photoz, n_gal_arcmin2=30.0, sigma_e=0.3)


def _bins(n_ell, ell_min, ell_max, n_chi, n_mass):
    return dict(n_ell=n_ell, ell_min=ell_min, ell_max=ell_max, f_sky=0.36,
                n_chi=n_chi, n_mass=n_mass, m_min=1.0e10, m_max=1.0e16, k_max=50.0)


def _wl(name, n_tomo, photoz, n_ell, ell_min, ell_max, n_chi, n_mass, terms):
    return dict(name=name, cosmology=dict(FIDUCIAL), nz=_nz(n_tomo, photoz),
                bins=_bins(n_ell, ell_min, ell_max, n_chi, n_mass), terms=terms)


WORKLOADS = {
    "cfg1_1bin": _wl("cfg1_1bin", 1, 0.0, 8, 20.0, 3000.0, 64, 64, TERM_G | TERM_1H),
    "cfg2_5bin": _wl("cfg2_5bin", 5, 0.05, 12, 10.0, 5000.0, 128, 96, TERMS_ALL),
    "cfg3_10bin": _wl("cfg3_10bin", 10, 0.05, 20, 10.0, 5000.0, 256, 128, TERMS_ALL),
    "cfg3_5bin": _wl("cfg3_5bin", 5, 0.05, 20, 10.0, 5000.0, 256, 128, TERMS_ALL),
    "cfg3_4bin": _wl("cfg3_4bin", 4, 0.05, 20, 10.0, 5000.0, 256, 128, TERMS_ALL),
    # small cases for element-by-element parity of whole matrices
    "tiny_2bin": _wl("tiny_2bin", 2, 0.05, 5, 100.0, 800.0, 16, 12, TERMS_ALL),
    "mid_2bin": _wl("mid_2bin", 2, 0.0, 8, 20.0, 3000.0, 40, 36, TERMS_ALL),
    "mid_3bin": _wl("mid_3bin", 3, 0.05, 6, 30.0, 4000.0, 48, 40, TERMS_ALL),
}


# The paper's own set-up (Sec. 1, Appendix A and Sec. 5.4): its cosmology, 14
# log-spaced ell bins on [10, 5000], n(z) with z0 = 0.9/sqrt(2) normalised on
# [0.001, 2.5], 30 sources per arcmin^2, sigma_e = 0.3, f_sky = 0.36, no
# photometric-redshift scatter, halo masses from 1e9 to 1e16 Msun/h and the
# Bullock et al. median concentration (conc_model 1).
PAPER_COSMOLOGY = dict(Om=0.238, Ob=0.042, h=0.732, ns=0.958, sigma8=0.76, w0=-1.0, Tcmb=2.7255)


def paper_workload(n_tomo, n_chi=128, n_mass=96, sigma_e=0.3, n_conc=0):
    """The paper's set-up with n_tomo equipopulated bins (sigma_e = 0: no shape noise)."""
    return dict(name=f"paper_{n_tomo}bin", cosmology=dict(PAPER_COSMOLOGY),
                nz=dict(n_tomo=n_tomo, z0=0.9 / math.sqrt(2.0), alpha=1.5, zmin=0.001, zmax=2.5,
                        photoz_sigma0=0.0, n_gal_arcmin2=30.0, sigma_e=sigma_e),
                bins=dict(n_ell=14, ell_min=10.0, ell_max=5000.0, f_sky=0.36, n_chi=n_chi, n_mass=n_mass,
                          m_min=1.0e9, m_max=1.0e16, k_max=50.0, conc_model=1, n_conc=n_conc,
                          sigma_lnc=SIGMA_LNC),
                terms=TERMS_ALL)


# the paper's set-up with 2 tomographic bins (M = 818) at reduced quadrature and
# concentration scatter: a parity case that spans several tiles
WORKLOADS["paper_2bin"] = paper_workload(2, n_chi=32, n_mass=24, n_conc=4)
# the same set-up at the paper-replica quadrature (N_chi = 128, N_M = 96), no scatter
WORKLOADS["paper_2bin_full"] = paper_workload(2)
# the 5-bin set-up on which the paper compares the concentration models (Sec. 5.4)
WORKLOADS["paper_5bin"] = paper_workload(5)


def get(name, **overrides):
    """A deep copy of a named workload, with top-level or nested overrides."""
    wl = copy.deepcopy(WORKLOADS[name])
    for key, val in overrides.items():
        if isinstance(val, dict):
            wl[key].update(val)
        else:
            wl[key] = val
    return wl


def serving_requests(n, rate_hz, seed=2024, n_chi=128, n_mass=96):
    """A seeded stream of survey set-ups for the serving loop: Poisson
    arrivals at rate_hz; tomographic bins uniform in 1..10; ell bins uniform
    in 8..24 on [10, 5000]; each cosmological parameter uniform within +-5% of
    the fiducial.  Returns [(arrival time in s, workload dict)].  The
    quadrature (N_chi, N_M) is that of cfg2_5bin unless given."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    out = []
    for k in range(n):
        nt = int(rng.integers(1, 11))
        nl = int(rng.integers(8, 25))
        cos = {p: v * (1.0 + rng.uniform(-0.05, 0.05)) for p, v in FIDUCIAL.items() if p != "Tcmb"}
        cos["Tcmb"] = FIDUCIAL["Tcmb"]
        wl = _wl(f"serve_{k}", nt, 0.05, nl, 10.0, 5000.0, n_chi, n_mass, TERMS_ALL)
        wl["cosmology"] = cos
        out.append((float(t[k]), wl))
    return out


def fisher_workload(n_tomo, n_ell=16, n_chi=256, n_mass=128):
    """The batched Fisher set-up: 16 log ell bins on [10, 5000], N_chi = 256,
    N_M = 128, photo-z scatter 0.05 (1+z), every covariance term."""
    return _wl(f"fisher_{n_tomo}bin", n_tomo, 0.05, n_ell, 10.0, 5000.0, n_chi, n_mass, TERMS_ALL)


def fisher_cosmologies(seed=12345, n=64):
    """The fiducial cosmology, +-1% and +-2% steps in each of Omega_m, sigma_8,
    w0, h, n_s and Omega_b (24 points), then uniform draws within +-5% of the
    fiducial in all six (seeded) up to n cosmologies."""
    import numpy as np
    keys = ["Om", "sigma8", "w0", "h", "ns", "Ob"]
    out = [dict(FIDUCIAL)]
    for k in keys:
        for step in (0.01, -0.01, 0.02, -0.02):
            c = dict(FIDUCIAL)
            c[k] *= 1.0 + step
            out.append(c)
    rng = np.random.default_rng(seed)
    while len(out) < n:
        c = dict(FIDUCIAL)
        for k in keys:
            c[k] *= 1.0 + rng.uniform(-0.05, 0.05)
        out.append(c)
    return out[:n]
