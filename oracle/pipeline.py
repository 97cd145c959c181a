"""One call that runs the oracle path for a workload dictionary.

Workload keys (plain parameters, no arithmetic):
  cosmology: Om, Ob, h, ns, sigma8, w0, Tcmb
  nz:        n_tomo, z0, alpha, zmin, zmax, photoz_sigma0, n_gal_arcmin2, sigma_e
  bins:      n_ell, ell_min, ell_max, f_sky, n_chi, n_mass, m_min, m_max, k_max
  terms:     bitmask of covariance terms (G=1, 1H=2, BBPT=4, PB=8, SSC=16)

coupling="exact" takes the BB+PT couplings as the exact lattice sums of
oracle/coupling.py (Eq. CovBB) instead of 1/N(l).
"""
import numpy as np

from . import counts as cnt
from . import coupling as cpl
from .covariance import Covariance
from .layout import data_layout
from .spectra import Spectra, Tables


class OracleRun:
    def __init__(self, wl, ntri=None, workers=None, coupling="modes"):
        self.wl = wl
        self.T = Tables(wl)
        nt = wl["nz"]["n_tomo"]
        self.rows, self.tris = data_layout(self.T.ell, nt)
        self.ell_f, self.s_lo, self.s_hi = cnt.lattice_thresholds(self.T.ell_edges, wl["bins"]["f_sky"])
        self.Nmodes = cnt.mode_counts(self.s_lo, self.s_hi)
        if ntri is None:
            ntri = cnt.triangle_counts(self.s_lo, self.s_hi, self.tris, workers=workers)
        self.Ntri = np.asarray(ntri, dtype=np.int64)
        self.S = Spectra(self.T, self.tris)
        kappa = None
        if coupling == "exact":
            _, self.col, self.G = cpl.grams(self.s_lo, self.s_hi, self.tris, workers=workers)
            kappa = cpl.kappa_table(self.col, self.G, self.Ntri, self.tris)
        elif coupling != "modes":
            raise ValueError(coupling)
        self.cov = Covariance(self.T, self.S, self.rows, self.tris, self.Nmodes, self.Ntri, kappa=kappa)
        self.D = np.array([self.S.data_value(r) for r in self.rows])

    @property
    def M(self):
        return len(self.rows)

    @property
    def n_P(self):
        return sum(1 for r in self.rows if r[0] == "P")
