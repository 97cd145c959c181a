"""Plain FP64 CPU oracle for the tomographic weak-lensing P+B covariance path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline and reference arm) may import or run it.  It shares no code with the
CUDA library under ``paper_1812_07437_gb300/``; the two sides meet only through
the plain workload dictionaries in ``paper_1812_07437_gb300/workloads.py``,
which hold parameters and no arithmetic of the method.

Every function follows the paper (Rizzato, Benabed, Bernardeau & Lacasa,
arXiv:1812.07437) step by step, in the paper's notation, with numpy/scipy
library primitives (Gauss-Legendre nodes, sici, j1, erf, FFT, matmul, solve)
used as single steps.  Where the paper is silent or garbled the oracle follows
a fixed reading; each reading is named in the docstring of the function that
takes it.

Pins (tests that fix the oracle against something other than itself) live in
``tests/test_oracle_*.py``.  Functions with no pin say so in their docstring
with the words "parity unpinned".

Modules
-------
cosmology   background, growth, Eisenstein-Hu no-wiggle P_lin, sigma(m)
halo        Sheth-Tormen mass function, PBS biases, regularisation, NFW u(k)
survey      n(z), equipopulated bins, lensing kernels W_i, ell bins, noise
counts      integer mode counts N(ell^b) and triangle counts N_tri
layout      data-vector ordering of P and B entries
spectra     halo-model 3D polyspectra, responses, Limber projection
covariance  Gaussian, 1-halo, BB+PT, PB and super-sample terms
snr         cumulative signal-to-noise
pca         principal components of the joint covariance (Sec. 6): one-sided
            Jacobi eigen-pairs, S/N per mode and cumulative
pipeline    one call that runs the whole path for a workload dictionary
"""
