"""Write the oracle's principal components of the joint covariance (Sec. 6,
Eqs. SNPCA, SNperEign, CumulSN) for the paper's own set-up.

Calls only ``oracle/`` (every table, the full FP64 covariance, and the
one-sided Jacobi eigen-solver of oracle/pca.py) and the parameter dictionaries
of the workloads module; the triangle counts are the stored oracle counts of
the paper's 14 ell bins (counts_paper_2bin_full.txt: they do not depend on the
tomography).  Output: tests/golden/pca_<name>.txt with the eigenvalues in
ascending order and the (S/N)^2 of each mode ("mode <a> <lambda_a> <snr2_a>"),
the total and the number of modes for 90/95/99% of the total S/N.

    python tests/golden/make_pca.py paper_1bin paper_2bin_full
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import make_counts  # noqa: E402
from oracle import pca  # noqa: E402
from oracle.covariance import TERMS_ALL  # noqa: E402
from oracle.pipeline import OracleRun  # noqa: E402
from paper_1812_07437_gb300 import workloads  # noqa: E402


def workload(name):
    if name == "paper_1bin":
        return workloads.paper_workload(1)
    return workloads.get(name)


def main(names):
    ntri = make_counts.load("paper_2bin_full")[1]
    for name in names:
        t0 = time.time()
        r = OracleRun(workload(name), ntri=ntri)
        out = pca.pca_snr(r.cov.full(TERMS_ALL), r.D)
        path = os.path.join(HERE, f"pca_{name}.txt")
        with open(path, "w") as fh:
            fh.write(f"# oracle PCA of the joint covariance of {name} (M = {r.M}), every term, written by "
                     f"make_pca.py from oracle/\n")
            fh.write(f"total {out['total']!r}\n")
            for f in (0.90, 0.95, 0.99):
                fh.write(f"modes {f} {pca.modes_for_fraction(out['snr2'], f)}\n")
            for a, (lam, s2) in enumerate(zip(out["lam"], out["snr2"])):
                fh.write(f"mode {a} {float(lam)!r} {float(s2)!r}\n")
        print(path, f"{time.time() - t0:.0f} s")


def load(name):
    """{'total': float, 'modes': {fraction: n}, 'lam': array, 'snr2': array}."""
    import numpy as np
    res = {"modes": {}, "lam": [], "snr2": []}
    with open(os.path.join(HERE, f"pca_{name}.txt")) as fh:
        for line in fh:
            p = line.split()
            if not p or p[0].startswith("#"):
                continue
            if p[0] == "total":
                res["total"] = float(p[1])
            elif p[0] == "modes":
                res["modes"][float(p[1])] = int(p[2])
            else:
                res["lam"].append(float(p[2]))
                res["snr2"].append(float(p[3]))
    res["lam"], res["snr2"] = np.array(res["lam"]), np.array(res["snr2"])
    return res


if __name__ == "__main__":
    main(sys.argv[1:])
