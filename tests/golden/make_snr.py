"""Write the oracle's cumulative S/N (P, B, joint) for a workload.

Calls only ``oracle/`` (every table, the full FP64 covariance in its block
form, and one scipy Cholesky per cumulative selection) and the parameter
dictionaries of the workloads module; the triangle counts are the stored
oracle counts of make_counts.py.  Output: tests/golden/snr_<workload>.txt with
one line "<which> <ell bin> <S/N>" per entry (which = P, B, J; NaN where the
selection is empty).

    python tests/golden/make_snr.py cfg2_5bin
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402

import make_counts  # noqa: E402
from oracle.covariance import TERMS_ALL  # noqa: E402
from oracle.pipeline import OracleRun  # noqa: E402
from oracle.snr import WHICH_B, WHICH_JOINT, WHICH_P, cumulative_snr  # noqa: E402
from paper_1812_07437_gb300 import workloads  # noqa: E402


def main(names):
    for name in names:
        t0 = time.time()
        ntri = make_counts.load(name)[1] if os.path.exists(os.path.join(HERE, f"counts_{name}.txt")) else None
        r = OracleRun(workloads.get(name), ntri=ntri)
        C = r.cov.full(TERMS_ALL)
        n_ell = len(r.T.ell)
        path = os.path.join(HERE, f"snr_{name}.txt")
        with open(path, "w") as fh:
            fh.write(f"# oracle cumulative S/N of workload {name} (M = {r.M}), every covariance term, "
                     f"written by make_snr.py from oracle/\n")
            for tag, w in (("P", WHICH_P), ("B", WHICH_B), ("J", WHICH_JOINT)):
                s = cumulative_snr(C, r.D, r.rows, n_ell, w)
                for c, v in enumerate(s):
                    fh.write(f"{tag} {c} {float(v)!r}\n")
        print(path, f"{time.time() - t0:.0f} s")


def load(name):
    """{'P'|'B'|'J': array[n_ell]} from a written file."""
    out = {}
    with open(os.path.join(HERE, f"snr_{name}.txt")) as fh:
        for line in fh:
            p = line.split()
            if not p or p[0].startswith("#"):
                continue
            out.setdefault(p[0], {})[int(p[1])] = float(p[2])
    return {k: np.array([v[c] for c in sorted(v)]) for k, v in out.items()}


if __name__ == "__main__":
    main(sys.argv[1:])
