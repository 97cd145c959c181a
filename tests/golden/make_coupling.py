"""Write the oracle's exact BB+PT coupling Gram matrices for benchmark binnings.

Calls only ``oracle/`` (lattice thresholds, closed triangles, the FFT leg
counts and integer Gram matrices of oracle/coupling.py) and the parameter
dictionaries of the workloads module.  Output:
tests/golden/coupling_<workload>.txt, per ell bin A a line
"A <bin> <ncol> <sha256>" (the sha256 of the ncol x ncol Gram matrix as
little-endian int64, row-major, columns in the order of the lines below),
then one line "C <Y> <Z> <G_cc> <sum_c' G_cc'>" per column (the row sum as an exact
integer: the entries reach 2^62.7 and a row sum can pass 2^63).

    python tests/golden/make_coupling.py cfg2_5bin cfg3_10bin
"""
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import counts as cnt  # noqa: E402
from oracle import coupling as cpl  # noqa: E402
from oracle.layout import closed_triangles  # noqa: E402
from oracle.survey import ell_bins  # noqa: E402
from paper_1812_07437_gb300 import workloads  # noqa: E402


def digest(G):
    return hashlib.sha256(np.ascontiguousarray(G, dtype="<i8").tobytes()).hexdigest()


def main(names):
    for name in names:
        b = workloads.get(name)["bins"]
        edges, centres, _ = ell_bins(b["n_ell"], b["ell_min"], b["ell_max"])
        _, s_lo, s_hi = cnt.lattice_thresholds(edges, b["f_sky"])
        tris = closed_triangles(centres)
        cols, _, G = cpl.grams(s_lo, s_hi, tris, workers=os.cpu_count())
        path = os.path.join(HERE, f"coupling_{name}.txt")
        with open(path, "w") as fh:
            fh.write(f"# exact BB+PT coupling Gram matrices of workload {name} written by make_coupling.py "
                     f"from oracle/\n")
            for A in range(len(s_lo)):
                fh.write(f"A {A} {len(cols[A])} {digest(G[A])}\n")
                for c, (Y, Z) in enumerate(cols[A]):
                    fh.write(f"C {Y} {Z} {int(G[A][c, c])} {sum(int(v) for v in G[A][c])}\n")
        print(path)


def load(name):
    """{bin: (sha256, [(Y, Z, G_cc, row sum), ...])} from a written file."""
    out = {}
    cur = None
    with open(os.path.join(HERE, f"coupling_{name}.txt")) as fh:
        for line in fh:
            p = line.split()
            if not p or p[0].startswith("#"):
                continue
            if p[0] == "A":
                cur = int(p[1])
                out[cur] = (p[3], [])
            elif p[0] == "C":
                out[cur][1].append(tuple(int(v) for v in p[1:5]))
    return out


if __name__ == "__main__":
    main(sys.argv[1:] or ["cfg2_5bin", "cfg3_10bin"])
