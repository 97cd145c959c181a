"""Write the oracle's exact integer counts for the benchmark workloads.

Calls only ``oracle/`` (lattice thresholds, direct mode enumeration, FFT
triangle counts) and the parameter dictionaries of the workloads module.
Output: tests/golden/counts_<workload>.txt with one line "N <b> <count>" per
ell bin and "T <t> <a> <b> <c> <count>" per closed bin triple.

    python tests/golden/make_counts.py cfg2_5bin cfg3_10bin
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import counts as cnt  # noqa: E402
from oracle.layout import closed_triangles  # noqa: E402
from oracle.survey import ell_bins  # noqa: E402
from paper_1812_07437_gb300 import workloads  # noqa: E402


def main(names):
    for name in names:
        b = workloads.get(name)["bins"]
        edges, centres, _ = ell_bins(b["n_ell"], b["ell_min"], b["ell_max"])
        ell_f, s_lo, s_hi = cnt.lattice_thresholds(edges, b["f_sky"])
        tris = closed_triangles(centres)
        N = cnt.mode_counts(s_lo, s_hi)
        T = cnt.triangle_counts(s_lo, s_hi, tris, workers=os.cpu_count())
        path = os.path.join(HERE, f"counts_{name}.txt")
        with open(path, "w") as fh:
            fh.write(f"# exact lattice counts of workload {name} written by make_counts.py from oracle/\n")
            for i, v in enumerate(N):
                fh.write(f"N {i} {int(v)}\n")
            for t, ((a, bb, c), v) in enumerate(zip(tris, T)):
                fh.write(f"T {t} {a} {bb} {c} {int(v)}\n")
        print(path)


def load(name):
    """(N(l^b) list, N_tri list) from a written file."""
    N, T = [], []
    with open(os.path.join(HERE, f"counts_{name}.txt")) as fh:
        for line in fh:
            p = line.split()
            if not p or p[0].startswith("#"):
                continue
            if p[0] == "N":
                N.append(int(p[2]))
            else:
                T.append(int(p[5]))
    return N, T


if __name__ == "__main__":
    main(sys.argv[1:] or ["cfg2_5bin", "cfg3_10bin"])
