"""Data-vector layout (oracle): Sec. 5, text after Eq. eq:SN2.

* P entries: ell bins in increasing order; for each, tomographic pairs
  (i, j) with i <= j, j the faster index.
* B entries: closed bin triples (l_a <= l_b <= l_c) ordered with l_b the
  fastest and l_c the slowest index; a triple is kept when the bin centres
  close, centre_c <= centre_a + centre_b (reading: inclusive closure on
  centres; it reproduces the paper's printed vector sizes).
* For each triple, tomographic triples (i, j, k) with k the fastest and i the
  slowest index; scalene triples keep all n_t^3, two equal ell bins keep the
  tomographic indices of the equal legs non-decreasing, equilateral triples
  keep i <= j <= k (reading of the symmetry reduction).
* The joint vector is P followed by B (Eq. eq:SN2).
"""


def closed_triangles(centres):
    n = len(centres)
    out = []
    for c in range(n):
        for a in range(c + 1):
            for b in range(a, c + 1):
                if centres[c] <= centres[a] + centres[b]:
                    out.append((a, b, c))
    return out


def tomo_triples(tri, nt):
    a, b, c = tri
    out = []
    for i in range(nt):
        for j in range(nt):
            for k in range(nt):
                if a == b == c:
                    ok = i <= j <= k
                elif a == b:
                    ok = i <= j
                elif b == c:
                    ok = j <= k
                else:
                    ok = True
                if ok:
                    out.append((i, j, k))
    return out


def data_layout(centres, nt):
    """Rows of the joint vector: ('P', b, (i, j)) then ('B', t, (a,b,c), (i,j,k))."""
    rows = []
    for b in range(len(centres)):
        for i in range(nt):
            for j in range(i, nt):
                rows.append(("P", b, (i, j)))
    tris = closed_triangles(centres)
    for t, tri in enumerate(tris):
        for ijk in tomo_triples(tri, nt):
            rows.append(("B", t, tri, ijk))
    return rows, tris


def max_bin(row):
    return row[1] if row[0] == "P" else row[2][2]
