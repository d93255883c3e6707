"""Write csrc/rbf_eps2_tables.cpp: the eps^2 coefficient of the universal
extension operator (Section 3.1, eq. defA) for Gaussians of small shape
parameter.

For Gaussians exp(-eps^2 |x - g|^2) centred at the points G, the universal
matrix A(eps) = Phi_{X,G} Phi_{G,G}^{-1} is a power series in eps^2 whose
constant term is the flat limit A0 (the Lagrange basis of the polynomials of
total degree <= q at G, which the library forms itself):

    A(eps) = A0 + eps^2 A2 + O(eps^4).

This script computes A2 = (A(eps1) - A0) / eps1^2 at eps1 = 1e-6 in
multiprecision (Phi_{G,G} has condition number ~ eps1^{-2q}; the error of A2 is
O(eps1^2) relative), on the reference square [-1,1]^2 and the point sets of the
library's universal stencil, in its order:

    X_S    K x K Gauss-Legendre nodes scaled by 1/3, index b*K + a (x fastest);
    X_Sbar Kbar x Kbar Chebyshev nodes of the first kind, Kbar = 3K/2;
    G      the Padua points of degree q = 10 (j outer, k inner, j + k even).

Run from the repository root:  python paper_2211_14537_gb300/tables/make_rbf_eps2.py
It needs mpmath and takes about a minute.
"""
import os
import sys

import mpmath as mp

Q = 10
KS = (6, 8, 16)
EPS1 = mp.mpf("1e-6")
DPS = 160

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "csrc", "rbf_eps2_tables.cpp")


def legendre_nodes(n):
    """Roots of P_n by Newton's method from the Chebyshev-like first guesses, ascending."""
    roots = []
    for k in range(n):
        x = mp.cos(mp.pi * (k + mp.mpf(3) / 4) / (n + mp.mpf(1) / 2))
        for _ in range(100):
            p0, p1 = mp.mpf(1), x
            for m in range(2, n + 1):
                p0, p1 = p1, ((2 * m - 1) * x * p1 - (m - 1) * p0) / m
            dp = n * (x * p1 - p0) / (x * x - 1)
            step = p1 / dp
            x -= step
            if abs(step) < mp.mpf(10) ** (-DPS + 10):
                break
        roots.append(x)
    return sorted(roots)


def points(K):
    kb = 3 * K // 2
    t = legendre_nodes(K)
    tc = [-mp.cos((2 * a + 1) * mp.pi / (2 * kb)) for a in range(kb)]
    X = [(t[a] / 3, t[b] / 3) for b in range(K) for a in range(K)]
    X += [(tc[a], tc[b]) for b in range(kb) for a in range(kb)]
    G = [(mp.cos(j * mp.pi / Q), mp.cos(k * mp.pi / (Q + 1)))
         for j in range(Q + 1) for k in range(Q + 2) if (j + k) % 2 == 0]
    return X + G, G


def a2_matrix(K):
    X, G = points(K)
    e2 = EPS1 * EPS1
    phi = lambda p, g: mp.exp(-e2 * ((p[0] - g[0]) ** 2 + (p[1] - g[1]) ** 2))
    mono = [(i, j) for i in range(Q + 1) for j in range(Q + 1 - i)]        # total degree <= q
    poly = lambda p: [p[0] ** i * p[1] ** j for i, j in mono]
    Wphi = mp.inverse(mp.matrix([[phi(gi, gj) for gj in G] for gi in G]))
    Wpol = mp.inverse(mp.matrix([poly(g) for g in G]))                      # rows: points, cols: monomials
    ng = len(G)
    rows = []
    for p in X:
        r_phi = [phi(p, g) for g in G]
        r_pol = poly(p)
        a_eps = [mp.fsum(r_phi[k] * Wphi[k, j] for k in range(ng)) for j in range(ng)]
        # A0 row: the interpolant through G of the monomials evaluated at p,
        # i.e. (V_p V_G^{-1}) with V the monomial Vandermonde rows
        a_0 = [mp.fsum(r_pol[m] * Wpol[m, j] for m in range(len(mono))) for j in range(ng)]
        rows.append([float((a_eps[j] - a_0[j]) / e2) for j in range(ng)])
    return rows


def main():
    mp.mp.dps = DPS
    parts = []
    for K in KS:
        rows = a2_matrix(K)
        nx, ng = len(rows), len(rows[0])
        vals = ",\n".join("    " + ", ".join("%.17g" % v for v in r) for r in rows)
        parts.append((K, nx, ng, "static const double kA2_K%d[%d * %d] = {\n%s};\n" % (K, nx, ng, vals)))
        print("K = %d: %d x %d" % (K, nx, ng), file=sys.stderr)
    with open(OUT, "w") as fh:
        fh.write("// rbf_eps2_tables.cpp -- written by tables/make_rbf_eps2.py; do not edit.\n")
        fh.write("//\n// A2, the eps^2 coefficient of the universal Gaussian operator\n")
        fh.write("// A(eps) = A0 + eps^2 A2 + O(eps^4) (Section 3.1, eq. defA) on [-1,1]^2, for the\n")
        fh.write("// universal stencil X_S u X_Sbar u G of leaf order K (row-major, NX x NG).\n")
        fh.write('#include "internal.h"\n\nnamespace vpx {\n\n')
        for _, _, _, body in parts:
            fh.write(body + "\n")
        fh.write("bool rbf_eps2_table(int K, const double **a2, int *nx, int *ng) {\n")
        fh.write("    switch (K) {\n")
        for K, nx, ng, _ in parts:
            fh.write("    case %d: *a2 = kA2_K%d; *nx = %d; *ng = %d; return true;\n" % (K, K, nx, ng))
        fh.write("    default: return false;\n    }\n}\n\n}  // namespace vpx\n")


if __name__ == "__main__":
    main()
