"""Pins of the CPU oracle against facts fixed by mathematics and the paper.

Each test checks the oracle against something other than itself:
Green's second identity (an independent boundary-integral evaluation of the
same area integrals), closed-form potentials (uniform and Gaussian sources),
exact reproduction of polynomials by the extension (Section 3.2: least squares
in a space that contains the data), brute-force tree invariants (Section 4)
and Lagrange-interpolation exactness.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import exp1

import workloads as W
from oracle import oracle as O

EPS = np.finfo(float).eps


def _green_area_integral(qfun, gradq, x, x0, x1, y0, y1):
    """int_B log|x-y| (Laplacian q)(y) dy by Green's second identity:
    2 pi q(x) [x in B] + sum over edges of int (log r dq/dn - q d(log r)/dn) ds,
    each edge integral by adaptive 1D quadrature split at the foot of x."""
    tot = 0.0
    corners = [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]
    normals = [(0, -1), (1, 0), (0, 1), (-1, 0)]
    for k in range(4):
        a = np.array(corners[k], float)
        b = np.array(corners[(k + 1) % 4], float)
        n = np.array(normals[k], float)
        L = np.linalg.norm(b - a)
        tdir = (b - a) / L
        s0 = float(np.clip(np.dot(x - a, tdir), 0.0, L))

        def integrand(s):
            y = a + s * tdir
            r = y - x
            r2 = r @ r
            return 0.5 * np.log(r2) * (gradq(y) @ n) - qfun(y) * (r @ n) / r2
        pts = [s0] if 0.0 < s0 < L else None
        v, _ = quad(integrand, 0.0, L, points=pts, epsabs=1e-15, epsrel=1e-14, limit=500)
        tot += v
    inside = x0 < x[0] < x1 and y0 < x[1] < y1
    return tot + (2.0 * math.pi * qfun(x) if inside else 0.0)


def _poly_q_tensor(K, cx, cy, h, seed):
    """q = sum c_ab u^(a+2) v^(b+2), a, b <= K-3: the Laplacian has degree up to
    K-1 in each variable (total degree up to 2K-4), i.e. it spans most of the
    leaf's tensor space Q_{K-1}, not only the total-degree subspace."""
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((K - 2, K - 2)) / (K * K)
    terms = [(a + 2, b + 2) for a in range(K - 2) for b in range(K - 2)]

    def q(y):
        u, v = (y[0] - cx) / h, (y[1] - cy) / h
        return sum(c[m - 2, n - 2] * u ** m * v ** n for m, n in terms)

    def gq(y):
        u, v = (y[0] - cx) / h, (y[1] - cy) / h
        gx = sum(c[m - 2, n - 2] * m * u ** (m - 1) * v ** n for m, n in terms) / h
        gy = sum(c[m - 2, n - 2] * n * u ** m * v ** (n - 1) for m, n in terms) / h
        return np.array([gx, gy])

    def lap(y):
        u, v = (y[0] - cx) / h, (y[1] - cy) / h
        return sum(c[m - 2, n - 2] * (m * (m - 1) * u ** (m - 2) * v ** n + n * (n - 1) * u ** m * v ** (n - 2))
                   for m, n in terms) / (h * h)
    return q, gq, lap


def _poly_q(K, cx, cy, h, seed):
    """Random q of total degree K+1 (so p = Laplacian q has total degree K-1)."""
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((K + 2, K + 2))
    terms = [(m, n) for m in range(K + 2) for n in range(K + 2 - m)]

    def q(y):
        u, v = (y[0] - cx) / h, (y[1] - cy) / h
        return sum(c[m, n] * u ** m * v ** n for m, n in terms)

    def gq(y):
        u, v = (y[0] - cx) / h, (y[1] - cy) / h
        gx = sum(c[m, n] * m * u ** (m - 1) * v ** n for m, n in terms if m >= 1) / h
        gy = sum(c[m, n] * n * u ** m * v ** (n - 1) for m, n in terms if n >= 1) / h
        return np.array([gx, gy])

    def lap(y):
        u, v = (y[0] - cx) / h, (y[1] - cy) / h
        s = 0.0
        for m, n in terms:
            if m >= 2:
                s += c[m, n] * m * (m - 1) * u ** (m - 2) * v ** n
            if n >= 2:
                s += c[m, n] * n * (n - 1) * u ** m * v ** (n - 2)
        return s / (h * h)
    return q, gq, lap


def test_gauss_legendre_exact_on_monomials():
    L = O.lib()
    for n in (4, 8, 12, 16, 20):
        x = np.zeros(n)
        w = np.zeros(n)
        L.orc_gauss_legendre(n, O._ptr(x), O._ptr(w))
        assert np.all(np.diff(x) > 0)
        for k in range(2 * n):
            exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
            assert abs(np.sum(w * x ** k) - exact) < 1e-14


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("K", [8, 16])
@pytest.mark.parametrize("where", ["self", "self_corner_node", "edge_near", "corner_near", "adjacent", "diag",
                                   "far", "far2", "far4"])
def test_leaf_integrals_match_green_identity(K, where, tensor):
    """Near/self/far leaf integrals of a polynomial density against Green's identity."""
    L = O.lib()
    t, _ = O.gauss_legendre(K)
    cx, cy, h = 0.1, -0.2, 0.05
    x = {
        "self": (cx + 0.3 * h, cy - 0.7 * h),
        "self_corner_node": (cx + h * t[-1], cy + h * t[0]),
        "edge_near": (cx + 1.003 * h, cy + 0.2 * h),
        "corner_near": (cx - 1.0001 * h, cy - 1.0002 * h),
        "adjacent": (cx + 2.5 * h, cy + 0.1 * h),
        "diag": (cx + 1.9 * h, cy + 1.9 * h),
        "far": (cx + 5.0 * h, cy - 3.1 * h),
        "far2": (cx + 3.05 * h, cy + 0.9 * h),
        "far4": (cx - 9.5 * h, cy + 2.0 * h),
    }[where]
    x = np.array(x)
    q, gq, lap = (_poly_q_tensor if tensor else _poly_q)(K, cx, cy, h, seed=K * 7 + len(where))
    X, Y = np.meshgrid(cx + h * t, cy + h * t, indexing="xy")
    nodes = np.stack([X.ravel(), Y.ravel()], axis=1)
    p = np.array([lap(y) for y in nodes])
    I = np.zeros(K * K)
    L.orc_leaf_basis_integrals(K, O._ptr(np.ascontiguousarray(t)), cx, cy, h, x[0], x[1], O._ptr(I))
    got = I @ p
    want = _green_area_integral(q, gq, x, cx - h, cx + h, cy - h, cy + h)
    scale = np.max(np.abs(p)) * h * h * (1 + abs(math.log(h)))
    assert abs(got - want) <= 1e-12 * scale, (got, want, scale)


def _uniform_tree(K, level, dom=None):
    dom = dom or W.WholeBoxDomain()
    return O.build_tree(dom, W.TreeOptions(K=K, min_level=level, max_level=level), lambda xy: 0 * xy[:, 0])


def test_potential_of_unit_source_on_D():
    """f = 1 on all of D: V(x) = (1/2pi) int_D log|x-y| dy, here evaluated by
    Green's identity with q = |y - x|^2 / 4 (Laplacian 1)."""
    tree = _uniform_tree(8, 3)
    vals = np.ones((tree.n_leaves, 1, 64))
    rng = np.random.default_rng(3)
    tg = np.concatenate([O.all_leaf_nodes(tree)[::97], rng.uniform(-0.5, 0.5, (8, 2))])
    V = O.volume_potential(tree, vals, tg)[:, 0]
    for k, x in enumerate(tg):
        q = lambda y, x=x: ((y[0] - x[0]) ** 2 + (y[1] - x[1]) ** 2) / 4.0
        gq = lambda y, x=x: np.array([(y[0] - x[0]) / 2.0, (y[1] - x[1]) / 2.0])
        want = _green_area_integral(q, gq, x, -0.5, 0.5, -0.5, 0.5) / (2 * math.pi)
        assert abs(V[k] - want) < 1e-14, (x, V[k], want)


def test_potential_of_gaussian_matches_closed_form():
    """f = exp(-r^2/s^2) has V(r) = (s^2/4)(ln r^2 + E1(r^2/s^2)); the source is
    negligible on the edge of D.  Error is the leaf interpolation error."""
    s, c = 0.05, np.array([0.03, -0.02])
    f = W.make_gaussian(c, s)
    tree = _uniform_tree(16, 4)
    nodes = O.all_leaf_nodes(tree)
    vals = f(nodes).reshape(tree.n_leaves, 1, 256)
    rng = np.random.default_rng(5)
    idx = rng.choice(len(nodes), 24, replace=False)
    tg = np.concatenate([nodes[idx], [[0.0301, -0.0199], [0.2, 0.3], [-0.41, 0.45]]])
    V = O.volume_potential(tree, vals, tg)[:, 0]
    r2 = np.sum((tg - c) ** 2, axis=1)
    want = (s * s / 4) * (np.log(r2) + exp1(r2 / (s * s)))
    assert np.max(np.abs(V - want)) < 1e-12 * np.max(np.abs(want)) * 10


def test_potential_linear_in_source_and_zero_leaves_skipped():
    tree = _uniform_tree(8, 2)
    rng = np.random.default_rng(11)
    a = rng.standard_normal((tree.n_leaves, 1, 64))
    b = rng.standard_normal((tree.n_leaves, 1, 64))
    a[3] = 0.0
    tg = rng.uniform(-0.5, 0.5, (5, 2))
    va = O.volume_potential(tree, a, tg)
    vb = O.volume_potential(tree, b, tg)
    vab = O.volume_potential(tree, np.concatenate([a, 2 * a - b], axis=1), tg)
    assert np.allclose(vab[:, 0], va[:, 0], rtol=0, atol=1e-14)
    assert np.allclose(vab[:, 1], 2 * va[:, 0] - vb[:, 0], rtol=0, atol=1e-13)


def _extension_operator_norm(tree, meta, i, targets):
    off, n, masks = meta[i]
    M, _ = O.extend_cut_leaf(tree.leaves[i], tree.K, tree.t, masks, np.eye(n), targets)
    return np.abs(M).sum(axis=1).max()


POLY_CASES = {
    "disk_l3_k8": lambda: W.disk_sincos(level=3, K=8),
    "disk_l4_k8": lambda: W.disk_sincos(level=4, K=8),
    "disk_l4_k16": lambda: W.disk_sincos(level=4, K=16),
    # multiply connected: Omega outside three inclusions, extension into each hole
    "exterior_l5_k8": lambda: W.exterior_three_stars(K=8, tol=0, min_level=5),
}


@pytest.mark.parametrize("wl", list(POLY_CASES))
def test_extension_reproduces_total_degree_q_polynomials(wl):
    """Section 3.2 least squares on P_q: a polynomial of total degree q = 10
    (N_G = 66) is reproduced at every extension node, up to rounding times the
    conditioning of the extrapolation, on every cut leaf whose interior
    stencil points determine P_q (all but a few, where a small part of the
    extension square lies in Omega)."""
    w = POLY_CASES[wl]()
    K = w.opts.K
    tree = O.build_tree(w.domain, w.opts, w.sources[0])
    q = O.stencil_params(K)[0]
    rng = np.random.default_rng(w.opts.min_level * 100 + K)
    cc = rng.standard_normal((q + 1, q + 1))

    def f(xy):
        x, y = 3 * xy[:, 0], 3 * xy[:, 1]
        return sum(cc[m, n] * x ** m * y ** n for m in range(q + 1) for n in range(q + 1 - m))
    pts, meta = O.stencil_points(tree, w.domain)
    vals, _ = O.leaf_values(tree, w.domain, f(pts)[:, None], meta)
    owned = {}
    for j, o in enumerate(tree.owner):
        if o >= 0:
            owned.setdefault(o, []).append(j)
    n_checked = 0
    for i in tree.cut_leaves():
        off, n, masks = meta[i]
        rank, cond = _poly_rank(pts[off:off + n], tree.leaves[i], q)
        if rank < (q + 1) * (q + 2) // 2:
            continue      # P_q is not determined by the interior points: the fit is the minimum-norm one
        n_checked += 1
        tg = np.concatenate([O.leaf_nodes(tree.leaves[i], tree.t)] +
                            [O.leaf_nodes(tree.leaves[j], tree.t) for j in owned.get(i, [])])
        got = np.concatenate([vals[i, 0]] + [vals[j, 0] for j in owned.get(i, [])])
        kappa = _extension_operator_norm(tree, meta, i, tg)
        # rounding of the least-squares solve grows with the conditioning of P_q on the data points
        tol = 100 * EPS * max(kappa, cond, 1.0) * np.max(np.abs(f(pts[off:off + n])))
        assert np.max(np.abs(got - f(tg))) <= tol, (tree.leaves[i], kappa, cond)
    assert n_checked >= 0.85 * len(tree.cut_leaves())


def _poly_rank(p, b, q):
    """Numerical rank and condition number of P_q (total degree <= q) sampled
    at the points p of cut leaf b's extension square, in the Chebyshev
    product basis on that square: the rank is N_G = (q+1)(q+2)/2 exactly when
    the interior data determine a unique least-squares polynomial."""
    c = np.array(O.box_center(b))
    z = (p - c) / (1.5 * O.box_side(b[0]))
    TX = np.polynomial.chebyshev.chebvander(z[:, 0], q)
    TY = np.polynomial.chebyshev.chebvander(z[:, 1], q)
    M = np.stack([TX[:, m] * TY[:, k] for m in range(q + 1) for k in range(q + 1 - m)], axis=1)
    sv = np.linalg.svd(M, compute_uv=False)
    rank = int(np.sum(sv > 1e-11 * sv[0]))
    return rank, sv[0] / sv[-1]


def test_extension_is_not_identity_on_nonpolynomial_data():
    """Guard against a vacuous pass: a degree q+3 polynomial is NOT reproduced."""
    w = W.disk_sincos(level=3, K=8)
    tree = O.build_tree(w.domain, w.opts, w.sources[0])
    f = lambda xy: (3 * xy[:, 0]) ** 13 + (3 * xy[:, 1]) ** 12 + np.exp(3 * xy[:, 0])
    pts, meta = O.stencil_points(tree, w.domain)
    vals, _ = O.leaf_values(tree, w.domain, f(pts)[:, None], meta)
    errs = [np.max(np.abs(vals[i, 0] - f(O.leaf_nodes(tree.leaves[i], tree.t)))) for i in tree.cut_leaves()]
    assert max(errs) > 1e-6


@pytest.mark.parametrize("which", ["disk3", "disk4", "starfish_k8", "lshape_small", "exterior_k8"])
def test_tree_invariants_brute_force(which):
    if which == "exterior_k8":
        w = W.exterior_three_stars(K=8, tol=1e-5, max_level=7)
    elif which == "disk3":
        w = W.disk_sincos(level=3)
    elif which == "disk4":
        w = W.disk_sincos(level=4)
    elif which == "starfish_k8":
        w = W.starfish_gaussian(K=8, tol=1e-8, max_level=8)
    else:
        w = W.lshape_expsin(K=8, base_level=4, max_level=7, corner_levels=4)
    tree = O.build_tree(w.domain, w.opts, w.sources[0])
    assert O.check_tree_invariants(tree) == []
    # classification is by the leaf's own nodes
    for b, c in zip(tree.leaves, tree.cls):
        ins = w.domain.inside(O.leaf_nodes(b, tree.t))
        assert c == (O.CUT if (ins.any() and not ins.all()) else (O.REGULAR if ins.all() else O.EXTERIOR))
    # owners are cut leaves and only exterior leaves are owned
    for j, o in enumerate(tree.owner):
        if o >= 0:
            assert tree.cls[o] == O.CUT and tree.cls[j] == O.EXTERIOR


def test_uniform_disk_tree_counts():
    """Uniform level-4 tree of the disk r = 0.35: 256 leaves; a leaf is cut
    exactly when its 64 nodes straddle the circle (checked by direct distance)."""
    w = W.disk_sincos(level=4)
    tree = O.build_tree(w.domain, w.opts, w.sources[0])
    assert tree.n_leaves == 256 and all(b[0] == 4 for b in tree.leaves)
    ncut = 0
    for b in tree.leaves:
        r = np.hypot(*O.leaf_nodes(b, tree.t).T)
        ncut += int((r < 0.35).any() and not (r < 0.35).all())
    assert ncut == len(tree.cut_leaves())


def test_interpolation_exact_for_tensor_polynomials():
    tree = _uniform_tree(8, 2)
    f = lambda xy: (1 + xy[:, 0]) ** 7 * (2 - xy[:, 1]) ** 7
    vals = f(O.all_leaf_nodes(tree)).reshape(tree.n_leaves, 64, 1)
    rng = np.random.default_rng(2)
    p = np.concatenate([rng.uniform(-0.5, 0.5, (30, 2)), [[0.25, 0.0], [0.5, 0.5], [-0.5, -0.5]]])
    got = O.interpolate_at(tree, vals, p)[:, 0]
    assert np.max(np.abs(got - f(p)) / np.abs(f(p))) < 1e-12


def _mono2cheb_exact(c):
    """Exact monomial -> Chebyshev coefficients (rationals):
    u^m = 2^(1-m) sum_k C(m,k) T_(m-2k), the T_0 term halved."""
    out = [Fraction(0)] * len(c)
    for m, cm in enumerate(c):
        if cm == 0:
            continue
        for k in range(m // 2 + 1):
            coef = Fraction(math.comb(m, k), 2 ** (m - 1)) if m > 0 else Fraction(1)
            j = m - 2 * k
            if j == 0 and m > 0:
                coef /= 2
            out[j] += cm * coef
    return out


def _cheb2d_exact(Q):
    n0, n1 = len(Q), len(Q[0])
    A = [_mono2cheb_exact([Q[i][j] for j in range(n1)]) for i in range(n0)]     # along v
    B = [[Fraction(0)] * n1 for _ in range(n0)]
    for j in range(n1):
        col = _mono2cheb_exact([A[i][j] for i in range(n0)])                     # along u
        for i in range(n0):
            B[i][j] = col[i]
    return np.array([[float(x) for x in row] for row in B])


def _basis_density_q(K, a, b, cx, cy, h):
    """Density p = l_a(u) l_b(v) (one tensor Lagrange basis function of the
    leaf, degree K-1 in each variable) and q with Laplacian q = p, built in
    exact rational arithmetic: monomial coefficients of l_a, l_b from the
    (exactly represented) nodes, the terminating series
    q = sum_k (-1)^k u^(m+2k+2) / ((m+1)...(m+2k+2)) d^2k/dv^2k v^n for every
    monomial u^m v^n, then an exact conversion to Chebyshev series that are
    evaluated in floating point (Clenshaw)."""
    t, _ = O.gauss_legendre(K)
    T = [Fraction(float(x)) for x in t]

    def lag(idx):
        c = [Fraction(1)]
        for m in range(K):
            if m == idx:
                continue
            d = T[idx] - T[m]
            nc = [Fraction(0)] * (len(c) + 1)
            for i, ci in enumerate(c):
                nc[i + 1] += ci / d
                nc[i] -= ci * T[m] / d
            c = nc
        return c
    la, lb = lag(a), lag(b)
    N = 2 * K + 3
    Q = [[Fraction(0)] * N for _ in range(N)]
    for m in range(K):
        for n in range(K):
            c = la[m] * lb[n]
            if c == 0:
                continue
            k = 0
            while 2 * k <= n:
                den = math.prod(range(m + 1, m + 2 * k + 3))
                dv = math.prod(range(n - 2 * k + 1, n + 1)) if k else 1
                Q[m + 2 * k + 2][n - 2 * k] += (-1) ** k * c * dv / den
                k += 1
    Qu = [[(i + 1) * Q[i + 1][j] for j in range(N)] for i in range(N - 1)] + [[Fraction(0)] * N]
    Qv = [[(j + 1) * Q[i][j + 1] for j in range(N - 1)] + [Fraction(0)] for i in range(N)]
    Cq, Cu, Cv = _cheb2d_exact(Q), _cheb2d_exact(Qu), _cheb2d_exact(Qv)
    ch = np.polynomial.chebyshev

    def q(y):
        return ch.chebval2d((y[0] - cx) / h, (y[1] - cy) / h, Cq) * h * h

    def gq(y):
        u, v = (y[0] - cx) / h, (y[1] - cy) / h
        return np.array([ch.chebval2d(u, v, Cu), ch.chebval2d(u, v, Cv)]) * h

    return q, gq


@pytest.mark.parametrize("K,a,b", [(16, 15, 0), (16, 7, 8), (16, 3, 12), (8, 7, 0), (8, 4, 3)])
@pytest.mark.parametrize("where", ["near_edge", "far1", "far2", "far4"])
def test_single_basis_integral_green_identity(K, a, b, where):
    """The integral of one Lagrange basis function times the log kernel (one
    table-like entry) against Green's identity: catches quadrature rules too
    short for the polynomial degree of the basis."""
    L = O.lib()
    t, _ = O.gauss_legendre(K)
    cx, cy, h = 0.0, 0.0, 1.0
    x = {"near_edge": (1.02, 0.3), "far1": (3.05, 0.9), "far2": (5.5, -2.0), "far4": (-9.5, 6.7)}[where]
    q, gq = _basis_density_q(K, a, b, cx, cy, h)
    I = np.zeros(K * K)
    L.orc_leaf_basis_integrals(K, O._ptr(np.ascontiguousarray(t)), cx, cy, h, x[0], x[1], O._ptr(I))
    want = _green_area_integral(q, gq, np.array(x), -1.0, 1.0, -1.0, 1.0)
    assert abs(I[b * K + a] - want) <= 1e-11 * max(1.0, abs(want)), (I[b * K + a], want)


def _golden(name):
    import os
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].split()
            if line:
                vals[line[0]] = int(line[1])
    return vals


def test_discretization_matches_section6():
    """The oracle's stencil and boundary rule take the sizes Section 6 states
    for K = 8: 66 Gaussians (points of G, columns of the universal operator),
    Kbar = 12 on the extension region, 16 Gauss-Legendre nodes per panel."""
    g = _golden("discretization_section6.txt")
    q, Kbar, NG = O.stencil_params(g["K"])
    assert (Kbar, NG) == (g["Kbar"], g["N_G"])
    assert len(O.padua_points(q)) == g["N_G"]
    A = O.universal_matrix(g["K"])
    assert A.shape[1] == g["N_G"]
    assert A.shape[0] == g["K"] ** 2 + g["Kbar"] ** 2 + g["N_G"]   # X = X_S u X_Sbar u G
    assert O.NQ_BOUNDARY == g["N_q"]
    dom = W.disk_sincos(level=3).domain
    assert len(O.boundary_nodes(dom)) == g["N_q"] * dom.n_panels


@pytest.mark.slow
def test_flat_limit_reading_against_finite_eps_operator():
    """The extension operator is read in the flat limit of the Gaussian basis
    (the Lagrange basis of P_10 at G).  The paper's operator has eps = 1e-5
    (Section 3.1, Section 6).  Formed in multiprecision, the finite-eps
    operator converges to the flat-limit one as eps^2 and differs from it by
    2.3e-11 in max norm at eps = 1e-5 (entries of order 1)."""
    pytest.importorskip("mpmath")
    A0 = O.universal_matrix(8)
    d3 = np.abs(O.universal_matrix_finite_eps(8, 1e-3) - A0).max()
    d5 = np.abs(O.universal_matrix_finite_eps(8, 1e-5) - A0).max()
    assert d5 <= 1e-10
    assert abs(d3 / d5 / 1e4 - 1.0) < 0.05      # eps^2 convergence


# ---------------------------------------------------------------- extension along lines (Section 6.4)

def test_fh_of_full_degree_is_polynomial_interpolation():
    """Floater-Hormann with d = n is the polynomial interpolant (textbook
    special case): against numpy's polynomial fit through the same nodes."""
    rng = np.random.Generator(np.random.PCG64(41))
    x = np.sort(rng.uniform(0.0, 1.0, 8))
    f = np.sin(3 * x) + x ** 2
    w = O.fh_weights(x, 7)
    c = np.polyfit(x, f, 7)
    for z in (0.05, 0.5, 0.97, 1.1, 1.25):
        assert abs(O.fh_eval(x, f, w, z) - np.polyval(c, z)) <= 1e-9 * max(1.0, abs(np.polyval(c, z)))


def test_fh_reproduces_polynomials_of_degree_d():
    """The Floater-Hormann interpolant of degree d reproduces polynomials of
    degree <= d, inside the nodes and beyond them."""
    rng = np.random.Generator(np.random.PCG64(42))
    x = np.sort(rng.uniform(0.2, 0.45, 8))
    for d in (0, 1, 2, 3):
        c = rng.standard_normal(d + 1)
        w = O.fh_weights(x, d)
        for z in (0.25, 0.33, 0.5, 0.6):
            assert abs(O.fh_eval(x, np.polyval(c, x), w, z) - np.polyval(c, z)) <= 1e-11 * np.abs(c).sum()


def test_fh_weights_on_equispaced_nodes_match_the_binomial_form():
    """On equispaced nodes the weights are, up to one common factor,
    (-1)^k sum_{i in J_k} binom(d, k - i)."""
    from math import comb
    x = 0.3 + 0.01 * np.arange(8)
    for d in (1, 2, 3, 4):
        w = O.fh_weights(x, d)
        ref = np.array([(-1.0) ** k * sum(comb(d, k - i) for i in range(max(0, k - d), min(k, 7 - d) + 1))
                        for k in range(8)])
        ratio = w / ref
        assert np.allclose(ratio, ratio[0], rtol=1e-12, atol=0)


def _star_workload(f):
    dom = W.StarDomain(0.35, [(3, 0.1, 0.3), (5, 0.05, 1.0)])
    return W.Workload("star_lines", 9, dom, W.TreeOptions(K=8, min_level=4, max_level=4), [f])


def _line_extension_error(f):
    wl = _star_workload(f)
    tree = O.build_tree(wl.domain, wl.opts, f)
    pts, meta = O.stencil_points_lines(tree, wl.domain)
    vals = O.leaf_values_lines(tree, wl.domain, f(pts), meta)
    err = 0.0
    for i, b in enumerate(tree.leaves):
        if tree.cls[i] == O.CUT or tree.owner[i] >= 0:
            nodes = O.leaf_nodes(b, tree.t)
            err = max(err, np.max(np.abs(vals[i, 0] - f(nodes))))
    return err, len(tree.cut_leaves())


def test_line_extension_exact_for_quadratic_along_rays():
    """f = x^2 + y^2 is quadratic along every line through the centre, so the
    degree-3 rational extension reproduces it at the exterior grid points, and
    the truncated Chebyshev expansion of a quadratic is exact: f^e = f at every
    node of every cut and extension-list leaf (Section 6.4 with the readings
    FH degree 3, 8 ray points over one leaf side)."""
    err, ncut = _line_extension_error(lambda xy: xy[:, 0] ** 2 + xy[:, 1] ** 2)
    assert ncut > 0 and err <= 1e-11


def test_line_extension_extrapolates_rather_than_sampling_f():
    """Along rays f = (x^2 + y^2)^3 is of degree 6 in the radius: the degree-3
    extension is no longer exact (so the exact case above is not f sampled
    outside Omega); the error stays below the size of f there (about 8e-3)."""
    err, _ = _line_extension_error(lambda xy: (xy[:, 0] ** 2 + xy[:, 1] ** 2) ** 3)
    assert 1e-10 < err < 1e-2


def _monomial_integral(m):
    """int_{-1/2}^{1/2} x^m dx as an exact fraction."""
    return Fraction(1, 2 ** (m + 1) * (m + 1)) * (1 - (-1) ** (m + 1))


def test_net_charge_exact_for_polynomials_on_an_adaptive_tree():
    """A tensor polynomial of degree <= 2K - 1 in each variable is integrated
    exactly by every leaf's K-point Gauss-Legendre rule, so the net charge
    over D equals the integral of the polynomial, whatever the leaf sizes."""
    K = 8
    tree = O.build_tree(W.WholeBoxDomain(), W.TreeOptions(K=K, min_level=2, max_level=6, refine_tol=1e-12),
                        W.make_gaussian((0.21, -0.13), 0.03))
    assert len({b[0] for b in tree.leaves}) >= 3
    terms = [(3.0, 6, 2), (-2.0, 15, 0), (0.5, 4, 14), (1.0, 0, 0), (7.0, 1, 5)]
    nodes = O.all_leaf_nodes(tree)
    f = sum(c * nodes[:, 0] ** m * nodes[:, 1] ** n for c, m, n in terms)
    got = O.net_charge(tree, f.reshape(tree.n_leaves, 1, K * K))[0]
    want = float(sum(Fraction(c) * _monomial_integral(m) * _monomial_integral(n) for c, m, n in terms))
    assert abs(got - want) <= 1e-14 * max(1.0, abs(want))


def test_net_charge_of_a_gaussian_is_pi_s_squared():
    """exp(-|x - c|^2 / s^2) integrates to pi s^2 over the plane; its mass
    outside D is below exp(-(0.45 / 0.05)^2)."""
    s, c = 0.05, (0.03, -0.02)
    tree = _uniform_tree(16, 4)
    vals = W.make_gaussian(c, s)(O.all_leaf_nodes(tree)).reshape(tree.n_leaves, 1, 256)
    got = O.net_charge(tree, vals)[0]
    assert abs(got - math.pi * s * s) <= 1e-13 * math.pi * s * s


def test_net_charge_is_the_growth_of_the_potential_at_infinity():
    """V[f](x) = (1/2 pi) int log|x - y| f(y) dy, and |log|x - y| - log|x||
    <= |y| / (|x| - |y|), so far from D the potential computed by the
    quadrature kernel is (A^e / 2 pi) log|x| within
    (1/2 pi) max|y| / (|x| - max|y|) int |f|.  Exterior workload, f^e from
    the oracle's extension (non-zero inside the holes)."""
    w = W.exterior_three_stars(K=8, tol=1e-5, max_level=7)
    tree = O.build_tree(w.domain, w.opts, w.sources[0])
    pts, meta = O.stencil_points(tree, w.domain)
    vals, _ = O.leaf_values(tree, w.domain, w.sources[0](pts)[:, None], meta)
    A = O.net_charge(tree, vals)[0]
    absmass = O.net_charge(tree, np.abs(vals))[0]
    for R, ang in [(1e3, 0.3), (1e4, 2.0), (3e5, -1.1)]:
        x = np.array([[R * math.cos(ang), R * math.sin(ang)]])
        V = O.volume_potential(tree, vals, x)[0, 0]
        ymax = math.sqrt(0.5)
        bound = absmass * ymax / (R - ymax) / (2 * math.pi)
        assert abs(V - A * math.log(R) / (2 * math.pi)) <= bound + 1e-12 * abs(V)
    # the bound is far from vacuous: at |x| = 1000 the growth term is much larger
    assert abs(A) * math.log(1e3) / (2 * math.pi) > 100 * absmass * ymax / (1e3 - ymax) / (2 * math.pi)
