"""CPU oracle for the particular-solution stage -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct FP64 implementation of what the library
computes, written from the paper (Sections 3.1, 3.2, 4, 4.1):

* quad-tree construction: resolution / cut-size refinement, level
  restriction (2:1 balance) and extension restriction (Section 4);
* leaf classification (regular / cut / exterior) and extension lists
  (Section 4, definition of the extension list);
* the universal stencil X_S u X_Sbar u G of every cut leaf and the
  least-squares extension f_E = A_{E,G} A_{I,G}^+ f_I (Section 3.2) in the
  flat limit of the Gaussian basis (A = Lagrange basis of P_q at G, formed
  with a Legendre Vandermonde matrix; A^+ by the SVD);
* the truncated Chebyshev expansion on the extension square and its
  evaluation on the extension-list leaves (Section 4.1, eq. chebexpbarS);
* the volume potential by direct quadrature (``vpx_oracle.c``) and its
  interpolation at boundary nodes (Section 4.1, last paragraph);
* the net charge A^e of the extended source (Section 6.2).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares no code with the CUDA library;
the two meet only through the seeded inputs of ``workloads``.

Conventions: D = [-0.5, 0.5]^2; a box is (level, ix, iy) with side 2^-level
and lower-left corner (-0.5 + ix*s, -0.5 + iy*s); leaf order is Z-order
(depth first, children SW, SE, NW, NE); leaf node (a, b) has index b*K + a.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field
from typing import Dict, List, Tuple

import numpy as np
from numpy.polynomial import chebyshev as npcheb
from numpy.polynomial import legendre as npleg

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libvpx_oracle.so")

REGULAR, CUT, EXTERIOR = 0, 1, 2
N_BOUNDARY_SAMPLES = 64   # boundary sample intervals per panel (classification)
NQ_BOUNDARY = 16          # Gauss-Legendre nodes per panel (boundary targets)


# --------------------------------------------------------------------------- build

def build_oracle(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, OpenMP) into oracle/_build."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    src = os.path.join(HERE, "vpx_oracle.c")
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(src):
        tmp = LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               src, "-o", tmp, "-lm"])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build_oracle()
        L = ctypes.CDLL(LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_volume_potential.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int, dp, ctypes.c_int, dp,
                                           ctypes.c_int, dp, dp, dp, ctypes.c_int]
        L.orc_volume_potential.restype = ctypes.c_int
        L.orc_leaf_basis_integrals.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        L.orc_leaf_basis_integrals.restype = None
        L.orc_rect_log_integral.argtypes = [ctypes.c_double] * 6
        L.orc_rect_log_integral.restype = ctypes.c_double
        L.orc_gauss_legendre.argtypes = [ctypes.c_int, dp, dp]
        L.orc_gauss_legendre.restype = None
        L.orc_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------------------------- point sets

def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1,1] (numpy's routine)."""
    return npleg.leggauss(n)


def chebyshev1_nodes(n: int) -> np.ndarray:
    """Chebyshev nodes of the first kind on [-1,1], ascending."""
    a = np.arange(n)
    return -np.cos((2 * a + 1) * math.pi / (2 * n))


def padua_points(q: int) -> np.ndarray:
    """Padua points of degree q: (cos(j pi/q), cos(k pi/(q+1))), j+k even.

    (q+1)(q+2)/2 points, unisolvent for polynomials of total degree <= q
    (our reading of the Gaussian support set G of Section 3.2)."""
    pts = []
    for j in range(q + 1):
        for k in range(q + 2):
            if (j + k) % 2 == 0:
                pts.append((math.cos(j * math.pi / q), math.cos(k * math.pi / (q + 1))))
    return np.asarray(pts)


PINV_RCOND = 1e-13   # singular values below this fraction of the largest are dropped


def stencil_params(K: int):
    """q, Kbar, N_G for leaf order K.

    N_G = 66 Gaussian support points (Section 6) for every K, i.e. the flat
    limit spans the polynomials of total degree q = 10; Kbar = 3K/2 (12 for
    K = 8 as in Section 6)."""
    q = 10
    Kbar = 3 * K // 2
    return q, Kbar, (q + 1) * (q + 2) // 2


_universal_A = {}


def universal_matrix(K: int):
    """A_{X,G} = Phi_{X,G} Phi_{G,G}^{-1} (eq. defA) on the reference extension
    square [-1,1]^2 in the flat limit: the Lagrange basis of P_q at the Padua
    points G evaluated at X = X_S u X_Sbar u G.  Written with the Legendre
    total-degree Vandermonde matrix (any basis of P_q gives the same A)."""
    if K not in _universal_A:
        q, Kbar, NG = stencil_params(K)
        t, _ = gauss_legendre(K)
        XS = np.stack(np.meshgrid(t / 3.0, t / 3.0, indexing="xy"), axis=-1).reshape(-1, 2)
        tc = chebyshev1_nodes(Kbar)
        XSb = np.stack(np.meshgrid(tc, tc, indexing="xy"), axis=-1).reshape(-1, 2)
        G = padua_points(q)
        VX = legendre_total_degree_vander(np.concatenate([XS, XSb, G]), q)
        VG = legendre_total_degree_vander(G, q)
        _universal_A[K] = np.linalg.solve(VG.T, VX.T).T
    return _universal_A[K]


def universal_matrix_finite_eps(K: int, eps: float) -> np.ndarray:
    """A_{X,G} = Phi_{X,G} Phi_{G,G}^{-1} (eq. defA) for Gaussians
    exp(-eps^2 |x - g|^2) of finite shape parameter eps on the reference square
    [-1,1]^2, the points X and G of universal_matrix.  Phi_{G,G} has condition
    number ~ eps^{-2q}, so the matrices are formed and the system solved in
    multiprecision (mpmath, 30 + 2q log10(1/eps) digits) and the result rounded
    to FP64.  As eps -> 0 this tends to the flat-limit operator of
    universal_matrix, the paper's operator at its small eps (Section 3.1,
    Section 6).  Slow (seconds); for checking the flat-limit reading only."""
    import mpmath as mp
    q, Kbar, NG = stencil_params(K)
    t, _ = gauss_legendre(K)
    XS = np.stack(np.meshgrid(t / 3.0, t / 3.0, indexing="xy"), axis=-1).reshape(-1, 2)
    tc = chebyshev1_nodes(Kbar)
    XSb = np.stack(np.meshgrid(tc, tc, indexing="xy"), axis=-1).reshape(-1, 2)
    G = padua_points(q)
    X = np.concatenate([XS, XSb, G])
    with mp.workdps(30 + int(math.ceil(2 * q * math.log10(1.0 / eps)))):
        e2 = mp.mpf(eps) ** 2
        Gm = [(mp.mpf(float(a)), mp.mpf(float(b))) for a, b in G]
        Xm = [(mp.mpf(float(a)), mp.mpf(float(b))) for a, b in X]
        phi = lambda p, g: mp.exp(-e2 * ((p[0] - g[0]) ** 2 + (p[1] - g[1]) ** 2))
        PGG = mp.matrix([[phi(gi, gj) for gj in Gm] for gi in Gm])
        W = mp.inverse(PGG)                       # Phi_GG is symmetric: A = Phi_XG W
        A = np.empty((len(Xm), len(Gm)))
        for i, x in enumerate(Xm):
            row = [phi(x, gj) for gj in Gm]
            for j in range(len(Gm)):
                A[i, j] = float(mp.fsum(row[k] * W[k, j] for k in range(len(Gm))))
    return A


_finite_eps_cache = {}


def _finite_eps_A(K: int, rbf_eps: float) -> np.ndarray:
    """The universal operator for Gaussians of shape parameter rbf_eps on the
    unit box: the extension square maps to [-1,1]^2, twice the unit box's side,
    so the reference-square parameter is rbf_eps / 2."""
    key = (K, float(rbf_eps))
    if key not in _finite_eps_cache:
        _finite_eps_cache[key] = universal_matrix_finite_eps(K, 0.5 * rbf_eps)
    return _finite_eps_cache[key]


def pseudo_inverse(M: np.ndarray, rcond: float = PINV_RCOND) -> np.ndarray:
    """Moore-Penrose pseudo-inverse by the SVD (numpy/LAPACK), singular values
    <= rcond * largest treated as zero."""
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    keep = s > rcond * s[0]
    return (Vt[keep].T / s[keep]) @ U[:, keep].T


# --------------------------------------------------------------------------- boxes

def box_side(level: int) -> float:
    return 2.0 ** (-level)


def box_bounds(b):
    l, ix, iy = b
    s = box_side(l)
    x0 = -0.5 + ix * s
    y0 = -0.5 + iy * s
    return x0, x0 + s, y0, y0 + s


def box_center(b):
    x0, x1, y0, y1 = box_bounds(b)
    return 0.5 * (x0 + x1), 0.5 * (y0 + y1)


def children(b):
    l, ix, iy = b
    return [(l + 1, 2 * ix + (c & 1), 2 * iy + (c >> 1)) for c in range(4)]


def ancestor(b, lev):
    l, ix, iy = b
    return (lev, ix >> (l - lev), iy >> (l - lev))


def morton_key(b, lmax: int) -> int:
    l, ix, iy = b
    ix <<= (lmax - l)
    iy <<= (lmax - l)
    key = 0
    for bit in range(lmax):
        key |= ((ix >> bit) & 1) << (2 * bit)
        key |= ((iy >> bit) & 1) << (2 * bit + 1)
    return key


def leaf_nodes(b, t: np.ndarray) -> np.ndarray:
    """K*K leaf nodes, index b*K + a."""
    cx, cy = box_center(b)
    h = 0.5 * box_side(b[0])
    X, Y = np.meshgrid(cx + h * t, cy + h * t, indexing="xy")
    return np.stack([X.ravel(), Y.ravel()], axis=1)


# --------------------------------------------------------------------------- the tree

@dataclass
class OracleTree:
    K: int
    leaves: List[Tuple[int, int, int]]          # Z-order
    cls: List[int]                              # REGULAR / CUT / EXTERIOR per leaf
    owner: List[int]                            # for exterior leaves: index of owning cut leaf or -1
    t: np.ndarray = None                        # leaf GL nodes
    index: Dict[Tuple[int, int, int], int] = field(default_factory=dict)

    @property
    def n_leaves(self):
        return len(self.leaves)

    def cut_leaves(self):
        return [i for i, c in enumerate(self.cls) if c == CUT]


class TreeError(RuntimeError):
    pass


class _Geometry:
    """Boundary samples and panel lengths used by the tree rules."""

    def __init__(self, dom):
        self.dom = dom
        n = getattr(dom, "n_panels", 0)
        tg, wg = npleg.leggauss(16)
        ts = -1.0 + 2.0 * np.arange(N_BOUNDARY_SAMPLES + 1) / N_BOUNDARY_SAMPLES
        samples, lens, pid = [], [], []
        for i in range(n):
            xy, _ = dom.curve(i, ts)
            _, d = dom.curve(i, tg)
            L = float(np.sum(wg * np.hypot(d[:, 0], d[:, 1])))
            samples.append(xy)
            lens.append(L)
            pid.append(np.full(len(ts), i))
        if n:
            self.samples = np.concatenate(samples)
            self.sample_panel = np.concatenate(pid)
        else:
            self.samples = np.zeros((0, 2))
            self.sample_panel = np.zeros(0, dtype=int)
        self.panel_len = np.asarray(lens)

    def samples_in(self, b):
        x0, x1, y0, y1 = box_bounds(b)
        p = self.samples
        m = (p[:, 0] >= x0) & (p[:, 0] <= x1) & (p[:, 1] >= y0) & (p[:, 1] <= y1)
        return m


def legendre_tail_max(F: np.ndarray, Vinv: np.ndarray, K: int) -> float:
    """Refinement measure of one leaf (Section 4, R8 reading): the largest
    |c_mn| over total degree m + n >= K-1 of the tensor Legendre coefficients
    of the leaf's K x K node values F[b][a] (b the y index), with
    Vinv = inverse Legendre Vandermonde matrix of the leaf nodes."""
    C = Vinv @ F @ Vinv.T          # C[n][m]: degree n in y, m in x
    mm, nn = np.meshgrid(np.arange(K), np.arange(K), indexing="xy")
    return float(np.max(np.abs(C[(mm + nn) >= K - 1])))


def build_tree(dom, opts, f_refine, verbose=False) -> OracleTree:
    """Quad-tree by the rules of Section 4 (our reading, applied literally).

    Phase A, level by level from the root: a box is split when its level is
    below ``min_level``; otherwise, when adaptive (refine_tol > 0) and below
    ``max_level``: exterior boxes are kept; a cut box is split when its side
    exceeds twice the length of the shortest panel sampled inside it
    (cut-size rule); a cut or regular box is split when f at its K x K nodes
    is not resolved: the largest Legendre coefficient of total degree >= K-1
    exceeds refine_tol * f_scale.
    Phase B, to a fixed point: 2:1 balance (split any leaf that is more than
    one level coarser than a leaf it touches), then the extension restriction
    (split any exterior leaf coarser than a cut leaf S that overlaps Sbar).
    """
    K = opts.K
    t, _ = gauss_legendre(K)
    geo = _Geometry(dom)
    Vinv = np.linalg.inv(npleg.legvander(t, K - 1))
    cls_cache: Dict = {}

    def classify(b):
        if b in cls_cache:
            return cls_cache[b]
        ins = dom.inside(leaf_nodes(b, t))
        if ins.any() and not ins.all():
            c = CUT
        elif ins.all():
            c = REGULAR
        else:
            c = EXTERIOR
        cls_cache[b] = c
        return c

    def unresolved(b):
        F = np.asarray(f_refine(leaf_nodes(b, t)), dtype=np.float64).reshape(K, K)  # [b][a]
        return legendre_tail_max(F, Vinv, K) > opts.refine_tol * opts.f_scale

    def split_phase_a(b):
        l = b[0]
        if l >= opts.max_level:
            return False
        if l < opts.min_level:
            return True
        if opts.refine_tol <= 0:
            return False
        c = classify(b)
        if c == EXTERIOR:
            return False
        if c == CUT:
            m = geo.samples_in(b)
            pl = geo.panel_len[np.unique(geo.sample_panel[m])]
            if len(pl) and box_side(l) > 2.0 * float(pl.min()):
                return True
        return unresolved(b)

    leaves = set()
    frontier = [(0, 0, 0)]
    while frontier:
        nxt = []
        for b in frontier:
            if split_phase_a(b):
                nxt.extend(children(b))
            else:
                leaves.add(b)
        frontier = nxt

    def leaf_containing(p):
        for lev in range(p[0], -1, -1):
            a = ancestor(p, lev)
            if a in leaves:
                return a
        return None

    def neighbour_positions(b):
        l, ix, iy = b
        n = 1 << l
        out = []
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx == 0 and dy == 0:
                    continue
                jx, jy = ix + dx, iy + dy
                if 0 <= jx < n and 0 <= jy < n:
                    out.append((l, jx, jy))
        return out

    def split(b):
        leaves.remove(b)
        for c in children(b):
            leaves.add(c)

    while True:
        changed = False
        while True:
            marks = set()
            for b in leaves:
                for p in neighbour_positions(b):
                    c = leaf_containing(p)
                    if c is not None and c[0] < b[0] - 1:
                        marks.add(c)
            if not marks:
                break
            for c in marks:
                split(c)
            changed = True
        marks = set()
        for b in leaves:
            if classify(b) != CUT:
                continue
            for p in neighbour_positions(b):
                c = leaf_containing(p)
                if c is not None and c[0] < b[0] and classify(c) == EXTERIOR:
                    marks.add(c)
        if marks:
            for c in marks:
                split(c)
            changed = True
        if not changed:
            break

    lmax = max(b[0] for b in leaves)
    order = sorted(leaves, key=lambda b: morton_key(b, lmax))
    cls = [classify(b) for b in order]
    # every cut leaf's extension square must lie inside D (R7 reading)
    for b, c in zip(order, cls):
        if c == CUT:
            l, ix, iy = b
            if ix < 1 or iy < 1 or ix > (1 << l) - 2 or iy > (1 << l) - 2:
                raise TreeError("extension square of cut leaf %s leaves D" % (b,))
    tree = OracleTree(K=K, leaves=order, cls=cls, owner=[-1] * len(order), t=t)
    tree.index = {b: i for i, b in enumerate(order)}
    tree.owner = extension_owners(tree)
    return tree


def extension_owners(tree: OracleTree) -> List[int]:
    """Extension lists (Section 4): each exterior leaf S' overlapping the
    extension square Sbar of some cut leaf S is owned by the cut leaf whose
    centre is closest to the centre of S'; on a tie the cut leaf later in
    leaf order wins.  Brute force over all cut leaves."""
    cut = tree.cut_leaves()
    owner = [-1] * tree.n_leaves
    if not cut:
        return owner
    cb = np.array([box_bounds(tree.leaves[i]) for i in cut])
    cs = cb[:, 1] - cb[:, 0]
    cc = np.stack([0.5 * (cb[:, 0] + cb[:, 1]), 0.5 * (cb[:, 2] + cb[:, 3])], axis=1)
    sb = np.stack([cc[:, 0] - 1.5 * cs, cc[:, 0] + 1.5 * cs, cc[:, 1] - 1.5 * cs, cc[:, 1] + 1.5 * cs], axis=1)
    for i, b in enumerate(tree.leaves):
        if tree.cls[i] != EXTERIOR:
            continue
        x0, x1, y0, y1 = box_bounds(b)
        ov = (np.minimum(x1, sb[:, 1]) > np.maximum(x0, sb[:, 0])) & \
             (np.minimum(y1, sb[:, 3]) > np.maximum(y0, sb[:, 2]))
        if not ov.any():
            continue
        c = np.array([0.5 * (x0 + x1), 0.5 * (y0 + y1)])
        d2 = (cc[:, 0] - c[0]) ** 2 + (cc[:, 1] - c[1]) ** 2
        best, bi = math.inf, -1
        for k in np.nonzero(ov)[0]:
            if d2[k] <= best:          # later cut leaf wins ties
                best, bi = d2[k], k
        owner[i] = cut[bi]
    return owner


def check_tree_invariants(tree: OracleTree):
    """Brute-force checks of the tree rules; returns a list of violations."""
    bad = []
    L = tree.leaves
    bounds = np.array([box_bounds(b) for b in L])
    lev = np.array([b[0] for b in L])
    n = len(L)
    for i in range(n):
        x0, x1, y0, y1 = bounds[i]
        touch = (bounds[:, 0] <= x1) & (bounds[:, 1] >= x0) & (bounds[:, 2] <= y1) & (bounds[:, 3] >= y0)
        touch[i] = False
        if np.any(np.abs(lev[touch] - lev[i]) > 1):
            bad.append(("balance", L[i]))
        if tree.cls[i] == CUT:
            s = x1 - x0
            sx0, sx1, sy0, sy1 = x0 - s, x1 + s, y0 - s, y1 + s
            ov = (np.minimum(bounds[:, 1], sx1) > np.maximum(bounds[:, 0], sx0)) & \
                 (np.minimum(bounds[:, 3], sy1) > np.maximum(bounds[:, 2], sy0))
            for j in np.nonzero(ov)[0]:
                if tree.cls[j] == EXTERIOR and lev[j] < lev[i]:
                    bad.append(("extension-restriction", L[i], L[j]))
    # owned leaves lie inside the owner's extension square
    for i, o in enumerate(tree.owner):
        if o < 0:
            continue
        x0, x1, y0, y1 = box_bounds(L[i])
        a0, a1, b0, b1 = box_bounds(L[o])
        s = a1 - a0
        if not (x0 >= a0 - s and x1 <= a1 + s and y0 >= b0 - s and y1 <= b1 + s):
            bad.append(("owner-containment", L[i], L[o]))
    # leaves tile D
    area = float(np.sum((bounds[:, 1] - bounds[:, 0]) * (bounds[:, 3] - bounds[:, 2])))
    if abs(area - 1.0) > 1e-14:
        bad.append(("tiling", area))
    return bad


# --------------------------------------------------------------------------- stencil

def cut_leaf_stencil(b, K: int, t: np.ndarray):
    """Universal stencil of cut leaf b in physical coordinates:
    X_S (K*K leaf nodes), X_Sbar (Kbar*Kbar Chebyshev-1 nodes on the 3x square),
    G (Padua points of degree q on the 3x square), in that order."""
    q, Kbar, NG = stencil_params(K)
    cx, cy = box_center(b)
    s = box_side(b[0])
    XS = leaf_nodes(b, t)
    tc = chebyshev1_nodes(Kbar)
    X, Y = np.meshgrid(cx + 1.5 * s * tc, cy + 1.5 * s * tc, indexing="xy")
    XSb = np.stack([X.ravel(), Y.ravel()], axis=1)
    P = padua_points(q)
    G = np.stack([cx + 1.5 * s * P[:, 0], cy + 1.5 * s * P[:, 1]], axis=1)
    return XS, XSb, G


def stencil_points(tree: OracleTree, dom):
    """All points where f is supplied: K*K nodes of each regular leaf (leaf
    order), then the interior stencil points of each cut leaf (leaf order;
    per leaf X_S^I, X_Sbar^I, G^I).  Returns (points, per-leaf metadata)."""
    K = tree.K
    pts, meta = [], {}
    off = 0
    for i, b in enumerate(tree.leaves):
        if tree.cls[i] == REGULAR:
            p = leaf_nodes(b, tree.t)
            meta[i] = (off, len(p))
            pts.append(p)
            off += len(p)
    for i, b in enumerate(tree.leaves):
        if tree.cls[i] == CUT:
            XS, XSb, G = cut_leaf_stencil(b, K, tree.t)
            m = [dom.inside(XS), dom.inside(XSb), dom.inside(G)]
            p = np.concatenate([XS[m[0]], XSb[m[1]], G[m[2]]])
            meta[i] = (off, len(p), m)
            pts.append(p)
            off += len(p)
    return (np.concatenate(pts) if pts else np.zeros((0, 2))), meta


# --------------------------------------------------------------------------- extension along lines

FH_DEGREE = 3        # Floater-Hormann blending degree d (the text leaves it open)
N_RAY_NODES = 8      # interior data points per ray (Section 6.4)


def fh_weights(x: np.ndarray, d: int) -> np.ndarray:
    """Floater-Hormann barycentric weights of degree d for the nodes x_0..x_n:
    w_k = (-1)^(k-d) sum over i in J_k of prod_{j=i..i+d, j != k} 1/|x_k - x_j|,
    J_k = {i : 0 <= i <= n-d, k-d <= i <= k}."""
    n = len(x) - 1
    w = np.zeros(n + 1)
    for k in range(n + 1):
        tot = 0.0
        for i in range(max(0, k - d), min(k, n - d) + 1):
            p = 1.0
            for j in range(i, i + d + 1):
                if j != k:
                    p /= abs(x[k] - x[j])
            tot += p
        w[k] = (-1.0) ** (k - d) * tot
    return w


def fh_eval(x: np.ndarray, f: np.ndarray, w: np.ndarray, z: float) -> float:
    """The barycentric rational interpolant sum w_k f_k/(z-x_k) / sum w_k/(z-x_k)."""
    dz = z - x
    hit = np.nonzero(dz == 0.0)[0]
    if len(hit):
        return float(f[hit[0]])
    c = w / dz
    return float(np.dot(c, f) / np.sum(c))


def ray_nodes(dom, p, L: float, n: int = N_RAY_NODES):
    """The data points for extending to p along the line through the star's
    centre c and p (Section 6.4): with r_b the boundary radius in the direction
    of p, the n points at radii r_b - j L / n, j = 1..n, inside Omega.
    Returns (points (n, 2), their radii, the radius of p)."""
    cx, cy = dom.center
    th = math.atan2(p[1] - cy, p[0] - cx)
    rb = float(dom.r(np.array([th]))[0])
    radii = rb - L * np.arange(1, n + 1) / n
    if radii[-1] <= 0.0:
        raise ValueError("ray nodes reach the centre")
    u = np.array([math.cos(th), math.sin(th)])
    return np.array([cx, cy]) + radii[:, None] * u, radii, math.hypot(p[0] - cx, p[1] - cy)


def stencil_points_lines(tree: OracleTree, dom):
    """Points where f is supplied for the extension along lines: the K*K nodes
    of each regular leaf, then per cut leaf X_S^I, X_Sbar^I and, for every
    exterior point of its Kbar x Kbar grid (grid order), the N_RAY_NODES ray
    points.  Returns (points, per-leaf metadata)."""
    K = tree.K
    pts, meta = [], {}
    off = 0
    for i, b in enumerate(tree.leaves):
        if tree.cls[i] == REGULAR:
            p = leaf_nodes(b, tree.t)
            meta[i] = (off, len(p))
            pts.append(p)
            off += len(p)
    for i, b in enumerate(tree.leaves):
        if tree.cls[i] == CUT:
            XS, XSb, _ = cut_leaf_stencil(b, K, tree.t)
            m = [dom.inside(XS), dom.inside(XSb)]
            L = box_side(b[0])
            rays = [ray_nodes(dom, XSb[e], L)[0] for e in np.nonzero(~m[1])[0]]
            p = np.concatenate([XS[m[0]], XSb[m[1]]] + rays)
            meta[i] = (off, len(p), m)
            pts.append(p)
            off += len(p)
    return (np.concatenate(pts) if pts else np.zeros((0, 2))), meta


def extend_cut_leaf_lines(b, K, t, dom, masks, fI: np.ndarray, targets: np.ndarray):
    """Extension along lines for cut leaf b (Section 6.4): the exterior points
    of the Kbar x Kbar grid take the Floater-Hormann interpolant (degree
    FH_DEGREE) of the data at their ray points, evaluated at their own radius;
    the interior grid points keep the data; then the truncated Chebyshev
    expansion of the grid (m + n < Kbar, eq. chebexpbarS) is evaluated at the
    targets, as in extend_cut_leaf.
    fI: (N, nrhs) data in the order of stencil_points_lines for this leaf."""
    q, Kbar, NG = stencil_params(K)
    _, XSb, _ = cut_leaf_stencil(b, K, t)
    cx, cy = box_center(b)
    r = 1.5 * box_side(b[0])
    L = box_side(b[0])
    nI_S, nI_Sb = int(masks[0].sum()), int(masks[1].sum())
    grid = np.zeros((Kbar * Kbar, fI.shape[1]))
    grid[masks[1]] = fI[nI_S:nI_S + nI_Sb]
    pos = nI_S + nI_Sb
    for e in np.nonzero(~masks[1])[0]:
        _, radii, rx = ray_nodes(dom, XSb[e], L)
        order = np.argsort(radii)
        w = fh_weights(radii[order], FH_DEGREE)
        for rr in range(fI.shape[1]):
            grid[e, rr] = fh_eval(radii[order], fI[pos:pos + N_RAY_NODES, rr][order], w, rx)
        pos += N_RAY_NODES
    tc = chebyshev1_nodes(Kbar)
    T = npcheb.chebvander(tc, Kbar - 1)
    Tinv = np.linalg.inv(T)
    zt = (targets - np.array([cx, cy])) / r
    TX = npcheb.chebvander(zt[:, 0], Kbar - 1)
    TY = npcheb.chebvander(zt[:, 1], Kbar - 1)
    mm, nn = np.meshgrid(np.arange(Kbar), np.arange(Kbar), indexing="ij")
    keep = (mm + nn) < Kbar
    out = np.zeros((len(targets), fI.shape[1]))
    for rr in range(fI.shape[1]):
        Fb = grid[:, rr].reshape(Kbar, Kbar).T
        alpha = np.where(keep, Tinv @ Fb @ Tinv.T, 0.0)
        out[:, rr] = np.einsum("im,mn,in->i", TX, alpha, TY)
    return out


def leaf_values_lines(tree: OracleTree, dom, f_stencil: np.ndarray, meta):
    """f^e at every leaf node with the extension along lines (Section 6.4) in
    place of the universal stencil; otherwise as leaf_values."""
    K = tree.K
    f_stencil = np.asarray(f_stencil, dtype=np.float64)
    if f_stencil.ndim == 1:
        f_stencil = f_stencil[:, None]
    nrhs = f_stencil.shape[1]
    out = np.zeros((tree.n_leaves, nrhs, K * K))
    owned: Dict[int, List[int]] = {}
    for i, o in enumerate(tree.owner):
        if o >= 0:
            owned.setdefault(o, []).append(i)
    for i, b in enumerate(tree.leaves):
        if tree.cls[i] == REGULAR:
            off, n = meta[i]
            out[i] = f_stencil[off:off + n].T
    for i, b in enumerate(tree.leaves):
        if tree.cls[i] != CUT:
            continue
        off, n, masks = meta[i]
        fI = f_stencil[off:off + n]
        own_nodes = leaf_nodes(b, tree.t)
        tg = [own_nodes[~masks[0]]] + [leaf_nodes(tree.leaves[j], tree.t) for j in owned.get(i, [])]
        vals = extend_cut_leaf_lines(b, K, tree.t, dom, masks, fI, np.concatenate(tg))
        nE = int((~masks[0]).sum())
        v = np.zeros((K * K, nrhs))
        v[masks[0]] = fI[:int(masks[0].sum())]
        v[~masks[0]] = vals[:nE]
        out[i] = v.T
        pos = nE
        for j in owned.get(i, []):
            out[j] = vals[pos:pos + K * K].T
            pos += K * K
    return out


# --------------------------------------------------------------------------- extension

def legendre_total_degree_vander(z: np.ndarray, q: int) -> np.ndarray:
    """Columns P_m(z1) P_n(z2), m + n <= q (ordered by m then n)."""
    V1 = npleg.legvander(z[:, 0], q)
    V2 = npleg.legvander(z[:, 1], q)
    cols = [V1[:, m] * V2[:, n] for m in range(q + 1) for n in range(q + 1 - m)]
    return np.stack(cols, axis=1)


def extend_cut_leaf(b, K, t, masks, fI: np.ndarray, targets: np.ndarray, rbf_eps: float = 0.0):
    """Section 3.2 + 4.1 for one cut leaf, flat-limit reading.

    fI: (N_I, nrhs) data at the interior stencil points (X_S^I, X_Sbar^I, G^I).
    f_{X_Sbar^E} = A_{X_Sbar^E,G} A_{X^I,G}^+ f_I fills the exterior nodes of
    the Kbar x Kbar Chebyshev grid, the interior nodes keep the data; the
    grid's Chebyshev expansion truncated to m+n < Kbar (eq. chebexpbarS) is
    evaluated at ``targets`` (physical coordinates inside Sbar).
    Returns (values at targets (n, nrhs), condition number of A_I).
    """
    q, Kbar, NG = stencil_params(K)
    XS, XSb, G = cut_leaf_stencil(b, K, t)
    cx, cy = box_center(b)
    r = 1.5 * box_side(b[0])
    A = universal_matrix(K) if rbf_eps == 0.0 else _finite_eps_A(K, rbf_eps)
    nS = K * K
    interior = np.concatenate(masks)
    AI = A[interior]
    AE = A[nS:nS + Kbar * Kbar][~masks[1]]
    fG = pseudo_inverse(AI) @ fI                  # values at G (the least-squares solution)
    sv = np.linalg.svd(AI, compute_uv=False)
    cond = sv[0] / sv[sv > PINV_RCOND * sv[0]][-1]
    # Kbar x Kbar grid: interior nodes keep the data, exterior nodes get the fit
    nI_S = int(masks[0].sum())
    nI_Sb = int(masks[1].sum())
    grid = np.zeros((Kbar * Kbar, fI.shape[1]))
    grid[masks[1]] = fI[nI_S:nI_S + nI_Sb]
    ext = ~masks[1]
    if ext.any():
        grid[ext] = AE @ fG
    # Chebyshev coefficients: grid[ax, by] = sum_mn alpha[m,n] T_m(x_ax) T_n(y_by)
    tc = chebyshev1_nodes(Kbar)
    T = npcheb.chebvander(tc, Kbar - 1)           # T[a, m] = T_m(tc[a])
    Tinv = np.linalg.inv(T)
    zt = (targets - np.array([cx, cy])) / r
    TX = npcheb.chebvander(zt[:, 0], Kbar - 1)
    TY = npcheb.chebvander(zt[:, 1], Kbar - 1)
    mm, nn = np.meshgrid(np.arange(Kbar), np.arange(Kbar), indexing="ij")
    keep = (mm + nn) < Kbar
    out = np.zeros((len(targets), fI.shape[1]))
    for rr in range(fI.shape[1]):
        Fb = grid[:, rr].reshape(Kbar, Kbar).T    # Fb[ax, by]  (grid index = by*Kbar + ax)
        alpha = Tinv @ Fb @ Tinv.T
        alpha = np.where(keep, alpha, 0.0)
        out[:, rr] = np.einsum("im,mn,in->i", TX, alpha, TY)
    return out, cond


def leaf_values(tree: OracleTree, dom, f_stencil: np.ndarray, meta, rbf_eps: float = 0.0):
    """f^e at every leaf node, shape (n_leaves, nrhs, K*K): data on regular
    leaves and on interior nodes of cut leaves, the extension on exterior
    nodes of cut leaves and on owned exterior leaves, zero elsewhere
    (Section 4.1).  rbf_eps > 0: Gaussians of that shape parameter on the unit
    box (Section 3.1) instead of their flat limit."""
    K = tree.K
    f_stencil = np.asarray(f_stencil, dtype=np.float64)
    if f_stencil.ndim == 1:
        f_stencil = f_stencil[:, None]
    nrhs = f_stencil.shape[1]
    out = np.zeros((tree.n_leaves, nrhs, K * K))
    conds = {}
    owned: Dict[int, List[int]] = {}
    for i, o in enumerate(tree.owner):
        if o >= 0:
            owned.setdefault(o, []).append(i)
    for i, b in enumerate(tree.leaves):
        if tree.cls[i] == REGULAR:
            off, n = meta[i]
            out[i] = f_stencil[off:off + n].T
    for i, b in enumerate(tree.leaves):
        if tree.cls[i] != CUT:
            continue
        off, n, masks = meta[i]
        fI = f_stencil[off:off + n]
        own_nodes = leaf_nodes(b, tree.t)
        tg = [own_nodes[~masks[0]]]
        for j in owned.get(i, []):
            tg.append(leaf_nodes(tree.leaves[j], tree.t))
        targets = np.concatenate(tg)
        vals, cond = extend_cut_leaf(b, K, tree.t, masks, fI, targets, rbf_eps)
        conds[i] = cond
        nE = int((~masks[0]).sum())
        v = np.zeros((K * K, nrhs))
        v[masks[0]] = fI[:int(masks[0].sum())]
        v[~masks[0]] = vals[:nE]
        out[i] = v.T
        pos = nE
        for j in owned.get(i, []):
            out[j] = vals[pos:pos + K * K].T
            pos += K * K
    return out, conds


# --------------------------------------------------------------------------- potential

def volume_potential(tree: OracleTree, values: np.ndarray, targets: np.ndarray, nthreads: int = 0):
    """V at targets (n, nrhs) by direct quadrature over all leaves."""
    L = lib()
    K = tree.K
    nrhs = values.shape[1]
    cen = np.array([box_center(b) for b in tree.leaves])
    h = np.array([0.5 * box_side(b[0]) for b in tree.leaves])
    cx = np.ascontiguousarray(cen[:, 0])
    cy = np.ascontiguousarray(cen[:, 1])
    t = np.ascontiguousarray(tree.t, dtype=np.float64)
    f = np.ascontiguousarray(values, dtype=np.float64)
    tx = np.ascontiguousarray(targets[:, 0], dtype=np.float64)
    ty = np.ascontiguousarray(targets[:, 1], dtype=np.float64)
    V = np.zeros((len(targets), nrhs))
    rc = L.orc_volume_potential(tree.n_leaves, _ptr(cx), _ptr(cy), _ptr(h), K, _ptr(t), nrhs, _ptr(f),
                                len(targets), _ptr(tx), _ptr(ty), _ptr(V), int(nthreads))
    if rc != 0:
        raise RuntimeError("orc_volume_potential failed: %d" % rc)
    return V


def net_charge(tree: OracleTree, values: np.ndarray) -> np.ndarray:
    """A^e = the integral of f^e over its support (Section 6.2, the growth
    constant of the particular solution at infinity): on every leaf the
    tensor Gauss-Legendre rule with the leaf's K x K nodes, Jacobian
    (side / 2)^2.  values: (n_leaves, nrhs, K*K).  Returns (nrhs,)."""
    _, w = gauss_legendre(tree.K)
    w2 = np.outer(w, w).ravel()                  # index b*K + a: w_b * w_a
    out = np.zeros(values.shape[1])
    for i, b in enumerate(tree.leaves):
        h = 0.5 * box_side(b[0])
        out += h * h * (values[i] @ w2)
    return out


def all_leaf_nodes(tree: OracleTree) -> np.ndarray:
    return np.concatenate([leaf_nodes(b, tree.t) for b in tree.leaves])


def boundary_nodes(dom, nq: int = NQ_BOUNDARY) -> np.ndarray:
    """y_ij = gamma_i(t_j) with t_j the nq-point Gauss-Legendre nodes (Section 5)."""
    t, _ = gauss_legendre(nq)
    n = getattr(dom, "n_panels", 0)
    if n == 0:
        return np.zeros((0, 2))
    return np.concatenate([dom.curve(i, t)[0] for i in range(n)])


def locate_leaf(tree: OracleTree, p) -> int:
    """Leaf containing p; a point on an edge belongs to the box with the larger
    index, except on the top/right edge of D."""
    lmax = max(b[0] for b in tree.leaves)
    for lev in range(0, lmax + 1):
        n = 1 << lev
        ix = min(int(math.floor((p[0] + 0.5) * n)), n - 1)
        iy = min(int(math.floor((p[1] + 0.5) * n)), n - 1)
        if (lev, ix, iy) in tree.index:
            return tree.index[(lev, ix, iy)]
    raise ValueError("point outside D")


def interpolate_at(tree: OracleTree, Vleaf: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Tensor Lagrange interpolation of leaf-node values (n_leaves, K*K, nrhs)
    at arbitrary points (Section 4.1: evaluation by interpolation on the
    containing leaf)."""
    K = tree.K
    t = tree.t
    out = np.zeros((len(pts), Vleaf.shape[2]))
    for k, p in enumerate(pts):
        i = locate_leaf(tree, p)
        cx, cy = box_center(tree.leaves[i])
        h = 0.5 * box_side(tree.leaves[i][0])
        u, v = (p[0] - cx) / h, (p[1] - cy) / h
        la = np.array([np.prod([(u - t[m]) / (t[a] - t[m]) for m in range(K) if m != a]) for a in range(K)])
        lb = np.array([np.prod([(v - t[m]) / (t[a] - t[m]) for m in range(K) if m != a]) for a in range(K)])
        w = np.outer(lb, la).ravel()    # index b*K + a
        out[k] = w @ Vleaf[i]
    return out


@dataclass
class OracleResult:
    tree: OracleTree
    stencil: np.ndarray
    f_stencil: np.ndarray
    values: np.ndarray          # (n_leaves, nrhs, K*K)
    v_leaf: np.ndarray          # (n_leaves*K*K, nrhs)
    v_bdry: np.ndarray          # (n_bdry, nrhs)
    conds: dict


def solve(workload, target_subset=None, nthreads: int = 0) -> OracleResult:
    """Whole particular-solution stage on the oracle's own tree.

    target_subset: optional index array into the leaf nodes; V is then
    computed only there (v_leaf holds NaN elsewhere) and boundary values are
    skipped.
    """
    dom = workload.domain
    tree = build_tree(dom, workload.opts, workload.sources[0])
    pts, meta = stencil_points(tree, dom)
    fs = np.stack([np.asarray(f(pts), dtype=np.float64) for f in workload.sources], axis=1) if len(pts) else \
        np.zeros((0, len(workload.sources)))
    vals, conds = leaf_values(tree, dom, fs, meta)
    nodes = all_leaf_nodes(tree)
    nrhs = vals.shape[1]
    if target_subset is None:
        V = volume_potential(tree, vals, nodes, nthreads)
        Vl = V.reshape(tree.n_leaves, tree.K * tree.K, nrhs)
        vb = interpolate_at(tree, Vl, boundary_nodes(dom))
    else:
        V = np.full((len(nodes), nrhs), np.nan)
        V[target_subset] = volume_potential(tree, vals, nodes[target_subset], nthreads)
        vb = np.zeros((0, nrhs))
    return OracleResult(tree, pts, fs, vals, V, vb, conds)
