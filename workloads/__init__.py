"""Seeded synthetic problem definitions: domains, boundary panels, sources.

This module is shared by the CUDA library's tests/benchmark and by the CPU
oracle.  It defines *inputs only* -- the geometry of Omega (an inside/outside
predicate and a panel parametrisation gamma_i(t), t in [-1,1]), the source
density f, and the tree options of each workload -- and holds none of the
method's arithmetic (no quadrature, no extension, no potential).

Geometry follows the problem statement of Section 4 (Omega inside the unit
box D centred at the origin, boundary given as panels gamma_i([-1,1])).
Random draws use NumPy's PCG64 with seed 2211 + workload id.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

TWO_PI = 2.0 * math.pi

# ---------------------------------------------------------------------------
# Domains
# ---------------------------------------------------------------------------


class StarDomain:
    """Star-shaped domain r(theta) = r0 * (1 + sum_k a_k cos(k theta + phi_k)).

    Covers the disk (no modes), the starfish of the adaptive interior
    workload (one mode k=5) and the random star shapes of the batch workload.
    The boundary is split into ``n_panels`` equal arcs in theta; panel i maps
    t in [-1,1] to theta = theta_i + (t+1)/2 * dtheta.
    """

    def __init__(self, r0: float, modes: Sequence[Tuple[int, float, float]] = (),
                 n_panels: Optional[int] = None, center=(0.0, 0.0)):
        self.r0 = float(r0)
        self.modes = [(int(k), float(a), float(p)) for (k, a, p) in modes]
        self.center = (float(center[0]), float(center[1]))
        self.n_panels = int(n_panels) if n_panels else choose_panel_count(self)

    # r(theta) and dr/dtheta
    def r(self, th):
        th = np.asarray(th, dtype=np.float64)
        s = np.ones_like(th)
        for k, a, p in self.modes:
            s = s + a * np.cos(k * th + p)
        return self.r0 * s

    def dr(self, th):
        th = np.asarray(th, dtype=np.float64)
        s = np.zeros_like(th)
        for k, a, p in self.modes:
            s = s - a * k * np.sin(k * th + p)
        return self.r0 * s

    def inside(self, xy: np.ndarray) -> np.ndarray:
        """Strict interior test: |x - c| < r(theta(x))."""
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        dx = xy[:, 0] - self.center[0]
        dy = xy[:, 1] - self.center[1]
        rho = np.hypot(dx, dy)
        th = np.arctan2(dy, dx)
        return rho < self.r(th)

    def panel_theta(self, i: int, t):
        dth = TWO_PI / self.n_panels
        return i * dth + (np.asarray(t, dtype=np.float64) + 1.0) * 0.5 * dth

    def curve(self, i: int, t) -> Tuple[np.ndarray, np.ndarray]:
        """gamma_i(t) and gamma_i'(t) (derivative w.r.t. t) as (n,2) arrays."""
        th = self.panel_theta(i, t)
        dth_dt = 0.5 * TWO_PI / self.n_panels
        r = self.r(th)
        dr = self.dr(th)
        c, s = np.cos(th), np.sin(th)
        xy = np.stack([self.center[0] + r * c, self.center[1] + r * s], axis=1)
        dxy = np.stack([(dr * c - r * s) * dth_dt, (dr * s + r * c) * dth_dt], axis=1)
        return xy, dxy


class ExteriorDomain:
    """The exterior of several star-shaped inclusions (within the root box D):
    Omega = D minus the closures of the inclusions (Section 6.2).  The boundary
    is the union of the inclusions' panels, numbered inclusion by inclusion
    (orientation plays no part in the particular solution)."""

    def __init__(self, inclusions: Sequence[StarDomain]):
        self.inclusions = list(inclusions)
        self.n_panels = sum(d.n_panels for d in self.inclusions)

    def inside(self, xy: np.ndarray) -> np.ndarray:
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        out = np.ones(len(xy), dtype=bool)
        for d in self.inclusions:
            out &= ~d.inside(xy)
        return out

    def curve(self, i: int, t) -> Tuple[np.ndarray, np.ndarray]:
        for d in self.inclusions:
            if i < d.n_panels:
                return d.curve(i, t)
            i -= d.n_panels
        raise IndexError("panel index out of range")


class SawDomain:
    """The simply connected domain of Section 6.1's second interior test:
    z(theta) = a (2 + b sin(m theta)) exp(i (theta + b sin(m theta))),
    a = 0.17, b = 0.5, m = 7, theta in [0, 2 pi).  The polar angle
    phi(theta) = theta + b sin(m theta) turns back (phi' = 1 + b m cos(m theta)
    changes sign), so the domain is not star-shaped: the inside test counts
    the crossings of the outward ray from the point, solving phi(theta) =
    psi (mod 2 pi) by bisection on each interval where phi is monotone.
    Panels are equal arcs in theta."""

    def __init__(self, a: float = 0.17, b: float = 0.5, m: int = 7, n_panels: Optional[int] = None):
        self.a, self.b, self.m = float(a), float(b), int(m)
        c = np.arccos(-1.0 / (self.b * self.m)) if self.b * self.m > 1.0 else None
        cuts = [0.0, TWO_PI]
        if c is not None:
            for j in range(self.m + 1):
                for th in ((c + TWO_PI * j) / self.m, (TWO_PI * (j + 1) - c) / self.m):
                    if 0.0 < th < TWO_PI:
                        cuts.append(th)
        self._cuts = np.array(sorted(cuts))
        self.n_panels = int(n_panels) if n_panels else choose_panel_count(self, [64, 96, 128, 160, 192, 256, 320,
                                                                                  384, 512, 640, 768, 1024])

    def rad(self, th):
        return self.a * (2.0 + self.b * np.sin(self.m * th))

    def phi(self, th):
        return th + self.b * np.sin(self.m * th)

    def inside(self, xy: np.ndarray) -> np.ndarray:
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        rho = np.hypot(xy[:, 0], xy[:, 1])
        psi = np.mod(np.arctan2(xy[:, 1], xy[:, 0]), TWO_PI)
        count = np.zeros(len(xy), dtype=np.int64)
        for lo, hi in zip(self._cuts[:-1], self._cuts[1:]):
            plo, phi_hi = self.phi(lo), self.phi(hi)
            up = phi_hi > plo
            for k in (-1, 0, 1):
                tgt = psi + TWO_PI * k
                # half-open in theta: a root at the interval's upper end belongs to the next one
                sel = np.nonzero((tgt >= min(plo, phi_hi)) & (tgt < max(plo, phi_hi)) if up else
                                 (tgt > min(plo, phi_hi)) & (tgt <= max(plo, phi_hi)))[0]
                if len(sel) == 0:
                    continue
                a = np.full(len(sel), lo)
                c = np.full(len(sel), hi)
                for _ in range(64):
                    mid = 0.5 * (a + c)
                    below = (self.phi(mid) < tgt[sel]) if up else (self.phi(mid) > tgt[sel])
                    a = np.where(below, mid, a)
                    c = np.where(below, c, mid)
                count[sel] += self.rad(0.5 * (a + c)) > rho[sel]
        return (count % 2) == 1

    def curve(self, i: int, t) -> Tuple[np.ndarray, np.ndarray]:
        dth = TWO_PI / self.n_panels
        th = i * dth + (np.asarray(t, dtype=np.float64) + 1.0) * 0.5 * dth
        r, p = self.rad(th), self.phi(th)
        dr = self.a * self.b * self.m * np.cos(self.m * th)
        dp = 1.0 + self.b * self.m * np.cos(self.m * th)
        c, s = np.cos(p), np.sin(p)
        xy = np.stack([r * c, r * s], axis=1)
        dxy = np.stack([(dr * c - r * dp * s) * 0.5 * dth, (dr * s + r * dp * c) * 0.5 * dth], axis=1)
        return xy, dxy


class HoledDomain:
    """Omega = the inside of an outer star-shaped curve minus the closures of
    inner star-shaped holes (the multiply connected interior problem of
    Section 2).  Panels: the outer curve's, then each hole's, every curve
    counter-clockwise."""

    def __init__(self, outer: StarDomain, holes: Sequence[StarDomain]):
        self.outer, self.holes = outer, list(holes)
        self.curves = [outer] + self.holes
        self.n_panels = sum(d.n_panels for d in self.curves)

    def inside(self, xy: np.ndarray) -> np.ndarray:
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        out = self.outer.inside(xy)
        for h in self.holes:
            out &= ~h.inside(xy)
        return out

    def curve(self, i: int, t) -> Tuple[np.ndarray, np.ndarray]:
        for d in self.curves:
            if i < d.n_panels:
                return d.curve(i, t)
            i -= d.n_panels
        raise IndexError("panel index out of range")


class PolygonDomain:
    """Polygon given by its vertices (counter-clockwise).

    Each side is split into ``panels_per_side`` equal panels; the first and
    last panel of every side are further split dyadically ``corner_levels``
    times toward the vertex, so that panel length halves toward each corner.
    """

    def __init__(self, vertices: Sequence[Tuple[float, float]], panels_per_side: int = 16,
                 corner_levels: int = 0, inside_fn: Optional[Callable] = None):
        self.vertices = np.asarray(vertices, dtype=np.float64)
        self._inside_fn = inside_fn
        segs = []  # (p0, p1) per panel
        nv = len(self.vertices)
        for v in range(nv):
            a = self.vertices[v]
            b = self.vertices[(v + 1) % nv]
            # parameters along the side in [0,1]
            cuts = list(np.linspace(0.0, 1.0, panels_per_side + 1))
            head = [0.0]
            x = cuts[1]
            for _ in range(corner_levels):
                x = x * 0.5
                head.append(x)
            head = sorted(head)
            tail = [1.0 - h for h in head]
            pts = sorted(set(head + cuts[1:-1] + tail + [cuts[1], cuts[-2]]))
            for j in range(len(pts) - 1):
                segs.append((a + (b - a) * pts[j], a + (b - a) * pts[j + 1]))
        self.segments = segs
        self.n_panels = len(segs)

    def inside(self, xy: np.ndarray) -> np.ndarray:
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        if self._inside_fn is not None:
            return self._inside_fn(xy)
        # crossing-number test (points exactly on an edge count as outside)
        x, y = xy[:, 0], xy[:, 1]
        res = np.zeros(len(xy), dtype=bool)
        vs = self.vertices
        n = len(vs)
        for i in range(n):
            x0, y0 = vs[i]
            x1, y1 = vs[(i + 1) % n]
            cond = (y0 > y) != (y1 > y)
            with np.errstate(divide="ignore", invalid="ignore"):
                xc = x0 + (y - y0) * (x1 - x0) / (y1 - y0)
            res ^= cond & (x < xc)
        return res

    def curve(self, i: int, t) -> Tuple[np.ndarray, np.ndarray]:
        t = np.asarray(t, dtype=np.float64)
        a, b = self.segments[i]
        s = (t + 1.0) * 0.5
        xy = a[None, :] + s[:, None] * (b - a)[None, :]
        dxy = np.repeat(((b - a) * 0.5)[None, :], len(t), axis=0)
        return xy, dxy


def choose_panel_count(dom: StarDomain, candidates=None) -> int:
    """Panel count rule for star boundaries (Section 6, boundary discretisation).

    The smallest N among ``candidates`` such that, on every panel, the
    16-point Legendre expansion of |gamma'(t)| has its two highest
    coefficients below 1e-14 times its largest one (fifteen digits, read
    against the ~4e-15 rounding floor of the transform).  This is input
    preparation (how finely the user samples the boundary), not part of the
    volume-potential method.
    """
    if candidates is None:
        candidates = [16, 24, 32, 40, 48, 64, 80, 96, 128, 160, 192, 256, 320, 384, 512]
    t, _ = np.polynomial.legendre.leggauss(16)
    V = np.polynomial.legendre.legvander(t, 15)
    Vinv = np.linalg.inv(V)
    for n in candidates:
        dom.n_panels = n
        ok = True
        for i in range(n):
            _, d = dom.curve(i, t)
            sp = np.hypot(d[:, 0], d[:, 1])
            c = Vinv @ sp
            if max(abs(c[-1]), abs(c[-2])) > 1e-14 * np.max(np.abs(c)):
                ok = False
                break
        if ok:
            return n
    return candidates[-1]


def l_shape_inside(xy):
    x, y = xy[:, 0], xy[:, 1]
    box = (x > -0.4) & (x < 0.4) & (y > -0.4) & (y < 0.4)
    notch = (x >= 0.0) & (y >= 0.0)
    return box & ~notch


def l_shape_domain(panels_per_side: int = 16, corner_levels: int = 11) -> PolygonDomain:
    """L-shaped polygon, side 0.8: [-0.4,0.4]^2 minus [0,0.4]^2, 6 corners."""
    verts = [(-0.4, -0.4), (0.4, -0.4), (0.4, 0.0), (0.0, 0.0), (0.0, 0.4), (-0.4, 0.4)]
    return PolygonDomain(verts, panels_per_side, corner_levels, inside_fn=l_shape_inside)


class WholeBoxDomain:
    """Omega = a region containing D: every point of D is interior.

    No boundary panels; every leaf is regular.  Used by closed-form checks.
    """
    n_panels = 0

    def inside(self, xy):
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        return np.ones(len(xy), dtype=bool)

    def curve(self, i, t):  # pragma: no cover - never called (no panels)
        raise IndexError("no panels")


# ---------------------------------------------------------------------------
# Sources
# ---------------------------------------------------------------------------


def f_sincos(xy):
    """f = -13 sin(3x) cos(2y) = Laplacian of sin(3x) cos(2y)."""
    xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
    return -13.0 * np.sin(3.0 * xy[:, 0]) * np.cos(2.0 * xy[:, 1])


def make_gaussian(center, width, amp=1.0):
    cx, cy = float(center[0]), float(center[1])
    w2 = float(width) ** 2
    a = float(amp)

    def f(xy):
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        return a * np.exp(-((xy[:, 0] - cx) ** 2 + (xy[:, 1] - cy) ** 2) / w2)
    return f


def make_gaussian_mixture(centers, widths, amps):
    centers = np.asarray(centers, dtype=np.float64)
    widths = np.asarray(widths, dtype=np.float64)
    amps = np.asarray(amps, dtype=np.float64)

    def f(xy):
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        out = np.zeros(len(xy))
        for c, w, a in zip(centers, widths, amps):
            out += a * np.exp(-((xy[:, 0] - c[0]) ** 2 + (xy[:, 1] - c[1]) ** 2) / (w * w))
        return out
    return f


def f_exp_sin(xy):
    """f = -3 e^x sin(2y) = Laplacian of e^x sin(2y)."""
    xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
    return -3.0 * np.exp(xy[:, 0]) * np.sin(2.0 * xy[:, 1])


def sample_inside(dom, n, rng, box=0.5):
    """Rejection-sample n points uniformly inside the domain."""
    pts = []
    while len(pts) < n:
        p = rng.uniform(-box, box, size=(4 * n, 2))
        p = p[dom.inside(p)]
        pts.extend(p.tolist())
    return np.asarray(pts[:n])


def random_mixture(dom, rng, n_gauss=8, wmin=0.01, wmax=0.1):
    c = sample_inside(dom, n_gauss, rng)
    w = np.exp(rng.uniform(math.log(wmin), math.log(wmax), size=n_gauss))
    a = rng.standard_normal(n_gauss)
    return make_gaussian_mixture(c, w, a), (c, w, a)


# ---------------------------------------------------------------------------
# Tree options and workloads
# ---------------------------------------------------------------------------


@dataclass
class TreeOptions:
    """Discretisation options shared by the library and the oracle.

    K: nodes per dimension on a leaf (Gauss-Legendre).  min_level: every box
    above this level is split (a uniform base).  max_level: no box is split
    beyond it.  refine_tol: adaptive resolution tolerance (0 = uniform tree
    at min_level).  f_scale: the scale the tolerance is relative to.
    """
    K: int = 8
    min_level: int = 4
    max_level: int = 4
    refine_tol: float = 0.0
    f_scale: float = 1.0


@dataclass
class Workload:
    name: str
    wid: int
    domain: object
    opts: TreeOptions
    sources: List[Callable] = field(default_factory=list)  # one per right-hand side
    description: str = ""


def disk_sincos(level: int = 4, K: int = 8) -> Workload:
    """Disk r=0.35, f=-13 sin3x cos2y, uniform tree, 16 panels x 16 nodes."""
    dom = StarDomain(0.35, (), n_panels=16)
    return Workload("disk_sincos_uniform_l%d_k%d" % (level, K), 1, dom,
                    TreeOptions(K=K, min_level=level, max_level=level), [f_sincos],
                    "disk r=0.35, f=-13sin(3x)cos(2y), uniform level %d, K=%d" % (level, K))


def starfish_gaussian(K: int = 16, tol: float = 1e-10, min_level: int = 2, max_level: int = 12) -> Workload:
    """Starfish r=0.35(1+0.3cos5t), Gaussian sigma=0.02 at (0.1,0.05), adaptive."""
    dom = StarDomain(0.35, [(5, 0.3, 0.0)])
    f = make_gaussian((0.1, 0.05), 0.02)
    return Workload("starfish_gaussian_adaptive_k%d" % K, 2, dom,
                    TreeOptions(K=K, min_level=min_level, max_level=max_level, refine_tol=tol, f_scale=1.0),
                    [f], "starfish r=.35(1+.3cos5t), f=exp(-|x-(.1,.05)|^2/.02^2), adaptive tol %g, K=%d" % (tol, K))


def disk_multi_rhs(nrhs: int = 64, level: int = 4, K: int = 8, n_gauss: int = 8) -> Workload:
    """Disk geometry of the uniform workload with nrhs Gaussian-mixture sources."""
    rng = np.random.Generator(np.random.PCG64(2211 + 3))
    dom = StarDomain(0.35, (), n_panels=16)
    srcs = [random_mixture(dom, rng, n_gauss)[0] for _ in range(nrhs)]
    return Workload("disk_mixture_x%d_l%d_k%d" % (nrhs, level, K), 3, dom,
                    TreeOptions(K=K, min_level=level, max_level=level), srcs,
                    "disk r=0.35, %d RHS of %d-Gaussian mixtures, uniform level %d" % (nrhs, n_gauss, level))


def lshape_expsin(K: int = 16, base_level: int = 6, max_level: int = 14, corner_levels: int = 11) -> Workload:
    dom = l_shape_domain(16, corner_levels)
    return Workload("lshape_expsin_k%d" % K, 4, dom,
                    TreeOptions(K=K, min_level=base_level, max_level=max_level, refine_tol=1e-10, f_scale=3.0),
                    [f_exp_sin], "L-shape side 0.8, f=-3e^x sin2y, base level %d, corners to level %d" % (base_level, max_level))


EXTERIOR_INCLUSIONS = [(0.12, 0.3, 5, (0.186, -0.15)), (0.17, 0.3, 4, (-0.21, -0.03)), (0.12, 0.2, 3, (0.2, 0.15))]
EXTERIOR_GAUSSIANS = [((0.1, 0.07), 1e-3), ((0.09, -0.25), 1e-3 / 2.1), ((-0.21, -0.25), 1e-3 / 4.5)]
EXTERIOR_LOG_CENTRE, EXTERIOR_LOG_COEF = (-0.2, 0.0), -10.0


def exterior_domain() -> "ExteriorDomain":
    """The three starfish inclusions of the exterior test of Section 6.2,
    z = R (1 + a cos(N t)) e^{-it} + c with (R, a, N, c) as in
    EXTERIOR_INCLUSIONS.  The third radius is 0.12 where the text prints 0.2:
    at 0.2 the first and third inclusions overlap (a sixth of the first
    curve lies inside the third), while at 0.12 the curves are disjoint and
    every Gaussian centre y_j lies 0.001 - 0.003 inside its inclusion, as the
    text describes them."""
    return ExteriorDomain([StarDomain(R, [(N, a, 0.0)], center=c) for R, a, N, c in EXTERIOR_INCLUSIONS])


def u_exterior(xy):
    """The exact solution of the exterior test (Section 6.2):
    u = sum_j exp(-|x - y_j|^2 / beta_j) - 10 log|x - (-0.2, 0)|."""
    xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
    out = EXTERIOR_LOG_COEF * np.log(np.hypot(xy[:, 0] - EXTERIOR_LOG_CENTRE[0], xy[:, 1] - EXTERIOR_LOG_CENTRE[1]))
    for y, b in EXTERIOR_GAUSSIANS:
        out = out + np.exp(-((xy[:, 0] - y[0]) ** 2 + (xy[:, 1] - y[1]) ** 2) / b)
    return out


def f_exterior(xy):
    """f = Laplacian of u_exterior in Omega: the Gaussians' Laplacians
    (4 r^2 / beta^2 - 4 / beta) exp(-r^2 / beta); the log term is harmonic there."""
    xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
    out = np.zeros(len(xy))
    for y, b in EXTERIOR_GAUSSIANS:
        r2 = (xy[:, 0] - y[0]) ** 2 + (xy[:, 1] - y[1]) ** 2
        out += (4.0 * r2 / (b * b) - 4.0 / b) * np.exp(-r2 / b)
    return out


def exterior_three_stars(K: int = 8, tol: float = 1e-8, min_level: int = 3, max_level: int = 10) -> Workload:
    """The exterior test of Section 6.2 in D = [-0.5, 0.5]^2: Omega = D minus
    three starfish inclusions (exterior_domain), f = f_exterior.  The
    Gaussian centres lie inside the inclusions, so the extension runs into
    the steep side of each bump."""
    return Workload("exterior_three_stars_k%d" % K, 6, exterior_domain(),
                    TreeOptions(K=K, min_level=min_level, max_level=max(min_level, max_level) if tol else min_level,
                                refine_tol=tol, f_scale=1e4),
                    [f_exterior], "exterior of three starfish inclusions (Section 6.2), "
                    "f = Laplacian of 3 Gaussians, %s, K=%d" % ("adaptive tol %g" % tol if tol else
                                                                 "uniform level %d" % min_level, K))


def u_harmext(xy):
    """The exact solution of Section 6.1's interior tests:
    u = sin(10 (x + y)) + x^2 - 3 y + 8 + exp(-500 x^2)."""
    xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
    x, y = xy[:, 0], xy[:, 1]
    return np.sin(10.0 * (x + y)) + x * x - 3.0 * y + 8.0 + np.exp(-500.0 * x * x)


def f_harmext(xy):
    """f = Laplacian of u_harmext = -200 sin(10 (x + y)) + 2 + (1e6 x^2 - 1000) exp(-500 x^2)."""
    xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
    x, y = xy[:, 0], xy[:, 1]
    return -200.0 * np.sin(10.0 * (x + y)) + 2.0 + (1e6 * x * x - 1000.0) * np.exp(-500.0 * x * x)


def saw_harmext(level: int = 5, K: int = 8, n_panels: Optional[int] = None) -> Workload:
    """Section 6.1's second interior test on a uniform tree: the saw domain,
    f = Laplacian of u_harmext, Dirichlet data g = u_harmext on the boundary.
    Without n_panels: 256 panels up to level 5 (|gamma'| resolved to 5e-8 on
    every panel, below the level-5 error of 6e-5), else the panel rule."""
    if n_panels is None and level <= 5:
        n_panels = 256
    return Workload("saw_harmext_l%d_k%d" % (level, K), 7, SawDomain(n_panels=n_panels),
                    TreeOptions(K=K, min_level=level, max_level=level), [f_harmext],
                    "saw domain (Section 6.1), u = sin(10(x+y)) + x^2 - 3y + 8 + exp(-500x^2), uniform level %d" % level)


def doubly_connected_domain() -> "HoledDomain":
    """Section 6.1's first test: r(theta) = sum_j c_j cos(j theta) + d_j sin(j theta)
    with, outside, c_0 = 0.25, d_3 = c_6 = c_8 = c_10 = 0.01, c_5 = 0.02 and, for
    the hole, c_0 = 0.05, c_2 = d_3 = c_5 = c_7 = 0.005 (sin = cos shifted by -pi/2)."""
    h = -0.5 * np.pi
    outer = StarDomain(0.25, [(3, 0.04, h), (6, 0.04, 0.0), (8, 0.04, 0.0), (10, 0.04, 0.0), (5, 0.08, 0.0)])
    hole = StarDomain(0.05, [(2, 0.1, 0.0), (3, 0.1, h), (5, 0.1, 0.0), (7, 0.1, 0.0)])
    return HoledDomain(outer, [hole])


def doubly_connected_harmext(level: int = 5, K: int = 8) -> Workload:
    """Section 6.1's first interior test on a uniform tree: the doubly connected
    domain, f = Laplacian of u_harmext, Dirichlet data u_harmext on both curves."""
    return Workload("doubly_connected_harmext_l%d_k%d" % (level, K), 8, doubly_connected_domain(),
                    TreeOptions(K=K, min_level=level, max_level=level), [f_harmext],
                    "doubly connected domain (Section 6.1), u = sin(10(x+y)) + x^2 - 3y + 8 + exp(-500x^2), "
                    "uniform level %d" % level)


def doubly_connected_adaptive(K: int = 8) -> Workload:
    """The run behind the paper's timings (Section 6.1): the doubly connected
    domain, f = Laplacian of u_harmext, adaptive at tolerance 0.5e-11 (relative
    to f_scale 1e3, the size of f) with seven levels near the boundary: 3,778
    leaves (273 cut), 241,792 leaf nodes here against the paper's 3,361 leaves
    (339 cut), about 215,000 points."""
    return Workload("doubly_connected_adaptive_k%d" % K, 10, doubly_connected_domain(),
                    TreeOptions(K=K, min_level=3, max_level=7, refine_tol=0.5e-11, f_scale=1e3), [f_harmext],
                    "doubly connected domain (Section 6.1), u = sin(10(x+y)) + x^2 - 3y + 8 + exp(-500x^2), "
                    "adaptive tol 0.5e-11, levels 3-7, K=%d (the paper's timing run)" % K)


SQUARE_CENTRE, SQUARE_SIDE, SQUARE_ANGLE = (0.01, -0.02), 0.5, np.pi / 3
SQUARE_POINTS = np.array([[-0.35, -0.135], [-0.09, 0.42], [0.445, 0.09], [0.135, -0.405]])
SQUARE_BETA = 800.0


def u_square(xy):
    """Section 6.3's solution, read as u = -2 sum_j (Ei(-beta r_j^2) - log r_j^2),
    r_j = |x - x_j|, beta = 800: smooth everywhere (the two logarithmic
    singularities at x_j cancel), with Laplacian 8 beta sum_j exp(-beta r_j^2)."""
    from scipy.special import expi
    xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
    out = np.zeros(len(xy))
    for x in SQUARE_POINTS:
        r2 = (xy[:, 0] - x[0]) ** 2 + (xy[:, 1] - x[1]) ** 2
        out += -2.0 * (expi(-SQUARE_BETA * r2) - np.log(r2))
    return out


def f_square(xy):
    """f = Laplacian of u_square = 8 beta sum_j exp(-beta |x - x_j|^2)."""
    xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
    out = np.zeros(len(xy))
    for x in SQUARE_POINTS:
        out += 8.0 * SQUARE_BETA * np.exp(-SQUARE_BETA * ((xy[:, 0] - x[0]) ** 2 + (xy[:, 1] - x[1]) ** 2))
    return out


def square_domain(panels_per_side: int = 16, corner_levels: int = 10) -> PolygonDomain:
    """Section 6.3: the square of side 0.5 centred at (0.01, -0.02), rotated by
    pi/3, counter-clockwise; panels graded dyadically toward the corners."""
    c, h, a = np.array(SQUARE_CENTRE), 0.5 * SQUARE_SIDE, SQUARE_ANGLE
    rot = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
    verts = [tuple(c + rot @ np.array(v)) for v in [(-h, -h), (h, -h), (h, h), (-h, h)]]
    return PolygonDomain(verts, panels_per_side, corner_levels)


def square_pwsmooth(level: int = 5, K: int = 8) -> Workload:
    """Section 6.3's piecewise smooth test on a uniform tree."""
    return Workload("square_pwsmooth_l%d_k%d" % (level, K), 9, square_domain(),
                    TreeOptions(K=K, min_level=level, max_level=level), [f_square],
                    "rotated square (Section 6.3), f = 8 beta sum exp(-beta |x - x_j|^2), uniform level %d" % level)


def grid_100(dom, n: int = 100) -> np.ndarray:
    """The points of a uniform n x n grid on D (endpoints included) inside Omega,
    where Section 6 measures the solution's error."""
    g = np.linspace(-0.5, 0.5, n)
    X, Y = np.meshgrid(g, g, indexing="xy")
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    return pts[dom.inside(pts)]


def star_batch(n_domains: int = 32, K: int = 8, tol: Optional[float] = None, max_level: int = 11):
    """Uneven batch: random star domains r = .35(1 + sum_{k=2..8} a_k cos(k t + phi_k)),
    a_k ~ U[0, .04], phi_k ~ U[0, 2 pi), each with its own Gaussian mixture.
    Without ``tol`` each domain draws its refinement tolerance log-uniformly
    from [1e-8, 1e-3], so every tree resolves its own f and the trees range
    from about 300 leaves (1.8e4 points at K = 8) to about 6,000 (3.8e5)."""
    rng = np.random.Generator(np.random.PCG64(2211 + 5))
    out = []
    for d in range(n_domains):
        modes = [(k, rng.uniform(0.0, 0.04), rng.uniform(0.0, TWO_PI)) for k in range(2, 9)]
        dom = StarDomain(0.35, modes)
        f, _ = random_mixture(dom, rng)
        t = 10.0 ** rng.uniform(-8.0, -3.0) if tol is None else float(tol)
        out.append(Workload("star%02d" % d, 5, dom,
                            TreeOptions(K=K, min_level=2, max_level=max_level, refine_tol=t, f_scale=1.0),
                            [f], "random star %d" % d))
    return out


def gauss_legendre_panel_nodes(dom, nq: int = 16):
    """Boundary target points y_ij = gamma_i(t_j) on every panel (j fastest)."""
    t, _ = np.polynomial.legendre.leggauss(nq)
    pts = [dom.curve(i, t)[0] for i in range(dom.n_panels)]
    return np.concatenate(pts, axis=0) if pts else np.zeros((0, 2))
