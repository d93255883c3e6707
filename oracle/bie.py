"""CPU oracle for the boundary correction -- TEST INFRASTRUCTURE ONLY.

Plain FP64 restatement of Section 5 for the interior Dirichlet problem on a
simply connected domain: u = V[f^e] + D[sigma] in Omega with

    D[sigma](x) = int_Gamma (1/2pi) (x - y).nu(y) / |x - y|^2 sigma(y) ds_y
                                                          (eq. dlpot, dblker),
    (-1/2 + D)[sigma] = g - V[f^e]   on Gamma             (eq. inteq),

nu the outward unit normal.  The Nystrom discretisation uses the panels'
16-point Gauss-Legendre nodes y_ij, speeds s_ij = |gamma_i'(t_j)| and weights
w_j (eq. discdblpotpanel); the diagonal takes the kernel's limit on the
boundary, -kappa(y) / (4 pi) with kappa the signed curvature.  The system is
solved directly (the paper uses GMRES on the same matrix; both give its
solution).  D[sigma] off the boundary is the same Gauss-Legendre sum, except
for targets close to a panel, where the panel's contribution is computed by
the Helsing-Ojala product integration that the paper names (Section 5): the
density is interpolated by a polynomial in the complex panel variable and
integrated against the Cauchy kernel exactly.

Readings (the paper's statements disagree with one another here): eq. inteq's
sign, -1/2 + D, holds for the kernel of eq. dblker with the outward normal, and
with it D[1] = -1 inside Omega; the discrete system's printed "+1/2" and the
extra 1/(2 pi) go with the opposite normal.  The kernel's boundary limit is
-kappa / (4 pi) for that kernel (a circle of radius R gives -1 / (4 pi R)).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg

NQ = 16            # Gauss-Legendre nodes per panel (Section 5, N_q)
NEAR_RADIUS = 2.0  # product integration when |zeta| < NEAR_RADIUS in panel coordinates


class BoundaryGeometry:
    """Nodes, outward normals, speeds, weights and curvatures of every panel.

    y (N, 2) with N = n_panels * NQ, panel-major; dy = gamma_i'(t_j) (N, 2);
    s = |dy|; nu = (dy_2, -dy_1) / s (outward for a counter-clockwise
    boundary); w = the Gauss-Legendre weight of each node; kappa the signed
    curvature (x'y'' - y'x'') / s^3, with gamma'' from differentiating the
    degree-15 Legendre interpolant of gamma' on the panel."""

    def __init__(self, dom, nq: int = NQ):
        t, w = npleg.leggauss(nq)
        V = npleg.legvander(t, nq - 1)
        Vinv = np.linalg.inv(V)
        n = dom.n_panels
        ys, dys, ddys = [], [], []
        for i in range(n):
            xy, d = dom.curve(i, t)
            ys.append(xy)
            dys.append(d)
            c = Vinv @ d                                   # Legendre coefficients of gamma'
            ddys.append(npleg.legval(t, npleg.legder(c)).T)
        self.nq, self.n_panels, self.t = nq, n, t
        self.y = np.concatenate(ys)
        self.dy = np.concatenate(dys)
        ddy = np.concatenate(ddys)
        self.s = np.hypot(self.dy[:, 0], self.dy[:, 1])
        self.nu = np.stack([self.dy[:, 1], -self.dy[:, 0]], axis=1) / self.s[:, None]
        self.w = np.tile(w, n)
        self.kappa = (self.dy[:, 0] * ddy[:, 1] - self.dy[:, 1] * ddy[:, 0]) / self.s ** 3
        ends = [dom.curve(i, np.array([-1.0, 1.0]))[0] for i in range(n)]
        self.a = np.array([e[0, 0] + 1j * e[0, 1] for e in ends])    # panel start gamma_i(-1)
        self.b = np.array([e[1, 0] + 1j * e[1, 1] for e in ends])    # panel end gamma_i(1)

    @property
    def n(self):
        return len(self.y)


def dlp_matrix(g: BoundaryGeometry) -> np.ndarray:
    """D (N x N): D[a, b] = (1/2pi) (y_a - y_b).nu_b / |y_a - y_b|^2 s_b w_b,
    D[a, a] = -kappa_a / (4 pi) s_a w_a (eq. discdblpotpanel at the nodes)."""
    dx = g.y[:, None, 0] - g.y[None, :, 0]
    dy = g.y[:, None, 1] - g.y[None, :, 1]
    r2 = dx * dx + dy * dy
    np.fill_diagonal(r2, 1.0)
    K = (dx * g.nu[None, :, 0] + dy * g.nu[None, :, 1]) / r2 / (2 * math.pi)
    np.fill_diagonal(K, -g.kappa / (4 * math.pi))
    return K * (g.s * g.w)[None, :]


def solve_density(g: BoundaryGeometry, rhs: np.ndarray) -> np.ndarray:
    """sigma with (-1/2 I + D) sigma = rhs (eq. inteq, Nystrom): rhs = g - V."""
    M = dlp_matrix(g) - 0.5 * np.eye(g.n)
    return np.linalg.solve(M, rhs)


def _panel_height_at(xi_nodes, t, re):
    """Imaginary part of the panel (in its own coordinates) where its real
    part equals re: Newton on the degree-15 Legendre interpolant xi(t)."""
    c = np.linalg.solve(npleg.legvander(t, len(t) - 1), xi_nodes)
    dc = npleg.legder(c)
    tt = float(np.clip(re, -1.0, 1.0))
    for _ in range(60):
        f = npleg.legval(tt, c).real - re
        step = f / npleg.legval(tt, dc).real
        tt -= step
        if abs(step) < 1e-16:
            break
    return npleg.legval(tt, c).imag


def _product_weights(tau, a, b, z, t):
    """Helsing-Ojala weights lam_j with sum_j lam_j sigma_j = int_panel
    sigma(tau) / (tau - z) dtau, sigma the polynomial (degree nq - 1 in the
    panel variable xi = (2 tau - a - b) / (b - a)) through the nodes."""
    n = len(tau)
    xi = (2 * tau - (a + b)) / (b - a)
    zeta = (2 * z - (a + b)) / (b - a)
    p = np.empty(n, dtype=complex)
    p[0] = np.log((1 - zeta) / (-1 - zeta))           # along the chord [-1, 1]
    if abs(zeta.real) < 1.0:
        # the curved panel and the chord enclose a sliver; inside it the two
        # integrals differ by the residue 2 pi i, with the loop's orientation
        h = _panel_height_at(xi, t, zeta.real)
        if h != 0.0 and 0.0 < zeta.imag / h < 1.0:
            p[0] += -2j * math.pi * np.sign(h)
    for k in range(1, n):
        p[k] = zeta * p[k - 1] + (1 - (-1) ** k) / k
    V = np.vander(xi, n, increasing=True)             # V[j, k] = xi_j^k
    return np.linalg.solve(V.T, p)


def dlp_eval(g: BoundaryGeometry, sigma: np.ndarray, targets: np.ndarray) -> np.ndarray:
    """D[sigma] at targets off the boundary: the Gauss-Legendre sum, with each
    panel within NEAR_RADIUS (in its own coordinates) of a target replaced by
    product integration.  In complex form the kernel times ds is
    Re(i dtau / (2 pi (tau - z))), so a panel contributes
    -(1/2pi) Im int sigma dtau / (tau - z)."""
    targets = np.asarray(targets, dtype=np.float64).reshape(-1, 2)
    sigma = np.asarray(sigma, dtype=np.float64)
    out = np.zeros(len(targets))
    sw = g.s * g.w * sigma
    tau = g.y[:, 0] + 1j * g.y[:, 1]
    nq = g.nq
    for k, x in enumerate(targets):
        dx = x[0] - g.y[:, 0]
        dy = x[1] - g.y[:, 1]
        direct = (dx * g.nu[:, 0] + dy * g.nu[:, 1]) / (dx * dx + dy * dy) * sw / (2 * math.pi)
        z = x[0] + 1j * x[1]
        zeta = (2 * z - (g.a + g.b)) / (g.b - g.a)
        near = np.nonzero(np.abs(zeta) < NEAR_RADIUS)[0]
        total = direct.sum()
        for i in near:
            sl = slice(i * nq, (i + 1) * nq)
            lam = _product_weights(tau[sl], g.a[i], g.b[i], z, g.t)
            total += -(lam @ sigma[sl]).imag / (2 * math.pi) - direct[sl].sum()
        out[k] = total
    return out


class ExteriorSolution:
    """u^H = D[sigma] + (1/2pi) int_Gamma sigma ds + sum_k A_k log|x - s_k| in
    the exterior of several closed curves (Section 2, exterior and multiply
    connected problems), the curves counter-clockwise so that nu points out
    of each inclusion, into Omega."""

    def __init__(self, g: BoundaryGeometry, sigma, A, centers):
        self.g, self.sigma, self.A, self.centers = g, sigma, np.asarray(A), np.asarray(centers, dtype=np.float64)

    def __call__(self, targets):
        targets = np.asarray(targets, dtype=np.float64).reshape(-1, 2)
        u = dlp_eval(self.g, self.sigma, targets) + np.sum(self.sigma * self.g.s * self.g.w) / (2 * math.pi)
        for A, c in zip(self.A, self.centers):
            u = u + A * np.log(np.hypot(targets[:, 0] - c[0], targets[:, 1] - c[1]))
        return u


def solve_exterior(g: BoundaryGeometry, curve_of_node, centers, rhs, growth) -> ExteriorSolution:
    """The exterior Dirichlet correction: on the boundary, the limit from
    Omega of the representation equals rhs = g - V,

        (1/2 + D) sigma + (1/2pi) int sigma ds + sum_k A_k log|y - s_k| = rhs,

    with int_{Gamma_k} sigma ds = 0 for every curve but the last and
    sum_k A_k = growth, the coefficient of log|x| that u^H must have at
    infinity: the solution's own growth A minus the particular solution's
    Q = (1/2pi) iint f^e (Section 2, alpha = A - Q).  s_k is a point inside
    curve k; curve_of_node gives the curve of every boundary node."""
    n, m = g.n, len(centers)
    sw = g.s * g.w
    M = np.zeros((n + m, n + m))
    M[:n, :n] = 0.5 * np.eye(n) + dlp_matrix(g) + np.outer(np.ones(n), sw) / (2 * math.pi)
    for k, c in enumerate(centers):
        M[:n, n + k] = np.log(np.hypot(g.y[:, 0] - c[0], g.y[:, 1] - c[1]))
    for k in range(m - 1):
        M[n + k, :n] = sw * (np.asarray(curve_of_node) == k)
    M[n + m - 1, n:] = 1.0
    b = np.concatenate([np.asarray(rhs, dtype=np.float64), np.zeros(m - 1), [float(growth)]])
    x = np.linalg.solve(M, b)
    return ExteriorSolution(g, x[:n], x[n:], centers)


class HoledSolution:
    """u^H = D[sigma] + sum_k A_k log|x - s_k| inside an outer curve with holes
    (Section 2, multiply connected interior problem), every curve
    counter-clockwise: D uses each curve's own outward normal, which points
    into Omega on the holes, so there the density is the paper's with its
    sign changed."""

    def __init__(self, g: BoundaryGeometry, sigma, A, centers):
        self.g, self.sigma, self.A, self.centers = g, sigma, np.asarray(A), np.asarray(centers, dtype=np.float64)

    def __call__(self, targets):
        targets = np.asarray(targets, dtype=np.float64).reshape(-1, 2)
        u = dlp_eval(self.g, self.sigma, targets)
        for A, c in zip(self.A, self.centers):
            u = u + A * np.log(np.hypot(targets[:, 0] - c[0], targets[:, 1] - c[1]))
        return u


def solve_holed(g: BoundaryGeometry, curve_of_node, hole_centers, rhs) -> HoledSolution:
    """The multiply connected interior correction: curve 0 is the outer
    boundary, curves 1..m the holes, s_k a point inside hole k.  On the
    boundary the limit from Omega equals rhs = g - V:

        (-1/2 on curve 0, +1/2 on the holes) sigma + D sigma + sum_k A_k log|y - s_k| = rhs,

    (the interior jump for the outer curve, the exterior jump of each hole's
    own double layer), with int_{Gamma_k} sigma ds = 0 on every hole
    (eq. densconst), which removes the m homogeneous solutions."""
    n, m = g.n, len(hole_centers)
    curve_of_node = np.asarray(curve_of_node)
    sw = g.s * g.w
    M = np.zeros((n + m, n + m))
    M[:n, :n] = dlp_matrix(g) + np.diag(np.where(curve_of_node == 0, -0.5, 0.5))
    for k, c in enumerate(hole_centers):
        M[:n, n + k] = np.log(np.hypot(g.y[:, 0] - c[0], g.y[:, 1] - c[1]))
        M[n + k, :n] = sw * (curve_of_node == k + 1)
    b = np.concatenate([np.asarray(rhs, dtype=np.float64), np.zeros(m)])
    x = np.linalg.solve(M, b)
    return HoledSolution(g, x[:n], x[n:], hole_centers)
