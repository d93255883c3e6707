"""Pins of the boundary-correction oracle (Section 5): each checks the oracle
against a fact that does not come from it -- eigenvalues of the circle's
Nystrom matrix, Gauss's law for the double layer, curvature in closed form,
recovery of harmonic functions (inside one curve, inside a curve with a hole,
and outside three curves, with their fluxes), and the paper's printed errors
for its saw domain and doubly connected (Section 6.1), exterior (Section 6.2),
square (Section 6.3) and extension-along-lines (Section 6.4) tests -- and the planted mistakes at the end must each
fail one of them."""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import bie as B
from oracle import oracle as O


def _printed(test):
    """{level: (linf, l2)} of one test from tests/golden/printed_errors_section6.txt."""
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "printed_errors_section6.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                name, lev, norm, val = line.split()
                if name == test:
                    out.setdefault(int(lev), {})[norm] = float(val)
    return {lev: (v["linf"], v["l2"]) for lev, v in out.items()}


def _near_points(dom, n, seed, dists=(1e-9, 1e-6, 1e-3, 3e-2)):
    """Points at the given distances on both sides of the boundary."""
    rng = np.random.default_rng(seed)
    out = []
    for i in rng.choice(dom.n_panels, n):
        xy, d = dom.curve(int(i), rng.uniform(-1.0, 1.0, 2))
        nrm = np.stack([d[:, 1], -d[:, 0]], axis=1) / np.hypot(d[:, 0], d[:, 1])[:, None]
        for h in dists:
            out += [xy - h * nrm, xy + h * nrm]
    return np.concatenate(out)


def test_circle_nystrom_eigenvalues():
    """On a circle of radius R the kernel is the constant -1/(4 pi R), so
    (-1/2 + D) has the eigenvalue -1 on constants and -1/2 on everything else."""
    g = B.BoundaryGeometry(W.StarDomain(0.35, (), n_panels=16))
    ev = np.sort(np.linalg.eigvals(B.dlp_matrix(g) - 0.5 * np.eye(g.n)).real)
    assert abs(ev[0] + 1.0) < 1e-13
    assert np.max(np.abs(ev[1:] + 0.5)) < 1e-13


def test_curvature_matches_the_polar_formula():
    """kappa = (r^2 + 2 r'^2 - r r'') / (r^2 + r'^2)^(3/2) for r(theta)."""
    d = W.StarDomain(0.35, [(5, 0.3, 0.0)])
    g = B.BoundaryGeometry(d)
    th = np.arctan2(g.y[:, 1], g.y[:, 0])
    r = 0.35 * (1 + 0.3 * np.cos(5 * th))
    r1 = -0.35 * 1.5 * np.sin(5 * th)
    r2 = -0.35 * 7.5 * np.cos(5 * th)
    want = (r * r + 2 * r1 * r1 - r * r2) / (r * r + r1 * r1) ** 1.5
    assert np.max(np.abs(g.kappa - want)) < 1e-9 * np.max(np.abs(want))


@pytest.mark.parametrize("which", ["starfish", "saw"])
def test_gauss_law_up_to_the_boundary(which):
    """D[1] = -1 inside Omega and 0 outside (Gauss), at distances down to 1e-9
    from the boundary, where the plain Gauss-Legendre sum is off by O(1)."""
    dom = W.StarDomain(0.35, [(5, 0.3, 0.0)]) if which == "starfish" else W.SawDomain(n_panels=256)
    g = B.BoundaryGeometry(dom)
    p = _near_points(dom, 24, 3)
    ins = dom.inside(p)
    assert ins.any() and (~ins).any()
    d1 = B.dlp_eval(g, np.ones(g.n), p)
    assert np.max(np.abs(d1[ins] + 1.0)) < 1e-11
    assert np.max(np.abs(d1[~ins])) < 1e-11
    # without product integration the near points are wrong: the pin is not vacuous
    plain = [np.sum(((x - g.y) * g.nu).sum(1) / ((x - g.y) ** 2).sum(1) * g.s * g.w) / (2 * math.pi)
             for x in p[ins][:8]]
    assert np.max(np.abs(np.array(plain) + 1.0)) > 1e-2


@pytest.mark.parametrize("which", ["starfish", "saw"])
def test_harmonic_dirichlet_data_are_reproduced(which):
    """f = 0: u = D[sigma] with (-1/2 + D) sigma = g is the harmonic function
    with boundary values g, here u = e^{3x} cos 3y + x y, at interior points
    far from and close to the boundary."""
    dom = W.StarDomain(0.35, [(5, 0.3, 0.0)]) if which == "starfish" else W.SawDomain(n_panels=256)
    g = B.BoundaryGeometry(dom)
    uh = lambda p: np.exp(3 * p[:, 0]) * np.cos(3 * p[:, 1]) + p[:, 0] * p[:, 1]
    sigma = B.solve_density(g, uh(g.y))
    p = _near_points(dom, 16, 4)
    p = np.concatenate([p[dom.inside(p)], [[0.0, 0.0], [0.1, -0.05]]])
    err = np.max(np.abs(B.dlp_eval(g, sigma, p) - uh(p)))
    assert err < (1e-12 if which == "starfish" else 1e-8)


def _saw_errors(level):
    wl = W.saw_harmext(level)
    tree = O.build_tree(wl.domain, wl.opts, wl.sources[0])
    pts, meta = O.stencil_points(tree, wl.domain)
    vals, _ = O.leaf_values(tree, wl.domain, wl.sources[0](pts)[:, None], meta)
    g = B.BoundaryGeometry(wl.domain)
    sigma = B.solve_density(g, W.u_harmext(g.y) - O.volume_potential(tree, vals, g.y)[:, 0])
    grid = W.grid_100(wl.domain)
    u = O.volume_potential(tree, vals, grid)[:, 0] + B.dlp_eval(g, sigma, grid)
    e, ue = u - W.u_harmext(grid), W.u_harmext(grid)
    return np.max(np.abs(e)) / np.max(np.abs(ue)), np.linalg.norm(e) / np.linalg.norm(ue)


@pytest.fixture(scope="module")
def saw_errors():
    return {lev: _saw_errors(lev) for lev in (4, 5)}


def test_saw_domain_poisson_meets_the_papers_printed_errors(saw_errors):
    """Section 6.1, second test, uniform trees: the paper prints relative
    errors (l_inf, l_2) of (1.57e-2, 7.0e-4) at N = 128 points per dimension
    (level 4) and (5.71e-5, 1.57e-6) at N = 256 (level 5) on the grid points
    in Omega.  The full solve (extension, volume potential, boundary
    correction) must be at least that accurate.  (Measured: 1.1e-4, 3.9e-6
    and 1.9e-7, 4.4e-9; the paper does not state its box D, which sets what a
    level means.)"""
    printed = _printed("saw")
    for lev, (linf, l2) in saw_errors.items():
        assert linf <= printed[lev][0] and l2 <= printed[lev][1], (lev, linf, l2)


def test_saw_domain_poisson_converges_at_high_order(saw_errors):
    """Eighth order would divide the error by 256 per level; require 100."""
    assert saw_errors[4][0] / saw_errors[5][0] > 100
    assert saw_errors[4][1] / saw_errors[5][1] > 100


def _exterior_setup():
    dom = W.exterior_domain()
    g = B.BoundaryGeometry(dom)
    curve = np.concatenate([np.full(d.n_panels * B.NQ, k) for k, d in enumerate(dom.inclusions)])
    return dom, g, curve, [d.center for d in dom.inclusions]


def test_exterior_harmonic_data_are_reproduced():
    """Exterior of the three inclusions of Section 6.2: for boundary data of
    u = sum_k c_k log|x - s_k| + Re 1/(z - s_1) + Re 0.01/(z - s_3)^2 (harmonic
    in Omega, growth sum_k c_k), the representation recovers the fluxes
    A_k = c_k (double layers carry none) and u itself, near the curves and
    far away."""
    dom, g, curve, centers = _exterior_setup()
    c = [1.5, -0.7, 2.0]
    s1, s3 = complex(*centers[0]), complex(*centers[2])

    def uh(p):
        z = p[:, 0] + 1j * p[:, 1]
        out = sum(ck * np.log(np.abs(z - complex(*s))) for ck, s in zip(c, centers))
        return out + (1 / (z - s1)).real + (0.01 / (z - s3) ** 2).real
    sol = B.solve_exterior(g, curve, centers, uh(g.y), sum(c))
    assert np.max(np.abs(sol.A - c)) < 1e-11
    p = _near_points(dom.inclusions[1], 12, 5)
    p = np.concatenate([p[dom.inside(p)], [[0.45, 0.45], [3.0, 1.0], [-20.0, 7.0], [100.0, -50.0]]])
    assert np.max(np.abs(sol(p) - uh(p))) < 1e-11


def _exterior_errors(level):
    wl = W.exterior_three_stars(K=8, tol=0, min_level=level)
    tree = O.build_tree(wl.domain, wl.opts, wl.sources[0])
    pts, meta = O.stencil_points(tree, wl.domain)
    vals, _ = O.leaf_values(tree, wl.domain, wl.sources[0](pts)[:, None], meta)
    _, g, curve, centers = _exterior_setup()
    Q = O.net_charge(tree, vals)[0] / (2 * math.pi)
    sol = B.solve_exterior(g, curve, centers, W.u_exterior(g.y) - O.volume_potential(tree, vals, g.y)[:, 0],
                           W.EXTERIOR_LOG_COEF - Q)
    grid = W.grid_100(wl.domain)
    e, ue = O.volume_potential(tree, vals, grid)[:, 0] + sol(grid) - W.u_exterior(grid), W.u_exterior(grid)
    return np.max(np.abs(e)) / np.max(np.abs(ue)), np.linalg.norm(e) / np.linalg.norm(ue)


def test_exterior_poisson_meets_the_papers_printed_errors():
    """Section 6.2 on uniform trees: extension into the holes, volume
    potential, net charge Q = (1/2pi) iint f^e and the exterior correction with
    sum_k A_k = -10 - Q (the exact solution grows like -10 log|x|).  The paper
    prints relative errors (l_inf, l_2) of (6.76e-2, 3.81e-3) at N = 128 points
    per dimension (level 4) and (2.59e-4, 5.90e-5) at N = 256 (level 5) on the
    grid points in Omega; the oracle must be at least that accurate (measured
    2.6e-4, 1.8e-5 and 4.4e-5, 2.8e-6)."""
    printed = _printed("exterior")
    for lev in (4, 5):
        linf, l2 = _exterior_errors(lev)
        assert linf <= printed[lev][0] and l2 <= printed[lev][1], (lev, linf, l2)


def _holed_setup():
    dom = W.doubly_connected_domain()
    g = B.BoundaryGeometry(dom)
    curve = np.concatenate([np.full(d.n_panels * B.NQ, k) for k, d in enumerate(dom.curves)])
    return dom, g, curve, [h.center for h in dom.holes]


def test_holed_harmonic_data_are_reproduced():
    """Inside the doubly connected domain of Section 6.1: boundary data of
    u = e^{3x} cos 3y + 0.7 log|x - a| (a inside the hole, harmonic in Omega,
    flux 0.7 through the hole) give A_1 = 0.7 and u, near both curves."""
    dom, g, curve, centers = _holed_setup()
    uh = lambda p: np.exp(3 * p[:, 0]) * np.cos(3 * p[:, 1]) + 0.7 * np.log(np.hypot(p[:, 0] - 0.01, p[:, 1] + 0.005))
    sol = B.solve_holed(g, curve, centers, uh(g.y))
    assert abs(sol.A[0] - 0.7) < 1e-12
    p = np.concatenate([_near_points(dom.outer, 8, 6), _near_points(dom.holes[0], 8, 7)])
    p = np.concatenate([p[dom.inside(p)], [[0.15, 0.0], [-0.1, 0.12]]])
    assert np.max(np.abs(sol(p) - uh(p))) < 1e-12


@pytest.fixture(scope="module")
def holed_errors():
    out = {}
    dom, g, curve, centers = _holed_setup()
    for lev in (4, 5):
        wl = W.doubly_connected_harmext(lev)
        tree = O.build_tree(wl.domain, wl.opts, wl.sources[0])
        pts, meta = O.stencil_points(tree, wl.domain)
        vals, _ = O.leaf_values(tree, wl.domain, wl.sources[0](pts)[:, None], meta)
        sol = B.solve_holed(g, curve, centers, W.u_harmext(g.y) - O.volume_potential(tree, vals, g.y)[:, 0])
        grid = W.grid_100(wl.domain)
        e, ue = O.volume_potential(tree, vals, grid)[:, 0] + sol(grid) - W.u_harmext(grid), W.u_harmext(grid)
        out[lev] = (np.max(np.abs(e)) / np.max(np.abs(ue)), np.linalg.norm(e) / np.linalg.norm(ue))
    return out


def test_doubly_connected_poisson_meets_the_papers_printed_errors(holed_errors):
    """Section 6.1, first test, uniform trees: the paper prints relative
    errors (l_inf, l_2) of (1.32e-4, 6.78e-6) at N = 128 (level 4) and
    (9.88e-7, 5.18e-8) at N = 256 (level 5); measured 1.8e-5, 1.3e-6 and
    1.8e-8, 1.3e-9."""
    printed = _printed("doubly")
    for lev, (linf, l2) in holed_errors.items():
        assert linf <= printed[lev][0] and l2 <= printed[lev][1], (lev, linf, l2)
    assert holed_errors[4][0] / holed_errors[5][0] > 100


def test_doubly_connected_with_the_analytic_extension(holed_errors):
    """Section 6.1's "analytic extension": f^e = the exact Laplacian on the
    same extended leaves (regular, cut and extension-list leaves), so the error
    is the volume potential's and the boundary correction's alone.  The paper
    prints relative (l_inf, l_2) = (2.58e-9, 8.41e-10) at N = 256 (level 5);
    measured 1.3e-11, 4.4e-12 -- and the numerical extension costs about three
    digits at this level (1.8e-8 l_inf, the holed_errors fixture)."""
    dom, g, curve, centers = _holed_setup()
    wl = W.doubly_connected_harmext(5)
    tree = O.build_tree(dom, wl.opts, wl.sources[0])
    nodes = O.all_leaf_nodes(tree)
    keep = np.array([(c != O.EXTERIOR) or (o >= 0) for c, o in zip(tree.cls, tree.owner)])
    vals = np.where(keep[:, None], W.f_harmext(nodes).reshape(tree.n_leaves, -1), 0.0)[:, None, :]
    sol = B.solve_holed(g, curve, centers, W.u_harmext(g.y) - O.volume_potential(tree, vals, g.y)[:, 0])
    grid = W.grid_100(dom)
    e, ue = O.volume_potential(tree, vals, grid)[:, 0] + sol(grid) - W.u_harmext(grid), W.u_harmext(grid)
    linf, l2 = np.max(np.abs(e)) / np.max(np.abs(ue)), np.linalg.norm(e) / np.linalg.norm(ue)
    printed = _printed("doubly_analytic")[5]
    assert linf <= printed[0] and l2 <= printed[1], (linf, l2)
    assert linf < holed_errors[5][0]


def test_square_poisson_meets_the_papers_printed_errors():
    """Section 6.3, the rotated square with corners, uniform trees: the paper
    prints relative errors (l_inf, l_2) of (6.93e-6, 3.47e-7) at N = 128
    (level 4) and (3.06e-8, 1.03e-9) at N = 256 (level 5), with RCIP at the
    corners; here the panels are graded dyadically toward each corner instead
    (measured 7.3e-7, 4.1e-8 and 9.9e-9, 2.8e-10).  The first pin checks that
    f is the Laplacian of the solution as read (second differences, h^2
    convergence)."""
    p = W.SQUARE_POINTS + np.array([[0.02, 0.01], [-0.015, -0.02], [0.01, 0.03], [0.0, 0.025]])
    rel = []
    for h in (1e-3, 5e-4):
        lap = (W.u_square(p + [h, 0]) + W.u_square(p - [h, 0]) + W.u_square(p + [0, h]) +
               W.u_square(p - [0, h]) - 4 * W.u_square(p)) / h ** 2
        rel.append(np.max(np.abs(lap - W.f_square(p)) / W.f_square(p)))
    assert rel[0] < 2e-4 and 3.5 < rel[0] / rel[1] < 4.5
    printed = _printed("square")
    g = None
    for lev in (4, 5):
        wl = W.square_pwsmooth(lev)
        g = g or B.BoundaryGeometry(wl.domain)
        tree = O.build_tree(wl.domain, wl.opts, wl.sources[0])
        pts, meta = O.stencil_points(tree, wl.domain)
        vals, _ = O.leaf_values(tree, wl.domain, wl.sources[0](pts)[:, None], meta)
        sigma = B.solve_density(g, W.u_square(g.y) - O.volume_potential(tree, vals, g.y)[:, 0])
        grid = W.grid_100(wl.domain)
        u = O.volume_potential(tree, vals, grid)[:, 0] + B.dlp_eval(g, sigma, grid)
        e, ue = u - W.u_square(grid), W.u_square(grid)
        linf, l2 = np.max(np.abs(e)) / np.max(np.abs(ue)), np.linalg.norm(e) / np.linalg.norm(ue)
        assert linf <= printed[lev][0] and l2 <= printed[lev][1], (lev, linf, l2)


@pytest.mark.parametrize("mode", ["stencil", "lines"])
def test_both_extensions_meet_the_papers_printed_errors_on_a_star(mode):
    """Section 6.4 compares the universal-stencil extension with the extension
    along lines through the origin on a star-shaped domain, u from eq.
    harmext; the paper prints relative l_inf (l_2) errors at N = 256 of
    6.25e-7 (2.90e-8) for the stencil and 2.07e-8 (3.20e-9) along lines.  Its
    star is not stated; the starfish of the adaptive workload stands in for
    it, at uniform level 5 (measured 1.2e-9 (5.1e-11) and 1.2e-8 (8.1e-10))."""
    printed = _printed("star_rbf" if mode == "stencil" else "star_lines")[5]
    dom = W.StarDomain(0.35, [(5, 0.3, 0.0)])
    tree = O.build_tree(dom, W.TreeOptions(K=8, min_level=5, max_level=5), W.f_harmext)
    if mode == "lines":
        pts, meta = O.stencil_points_lines(tree, dom)
        vals = O.leaf_values_lines(tree, dom, W.f_harmext(pts)[:, None], meta)
    else:
        pts, meta = O.stencil_points(tree, dom)
        vals, _ = O.leaf_values(tree, dom, W.f_harmext(pts)[:, None], meta)
    g = B.BoundaryGeometry(dom)
    sigma = B.solve_density(g, W.u_harmext(g.y) - O.volume_potential(tree, vals, g.y)[:, 0])
    grid = W.grid_100(dom)
    e = O.volume_potential(tree, vals, grid)[:, 0] + B.dlp_eval(g, sigma, grid) - W.u_harmext(grid)
    ue = W.u_harmext(grid)
    linf, l2 = np.max(np.abs(e)) / np.max(np.abs(ue)), np.linalg.norm(e) / np.linalg.norm(ue)
    assert linf <= printed[0] and l2 <= printed[1], (linf, l2)


# ---------------------------------------------------------------- planted mistakes

def test_wrong_jump_sign_is_caught(monkeypatch):
    monkeypatch.setattr(B, "solve_density",
                        lambda g, rhs: np.linalg.solve(B.dlp_matrix(g) + 0.5 * np.eye(g.n), rhs))
    with pytest.raises(AssertionError):
        test_harmonic_dirichlet_data_are_reproduced("starfish")


def test_dropped_curvature_diagonal_is_caught(monkeypatch):
    real = B.dlp_matrix

    def no_diag(g):
        M = real(g)
        np.fill_diagonal(M, 0.0)
        return M
    monkeypatch.setattr(B, "dlp_matrix", no_diag)
    with pytest.raises(AssertionError):
        test_circle_nystrom_eigenvalues()
    with pytest.raises(AssertionError):
        test_harmonic_dirichlet_data_are_reproduced("starfish")


def test_missing_residue_in_product_integration_is_caught(monkeypatch):
    real = B._panel_height_at
    monkeypatch.setattr(B, "_panel_height_at", lambda xi, t, re: 0.0 * real(xi, t, re))
    with pytest.raises(AssertionError):
        test_gauss_law_up_to_the_boundary("starfish")


def test_exterior_jump_of_the_wrong_side_is_caught(monkeypatch):
    real = B.dlp_matrix
    monkeypatch.setattr(B, "dlp_matrix", lambda g: real(g) - np.eye(g.n))     # planted: -1/2 + D outside
    with pytest.raises(AssertionError):
        test_exterior_harmonic_data_are_reproduced()


def test_holes_with_the_interior_jump_are_caught(monkeypatch):
    real = B.dlp_matrix
    monkeypatch.setattr(B, "dlp_matrix", lambda g: real(g) - np.diag(np.where(np.arange(g.n) >= 160 * B.NQ, 1.0, 0.0)))
    with pytest.raises(AssertionError):        # planted: -1/2 on the hole's curve too
        test_holed_harmonic_data_are_reproduced()
