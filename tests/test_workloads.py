"""Checks of the seeded inputs: the geometry the tests and the benchmark are
built on (inside tests, orientation, the exterior test's reading of its third
radius) and the sources against their stated Laplacians."""
import math

import numpy as np
import pytest

import workloads as W


def _winding(poly, p):
    v = poly - p
    a = np.arctan2(v[:, 1], v[:, 0])
    d = np.diff(np.concatenate([a, a[:1]]))
    d = (d + np.pi) % (2 * np.pi) - np.pi
    return int(round(d.sum() / (2 * np.pi)))


def test_saw_inside_test_agrees_with_the_winding_number():
    """The saw domain is not star-shaped; its ray-crossing inside test must
    agree with the winding number of a dense polygon of the curve, and decide
    points 1e-12 off the curve by the side they lie on."""
    d = W.SawDomain(n_panels=64)
    th = np.linspace(0.0, 2 * np.pi, 100001)[:-1]
    poly = np.stack([d.rad(th) * np.cos(d.phi(th)), d.rad(th) * np.sin(d.phi(th))], axis=1)
    rng = np.random.default_rng(1)
    p = rng.uniform(-0.5, 0.5, (1500, 2))
    ins = d.inside(p)
    assert 0.2 < ins.mean() < 0.6
    assert all((_winding(poly, q) != 0) == bool(s) for q, s in zip(p, ins))
    for i in range(0, 64, 7):
        xy, dxy = d.curve(i, np.array([-0.4, 0.3]))
        nu = np.stack([dxy[:, 1], -dxy[:, 0]], axis=1) / np.hypot(dxy[:, 0], dxy[:, 1])[:, None]
        assert d.inside(xy - 1e-12 * nu).all() and not d.inside(xy + 1e-12 * nu).any()


@pytest.mark.parametrize("make", [lambda: W.StarDomain(0.35, [(5, 0.3, 0.0)]), lambda: W.SawDomain(n_panels=64),
                                  W.doubly_connected_domain, W.exterior_domain, W.square_domain])
def test_curves_are_closed_and_counter_clockwise(make):
    """Every curve of every domain: panel ends meet, and the signed area by
    the 16-point rule is positive."""
    dom = make()
    t, w = np.polynomial.legendre.leggauss(16)
    curves = getattr(dom, "curves", None) or getattr(dom, "inclusions", None) or [dom]
    start = 0
    for c in curves:
        n = c.n_panels
        area = 0.0
        for i in range(n):
            xy, d = dom.curve(start + i, t)
            area += 0.5 * np.sum(w * (xy[:, 0] * d[:, 1] - xy[:, 1] * d[:, 0]))
            end = dom.curve(start + i, np.array([1.0]))[0][0]
            nxt = dom.curve(start + (i + 1) % n, np.array([-1.0]))[0][0]
            assert np.hypot(*(end - nxt)) < 1e-12
        assert area > 0
        start += n


def test_exterior_inclusions_are_disjoint_and_hold_the_gaussian_centres():
    """The reading of the exterior test's third radius (0.12, printed 0.2):
    the three inclusions are disjoint, at least 0.03 apart, and each Gaussian
    centre y_j lies inside an inclusion within 0.005 of its boundary, as the
    text says; with the printed 0.2 the first and third inclusions overlap."""
    dom = W.exterior_domain()
    t = np.linspace(0.0, 2 * np.pi, 4001)[:-1]
    pts = [np.stack([d.center[0] + d.r(t) * np.cos(t), d.center[1] + d.r(t) * np.sin(t)], axis=1)
           for d in dom.inclusions]
    for a in range(3):
        for b in range(a + 1, 3):
            assert not dom.inclusions[b].inside(pts[a]).any()
            assert np.min(np.hypot(*(pts[a][:, None, :] - pts[b][None, ::4, :]).transpose(2, 0, 1))) > 0.03
    for y, _ in W.EXTERIOR_GAUSSIANS:
        y = np.array([y])
        holders = [k for k, d in enumerate(dom.inclusions) if d.inside(y)[0]]
        assert len(holders) == 1
        assert np.min(np.hypot(*(pts[holders[0]] - y).T)) < 0.005
    printed = W.StarDomain(0.2, [(3, 0.2, 0.0)], center=(0.2, 0.15))
    assert printed.inside(pts[0]).any()


@pytest.mark.parametrize("u,f,pts", [
    (W.u_harmext, W.f_harmext, [[0.05, 0.02], [-0.1, 0.2], [0.01, -0.03]]),
    (W.u_exterior, W.f_exterior, [[0.1, 0.08], [0.1, -0.24], [0.3, 0.3]]),
    (W.u_square, W.f_square, [[-0.33, -0.12], [0.0, 0.0], [0.42, 0.1]]),
])
def test_sources_are_the_laplacians_of_the_solutions(u, f, pts):
    """Second differences of u converge to f at the rate h^2."""
    p = np.array(pts)
    errs = []
    for h in (2e-3, 1e-3):
        lap = (u(p + [h, 0]) + u(p - [h, 0]) + u(p + [0, h]) + u(p - [0, h]) - 4 * u(p)) / h ** 2
        errs.append(np.max(np.abs(lap - f(p))) / max(1.0, np.max(np.abs(f(p)))))
    assert errs[1] < 1e-3 and (errs[1] < 1e-9 or 3.0 < errs[0] / errs[1] < 5.0)
