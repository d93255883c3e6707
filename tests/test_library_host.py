"""CPU-side checks of the library: the shared object loads and exports every
function declared in include/vpx.h, and a C99 program links against it; the
host tree (Section 4 rules) equals the oracle's tree; the interaction lists
(built on the host and uploaded) count every (target leaf, source leaf) pair
exactly once across near, list i, list i+ and list i- (Fig. tree_levels); the
stencil, the operators and the boundary-correction host part equal the
oracle's."""
import os
import re
from collections import defaultdict

import numpy as np
import pytest

EPS = np.finfo(float).eps

import workloads as W
from oracle import bie as B
from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def V():
    import __graft_entry__ as g
    g.build_library()
    from paper_2211_14537_gb300 import vpx
    return vpx


def test_library_exports_every_declared_symbol(V):
    with open(os.path.join(ROOT, "include", "vpx.h")) as fh:
        hdr = fh.read()
    names = set(re.findall(r"^(?:int|void|const char \*)\s*\*?\s*(vpx_\w+)\s*\(", hdr, flags=re.M))
    assert len(names) >= 20
    L = V.load_library()
    for n in names:
        assert hasattr(L, n), n
    assert set(V.EXPORTED) == names


def test_c99_program_links_against_the_library(V, tmp_path):
    """The header is plain C (C99, pedantic, warnings as errors) and a C caller
    gets the defaults and the error strings without a GPU."""
    import subprocess
    src = tmp_path / "caller.c"
    src.write_text(
        '#include <stdio.h>\n#include "vpx.h"\n'
        "int main(void) {\n"
        "    vpx_options o;\n"
        "    if (vpx_default_options(&o) != VPX_OK) return 1;\n"
        '    printf("%d %d %d %s\\n", o.K, o.p, o.n_quad_bdry, vpx_error_string(VPX_ERR_DOMAIN));\n'
        "    return vpx_default_options(NULL) == VPX_ERR_ARG ? 0 : 2;\n"
        "}\n")
    lib = os.path.dirname(V.LIB_PATH)
    exe = tmp_path / "caller"
    subprocess.run(["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", str(src), "-I",
                    os.path.join(ROOT, "include"), "-L", lib, "-lvpx", "-Wl,-rpath," + lib, "-o", str(exe)],
                   check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    K, p, nq, msg = r.stdout.split(maxsplit=3)
    o = V.vpx_default_options()
    assert (int(K), int(p), int(nq)) == (o.K, o.p, o.n_quad_bdry) and "root box" in msg


def _plan(V, wl, host_only=True):
    o = V.vpx_default_options(K=wl.opts.K, min_level=wl.opts.min_level, max_level=wl.opts.max_level,
                              refine_tol=wl.opts.refine_tol, f_scale=wl.opts.f_scale)
    return V.vpx_plan_create(o, wl.domain, wl.sources[0], host_only=host_only)


WORKLOADS = {
    "disk_l4": lambda: W.disk_sincos(level=4),
    "disk_l3_k16": lambda: W.disk_sincos(level=3, K=16),
    "starfish_k8": lambda: W.starfish_gaussian(K=8, tol=1e-8, max_level=8),
    "lshape_small": lambda: W.lshape_expsin(K=8, base_level=4, max_level=8, corner_levels=5),
    "star_batch_03": lambda: W.star_batch(4)[3],   # adaptive K = 8 star of the uneven batch (3,844 leaves)
    "exterior_k8": lambda: W.exterior_three_stars(K=8, tol=1e-5, max_level=7),   # three holes, 1,726 leaves
    "doubly_connected_l5": lambda: W.doubly_connected_harmext(5),                  # a hole in a star
    "square_l5": lambda: W.square_pwsmooth(5),                                      # rotated square, graded corners
    "doubly_connected_adaptive": W.doubly_connected_adaptive,                       # the paper's timing run: 3,778 leaves
}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_tree_matches_oracle_exactly(V, name):
    wl = WORKLOADS[name]()
    plan = _plan(V, wl)
    L = plan.leaves()
    tr = O.build_tree(wl.domain, wl.opts, wl.sources[0])
    assert [tuple(x) for x in zip(L["level"], L["ix"], L["iy"])] == tr.leaves
    assert list(L["cls"]) == tr.cls
    assert list(L["owner"]) == tr.owner
    sp = plan.stencil_points()
    so, _ = O.stencil_points(tr, wl.domain)
    assert sp.shape == so.shape and np.max(np.abs(sp - so)) < 1e-15
    ln = plan.leaf_nodes()
    assert np.max(np.abs(ln - O.all_leaf_nodes(tr))) < 1e-15
    bn = plan.boundary_nodes()
    assert np.max(np.abs(bn - O.boundary_nodes(wl.domain))) < 1e-15


def test_plan_rejects_bad_options(V):
    o = V.vpx_default_options(K=7)
    with pytest.raises(V.VpxError) as e:
        V.vpx_plan_create(o, W.WholeBoxDomain(), lambda xy: 0 * xy[:, 0], host_only=True)
    assert e.value.code == -1
    o = V.vpx_default_options(K=8, min_level=2, max_level=2)
    with pytest.raises(V.VpxError) as e:   # disk cut leaves touch the edge of D at level 2
        V.vpx_plan_create(o, W.disk_sincos(level=2).domain, lambda xy: 0 * xy[:, 0], host_only=True)
    assert e.value.code == -5


def test_callback_failure_is_reported(V):
    o = V.vpx_default_options(K=8, min_level=2, max_level=6, refine_tol=1e-8)

    def bad(xy):
        raise ValueError("boom")
    with pytest.raises(V.VpxError) as e:
        V.vpx_plan_create(o, W.WholeBoxDomain(), bad, host_only=True)
    assert e.value.code == -9


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_lists_cover_every_pair_exactly_once(V, name):
    wl = WORKLOADS[name]()
    plan = _plan(V, wl)
    Ls = plan.lists()
    lv = plan.leaves()
    nl = len(lv["level"])
    nz = (lv["cls"] != 2) | (lv["owner"] >= 0)
    blev, bix, biy, bleaf = Ls["box_level"], Ls["box_ix"], Ls["box_iy"], Ls["box_leaf"]
    nb = len(blev)
    key = {(int(blev[b]), int(bix[b]), int(biy[b])): b for b in range(nb)}
    parent = np.full(nb, -1)
    for b in range(nb):
        if blev[b] > 0:
            parent[b] = key[(blev[b] - 1, bix[b] >> 1, biy[b] >> 1)]
    desc = defaultdict(list)          # box -> descendant leaves
    leaf_box = np.zeros(nl, dtype=int)
    for b in range(nb):
        if bleaf[b] >= 0:
            leaf_box[bleaf[b]] = b
            a = b
            while a >= 0:
                desc[a].append(bleaf[b])
                a = parent[a]
    near, vl, xl, wlst = Ls["near"], Ls["vlist"], Ls["xlist"], Ls["wlist"]
    for t in range(nl):
        cnt = np.zeros(nl, dtype=int)
        for s in near[t]:
            if s >= 0:
                cnt[s] += 1
        for s in wlst[t]:
            if s >= 0:
                cnt[desc[s]] += 1
        a = leaf_box[t]
        while a >= 0:
            for s in vl[a]:
                if s >= 0:
                    cnt[desc[s]] += 1
            for s in xl[a]:
                if s >= 0:
                    cnt[s] += 1
            a = parent[a]
        assert np.all(cnt[nz] == 1), (name, t, np.nonzero(cnt[nz] != 1)[0][:10])
        assert np.all(cnt[~nz] <= 1)   # zero leaves only ever appear inside a listed box
    # near configurations are geometrically right: colleague slots are same-level offsets
    for t in range(nl):
        for c in range(9):
            s = near[t, c]
            if s >= 0:
                dx, dy = c % 3 - 1, c // 3 - 1
                assert (lv["level"][s], lv["ix"][s], lv["iy"][s]) == (lv["level"][t], lv["ix"][t] + dx, lv["iy"][t] + dy)
        for c in range(9, 21):
            s = near[t, c]
            if s >= 0:
                assert lv["level"][s] == lv["level"][t] - 1
        for c in range(21, 33):
            s = near[t, c]
            if s >= 0:
                assert lv["level"][s] == lv["level"][t] + 1


def test_batch_refuses_host_only_plans_and_bad_arrays(V):
    """vpx_execute_batch validates every entry before anything is launched:
    a host-only plan is a state error, a plan listed twice an argument error."""
    wls = W.star_batch(2)
    plans = [_plan(V, wl) for wl in wls]
    torch = pytest.importorskip("torch")
    f = [torch.zeros(p.sizes()[2], dtype=torch.float64) for p in plans]
    v = [torch.zeros(p.sizes()[1], dtype=torch.float64) for p in plans]
    with pytest.raises(V.VpxError) as e:
        V.vpx_execute_batch(plans, f, v, None, stream=0)
    assert e.value.code == V.VPX_ERR_STATE
    with pytest.raises(V.VpxError) as e:
        V.vpx_execute_batch([plans[0], plans[0]], f, v, None, stream=0)
    assert e.value.code == V.VPX_ERR_ARG
    L = V.load_library()
    assert L.vpx_execute_batch(0, None, None, None, None, None, None, None, None, None) == V.VPX_ERR_ARG


def test_potential_static_refuses_too_many_columns_before_any_launch(V):
    """vpx_potential_static bounds nrhs by the plan's max_rhs before it looks at
    the device state: the mixed form's slice buffers are plan workspace sized by
    max_rhs, so more columns than that would write past them."""
    torch = pytest.importorskip("torch")
    wl = W.disk_sincos(level=3)
    plan = _plan(V, wl)   # host-only, max_rhs = 1
    nt = plan.sizes()[1]
    fe = torch.zeros((2, nt), dtype=torch.float64)
    v = torch.zeros((2, nt), dtype=torch.float64)
    with pytest.raises(V.VpxError) as e:
        V.vpx_potential_static(plan, fe, v, stream=0)
    assert e.value.code == V.VPX_ERR_ARG
    # within range, the host-only plan is a state error as for vpx_potential
    with pytest.raises(V.VpxError) as e:
        V.vpx_potential_static(plan, fe[:1], v[:1], stream=0)
    assert e.value.code == V.VPX_ERR_STATE


def test_autotune_refuses_host_only_plan(V):
    torch = pytest.importorskip("torch")
    wl = W.disk_sincos(level=3)
    plan = _plan(V, wl)
    f = torch.zeros(plan.sizes()[2], dtype=torch.float64)
    with pytest.raises(V.VpxError) as e:
        V.vpx_autotune(plan, f, stream=0)
    assert e.value.code == V.VPX_ERR_STATE


def test_boundary_targets_follow_section6(V):
    """16 Gauss-Legendre nodes per boundary panel (Section 6), as in the
    oracle and the golden fixture."""
    import os
    n_q = None
    with open(os.path.join(ROOT, "tests", "golden", "discretization_section6.txt")) as fh:
        for line in fh:
            w = line.split("#", 1)[0].split()
            if w and w[0] == "N_q":
                n_q = int(w[1])
    for wl in (W.disk_sincos(level=3), W.starfish_gaussian(K=8, tol=1e-6, max_level=6)):
        plan = _plan(V, wl)
        assert plan.sizes()[3] == n_q * wl.domain.n_panels


def test_star_batch_is_seeded_and_uneven(V):
    """The uneven batch: 32 domains, the same on every call; each draws its own
    refinement tolerance in [1e-8, 1e-3]; the trees (host-only plans) span more
    than a factor of ten in leaf targets."""
    a, b = W.star_batch(32), W.star_batch(32)
    assert len(a) == 32
    xy = np.random.Generator(np.random.PCG64(3)).uniform(-0.3, 0.3, size=(50, 2))
    for wa, wb in zip(a, b):
        assert wa.opts.refine_tol == wb.opts.refine_tol
        assert 1e-8 <= wa.opts.refine_tol <= 1e-3
        assert np.array_equal(wa.sources[0](xy), wb.sources[0](xy))
        assert np.array_equal(wa.domain.inside(xy), wb.domain.inside(xy))
    sizes = [_plan(V, wl).sizes()[1] for wl in a[:8]]
    assert max(sizes) > 10 * min(sizes)


@pytest.mark.slow
@pytest.mark.parametrize("K", [6, 8])
def test_universal_operator_matches_oracle(V, K):
    """The library's universal operator (flat limit + the tabulated eps^2 term
    of the Gaussian operator) against the oracle's, formed independently (its
    own basis; the finite-eps operator directly in multiprecision): the flat
    limit to 1e-13; at the paper's eps = 1e-5 on the unit box to 1e-13; the
    eps^2 term at eps = 1e-3 to 1e-5 of its size (the O(eps^4) remainder)."""
    pytest.importorskip("mpmath")
    from oracle import oracle as O
    A0 = V.vpx_universal_matrix(K)
    assert np.abs(A0 - O.universal_matrix(K)).max() <= 1e-13
    A5 = V.vpx_universal_matrix(K, 1e-5)
    assert np.abs(A5 - O.universal_matrix_finite_eps(K, 0.5e-5)).max() <= 1e-13
    D_lib = V.vpx_universal_matrix(K, 1e-3) - A0
    D_orc = O.universal_matrix_finite_eps(K, 0.5e-3) - O.universal_matrix(K)
    assert np.abs(D_lib - D_orc).max() <= 1e-5 * np.abs(D_orc).max()


def test_rbf_eps_option_is_checked(V):
    with pytest.raises(V.VpxError):
        V.vpx_universal_matrix(10, 1e-5)          # no Gaussian table for K = 10
    with pytest.raises(V.VpxError):
        V.vpx_universal_matrix(8, -1e-5)
    with pytest.raises(V.VpxError):
        V.vpx_universal_matrix(8, 2e-3)
    wl = W.disk_sincos(level=3)
    o = V.vpx_default_options(K=10, min_level=3, max_level=3, rbf_eps=1e-5)
    with pytest.raises(V.VpxError):
        V.vpx_plan_create(o, wl.domain, wl.sources[0], host_only=True)


def test_ray_stencil_matches_oracle(V):
    """Extension along lines (Section 6.4), host part: the points where f is
    needed -- interior leaf nodes and grid points of each cut leaf, then eight
    points per exterior grid point on its line through the origin -- equal the
    oracle's (the library finds the boundary radius by bisection on the inside
    test, the oracle takes it from the analytic r(theta))."""
    from oracle import oracle as O
    f = lambda xy: xy[:, 0] ** 2 + xy[:, 1] ** 2
    dom = W.StarDomain(0.35, [(3, 0.1, 0.3), (5, 0.05, 1.0)])
    wl = W.Workload("star_lines", 9, dom, W.TreeOptions(K=8, min_level=4, max_level=4), [f])
    o = V.vpx_default_options(K=8, min_level=4, max_level=4, ext_mode=1)
    plan = V.vpx_plan_create(o, wl.domain, f, host_only=True)
    lib = plan.stencil_points()
    tree = O.build_tree(dom, wl.opts, f)
    orc, _ = O.stencil_points_lines(tree, dom)
    assert lib.shape == orc.shape and np.abs(lib - orc).max() <= 1e-14


def test_line_extension_mode_takes_no_shape_parameter(V):
    wl = W.disk_sincos(level=3)
    o = V.vpx_default_options(K=8, min_level=3, max_level=3, ext_mode=1, rbf_eps=1e-5)
    with pytest.raises(V.VpxError) as e:
        V.vpx_plan_create(o, wl.domain, wl.sources[0], host_only=True)
    assert e.value.code == V.VPX_ERR_ARG
    o = V.vpx_default_options(K=8, min_level=3, max_level=3, ext_mode=2)
    with pytest.raises(V.VpxError):
        V.vpx_plan_create(o, wl.domain, wl.sources[0], host_only=True)


def test_line_extension_refuses_a_domain_not_star_shaped_about_the_origin(V):
    """Lines through the origin reach Omega's boundary once only in a domain
    star-shaped about the origin; exteriors of inclusions are not, and their
    rays run through the holes."""
    wl = W.exterior_three_stars(K=8, tol=0, min_level=4)     # the origin lies in a hole
    o = V.vpx_default_options(K=8, min_level=4, max_level=4, ext_mode=1)
    with pytest.raises(V.VpxError) as e:
        V.vpx_plan_create(o, wl.domain, wl.sources[0], host_only=True)
    assert e.value.code == V.VPX_ERR_STENCIL and "origin" in str(e.value)
    # two holes on the positive x axis, the origin in Omega: a ray to a point of
    # the far hole meets the boundary first at the near edge of the far hole,
    # and its data points, one leaf side back from there, fall into the small hole
    holes = W.ExteriorDomain([W.StarDomain(0.03, (), n_panels=16, center=(0.1, 0.0)),
                              W.StarDomain(0.08, (), n_panels=16, center=(0.25, 0.0))])
    assert holes.inside(np.zeros((1, 2)))[0]
    with pytest.raises(V.VpxError) as e:
        V.vpx_plan_create(o, holes, W.f_sincos, host_only=True)
    assert e.value.code == V.VPX_ERR_STENCIL and "star-shaped" in str(e.value)
    o = V.vpx_default_options(K=8, min_level=4, max_level=4)     # the universal stencil takes both
    V.vpx_plan_create(o, wl.domain, wl.sources[0], host_only=True)
    V.vpx_plan_create(o, holes, W.f_sincos, host_only=True)


def test_ray_operator_matches_oracle_floater_hormann(V):
    """The library's line-extension operator (coefficients on the host, from the
    Floater-Hormann weights' definition) gives the oracle's exterior grid
    values: sum_q coef[q] f[ray_src + q] against the oracle's barycentric
    interpolant through the same line points, for a non-polynomial f."""
    from oracle import oracle as O
    f = lambda xy: np.sin(3 * xy[:, 0]) * np.cos(2 * xy[:, 1]) + (xy[:, 0] ** 2 + xy[:, 1] ** 2) ** 3
    dom = W.StarDomain(0.35, [(3, 0.1, 0.3), (5, 0.05, 1.0)])
    wl = W.Workload("star_lines", 9, dom, W.TreeOptions(K=8, min_level=4, max_level=4), [f])
    o = V.vpx_default_options(K=8, min_level=4, max_level=4, ext_mode=1)
    plan = V.vpx_plan_create(o, wl.domain, f, host_only=True)
    fs = f(plan.stencil_points())
    rc, rg, src, coef = V.vpx_plan_ray_operator(plan)
    got = np.array([np.dot(coef[k], fs[src[k]:src[k] + 8]) for k in range(len(rc))])
    tree = O.build_tree(dom, wl.opts, f)
    cuts = tree.cut_leaves()
    want = np.empty(len(rc))
    for k in range(len(rc)):
        b = tree.leaves[cuts[rc[k]]]
        _, XSb, _ = O.cut_leaf_stencil(b, 8, tree.t)
        pts, radii, rx = O.ray_nodes(dom, XSb[rg[k]], O.box_side(b[0]))
        order = np.argsort(radii)
        want[k] = O.fh_eval(radii[order], f(pts)[order], O.fh_weights(radii[order], O.FH_DEGREE), rx)
    assert len(rc) > 100
    # rounding of an extrapolation: 64 eps times the coefficients' absolute sum
    # (a Lebesgue-type constant) times the data's size along the line
    lam = np.abs(coef).sum(axis=1)
    fmag = np.array([np.abs(fs[src[k]:src[k] + 8]).max() for k in range(len(rc))])
    assert np.all(np.abs(got - want) <= 64 * EPS * lam * fmag)


@pytest.mark.parametrize("name", ["starfish_k8", "saw_l5", "square_l5"])
def test_bie_host_part_matches_oracle(V, name):
    """Boundary correction, host part (Section 5): normals, s*w and curvature
    equal the oracle's; the plain sum plus the library's product-integration
    corrections reproduces the oracle's D[sigma] at leaf nodes near and far
    from the boundary, for the density of harmonic Dirichlet data."""
    wl = {"starfish_k8": lambda: W.starfish_gaussian(K=8, tol=1e-8, max_level=8), "saw_l5": lambda: W.saw_harmext(5),
          "square_l5": lambda: W.square_pwsmooth(5)}[name]()
    plan = _plan(V, wl)
    with pytest.raises(V.VpxError) as e:
        V.vpx_bie_geometry(plan)
    assert e.value.code == V.VPX_ERR_STATE
    V.vpx_bie_setup(plan)
    nc, oc, _, jp = V.vpx_bie_topology(plan)
    assert nc == 1 and oc == 0 and np.all(jp == -0.5) and V.vpx_bie_log_terms(plan)[2] == len(jp)
    nu, sw, ka = V.vpx_bie_geometry(plan)
    g = B.BoundaryGeometry(wl.domain)
    assert np.abs(nu - g.nu).max() < 1e-15 and np.abs(sw - g.s * g.w).max() < 1e-16
    # the square's flat panels have kappa = 0; both sides then return the rounding
    # of differentiating a constant gamma' on panels down to 2^-10 of a side
    assert np.abs(ka - g.kappa).max() < 1e-12 * np.abs(g.kappa).max() + 1e-9
    off, pan, w = V.vpx_bie_corrections(plan)
    uh = lambda p: np.exp(3 * p[:, 0]) * np.cos(3 * p[:, 1]) + p[:, 0] * p[:, 1]
    sigma = B.solve_density(g, uh(g.y))
    X = plan.leaf_nodes()
    rng = np.random.default_rng(9)
    near = np.nonzero(np.diff(off) > 0)[0]
    sel = np.concatenate([rng.choice(near, 200, replace=False), rng.choice(len(X), 60, replace=False)])
    got = np.empty(len(sel))
    for k, q in enumerate(sel):
        d = X[q] - g.y
        got[k] = np.sum((d * nu).sum(1) / (d * d).sum(1) * sw * sigma) / (2 * np.pi)
        for e in range(off[q], off[q + 1]):
            got[k] += w[e] @ sigma[pan[e] * 16:(pan[e] + 1) * 16]
    want = B.dlp_eval(g, sigma, X[sel])
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()
    ins = wl.domain.inside(X[sel])
    assert np.abs(got[ins] - uh(X[sel][ins])).max() < {"starfish_k8": 1e-11, "saw_l5": 1e-8, "square_l5": 1e-8}[name]


@pytest.mark.parametrize("name", ["exterior", "doubly_connected"])
def test_bie_host_part_on_several_curves(V, name):
    """Closed curves and the side of Omega: the exterior of three inclusions
    (no outer curve, +1/2 on all three) and the domain with a hole (outer
    curve 0 at -1/2, the hole at +1/2); the corrected D[sigma] equals the
    oracle's for the densities that reproduce harmonic data there."""
    if name == "exterior":
        wl = W.exterior_three_stars(K=8, tol=1e-5, max_level=7)
        curves, outer = wl.domain.inclusions, -1
    else:
        wl = W.doubly_connected_harmext(5)
        curves, outer = wl.domain.curves, 0
    plan = _plan(V, wl)
    V.vpx_bie_setup(plan)
    nc, oc, cn, jp = V.vpx_bie_topology(plan)
    want_cn = np.concatenate([np.full(d.n_panels * 16, k) for k, d in enumerate(curves)])
    assert nc == len(curves) and oc == outer and np.array_equal(cn, want_cn)
    assert np.array_equal(jp, np.where(cn == outer, -0.5, 0.5))
    # one log term per curve that Omega surrounds, centred inside that curve
    lc, centre, n_unknowns = V.vpx_bie_log_terms(plan)
    assert list(lc) == [c for c in range(nc) if c != outer] and n_unknowns == len(cn) + len(lc)
    for c, p in zip(lc, centre):
        assert curves[c].inside(p[None, :])[0] and not wl.domain.inside(p[None, :])[0]
    g = B.BoundaryGeometry(wl.domain)
    if name == "exterior":
        cs = [d.center for d in curves]
        uh = lambda p: sum(c * np.log(np.hypot(p[:, 0] - s[0], p[:, 1] - s[1])) for c, s in zip([1.5, -0.7, 2.0], cs))
        sol = B.solve_exterior(g, cn, cs, uh(g.y), 0.8)
    else:
        uh = lambda p: np.exp(3 * p[:, 0]) * np.cos(3 * p[:, 1]) + 0.7 * np.log(np.hypot(p[:, 0], p[:, 1]))
        sol = B.solve_holed(g, cn, [curves[1].center], uh(g.y))
    nu, sw, _ = V.vpx_bie_geometry(plan)
    off, pan, w = V.vpx_bie_corrections(plan)
    X = plan.leaf_nodes()
    rng = np.random.default_rng(10)
    sel = rng.choice(np.nonzero(np.diff(off) > 0)[0], 150, replace=False)
    got = np.empty(len(sel))
    for k, q in enumerate(sel):
        d = X[q] - g.y
        got[k] = np.sum((d * nu).sum(1) / (d * d).sum(1) * sw * sol.sigma) / (2 * np.pi)
        for e in range(off[q], off[q + 1]):
            got[k] += w[e] @ sol.sigma[pan[e] * 16:(pan[e] + 1) * 16]
    want = B.dlp_eval(g, sol.sigma, X[sel])
    assert np.abs(got - want).max() < 1e-13 * max(1.0, np.abs(want).max())


def test_bie_setup_refuses_what_it_cannot_solve(V):
    """A clockwise curve, panels that do not close into curves, no boundary
    at all, and a hole without a log centre are refused with VPX_ERR_STATE."""
    class Clockwise(W.StarDomain):
        def curve(self, i, t):
            xy, d = W.StarDomain.curve(self, self.n_panels - 1 - i, -np.asarray(t))
            return xy, -d
    cw = Clockwise(0.35, (), n_panels=16)
    o = V.vpx_default_options(K=8, min_level=3, max_level=3)
    plan = V.vpx_plan_create(o, cw, W.f_sincos, host_only=True)
    with pytest.raises(V.VpxError) as e:
        V.vpx_bie_setup(plan)
    assert e.value.code == V.VPX_ERR_STATE and "counter-clockwise" in str(e.value)

    class Open(W.StarDomain):            # the last panel stops half way
        def curve(self, i, t):
            if i == self.n_panels - 1:
                t = (np.asarray(t) - 1.0) * 0.5
            return W.StarDomain.curve(self, i, t)
    plan = V.vpx_plan_create(o, Open(0.35, (), n_panels=16), W.f_sincos, host_only=True)
    with pytest.raises(V.VpxError) as e:
        V.vpx_bie_setup(plan)
    assert e.value.code == V.VPX_ERR_STATE and "closed curves" in str(e.value)
    o = V.vpx_default_options(K=8, min_level=2, max_level=2)
    plan = V.vpx_plan_create(o, W.WholeBoxDomain(), W.f_sincos, host_only=True)
    with pytest.raises(V.VpxError) as e:
        V.vpx_bie_setup(plan)
    assert e.value.code == V.VPX_ERR_STATE
    # a C-shaped hole: its centroid lies in the opening, i.e. in Omega, so the
    # hole has no log centre there
    c_hole = W.PolygonDomain([(0.1, 0.1), (-0.1, 0.1), (-0.1, -0.1), (0.1, -0.1), (0.1, -0.06), (-0.06, -0.06),
                              (-0.06, 0.06), (0.1, 0.06)], panels_per_side=2)
    holed = W.HoledDomain(W.StarDomain(0.4, (), n_panels=32), [c_hole])
    o = V.vpx_default_options(K=8, min_level=4, max_level=4)
    plan = V.vpx_plan_create(o, holed, W.f_sincos, host_only=True)
    with pytest.raises(V.VpxError) as e:
        V.vpx_bie_setup(plan)
    assert e.value.code == V.VPX_ERR_STATE and "centroid" in str(e.value)


@pytest.mark.parametrize("name", ["starfish", "doubly_connected", "exterior"])
def test_bie_system_from_the_library_data_reproduces_harmonic_data(V, name):
    """The Nystrom system that vpx_bie_solve inverts, written out as the header
    defines it from the library's own geometry, jumps, log centres and
    corrections (numpy here; the device assembles the same rows): solved for
    the boundary values of a harmonic u, it returns the fluxes through holes
    and inclusions and reproduces u at leaf nodes in Omega, near the boundary
    and far from it."""
    if name == "starfish":
        wl, growth = W.starfish_gaussian(K=8, tol=1e-8, max_level=8), 0.0
        uh = lambda p: np.exp(3 * p[:, 0]) * np.cos(3 * p[:, 1]) + p[:, 0] * p[:, 1]
        flux = []
    elif name == "doubly_connected":
        wl, growth, flux = W.doubly_connected_harmext(5), 0.0, [0.7]
        uh = lambda p: np.exp(3 * p[:, 0]) * np.cos(3 * p[:, 1]) + 0.7 * np.log(np.hypot(p[:, 0] - 0.01, p[:, 1]))
    else:
        wl = W.exterior_three_stars(K=8, tol=1e-5, max_level=7)
        cs, flux = [d.center for d in wl.domain.inclusions], [1.5, -0.7, 2.0]
        growth = sum(flux)
        uh = lambda p: (sum(c * np.log(np.hypot(p[:, 0] - s[0], p[:, 1] - s[1])) for c, s in zip(flux, cs)) +
                        (1 / ((p[:, 0] + 1j * p[:, 1]) - complex(*cs[0]))).real)
    plan = _plan(V, wl)
    V.vpx_bie_setup(plan)
    _, oc, cn, jp = V.vpx_bie_topology(plan)
    lc, centre, nunk = V.vpx_bie_log_terms(plan)
    nu, sw, ka = V.vpx_bie_geometry(plan)
    off, pan, w = V.vpx_bie_corrections(plan)
    y = plan.boundary_nodes()
    N, nl, ext = len(y), len(lc), oc < 0
    d = y[:, None, :] - y[None, :, :]
    r2 = (d * d).sum(2)
    np.fill_diagonal(r2, 1.0)
    M = np.zeros((nunk, nunk))
    M[:N, :N] = (d * nu[None, :, :]).sum(2) / r2 / (2 * np.pi) * sw[None, :]
    np.fill_diagonal(M[:N, :N], -ka / (4 * np.pi) * sw)
    M[:N, :N] += np.diag(jp) + (np.outer(np.ones(N), sw) / (2 * np.pi) if ext else 0.0)
    for k in range(nl):
        M[:N, N + k] = np.log(np.hypot(y[:, 0] - centre[k, 0], y[:, 1] - centre[k, 1]))
        if ext and k == nl - 1:
            M[N + k, N:] = 1.0
        else:
            M[N + k, :N] = sw * (cn == lc[k])
    rhs = np.concatenate([uh(y), np.zeros(nl)])
    if ext:
        rhs[-1] = growth
    sol = np.linalg.solve(M, rhs)
    sig, A = sol[:N], sol[N:]
    assert np.allclose(A, flux, atol=1e-10, rtol=0)
    X = plan.leaf_nodes()
    ins = wl.domain.inside(X)
    rng = np.random.default_rng(11)
    sel = np.concatenate([rng.choice(np.nonzero((np.diff(off) > 0) & ins)[0], 120, replace=False),
                          rng.choice(np.nonzero(ins)[0], 40, replace=False)])
    u = np.empty(len(sel))
    for k, q in enumerate(sel):
        dq = X[q] - y
        u[k] = np.sum((dq * nu).sum(1) / (dq * dq).sum(1) * sw * sig) / (2 * np.pi)
        for e in range(off[q], off[q + 1]):
            u[k] += w[e] @ sig[pan[e] * 16:(pan[e] + 1) * 16]
        u[k] += sum(A[j] * np.log(np.hypot(*(X[q] - centre[j]))) for j in range(nl))
        if ext:
            u[k] += np.sum(sw * sig) / (2 * np.pi)
    assert np.abs(u - uh(X[sel])).max() < 1e-11


def test_bie_device_calls_refuse_host_only_plans_and_missing_setup(V):
    """vpx_bie_solve and vpx_bie_eval check their plan before touching any
    pointer: a host-only plan, or a plan without vpx_bie_setup, is refused."""
    torch = pytest.importorskip("torch")
    wl = W.disk_sincos(level=3)
    plan = _plan(V, wl)
    x = torch.zeros(8, dtype=torch.float64)
    calls = (lambda: V.vpx_bie_solve(plan, x, x, x, stream=0), lambda: V.vpx_bie_eval(plan, x, x, x, stream=0))
    for call in calls:
        with pytest.raises(V.VpxError) as e:
            call()
        assert e.value.code == V.VPX_ERR_STATE
    V.vpx_bie_setup(plan)
    for call in calls:
        with pytest.raises(V.VpxError) as e:
            call()
        assert e.value.code == V.VPX_ERR_STATE and "host-only" in str(e.value)
    assert V.load_library().vpx_bie_solve(plan.handle, None, None, 0.0, None, None) == V.VPX_ERR_ARG


def test_dipole_multipoles_reproduce_the_double_layer_far_away(V):
    """The density enters the box FMM through each boundary node's multipole
    about its leaf: summed over a leaf's nodes and evaluated 2 to 5 leaf sides
    away, (1/2pi) Re sum_k at_k (L / (z - c))^k equals the direct sum of the
    double-layer kernel over those nodes (p = 40: to rounding); so does the
    local expansion of the same nodes about a box three sides away (list i+)."""
    wl = W.starfish_gaussian(K=8, tol=1e-8, max_level=8)
    o = V.vpx_default_options(K=8, min_level=wl.opts.min_level, max_level=wl.opts.max_level,
                              refine_tol=wl.opts.refine_tol, f_scale=wl.opts.f_scale, p=40)
    plan = V.vpx_plan_create(o, wl.domain, wl.sources[0], host_only=True)
    V.vpx_bie_setup(plan)
    M = V.vpx_bie_dipole_multipoles(plan)
    assert M.shape[1] == 41 and np.all(M[:, 0] == 0)
    nu, sw, _ = V.vpx_bie_geometry(plan)
    y = plan.boundary_nodes()
    tree = O.build_tree(wl.domain, wl.opts, wl.sources[0])
    leaf_of = np.array([O.locate_leaf(tree, p) for p in y])
    sigma = np.cos(3 * np.arange(len(y)) * 2 * np.pi / len(y)) + 0.3
    rng = np.random.default_rng(12)
    for li in rng.choice(np.unique(leaf_of), 6, replace=False):
        nodes = np.nonzero(leaf_of == li)[0]
        lev, ix, iy = tree.leaves[li]
        L = 2.0 ** -lev
        c = complex(-0.5 + (ix + 0.5) * L, -0.5 + (iy + 0.5) * L)
        a = M[nodes].T @ sigma[nodes]
        for dist in (2.0, 3.5, 5.0):
            ang = rng.uniform(0, 2 * np.pi)
            z = c + dist * L * np.exp(1j * ang)
            k = np.arange(41)
            phi = np.sum(a[1:] * (L / (z - c)) ** k[1:])
            d = np.array([z.real, z.imag]) - y[nodes]
            direct = np.sum((d * nu[nodes]).sum(1) / (d * d).sum(1) * sw[nodes] * sigma[nodes]) / (2 * np.pi)
            assert abs(phi.real / (2 * np.pi) - direct) <= 1e-13 * np.sum(np.abs(sw[nodes] * sigma[nodes])) / L
        # the same nodes as a local expansion about a box of side L two to four
        # sides away (list i+): bt_l = i gamma' w L^l / (tau - c)^(l+1), with
        # gamma' w = s w (-nu_y + i nu_x) on a counter-clockwise curve
        gw = sw[nodes] * (-nu[nodes, 1] + 1j * nu[nodes, 0])
        tau = y[nodes, 0] + 1j * y[nodes, 1]
        cT = c + 3.0 * L * np.exp(1j * rng.uniform(0, 2 * np.pi))
        b = np.array([np.sum(1j * gw * sigma[nodes] * L ** l / (tau - cT) ** (l + 1)) for l in range(41)])
        for _ in range(3):
            z = cT + 0.5 * L * rng.uniform(-1, 1) + 0.5j * L * rng.uniform(-1, 1)
            psi = np.sum(b * ((z - cT) / L) ** np.arange(41))
            d = np.array([z.real, z.imag]) - y[nodes]
            direct = np.sum((d * nu[nodes]).sum(1) / (d * d).sum(1) * sw[nodes] * sigma[nodes]) / (2 * np.pi)
            assert abs(psi.real / (2 * np.pi) - direct) <= 1e-12 * np.sum(np.abs(sw[nodes] * sigma[nodes])) / L
