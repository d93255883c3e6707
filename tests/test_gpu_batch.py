"""Uneven batch of trees in one captured graph (vpx_execute_batch): 32 random
star domains, each with its own Gaussian mixture and its own adaptive tree
(refinement tolerance drawn from [1e-8, 1e-3]: 1.8e4 to 3.8e5 leaf targets
per tree), in the mixed form.

The batch must give every tree what a single vpx_execute gives (the same
kernels on the same data), and three trees are checked stage by stage against
the oracle: the extension (Section 3) against the oracle's, and the potential
of the oracle's extended values against its direct quadrature (Eq. 2).
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from bounds import MIXED_EXT_EPS, MIXED_SCHEDULE_TOL, extension_bounds

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import __graft_entry__ as g
    g.build_library()
    from paper_2211_14537_gb300 import vpx
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return vpx


def _plan(V, wl, precision=1):
    o = V.vpx_default_options(K=wl.opts.K, min_level=wl.opts.min_level, max_level=wl.opts.max_level,
                              refine_tol=wl.opts.refine_tol, f_scale=wl.opts.f_scale, p=40, precision=precision)
    return V.vpx_plan_create(o, wl.domain, wl.sources[0])


@pytest.fixture(scope="module")
def batch(V):
    wls = W.star_batch(32)
    plans = [_plan(V, wl) for wl in wls]
    sizes = [p.sizes() for p in plans]
    fs = [torch.tensor(wl.sources[0](p.stencil_points()), dtype=torch.float64, device="cuda")
          for wl, p in zip(wls, plans)]
    return wls, plans, sizes, fs


def _outputs(sizes):
    vs = [torch.full((sz[1],), float("nan"), dtype=torch.float64, device="cuda") for sz in sizes]
    vbs = [torch.full((sz[3],), float("nan"), dtype=torch.float64, device="cuda") for sz in sizes]
    return vs, vbs


def test_c5_batch_matches_single_executes(V, batch):
    wls, plans, sizes, fs = batch
    npts = [sz[1] for sz in sizes]
    assert min(npts) < 20000 and max(npts) > 100000          # uneven
    stream = torch.cuda.Stream()
    vs, vbs = _outputs(sizes)
    V.vpx_execute_batch(plans, fs, vs, vbs, stream=stream)
    for p in plans:
        assert V.vpx_sync_status(p) == 0
    # replay of the cached graph on fresh contents of the same buffers
    for v in vs:
        v.fill_(float("nan"))
    V.vpx_execute_batch(plans, fs, vs, vbs, stream=stream)
    stream.synchronize()
    worst = 0.0
    for i, p in enumerate(plans):
        v1 = torch.empty(sizes[i][1], dtype=torch.float64, device="cuda")
        vb1 = torch.empty(sizes[i][3], dtype=torch.float64, device="cuda")
        V.vpx_execute(p, fs[i], v1, vb1, stream=stream)
        assert V.vpx_sync_status(p) == 0
        assert torch.isfinite(vs[i]).all() and torch.isfinite(vbs[i]).all()
        d = max(float((vs[i] - v1).abs().max()) / float(v1.abs().max()),
                float((vbs[i] - vb1).abs().max()) / float(vb1.abs().max()))
        worst = max(worst, d)
    # targets and expansions accumulate with FP64 atomics, whose order varies
    print("C5 batch vs single executes: max rel diff %.3e over %d trees" % (worst, len(plans)))
    assert worst <= MIXED_SCHEDULE_TOL


def test_c5_batch_sampled_against_oracle(V, batch):
    """The smallest, a middle and the largest tree of the batch, stage by stage
    against the oracle: the extension within 64 units of the mixed form's
    extension arithmetic (2^-40 for its five-slice grid stage) times each
    cut leaf's forward-error factor kappa, and the potential of the
    oracle's own extended values on sampled leaf targets (direct quadrature)
    and boundary targets (interpolation of the leaf values on the containing
    leaf, Section 4.1) within 1e-9 of max |V|.  The batch's end-to-end error is reported: for these
    mixtures (Gaussians of width down to 0.01 crossing the boundary) kappa
    reaches 1e12, so no useful end-to-end bound follows from it."""
    wls, plans, sizes, fs = batch
    stream = torch.cuda.Stream()
    vs, vbs = _outputs(sizes)
    V.vpx_execute_batch(plans, fs, vs, vbs, stream=stream)
    for p in plans:
        assert V.vpx_sync_status(p) == 0
    order = np.argsort([sz[1] for sz in sizes])
    picks = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    for i in picks:
        wl, plan = wls[i], plans[i]
        tree = O.build_tree(wl.domain, wl.opts, wl.sources[0])
        assert tree.n_leaves == sizes[i][0]
        pts, meta = O.stencil_points(tree, wl.domain)
        f = wl.sources[0](pts)
        vals, _ = O.leaf_values(tree, wl.domain, f[:, None], meta)
        # extension
        fe = torch.empty(sizes[i][1], dtype=torch.float64, device="cuda")
        V.vpx_extend(plan, fs[i], fe, stream=stream)
        assert V.vpx_sync_status(plan) == 0
        got = fe.cpu().numpy().reshape(tree.n_leaves, -1)
        kappa = extension_bounds(tree, wl.domain, meta)
        fmax = np.max(np.abs(f))
        worst = 0.0
        for j, k in kappa.items():
            d = np.max(np.abs(got[j] - vals[j, 0])) / (64 * MIXED_EXT_EPS * max(k, 1.0) * fmax)
            worst = max(worst, d)
        reg = [j for j in range(tree.n_leaves) if tree.cls[j] == O.REGULAR]
        assert np.max(np.abs(got[reg] - vals[reg, 0])) <= 1e-14 * fmax
        assert worst <= 1.0, (wl.name, worst)
        # potential of the oracle's extended values
        nodes = O.all_leaf_nodes(tree)
        bnodes = plan.boundary_nodes()
        rng = np.random.Generator(np.random.PCG64(2215 + i))
        sub = np.sort(rng.choice(len(nodes), 60, replace=False))
        bsub = np.sort(rng.choice(len(bnodes), 20, replace=False))
        want = O.volume_potential(tree, vals, nodes[sub])[:, 0]
        # boundary values interpolate V on the containing leaf (Section 4.1):
        # V at the nodes of those leaves, then the oracle's interpolation
        KK = tree.K * tree.K
        bl = sorted({O.locate_leaf(tree, q) for q in bnodes[bsub]})
        Vl = np.full((tree.n_leaves, KK, 1), np.nan)
        for j in bl:
            Vl[j] = O.volume_potential(tree, vals, nodes[j * KK:(j + 1) * KK])
        wantb = O.interpolate_at(tree, Vl, bnodes[bsub])[:, 0]
        scale = max(np.max(np.abs(want)), np.max(np.abs(wantb)))
        fe_o = torch.tensor(vals[:, 0, :].ravel(), dtype=torch.float64, device="cuda")
        v = torch.empty(sizes[i][1], dtype=torch.float64, device="cuda")
        vb = torch.empty(sizes[i][3], dtype=torch.float64, device="cuda")
        V.vpx_potential(plan, fe_o, v, vb, stream=stream)
        assert V.vpx_sync_status(plan) == 0
        dv = max(np.max(np.abs(v.cpu().numpy()[sub] - want)), np.max(np.abs(vb.cpu().numpy()[bsub] - wantb)))
        e2e = max(np.max(np.abs(vs[i].cpu().numpy()[sub] - want)),
                  np.max(np.abs(vbs[i].cpu().numpy()[bsub] - wantb))) / scale
        print("C5 tree %s (%d leaf targets): extension err / bound %.3e, potential rel err %.3e, "
              "batch end to end rel err %.3e" % (wl.name, sizes[i][1], worst, dv / scale, e2e))
        assert dv <= 1e-9 * scale, (wl.name, dv / scale)


def test_c5_batch_graph_follows_its_arguments(V, batch):
    """A different selection or order of plans, or other buffers, is a new
    graph; the results do not depend on the batch the tree is in."""
    wls, plans, sizes, fs = batch
    stream = torch.cuda.Stream()
    sel = [5, 1, 23]
    vs, vbs = _outputs([sizes[i] for i in sel])
    V.vpx_execute_batch([plans[i] for i in sel], [fs[i] for i in sel], vs, vbs, stream=stream)
    ref = []
    for k, i in enumerate(sel):
        assert V.vpx_sync_status(plans[i]) == 0
        v1 = torch.empty(sizes[i][1], dtype=torch.float64, device="cuda")
        V.vpx_execute(plans[i], fs[i], v1, stream=stream)
        assert V.vpx_sync_status(plans[i]) == 0
        assert float((vs[k] - v1).abs().max()) <= MIXED_SCHEDULE_TOL * float(v1.abs().max())
        ref.append(v1)
    rev = sel[::-1]
    vs2, _ = _outputs([sizes[i] for i in rev])
    V.vpx_execute_batch([plans[i] for i in rev], [fs[i] for i in rev], vs2, None, stream=stream)
    for k, i in enumerate(rev):
        assert V.vpx_sync_status(plans[i]) == 0
        r = ref[len(sel) - 1 - k]
        assert float((vs2[k] - r).abs().max()) <= MIXED_SCHEDULE_TOL * float(r.abs().max())
    # a plan created after the cached graph was captured
    extra = _plan(V, wls[1])
    f_extra = torch.tensor(wls[1].sources[0](extra.stencil_points()), dtype=torch.float64, device="cuda")
    vs3, _ = _outputs([sizes[1]])
    V.vpx_execute_batch([extra], [f_extra], vs3, None, stream=stream)
    assert V.vpx_sync_status(extra) == 0
    assert float((vs3[0] - ref[1]).abs().max()) <= MIXED_SCHEDULE_TOL * float(ref[1].abs().max())


def test_c5_batch_rejects_bad_arguments(V, batch):
    wls, plans, sizes, fs = batch
    vs, vbs = _outputs(sizes[:2])
    with pytest.raises(V.VpxError):
        V.vpx_execute_batch([plans[0], plans[0]], [fs[0], fs[0]], [vs[0], vs[0]], None)
    with pytest.raises(V.VpxError):
        V.vpx_execute_batch([plans[0], plans[1]], [fs[0], fs[1]], [vs[1], vs[0]], None)   # short buffers


def test_c5_batch_autotune_keeps_results(V, batch):
    """The batch autotuner (one engine / tile choice per pass role, timed on the
    batch graph) leaves every tree's result unchanged to MIXED_SCHEDULE_TOL."""
    wls, plans, sizes, fs = batch
    stream = torch.cuda.Stream()
    vs, vbs = _outputs(sizes)
    V.vpx_execute_batch(plans, fs, vs, vbs, stream=stream)
    stream.synchronize()
    npass, nchg = V.vpx_autotune_batch(plans, fs, stream=stream)
    print("C5 batch autotune: %d passes tuned, %d changed" % (npass, nchg))
    assert npass >= 4 * len(plans)
    vs2, vbs2 = _outputs(sizes)
    V.vpx_execute_batch(plans, fs, vs2, vbs2, stream=stream)
    for i, p in enumerate(plans):
        assert V.vpx_sync_status(p) == 0
        scale = float(vs[i].abs().max())
        assert float((vs2[i] - vs[i]).abs().max()) <= MIXED_SCHEDULE_TOL * scale
        assert float((vbs2[i] - vbs[i]).abs().max()) <= MIXED_SCHEDULE_TOL * scale
