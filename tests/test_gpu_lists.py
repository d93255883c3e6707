"""The interaction lists built on the device (one launch per level, Section 4's
near, i, i+ and i- lists) against the host builder, bit for bit: a device
plan's lists (the ones its passes use) equal a host-only plan's lists of the
same tree, on every workload of the tests and the benchmark, including the
uneven star batches.  The host builder itself is pinned on the CPU (every
(target, source) pair covered exactly once, slots geometrically right)."""
import numpy as np
import pytest

import workloads as W

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


def _box(K, level):
    return W.Workload("box%d" % level, 0, W.WholeBoxDomain(), W.TreeOptions(K=K, min_level=level, max_level=level),
                      [lambda xy: 0 * xy[:, 0]])


SINGLE = {
    "box_l1": lambda: _box(8, 1),
    "box_l2": lambda: _box(8, 2),
    "disk_l4": lambda: W.disk_sincos(level=4),
    "starfish_k16": lambda: W.starfish_gaussian(K=16),
    "lshape_c4": lambda: W.lshape_expsin(),
    "exterior": lambda: W.exterior_three_stars(K=8, tol=1e-5, max_level=7),
    "doubly_connected": lambda: W.doubly_connected_adaptive(),
}


def _same_lists(V, wl):
    o = V.vpx_default_options(K=wl.opts.K, min_level=wl.opts.min_level, max_level=wl.opts.max_level,
                              refine_tol=wl.opts.refine_tol, f_scale=wl.opts.f_scale, p=40)
    dev = V.vpx_plan_create(o, wl.domain, wl.sources[0])
    host = V.vpx_plan_create(o, wl.domain, wl.sources[0], host_only=True)
    a, b = dev.lists(), host.lists()
    for k in ("box_level", "box_ix", "box_iy", "box_leaf", "near", "vlist", "xlist", "wlist"):
        assert np.array_equal(a[k], b[k]), k
    assert dev.list_counts() == host.list_counts()
    return len(a["box_level"])


@pytest.mark.parametrize("name", list(SINGLE))
def test_device_lists_equal_host_lists(V, name):
    nb = _same_lists(V, SINGLE[name]())
    assert nb > 0


@pytest.mark.parametrize("deep", [False, True])
def test_device_lists_equal_host_lists_star_batches(V, deep):
    """The 32 trees of the uneven batch, and 32 star trees allowed to refine to
    level 12 (up to 10 levels and 7.8 k boxes)."""
    wls = W.star_batch(32, max_level=12) if deep else W.star_batch(32)
    sizes = [_same_lists(V, wl) for wl in wls]
    assert max(sizes) > (5000 if deep else 500)
