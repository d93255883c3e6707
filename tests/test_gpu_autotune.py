"""The autotuner (vpx_autotune) changes only the schedule of the mixed-form
passes (engine, pairs per tile): results after tuning equal those before to
bounds.MIXED_SCHEDULE_TOL of the maximum (re-sliced expansions may round to
the neighbouring last digit), captured graphs pick the new choices up, and an FP64-form
plan has nothing to tune."""
import numpy as np
import pytest

import workloads as W
from bounds import MIXED_SCHEDULE_TOL

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


def _plan(V, wl, precision, p=40):
    o = V.vpx_default_options(K=wl.opts.K, min_level=wl.opts.min_level, max_level=wl.opts.max_level,
                              refine_tol=wl.opts.refine_tol, f_scale=wl.opts.f_scale, p=p, precision=precision)
    return V.vpx_plan_create(o, wl.domain, wl.sources[0])


@pytest.mark.parametrize("name", ["starfish_k16", "star_batch_tree"])
def test_autotune_keeps_results(V, name):
    wl = W.starfish_gaussian(K=16) if name == "starfish_k16" else W.star_batch(32)[26]
    plan = _plan(V, wl, V.VPX_PREC_MIXED)
    _, nt, _, nb = plan.sizes()
    f = torch.tensor(wl.sources[0](plan.stencil_points()), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    v0 = torch.empty(nt, dtype=torch.float64, device="cuda")
    b0 = torch.empty(nb, dtype=torch.float64, device="cuda")
    V.vpx_execute(plan, f, v0, b0, stream=stream)      # captures the graph with the defaults
    assert V.vpx_sync_status(plan) == 0
    npass, nchg = V.vpx_autotune(plan, f, stream=stream)
    print("%s: %d passes tuned, %d changed" % (name, npass, nchg))
    assert npass >= 4 and 0 <= nchg <= npass
    v1 = torch.empty_like(v0)
    b1 = torch.empty_like(b0)
    for _ in range(2):                                  # recapture, then replay
        V.vpx_execute(plan, f, v1, b1, stream=stream)
        assert V.vpx_sync_status(plan) == 0
    scale = float(v0.abs().max())
    print("%s: after tuning max diff %.3e, boundary %.3e (scale %.3e)"
          % (name, float((v1 - v0).abs().max()), float((b1 - b0).abs().max()), scale))
    assert float((v1 - v0).abs().max()) <= MIXED_SCHEDULE_TOL * scale
    assert float((b1 - b0).abs().max()) <= MIXED_SCHEDULE_TOL * scale
    # a second plan of the same shapes takes the cached choices without timing
    plan2 = _plan(V, wl, V.VPX_PREC_MIXED)
    assert V.vpx_autotune(plan2, f, stream=stream) == (npass, nchg)


def test_autotune_fp64_plan_has_nothing_to_tune(V):
    wl = W.disk_sincos(level=3)
    plan = _plan(V, wl, V.VPX_PREC_FP64)
    f = torch.tensor(wl.sources[0](plan.stencil_points()), dtype=torch.float64, device="cuda")
    assert V.vpx_autotune(plan, f) == (0, 0)
