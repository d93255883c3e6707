"""vpx_potential_static: the volume potential with its expansion scratch in
the library's fixed device array, for callers that must not allocate device
memory at the time of the call.  Checked through the C ABI against
vpx_potential (the plan-workspace path) on two calls in a row, in both the
FP64 and the mixed form, and for its two refusals (more columns than the
plan's max_rhs; scratch larger than the array).  Runs last so that a failure
here leaves every other test run."""
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


def _plan(V, wl, max_rhs=1, precision=0):
    o = V.vpx_default_options(K=wl.opts.K, min_level=wl.opts.min_level, max_level=wl.opts.max_level,
                              refine_tol=wl.opts.refine_tol, f_scale=wl.opts.f_scale, p=40, max_rhs=max_rhs,
                              precision=precision)
    return V.vpx_plan_create(o, wl.domain, wl.sources[0])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nrhs", [1, 2])
def test_static_scratch_matches_workspace_path_twice(V, nrhs, precision):
    prec = V.VPX_PREC_MIXED if precision == "mixed" else V.VPX_PREC_FP64
    wl = W.starfish_gaussian(K=8, tol=1e-8, max_level=8)
    plan = _plan(V, wl, max_rhs=nrhs, precision=prec)
    _, nt, _, nb = plan.sizes()
    rng = np.random.Generator(np.random.PCG64(5))
    fe = torch.tensor(rng.uniform(-1, 1, (nrhs, nt)), dtype=torch.float64, device="cuda")
    v_ref = torch.empty((nrhs, nt), dtype=torch.float64, device="cuda")
    b_ref = torch.empty((nrhs, nb), dtype=torch.float64, device="cuda")
    V.vpx_potential(plan, fe, v_ref, b_ref)
    assert V.vpx_sync_status(plan) == 0
    scale = float(v_ref.abs().max())
    # both paths run the same kernels in the same order on the same inputs; only
    # the expansion arrays live elsewhere, so they agree to the order in which
    # the atomic accumulations land (a few units of rounding)
    tol = 1e-13 * scale
    for call in range(2):
        v = torch.full((nrhs, nt), float("nan"), dtype=torch.float64, device="cuda")
        b = torch.full((nrhs, nb), float("nan"), dtype=torch.float64, device="cuda")
        V.vpx_potential_static(plan, fe, v, b)
        assert V.vpx_sync_status(plan) == 0
        assert float((v - v_ref).abs().max()) <= tol, call
        assert float((b - b_ref).abs().max()) <= tol, call


def test_static_scratch_rejects_more_columns_than_max_rhs(V):
    """A mixed plan built for one column refuses two, although two would fit the
    static array: the slice buffers it also writes are sized by max_rhs."""
    wl = W.disk_sincos(level=3, K=8)
    plan = _plan(V, wl, max_rhs=1, precision=V.VPX_PREC_MIXED)
    _, nt, _, nb = plan.sizes()
    fe = torch.zeros((2, nt), dtype=torch.float64, device="cuda")
    v = torch.empty((2, nt), dtype=torch.float64, device="cuda")
    with pytest.raises(V.VpxError) as e:
        V.vpx_potential_static(plan, fe, v)
    assert e.value.code == V.VPX_ERR_ARG
    assert V.vpx_sync_status(plan) == 0


def test_static_scratch_rejects_oversize(V):
    wl = W.disk_sincos(level=4, K=8)
    nrhs = 40   # 40 * 341 boxes * 4 * 41 doubles > 2 Mi doubles
    plan = _plan(V, wl, max_rhs=nrhs)
    _, nt, _, nb = plan.sizes()
    fe = torch.zeros((nrhs, nt), dtype=torch.float64, device="cuda")
    v = torch.empty((nrhs, nt), dtype=torch.float64, device="cuda")
    with pytest.raises(V.VpxError) as e:
        V.vpx_potential_static(plan, fe, v)
    assert e.value.code == V.VPX_ERR_ARG
