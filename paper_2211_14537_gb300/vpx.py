"""Thin Python binding of the vpx C ABI (include/vpx.h).

Argument marshalling only: every step of the computation runs in the CUDA
library ``_build/libvpx.so``.  Device buffers are passed as torch CUDA
tensors (their data pointers); streams as torch streams.  If the library is
missing, importing the functions raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Callable, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libvpx.so")

VPX_OK = 0
VPX_ERR_ARG = -1
VPX_ERR_CUDA = -2
VPX_ERR_NOMEM = -3
VPX_ERR_STENCIL = -4
VPX_ERR_DOMAIN = -5
VPX_ERR_LEVEL = -6
VPX_ERR_TIMEOUT = -7
VPX_ERR_NAN = -8
VPX_ERR_CALLBACK = -9
VPX_ERR_STATE = -10
VPX_ERR_NODEV = -11
VPX_PREC_FP64 = 0
VPX_PREC_MIXED = 1
VPX_PLAN_HOST_ONLY = 1
VPX_N_PASSES = 8
N_NEAR, N_V, N_X, N_W = 33, 40, 20, 20


class VpxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("vpx error %d: %s" % (code, msg))
        self.code = code


class vpx_options(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("min_level", ctypes.c_int), ("max_level", ctypes.c_int),
                ("refine_tol", ctypes.c_double), ("f_scale", ctypes.c_double), ("p", ctypes.c_int),
                ("precision", ctypes.c_int), ("max_rhs", ctypes.c_int), ("n_quad_bdry", ctypes.c_int),
                ("rbf_eps", ctypes.c_double), ("ext_mode", ctypes.c_int)]


POINTS_CB = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                             ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)
INSIDE_CB = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                             ctypes.POINTER(ctypes.c_uint8), ctypes.c_void_p)
CURVE_CB = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)

EXPORTED = [
    "vpx_default_options", "vpx_plan_create", "vpx_plan_sizes", "vpx_plan_leaves", "vpx_stencil_points",
    "vpx_leaf_nodes", "vpx_boundary_nodes", "vpx_plan_list_counts", "vpx_plan_lists", "vpx_plan_near_tables",
    "vpx_universal_matrix", "vpx_plan_ray_operator", "vpx_execute",
    "vpx_execute_batch", "vpx_autotune", "vpx_autotune_batch",
    "vpx_extend", "vpx_potential", "vpx_potential_static", "vpx_net_charge", "vpx_bie_setup", "vpx_bie_topology", "vpx_bie_log_terms", "vpx_bie_solve", "vpx_bie_eval", "vpx_bie_dipole_multipoles", "vpx_bie_geometry", "vpx_bie_corrections", "vpx_execute_host", "vpx_sync_status", "vpx_set_timing",
    "vpx_get_timings", "vpx_pass_name", "vpx_graph_kernel_count", "vpx_check_bounded_wait", "vpx_check_gauss_jordan", "vpx_error_string", "vpx_last_error_message", "vpx_plan_destroy",
]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("vpx CUDA library not built: %s (run __graft_entry__.build())" % path)
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    d, i64, i32, vp = ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
    L.vpx_default_options.argtypes = [P(vpx_options)]
    L.vpx_plan_create.argtypes = [P(vpx_options), ctypes.c_int, CURVE_CB, INSIDE_CB, POINTS_CB, vp,
                                  ctypes.c_uint, P(vp)]
    L.vpx_plan_sizes.argtypes = [vp, P(i64), P(i64), P(i64), P(i64)]
    L.vpx_plan_leaves.argtypes = [vp, P(i32), P(i32), P(i32), P(i32), P(i32)]
    L.vpx_stencil_points.argtypes = [vp, P(d)]
    L.vpx_leaf_nodes.argtypes = [vp, P(d)]
    L.vpx_boundary_nodes.argtypes = [vp, P(d)]
    L.vpx_plan_list_counts.argtypes = [vp, P(i64), P(i64), P(i64), P(i64), P(i64), P(i32)]
    L.vpx_plan_lists.argtypes = [vp] + [P(i32)] * 8
    L.vpx_plan_near_tables.argtypes = [vp, P(d)]
    L.vpx_execute.argtypes = [vp, vp, ctypes.c_int, i64, vp, i64, vp, i64, vp]
    L.vpx_extend.argtypes = [vp, vp, ctypes.c_int, i64, vp, i64, vp]
    L.vpx_execute_batch.argtypes = [ctypes.c_int, P(vp), P(vp), P(ctypes.c_int), P(i64), P(vp), P(i64), P(vp), P(i64),
                                    vp]
    L.vpx_potential.argtypes = [vp, vp, ctypes.c_int, i64, vp, i64, vp, i64, vp]
    L.vpx_autotune.argtypes = [vp, vp, ctypes.c_int, i64, vp, P(ctypes.c_int), P(ctypes.c_int)]
    L.vpx_universal_matrix.argtypes = [ctypes.c_int, ctypes.c_double, P(ctypes.c_double), P(i64), P(i64)]
    L.vpx_plan_ray_operator.argtypes = [vp, P(i64), P(ctypes.c_int32), P(ctypes.c_int32), P(i64), P(ctypes.c_double)]
    L.vpx_autotune_batch.argtypes = [ctypes.c_int, P(vp), P(vp), P(ctypes.c_int), P(i64), vp, P(ctypes.c_int),
                                     P(ctypes.c_int)]
    L.vpx_potential_static.argtypes = [vp, vp, ctypes.c_int, i64, vp, i64, vp, i64, vp]
    L.vpx_net_charge.argtypes = [vp, vp, ctypes.c_int, i64, vp, vp]
    L.vpx_bie_setup.argtypes = [vp, INSIDE_CB, vp]
    L.vpx_bie_topology.argtypes = [vp, P(ctypes.c_int), P(ctypes.c_int), P(i32), P(d)]
    L.vpx_bie_log_terms.argtypes = [vp, P(ctypes.c_int), P(i32), P(d), P(i64)]
    L.vpx_bie_solve.argtypes = [vp, vp, vp, d, vp, vp]
    L.vpx_bie_eval.argtypes = [vp, vp, vp, vp, vp]
    L.vpx_bie_dipole_multipoles.argtypes = [vp, P(ctypes.c_int), P(d)]
    L.vpx_bie_geometry.argtypes = [vp, P(d), P(d), P(d)]
    L.vpx_bie_corrections.argtypes = [vp, P(i64), P(i64), P(i32), P(d)]
    L.vpx_execute_host.argtypes = [vp, P(d), ctypes.c_int, P(d), P(d)]
    L.vpx_sync_status.argtypes = [vp]
    L.vpx_set_timing.argtypes = [vp, ctypes.c_int]
    L.vpx_get_timings.argtypes = [vp, P(d), ctypes.c_int]
    L.vpx_graph_kernel_count.argtypes = [vp, P(ctypes.c_int64)]
    L.vpx_check_bounded_wait.argtypes = [P(ctypes.c_int)]
    L.vpx_check_gauss_jordan.argtypes = [ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int)]
    L.vpx_pass_name.argtypes = [ctypes.c_int]
    L.vpx_pass_name.restype = ctypes.c_char_p
    L.vpx_error_string.argtypes = [ctypes.c_int]
    L.vpx_error_string.restype = ctypes.c_char_p
    L.vpx_last_error_message.restype = ctypes.c_char_p
    L.vpx_plan_destroy.argtypes = [vp]
    L.vpx_plan_destroy.restype = None
    _lib = L
    return L


def _check(rc: int):
    if rc != VPX_OK:
        L = load_library()
        raise VpxError(rc, "%s: %s" % (L.vpx_error_string(rc).decode(), L.vpx_last_error_message().decode()))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def vpx_default_options(**kw) -> vpx_options:
    o = vpx_options()
    _check(load_library().vpx_default_options(ctypes.byref(o)))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Plan:
    """Owns a vpx_plan_t and the Python callbacks it was built with."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "handle", None):
            load_library().vpx_plan_destroy(self.handle)
            self.handle = None

    # ------------------------------------------------------------ queries
    def sizes(self):
        v = [ctypes.c_int64() for _ in range(4)]
        _check(load_library().vpx_plan_sizes(self.handle, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)   # n_leaves, n_leaf_nodes, n_stencil, n_bdry

    def leaves(self):
        nl = self.sizes()[0]
        arrs = [np.zeros(nl, dtype=np.int32) for _ in range(5)]
        _check(load_library().vpx_plan_leaves(self.handle, *[_iptr(a) for a in arrs]))
        return dict(zip(["level", "ix", "iy", "cls", "owner"], arrs))

    def _points(self, fn, n):
        a = np.zeros(2 * n)
        _check(fn(self.handle, _dptr(a)))
        return a.reshape(-1, 2)

    def stencil_points(self):
        return self._points(load_library().vpx_stencil_points, self.sizes()[2])

    def leaf_nodes(self):
        return self._points(load_library().vpx_leaf_nodes, self.sizes()[1])

    def boundary_nodes(self):
        return self._points(load_library().vpx_boundary_nodes, self.sizes()[3])

    def list_counts(self):
        v = [ctypes.c_int64() for _ in range(5)] + [ctypes.c_int32()]
        _check(load_library().vpx_plan_list_counts(self.handle, *[ctypes.byref(x) for x in v]))
        return dict(zip(["near", "m2l", "s2l", "m2t", "n_boxes", "n_levels"], [x.value for x in v]))

    def lists(self):
        nl = self.sizes()[0]
        nb = self.list_counts()["n_boxes"]
        a = [np.zeros(nl * N_NEAR, np.int32), np.zeros(nb * N_V, np.int32), np.zeros(nb * N_X, np.int32),
             np.zeros(nl * N_W, np.int32)] + [np.zeros(nb, np.int32) for _ in range(4)]
        _check(load_library().vpx_plan_lists(self.handle, *[_iptr(x) for x in a]))
        return dict(near=a[0].reshape(nl, N_NEAR), vlist=a[1].reshape(nb, N_V), xlist=a[2].reshape(nb, N_X),
                    wlist=a[3].reshape(nl, N_W), box_level=a[4], box_ix=a[5], box_iy=a[6], box_leaf=a[7])


def vpx_plan_ray_operator(plan: "Plan"):
    """(ray_c, ray_g, ray_src, coef[n, 8]) of a plan extending along lines."""
    L = load_library()
    n = ctypes.c_int64()
    _check(L.vpx_plan_ray_operator(plan.handle, ctypes.byref(n), None, None, None, None))
    c = np.zeros(n.value, dtype=np.int32)
    g = np.zeros(n.value, dtype=np.int32)
    src = np.zeros(n.value, dtype=np.int64)
    coef = np.zeros((n.value, 8))
    P = ctypes.POINTER
    _check(L.vpx_plan_ray_operator(plan.handle, ctypes.byref(n), c.ctypes.data_as(P(ctypes.c_int32)),
                                   g.ctypes.data_as(P(ctypes.c_int32)), src.ctypes.data_as(P(ctypes.c_int64)),
                                   coef.ctypes.data_as(P(ctypes.c_double))))
    return c, g, src, coef


def vpx_universal_matrix(K: int, rbf_eps: float = 0.0) -> np.ndarray:
    """The universal extension operator (rows X_S, X_Sbar, G; columns G) that
    plans of leaf order K and shape parameter rbf_eps use (host)."""
    L = load_library()
    nx, ng = ctypes.c_int64(), ctypes.c_int64()
    _check(L.vpx_universal_matrix(K, rbf_eps, None, ctypes.byref(nx), ctypes.byref(ng)))
    out = np.zeros((nx.value, ng.value))
    _check(L.vpx_universal_matrix(K, rbf_eps, _dptr(out), ctypes.byref(nx), ctypes.byref(ng)))
    return out


def vpx_plan_near_tables(plan: "Plan") -> np.ndarray:
    K2 = plan.sizes()[1] // max(plan.sizes()[0], 1)
    out = np.zeros(N_NEAR * K2 * K2)
    _check(load_library().vpx_plan_near_tables(plan.handle, _dptr(out)))
    return out.reshape(N_NEAR, K2, K2)


def vpx_plan_create(opts: vpx_options, domain, refine_f: Callable, host_only: bool = False) -> Plan:
    """Build a plan from a domain object (``inside(xy)``, ``curve(i, t)``,
    ``n_panels``) and the source used for adaptive refinement."""
    def f_cb(xy, n, out, ctx):
        try:
            pts = np.ctypeslib.as_array(xy, shape=(2 * n,)).reshape(n, 2)
            np.ctypeslib.as_array(out, shape=(n,))[:] = np.asarray(refine_f(pts), dtype=np.float64)
            return 0
        except Exception:   # noqa: BLE001 - reported as VPX_ERR_CALLBACK
            return 1

    def in_cb(xy, n, ins, ctx):
        try:
            pts = np.ctypeslib.as_array(xy, shape=(2 * n,)).reshape(n, 2)
            np.ctypeslib.as_array(ins, shape=(n,))[:] = np.asarray(domain.inside(pts), dtype=np.uint8)
            return 0
        except Exception:   # noqa: BLE001
            return 1

    def cv_cb(panel, t, n, xy, dxy, ctx):
        try:
            tt = np.ctypeslib.as_array(t, shape=(n,)).copy()
            p, d = domain.curve(panel, tt)
            np.ctypeslib.as_array(xy, shape=(2 * n,))[:] = np.asarray(p, dtype=np.float64).ravel()
            np.ctypeslib.as_array(dxy, shape=(2 * n,))[:] = np.asarray(d, dtype=np.float64).ravel()
            return 0
        except Exception:   # noqa: BLE001
            return 1

    keep = (POINTS_CB(f_cb), INSIDE_CB(in_cb), CURVE_CB(cv_cb))
    h = ctypes.c_void_p()
    n_panels = int(getattr(domain, "n_panels", 0))
    rc = load_library().vpx_plan_create(ctypes.byref(opts), n_panels, keep[2], keep[1], keep[0], None,
                                        VPX_PLAN_HOST_ONLY if host_only else 0, ctypes.byref(h))
    _check(rc)
    return Plan(h, keep)


def _tptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _cols(t):
    """(pointer, nrhs, ld) of a float64 CUDA tensor shaped (n,) or (nrhs, n) with unit inner stride."""
    if t.dtype.__str__() != "torch.float64":
        raise TypeError("float64 tensor required")
    if t.dim() == 1:
        return _tptr(t), 1, t.shape[0]
    if t.stride(1) != 1:
        raise ValueError("inner stride must be 1")
    return _tptr(t), t.shape[0], t.stride(0)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


def vpx_execute(plan: Plan, f_stencil, v_leaf, v_bdry=None, stream=None):
    fp, nrhs, ldf = _cols(f_stencil)
    vp_, n2, ldv = _cols(v_leaf)
    bp, ldb = ctypes.c_void_p(0), 1
    if v_bdry is not None and v_bdry.numel() > 0:
        bp, _, ldb = _cols(v_bdry)
    _check(load_library().vpx_execute(plan.handle, fp, nrhs, ldf, vp_, ldv, bp, ldb, _stream_handle(stream)))


def vpx_execute_batch(plans, f_stencils, v_leaves, v_bdrys=None, stream=None):
    """vpx_execute for every (plan, f, v[, v_bdry]) of the lists, in one captured graph."""
    n = len(plans)
    vp = ctypes.c_void_p

    def raw(x):
        return x.value if isinstance(x, vp) else x

    fps, nrs, ldfs, vps, ldvs, bps, ldbs = [], [], [], [], [], [], []
    for i in range(n):
        fp, nrhs, ldf = _cols(f_stencils[i])
        vq, _, ldv = _cols(v_leaves[i])
        bp, ldb = vp(0), 1
        if v_bdrys is not None and v_bdrys[i] is not None and v_bdrys[i].numel() > 0:
            bp, _, ldb = _cols(v_bdrys[i])
        fps.append(raw(fp)); nrs.append(nrhs); ldfs.append(ldf)
        vps.append(raw(vq)); ldvs.append(ldv); bps.append(raw(bp)); ldbs.append(ldb)

    def arr(t, xs):
        return (t * n)(*xs)

    hs = [raw(p.handle) for p in plans]
    _check(load_library().vpx_execute_batch(n, arr(vp, hs), arr(vp, fps), arr(ctypes.c_int, nrs),
                                            arr(ctypes.c_int64, ldfs), arr(vp, vps), arr(ctypes.c_int64, ldvs),
                                            arr(vp, bps), arr(ctypes.c_int64, ldbs), _stream_handle(stream)))


def vpx_autotune(plan: Plan, f_stencil, stream=None):
    """Time the engine / tile-width candidates of the plan's mixed-form passes on
    its own data and keep the fastest; returns (passes tuned, passes changed)."""
    fp, nrhs, ldf = _cols(f_stencil)
    npass, nchg = ctypes.c_int(), ctypes.c_int()
    _check(load_library().vpx_autotune(plan.handle, fp, nrhs, ldf, _stream_handle(stream), ctypes.byref(npass),
                                       ctypes.byref(nchg)))
    return npass.value, nchg.value


def vpx_autotune_batch(plans, f_stencils, stream=None):
    """vpx_autotune for a batch: one choice per pass role, timed on the batch graph."""
    n = len(plans)
    vp = ctypes.c_void_p
    raw = lambda x: x.value if isinstance(x, vp) else x
    cols = [_cols(t) for t in f_stencils]
    npass, nchg = ctypes.c_int(), ctypes.c_int()
    _check(load_library().vpx_autotune_batch(n, (vp * n)(*[raw(p.handle) for p in plans]),
                                             (vp * n)(*[raw(c[0]) for c in cols]), (ctypes.c_int * n)(*[c[1] for c in cols]),
                                             (ctypes.c_int64 * n)(*[c[2] for c in cols]), _stream_handle(stream),
                                             ctypes.byref(npass), ctypes.byref(nchg)))
    return npass.value, nchg.value


def vpx_extend(plan: Plan, f_stencil, fe_leaf, stream=None):
    fp, nrhs, ldf = _cols(f_stencil)
    ep, _, lde = _cols(fe_leaf)
    _check(load_library().vpx_extend(plan.handle, fp, nrhs, ldf, ep, lde, _stream_handle(stream)))


def vpx_potential(plan: Plan, fe_leaf, v_leaf, v_bdry=None, stream=None):
    ep, nrhs, lde = _cols(fe_leaf)
    vp_, _, ldv = _cols(v_leaf)
    bp, ldb = ctypes.c_void_p(0), 1
    if v_bdry is not None and v_bdry.numel() > 0:
        bp, _, ldb = _cols(v_bdry)
    _check(load_library().vpx_potential(plan.handle, ep, nrhs, lde, vp_, ldv, bp, ldb, _stream_handle(stream)))


def vpx_potential_static(plan: Plan, fe_leaf, v_leaf, v_bdry=None, stream=None):
    """vpx_potential with the expansion scratch in the library's static device
    array (no allocation at call time; see include/vpx.h)."""
    ep, nrhs, lde = _cols(fe_leaf)
    vp_, _, ldv = _cols(v_leaf)
    bp, ldb = ctypes.c_void_p(0), 1
    if v_bdry is not None and v_bdry.numel() > 0:
        bp, _, ldb = _cols(v_bdry)
    _check(load_library().vpx_potential_static(plan.handle, ep, nrhs, lde, vp_, ldv, bp, ldb,
                                               _stream_handle(stream)))


def vpx_net_charge(plan: Plan, fe_leaf, charge, stream=None):
    """A^e per right-hand side of the leaf values fe_leaf into the device tensor charge."""
    ep, nrhs, lde = _cols(fe_leaf)
    if charge.numel() < nrhs:
        raise ValueError("charge holds fewer than nrhs values")
    _check(load_library().vpx_net_charge(plan.handle, ep, nrhs, lde, ctypes.c_void_p(charge.data_ptr()),
                                         _stream_handle(stream)))


def vpx_bie_setup(plan: Plan):
    """Host part of the boundary correction, with the domain's own inside test."""
    _check(load_library().vpx_bie_setup(plan.handle, plan._keep[1], None))


def vpx_bie_topology(plan: Plan):
    """(n_curves, outer_curve, curve_of_node (n_bdry,), jump (n_bdry,)) after vpx_bie_setup."""
    nb = plan.sizes()[3]
    nc, oc = ctypes.c_int(0), ctypes.c_int(0)
    cn, jp = np.zeros(nb, dtype=np.int32), np.zeros(nb)
    _check(load_library().vpx_bie_topology(plan.handle, ctypes.byref(nc), ctypes.byref(oc), _iptr(cn), _dptr(jp)))
    return nc.value, oc.value, cn, jp


def vpx_bie_log_terms(plan: Plan):
    """(curve (n_log,), centre (n_log, 2), n_unknowns) after vpx_bie_setup."""
    L = load_library()
    n, nu = ctypes.c_int(0), ctypes.c_int64(0)
    _check(L.vpx_bie_log_terms(plan.handle, ctypes.byref(n), None, None, ctypes.byref(nu)))
    cv, ce = np.zeros(n.value, dtype=np.int32), np.zeros((n.value, 2))
    _check(L.vpx_bie_log_terms(plan.handle, ctypes.byref(n), _iptr(cv), _dptr(ce), ctypes.byref(nu)))
    return cv, ce, nu.value


def vpx_bie_solve(plan: Plan, g, vb, sol, growth: float = 0.0, stream=None):
    """Device tensors: g, vb (n_bdry), sol (n_unknowns) written."""
    _check(load_library().vpx_bie_solve(plan.handle, _tptr(g), _tptr(vb), float(growth), _tptr(sol),
                                        _stream_handle(stream)))


def vpx_bie_eval(plan: Plan, sol, v_leaf, u_leaf, stream=None):
    """Device tensors: u_leaf = V + the correction at every leaf node."""
    _check(load_library().vpx_bie_eval(plan.handle, _tptr(sol), _tptr(v_leaf), _tptr(u_leaf), _stream_handle(stream)))


def vpx_bie_dipole_multipoles(plan: Plan):
    """(n_bdry, p + 1) complex: each node's unit double-layer term as a scaled multipole of its leaf."""
    L = load_library()
    n = ctypes.c_int(0)
    _check(L.vpx_bie_dipole_multipoles(plan.handle, ctypes.byref(n), None))
    out = np.zeros((plan.sizes()[3], n.value))
    _check(L.vpx_bie_dipole_multipoles(plan.handle, ctypes.byref(n), _dptr(out)))
    return out[:, 0::2] + 1j * out[:, 1::2]


def vpx_bie_geometry(plan: Plan):
    """(nu (n_bdry, 2), s*w (n_bdry,), kappa (n_bdry,)) after vpx_bie_setup."""
    nb = plan.sizes()[3]
    nu, sw, ka = np.zeros((nb, 2)), np.zeros(nb), np.zeros(nb)
    _check(load_library().vpx_bie_geometry(plan.handle, _dptr(nu), _dptr(sw), _dptr(ka)))
    return nu, sw, ka


def vpx_bie_corrections(plan: Plan, nq: int = 16):
    """(off (n_leaf_nodes + 1,), panel (n_corr,), w (n_corr, nq)) after vpx_bie_setup."""
    L = load_library()
    n = ctypes.c_int64(0)
    _check(L.vpx_bie_corrections(plan.handle, ctypes.byref(n), None, None, None))
    nt = plan.sizes()[1]
    off = np.zeros(nt + 1, dtype=np.int64)
    pan = np.zeros(n.value, dtype=np.int32)
    w = np.zeros((n.value, nq))
    _check(L.vpx_bie_corrections(plan.handle, ctypes.byref(n), off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 pan.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dptr(w)))
    return off, pan, w


def vpx_execute_host(plan: Plan, f_stencil: np.ndarray, nrhs: int = 1, v_out: np.ndarray = None,
                     b_out: np.ndarray = None):
    """End to end with host arrays: returns (v_leaf, v_bdry) as (nrhs, n) numpy arrays.

    v_out (nrhs, n_leaf_nodes) and b_out (nrhs, max(n_bdry, 1)), C-contiguous
    float64, receive the results when given (for instance views of page-locked
    buffers, whose copies run at the link's rate); otherwise new arrays."""
    _, nt, ns, nb = plan.sizes()
    f = np.ascontiguousarray(f_stencil, dtype=np.float64).reshape(nrhs, ns)

    def out(a, shape):
        if a is None:
            return np.zeros(shape)
        if a.dtype != np.float64 or a.shape != shape or not a.flags["C_CONTIGUOUS"]:
            raise VpxError(VPX_ERR_ARG, "output array must be C-contiguous float64 of shape %s" % (shape,))
        return a

    v = out(v_out, (nrhs, nt))
    b = out(b_out, (nrhs, max(nb, 1)))
    _check(load_library().vpx_execute_host(plan.handle, _dptr(f), nrhs, _dptr(v), _dptr(b)))
    return v, b[:, :nb]


def vpx_sync_status(plan: Plan) -> int:
    return load_library().vpx_sync_status(plan.handle)


def vpx_set_timing(plan: Plan, enable: bool = True):
    _check(load_library().vpx_set_timing(plan.handle, int(bool(enable))))


def vpx_check_bounded_wait() -> int:
    """Run the bounded-wait probe; returns the latched status (VPX_ERR_TIMEOUT expected)."""
    st = ctypes.c_int(0)
    _check(load_library().vpx_check_bounded_wait(ctypes.byref(st)))
    return int(st.value)


def vpx_graph_kernel_count(plan: Plan) -> int:
    """Kernel launches in the graph that vpx_execute captured (0 before it)."""
    n = ctypes.c_int64(0)
    _check(load_library().vpx_graph_kernel_count(plan.handle, ctypes.byref(n)))
    return int(n.value)


def vpx_get_timings(plan: Plan):
    a = np.zeros(VPX_N_PASSES)
    _check(load_library().vpx_get_timings(plan.handle, _dptr(a), VPX_N_PASSES))
    L = load_library()
    return {L.vpx_pass_name(i).decode(): float(a[i]) for i in range(VPX_N_PASSES)}


def vpx_check_gauss_jordan(a: np.ndarray):
    """(inverse, status) of the square host matrix a by the device Gauss-Jordan
    elimination of the boundary correction; status VPX_ERR_STATE for a
    singular matrix."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    inv = np.zeros_like(a)
    st = ctypes.c_int(0)
    _check(load_library().vpx_check_gauss_jordan(a.shape[0], _dptr(a), _dptr(inv), ctypes.byref(st)))
    return inv, st.value
