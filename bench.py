"""Benchmark: volume-potential targets/s of the particular-solution stage.

Default workload: the largest single-GPU configuration, the L-shaped polygon
[-0.4,0.4]^2 minus [0,0.4]^2 with f = Laplacian of exp(x) sin(2y), a uniform
level-6 tree refined toward the six corners to level 14, K = 16
Gauss-Legendre nodes per leaf (5,407 leaves, 1.38 M leaf targets).  One step =
one call of vpx_execute: extension of f on the cut leaves plus the box-FMM
volume potential at every leaf node and boundary node, on device-resident
inputs.  The line also carries the uneven 32-tree batch (one graph) as the
key "batch" (skip with --no-batch).

Prints one JSON line (rank 0).  `--impl reference` times the CPU FP64 oracle
(direct quadrature) on a bounded sample of the same targets instead.
Multi-GPU runs are independent replicas (one tree per GPU, no collective on
the data path); value = targets of all ranks / max rank time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "volume-potential targets/sec at rel err 1e-10 (FP64 vs mixed/batched), % of roofline"
UNIT = "targets/s"
FP64_PEAK_TFLOPS = 1.25   # GB300 FP64 (nominal; an FMA probe measured 1.20 at 1.99 GHz)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--p", type=int, default=27,
                    help="expansion order: 27 keeps the potential error at the arithmetic's floor (below 1e-12) on the L-shape and the starfish")
    ap.add_argument("--precision", default="both", choices=["fp64", "mixed", "both"])
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--oracle-sample", type=int, default=0,
                    help="targets of the oracle's sample (0: sized for about 15 s of oracle work on all cores)")
    ap.add_argument("--no-batch", action="store_true", help="leave the uneven 32-tree batch out of the line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default engine / tile choices")
    ap.add_argument("--ext-mode", default="stencil", choices=["stencil", "lines"],
                    help="extension: universal stencil (default) or along lines through the origin (star domains)")
    ap.add_argument("--workload", default="lshape",
                    choices=["starfish", "lshape", "exterior", "doubly-connected", "disk-multi-rhs", "star-batch"],
                    help="lshape: the L-shape refined to level 14 (1.4 M targets); disk-multi-rhs: the disk tree "
                         "with 64 distinct right-hand sides, split into column blocks over the ranks; "
                         "doubly-connected: the run behind the paper's timings (242 k targets); "
                         "exterior: D minus three "
                         "starfish inclusions (Section 6.2, 248 k targets); star-batch: the uneven "
                         "batch of 32 star domains in one graph (mixed form), against the same trees run one "
                         "after another in both forms")
    return ap.parse_args()


DOMAIN_LABEL = {"starfish": "starfish", "lshape": "L-shape", "exterior": "exterior of three inclusions",
                "disk-multi-rhs": "disk (64 right-hand sides)", "doubly-connected": "doubly connected"}
MULTI_RHS_COLUMNS = 64


def workload(name="starfish"):
    """The single-tree workloads: the L-shape refined to level 14 toward its
    corners (1.4 M targets, the default line), the adaptive starfish (185 k
    targets) and the exterior of three starfish inclusions (Section 6.2, 248 k
    targets)."""
    import workloads as W
    if name == "lshape":
        return W.lshape_expsin()
    if name == "exterior":
        return W.exterior_three_stars()
    if name == "disk-multi-rhs":
        return W.disk_multi_rhs(nrhs=MULTI_RHS_COLUMNS)
    if name == "doubly-connected":
        return W.doubly_connected_adaptive()
    return W.starfish_gaussian(K=16)


def rhs_block(n_columns, rank, world):
    """The contiguous block of right-hand-side columns of one rank: the first
    n_columns % world ranks take one column more; every column lands on
    exactly one rank."""
    q, r = divmod(n_columns, world)
    lo = rank * q + min(rank, r)
    return list(range(lo, lo + q + (1 if rank < r else 0)))


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:   # noqa: BLE001 - no nvidia-smi: no clock record
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:   # noqa: BLE001
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def plan_options(V, wl, args, precision):
    """Plan options of the single-tree workloads: the workload's tree, the
    expansion order, the form, the right-hand sides and the extension mode
    (universal stencil, or along lines through the origin)."""
    return V.vpx_default_options(K=wl.opts.K, min_level=wl.opts.min_level, max_level=wl.opts.max_level,
                                 refine_tol=wl.opts.refine_tol, f_scale=wl.opts.f_scale, p=args.p,
                                 precision=V.VPX_PREC_MIXED if precision == "mixed" else V.VPX_PREC_FP64,
                                 max_rhs=args.nrhs, ext_mode=1 if args.ext_mode == "lines" else 0)


def run_gpu(args, rank, world, precision):
    import torch
    from paper_2211_14537_gb300 import vpx as V

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl = workload(args.workload)
    columns = rhs_block(len(wl.sources), rank, world) if args.workload == "disk-multi-rhs" else None
    if columns is not None:
        args.nrhs = len(columns)
    t0 = time.perf_counter()
    o = plan_options(V, wl, args, precision)
    plan = V.vpx_plan_create(o, wl.domain, wl.sources[0])
    setup_s = time.perf_counter() - t0
    n_leaves, nt, ns, nb = plan.sizes()
    lc = plan.list_counts()
    K = wl.opts.K
    KK = K * K
    nrhs = args.nrhs
    if columns is not None:
        f_host = np.stack([wl.sources[c](plan.stencil_points()) for c in columns])
    else:
        f_host = np.stack([wl.sources[0](plan.stencil_points())] * nrhs)
    f = torch.tensor(f_host, dtype=torch.float64, device=dev)
    v = torch.empty((nrhs, nt), dtype=torch.float64, device=dev)
    vb = torch.empty((nrhs, max(nb, 1)), dtype=torch.float64, device=dev)[:, :nb]
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2

    def step():
        V.vpx_execute(plan, f, v, vb if nb else None, stream=stream)

    tune = (0, 0)
    if precision == "mixed" and not args.no_autotune:
        tune = V.vpx_autotune(plan, f, stream=stream)   # engine / tile choices on this plan's data
    V.vpx_set_timing(plan, False)
    for _ in range(max(args.warmup, 3)):
        step()
    if V.vpx_sync_status(plan) != 0:
        raise RuntimeError("device status error during warm-up")
    torch.cuda.synchronize(dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)   # let the sampler come up before the timed region
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))                  # evict L2 between timed steps (outside the events)
            ev0[i].record(stream)
        step()
        with torch.cuda.stream(stream):
            ev1[i].record(stream)
    torch.cuda.synchronize(dev)
    st = V.vpx_sync_status(plan)
    if st != 0:
        raise RuntimeError("device status %d" % st)
    time.sleep(0.15)
    cl = clocks.stop()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    times = [ev0[i].elapsed_time(ev1[i]) for i in range(args.steps)]
    graph_kernels = V.vpx_graph_kernel_count(plan)   # kernel launches of one replayed step
    ms = statistics.mean(times)
    # per-pass breakdown (separate short loop with the pass events enabled)
    V.vpx_set_timing(plan, True)
    passes = []
    for i in range(5):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        step()
        V.vpx_sync_status(plan)
        passes.append(V.vpx_get_timings(plan))
    V.vpx_set_timing(plan, False)
    # e2e through the public host-buffer call (copies in the timed region),
    # input and outputs in page-locked host memory
    f_pin = torch.tensor(np.ascontiguousarray(f_host)).pin_memory()
    v_pin = torch.empty((nrhs, nt), dtype=torch.float64).pin_memory()
    b_pin = torch.empty((nrhs, max(nb, 1)), dtype=torch.float64).pin_memory()
    f_np, v_np, b_np = f_pin.numpy(), v_pin.numpy(), b_pin.numpy()
    for _ in range(3):
        V.vpx_execute_host(plan, f_np, nrhs, v_np, b_np)
    te = []
    for _ in range(20):
        t1 = time.perf_counter()
        vh, bh = V.vpx_execute_host(plan, f_np, nrhs, v_np, b_np)
        te.append(time.perf_counter() - t1)
    vh, bh = vh.copy(), bh.copy()
    e2e_s = statistics.median(te)
    tg = (nt + nb) * nrhs
    pass_ms = {k: statistics.median([p[k] for p in passes]) for k in passes[0]}
    near_flops = 2.0 * KK * KK * lc["near"] * nrhs
    near_ms = pass_ms.get("near", float("nan"))
    return dict(plan=plan, wl=wl, ms=ms, times=times, setup_s=setup_s, tg=tg, nt=nt, nb=nb, ns=ns,
                n_leaves=n_leaves, lc=lc, pass_ms=pass_ms, near_flops=near_flops, near_ms=near_ms,
                clocks=cl, e2e_s=e2e_s, v=v[0].cpu().numpy(), vh=vh, K=K, graph_kernels=graph_kernels, tune=tune)


def latency_floor_us(device="cuda"):
    """Replay time of a captured graph holding one trivial kernel: the floor
    under any captured pipeline on this GPU (CUDA events over 200 replays).
    None when it cannot be measured; it never stops the benchmark line."""
    try:
        import torch
        x = torch.zeros(1, device=device)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(device=device)
        with torch.cuda.stream(s):
            x.add_(1.0)                       # warm-up outside the capture
            torch.cuda.synchronize(device)
            with torch.cuda.graph(g, stream=s):
                x.add_(1.0)
            for _ in range(10):
                g.replay()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(200):
                g.replay()
            e1.record(s)
        torch.cuda.synchronize(device)
        return e0.elapsed_time(e1) / 200 * 1e3
    except Exception:   # noqa: BLE001 - a measurement aid only
        return None


def shard_by_size(sizes, world):
    """Trees to ranks for the batch: largest first, each to the rank with the
    least work so far (ties: the lower rank).  Returns one sorted index list
    per rank; every tree lands on exactly one rank."""
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += sizes[i]
    return [sorted(x) for x in out]


def reduce_over_ranks(ms, units, device, world):
    """(max of ms, sum of units) over the ranks: the job's time is its slowest
    rank's, its work all ranks' work.  No collective on one rank."""
    if world == 1:
        return float(ms), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_batch(args, rank=0, world=1, as_key=False):
    """Uneven batch: 32 random star domains, each with its own mixture and tree,
    in one vpx_execute_batch graph (mixed form), against the same trees run one
    after another (mixed, and FP64 as in a plain sequential solver).  On N
    ranks each takes a size-balanced share of the trees (no collective on the
    data path); value = all ranks' targets / the slowest rank's time.  With
    as_key, returns the batch's figures (rank 0) instead of printing a line."""
    import torch
    import workloads as W
    from paper_2211_14537_gb300 import vpx as V

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wls_all = W.star_batch(32)
    shard = list(range(len(wls_all)))
    if world > 1:
        # tree sizes from host-only plans (no device work), then the share of this rank
        sizes_all = []
        for wl in wls_all:
            o = V.vpx_default_options(K=wl.opts.K, min_level=wl.opts.min_level, max_level=wl.opts.max_level,
                                      refine_tol=wl.opts.refine_tol, f_scale=wl.opts.f_scale, p=args.p)
            sizes_all.append(V.vpx_plan_create(o, wl.domain, wl.sources[0], host_only=True).sizes()[1])
        shard = shard_by_size(sizes_all, world)[rank]
    wls = [wls_all[i] for i in shard]
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def make(prec):
        t0 = time.perf_counter()
        plans = []
        for wl in wls:
            o = V.vpx_default_options(K=wl.opts.K, min_level=wl.opts.min_level, max_level=wl.opts.max_level,
                                      refine_tol=wl.opts.refine_tol, f_scale=wl.opts.f_scale, p=args.p,
                                      precision=prec)
            plans.append(V.vpx_plan_create(o, wl.domain, wl.sources[0]))
        return plans, time.perf_counter() - t0

    def timed(step, steps):
        for _ in range(max(args.warmup, 3)):
            step()
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for i in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
                e0[i].record(stream)
            step()
            with torch.cuda.stream(stream):
                e1[i].record(stream)
        torch.cuda.synchronize(dev)
        ms = statistics.mean([e0[i].elapsed_time(e1[i]) for i in range(steps)])
        return reduce_over_ranks(ms, 0, dev, world)[0]

    mixed, setup_mixed = make(V.VPX_PREC_MIXED)
    sizes = [p.sizes() for p in mixed]
    fs = [torch.tensor(wl.sources[0](p.stencil_points()), dtype=torch.float64, device=dev)
          for wl, p in zip(wls, mixed)]
    vs = [torch.empty(sz[1], dtype=torch.float64, device=dev) for sz in sizes]
    vbs = [torch.empty(sz[3], dtype=torch.float64, device=dev) for sz in sizes]
    targets = reduce_over_ranks(0.0, sum(sz[1] + sz[3] for sz in sizes), dev, world)[1]
    tuned = [0, 0]
    if not args.no_autotune:
        t0 = time.perf_counter()
        tuned = list(V.vpx_autotune_batch(mixed, fs, stream=stream))   # one choice per pass role, on the batch graph
        tune_s = time.perf_counter() - t0
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)
    ms_batch = timed(lambda: V.vpx_execute_batch(mixed, fs, vs, vbs, stream=stream), args.steps)
    time.sleep(0.15)
    cl = clocks.stop()
    for p in mixed:
        if V.vpx_sync_status(p) != 0:
            raise RuntimeError("device status error in the batch")

    def sequence(plans):
        def step():
            for i, p in enumerate(plans):
                V.vpx_execute(p, fs[i], vs[i], vbs[i], stream=stream)
        return step

    ms_seq_mixed = timed(sequence(mixed), max(args.steps // 4, 5))
    kernels = sum(V.vpx_graph_kernel_count(p) for p in mixed)
    del mixed
    fp64, setup_fp64 = make(V.VPX_PREC_FP64)
    ms_seq_fp64 = timed(sequence(fp64), 5)
    for p in fp64:
        if V.vpx_sync_status(p) != 0:
            raise RuntimeError("device status error in the FP64 sequence")
    rate = lambda ms: targets / (ms * 1e-3)
    leaf_all = reduce_over_ranks(0.0, sum(sz[1] for sz in sizes), dev, world)[1]
    bdry_all = reduce_over_ranks(0.0, sum(sz[3] for sz in sizes), dev, world)[1]
    kernels = reduce_over_ranks(0.0, kernels, dev, world)[1]
    if rank != 0:
        return None
    if as_key:
        return {"workload": "star_batch_32", "trees": len(wls_all), "leaf_targets": int(leaf_all),
                "boundary_targets": int(bdry_all), "value": rate(ms_batch), "unit": UNIT, "ms_per_step": ms_batch,
                "mixed_sequential": {"value": rate(ms_seq_mixed), "ms_per_step": ms_seq_mixed},
                "fp64_sequential": {"value": rate(ms_seq_fp64), "ms_per_step": ms_seq_fp64},
                "kernels_per_step": int(kernels),
                "autotune": {"passes_tuned": tuned[0], "passes_changed": tuned[1]},
                "setup_s": {"mixed": round(setup_mixed, 2), "fp64": round(setup_fp64, 2)}, "clocks": cl}
    out = {
        "metric": METRIC, "value": rate(ms_batch), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_batch, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 (exact 8-bit slices) + f64",
        "data": "synthetic (32 seeded random star domains, each with its own Gaussian mixture)",
        "config": {"workload": "star_batch_32", "K": 8, "p": args.p, "trees": len(wls_all),
                   "trees_per_rank": "size-balanced shares" if world > 1 else "all",
                   "leaf_targets": int(leaf_all), "boundary_targets": int(bdry_all),
                   "leaf_targets_min_rank0": min(sz[1] for sz in sizes),
                   "leaf_targets_max_rank0": max(sz[1] for sz in sizes),
                   "l2": "flushed between timed steps (256 MB write, outside the events)",
                   "graph": "one vpx_execute_batch graph replay per step",
                   "setup_s": {"mixed": round(setup_mixed, 2), "fp64": round(setup_fp64, 2)},
                   "autotune": {"passes_tuned": tuned[0], "passes_changed": tuned[1],
                                "seconds": round(tune_s, 2) if not args.no_autotune else 0.0}},
        "forms": {"mixed_batch": {"value": rate(ms_batch), "ms_per_step": ms_batch},
                  "mixed_sequential": {"value": rate(ms_seq_mixed), "ms_per_step": ms_seq_mixed},
                  "fp64_sequential": {"value": rate(ms_seq_fp64), "ms_per_step": ms_seq_fp64}},
        "gpu_launches": int(kernels) * args.steps,
        "clocks": cl,
    }
    print(json.dumps(out), flush=True)


def algorithmic_flops(K, p, n_leaves, lc):
    """Real flops per right-hand side of each pass from the list sizes
    (complex multiply-add = 8): near 2K^4 + 2K^2 per pair, L2M and L2T
    4(p+1)K^2 per leaf, lists i+ and i- 4(p+1)K^2 per pair, M2M and L2L
    4(p+1)^2 per child box, M2L 8(p+1)^2 per pair."""
    P = p + 1
    children = max(int(lc.get("n_boxes", 0)) - 1, 0)
    out = {"near": lc["near"] * (2 * K ** 4 + 2 * K * K), "l2m": 4 * P * K * K * n_leaves,
           "m2m": 4 * P * P * children, "m2l": 8 * P * P * lc["m2l"], "s2l": 4 * P * K * K * lc["s2l"],
           "m2t": 4 * P * K * K * lc["m2t"], "l2l": 4 * P * P * children, "l2t": 4 * P * K * K * n_leaves}
    out["total"] = sum(out.values())
    return out


def oracle_sample(wl, n_sample=0, seconds=15.0, seed=2213, lines=False, one_core_s=0.0):
    """Oracle: own tree + extension (the universal stencil, or along lines),
    then V at a seeded sample of leaf nodes on all host cores and, if
    one_core_s > 0, on one core at an evenly spread subset of the same sample
    (about one_core_s seconds).  n_sample = 0 sizes the sample for about
    `seconds` of oracle work, calibrated on 64 targets.  Returns a dict: the
    oracle's leaf values (leaf-major, the library's layout), the sample
    indices, V there, the seconds and threads of the all-core run and the
    one-core (targets, seconds) or None."""
    from oracle import oracle as O
    tree = O.build_tree(wl.domain, wl.opts, wl.sources[0])
    if lines:
        pts, meta = O.stencil_points_lines(tree, wl.domain)
        vals = O.leaf_values_lines(tree, wl.domain, wl.sources[0](pts)[:, None], meta)
    else:
        pts, meta = O.stencil_points(tree, wl.domain)
        vals, _ = O.leaf_values(tree, wl.domain, wl.sources[0](pts)[:, None], meta)
    nodes = O.all_leaf_nodes(tree)
    threads = O.lib().orc_max_threads()     # all host cores, read before any one-core run
    rng = np.random.Generator(np.random.PCG64(seed))
    perm = rng.permutation(len(nodes))
    if n_sample <= 0:
        t0 = time.perf_counter()
        O.volume_potential(tree, vals, nodes[np.sort(perm[:64])], threads)
        per = (time.perf_counter() - t0) / 64
        n_sample = int(min(max(seconds / per, 128), len(nodes)))
    idx = np.sort(perm[:min(n_sample, len(nodes))])
    t0 = time.perf_counter()
    Vs = O.volume_potential(tree, vals, nodes[idx], threads)[:, 0]
    dt = time.perf_counter() - t0
    one = None
    if one_core_s > 0:
        n1 = int(max(16, min(len(idx), one_core_s / (dt / len(idx) * threads))))
        sub1 = idx[::max(1, len(idx) // n1)]
        t1 = time.perf_counter()
        O.volume_potential(tree, vals, nodes[sub1], 1)
        one = (len(sub1), time.perf_counter() - t1)
    return {"vals": vals, "idx": idx, "V": Vs, "seconds": dt, "threads": threads, "one_core": one,
            "n_leaves": tree.n_leaves}


def measured_peaks():
    """The measured peaks of this GPU pool (MEASURED_PEAKS.json beside
    this file), else the profiling recipe's fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return {"bf16_tflops": float(d["bf16_tflops"]), "bf16_tflops_sustained": float(d["bf16_tflops_sustained"]),
                "hbm_gbs": float(d["hbm_gbs"]), "source": "measured (MEASURED_PEAKS.json)"}
    except (OSError, KeyError, ValueError):
        return {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0,
                "source": "fallback (recipe: one earlier GB300 measurement)"}


# DRAM bytes (read + written) of one launch of the near-field kernel, from an
# ncu capture, keyed by (workload, right-hand sides, SHA-256 prefix of the
# kernel's source file and the headers it compiles with).  A changed kernel
# source matches no key, so the line then reports traffic as null until the
# kernel is captured again.
NEAR_TRAFFIC = {
    # profiles/k_gemm_ws_near_lshape_k16.md: 37,000,192 B read + 2,816 B written
    ("lshape_expsin_k16", 1, "d3b48934915bcaa5"): 37003008,
}

KERNEL_HEADERS = ("gemm.cuh", "slice_math.cuh", "bulk.cuh")


def kernel_source_key(fname="gemm_ws.cu"):
    import hashlib
    h = hashlib.sha256()
    for name in (fname,) + KERNEL_HEADERS:
        with open(os.path.join(ROOT, "paper_2211_14537_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def potential_error(V, plan, vals, idx, Vs):
    """Relative max-norm error at the sampled targets of the library's volume
    potential of the oracle's own leaf values (the potential alone, without the
    extension's conditioning)."""
    import torch
    nt = vals.shape[0] * vals.shape[2]
    fe = torch.tensor(np.ascontiguousarray(vals[:, 0, :].ravel()), dtype=torch.float64, device="cuda")
    v = torch.empty(nt, dtype=torch.float64, device="cuda")
    V.vpx_potential(plan, fe, v, None, stream=0)
    torch.cuda.synchronize()
    if V.vpx_sync_status(plan) != 0:
        raise RuntimeError("device status error in the potential check")
    return float(np.max(np.abs(v.cpu().numpy()[idx] - Vs)) / np.max(np.abs(Vs)))


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "gb300" else "gloo")
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, world)
        return
    if args.workload == "star-batch":
        run_batch(args, rank, world)
        return
    forms = ["fp64", "mixed"] if args.precision == "both" else [args.precision]
    res = {f: run_gpu(args, rank, world, f) for f in forms}
    errs, errs_e2e = {}, {}
    cpu = None
    if rank == 0 and world == 1:
        try:
            o = oracle_sample(res[forms[0]]["wl"], args.oracle_sample, lines=args.ext_mode == "lines",
                              one_core_s=0.0 if args.no_cpu_baseline else 5.0)
            idx, Vs = o["idx"], o["V"]
            for f in forms:
                # the potential of the oracle's own f^e (the metric's error), and
                # end to end from the stencil data, where the two sides' extension
                # fits (two backward-stable least-squares solutions) also differ
                errs[f] = potential_error(V_module(), res[f]["plan"], o["vals"], idx, Vs)
                errs_e2e[f] = float(np.max(np.abs(res[f]["v"][idx] - Vs)) / np.max(np.abs(Vs)))
            if not args.no_cpu_baseline:
                dt = o["seconds"]
                cpu = {"value": len(idx) / dt, "unit": UNIT, "cores": o["threads"], "kind": "oracle",
                       "sample": "direct-quadrature V at %d of %d leaf nodes (seeded) on %d threads, oracle "
                                 "tree+extension excluded, %.1f s" % (len(idx), res[forms[0]]["nt"], o["threads"], dt),
                       "extrapolated_full_s": res[forms[0]]["tg"] * dt / len(idx)}
                if o["one_core"]:
                    n1, t1 = o["one_core"]
                    cpu["one_core"] = {"value": n1 / t1, "unit": UNIT, "cores": 1,
                                       "sample": "%d targets spread evenly over the same sample, one thread, %.1f s"
                                                 % (n1, t1)}
        except Exception as e:   # noqa: BLE001 - report, do not hide the GPU number
            cpu = {"value": None, "error": repr(e)}
    # headline: the fastest form whose potential error against the oracle meets 1e-10
    ok = [f for f in forms if errs.get(f, 0.0) <= 1e-10]
    head = min(ok or forms, key=lambda f: res[f]["ms"])
    r = res[head]
    ms_max, tg_all = reduce_over_ranks(r["ms"], r["tg"], "cuda", world)   # replicas: every rank one tree
    value = tg_all / (ms_max * 1e-3)
    peaks = measured_peaks()
    method_flops = r["near_flops"] + 2.0 * r["K"] ** 2 * r["lc"]["near"] * args.nrhs   # 2K^4 + 2K^2 per pair
    near_s = r["near_ms"] * 1e-3
    if head == "mixed":
        tc = not os.environ.get("VPX_NO_TC")
        achieved = method_flops / near_s / 1e12
        peak = peaks["bf16_tflops"]
        key = (r["wl"].name, args.nrhs, kernel_source_key("gemm_ws.cu" if tc else "gemm_frag.cu"))
        roof = {"kernel": ("k_gemm_ws (near-field pass: exact bf16 slices on tcgen05, TMA tables, TMEM accumulators)"
                           if tc else "k_gemm_frag (near-field pass: exact bf16 slices on mma.sync)"),
                "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": NEAR_TRAFFIC.get(key), "traffic_unit": "bytes per launch (ncu dram__bytes read+write)",
                "work": "method flops 2K^4 + 2K^2 per near pair (%d pairs), per launch" % r["lc"]["near"],
                "peak_source": "bf16 dense burst, %s" % peaks["source"],
                "slice_products_tflops": 15 * r["near_flops"] / near_s / 1e12,
                "slice_products_note": "the 15 exact bf16 slice products per FP64-equivalent product the "
                                       "tensor pipe executes, per second"}
    else:
        achieved = method_flops / near_s / 1e12
        roof = {"kernel": "k_gemm_fp64 (near-field pass)", "bound": "alu", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "work": "method flops 2K^4 + 2K^2 per near pair, per launch",
                "peak_source": "nominal GB300 FP64 (recipe); an FMA probe measured 1.20"}
    ext_modes = None
    if not args.no_batch and args.nrhs == 1 and rank == 0:
        try:
            ext_modes = extension_modes(args)
        except Exception as e:   # noqa: BLE001 - the single-tree line stands on its own
            ext_modes = {"error": repr(e)}
    batch = None
    if not args.no_batch and args.nrhs == 1:
        try:
            batch = run_batch(args, rank, world, as_key=True)
        except Exception as e:   # noqa: BLE001 - the single-tree line stands on its own
            batch = {"error": repr(e)}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "strong" if args.workload == "disk-multi-rhs" else "weak",
        "vs_baseline": None, "dtype": "f64" if head == "fp64" else "bf16 (exact 8-bit slices) + f64",
        "data": "synthetic (seeded analytic source on the %s domain)" % DOMAIN_LABEL[args.workload],
        "config": {"workload": r["wl"].name, "description": r["wl"].description, "K": r["K"], "p": args.p,
                   "refine_tol": r["wl"].opts.refine_tol, "n_leaves": r["n_leaves"], "leaf_targets": r["nt"],
                   "boundary_targets": r["nb"], "stencil_points": r["ns"], "nrhs": args.nrhs,
                   "nrhs_all_ranks": MULTI_RHS_COLUMNS if args.workload == "disk-multi-rhs" else args.nrhs * world,
                   "precision": head, "near_pairs": r["lc"]["near"], "m2l_pairs": r["lc"]["m2l"],
                   "s2l_pairs": r["lc"]["s2l"], "m2t_pairs": r["lc"]["m2t"], "levels": r["lc"]["n_levels"],
                   "algorithmic_flops_per_rhs": algorithmic_flops(r["K"], args.p, r["n_leaves"], r["lc"]),
                   "l2": "flushed between timed steps (256 MB write, outside the events)",
                   "graph": "vpx_execute replays a captured CUDA graph",
                   "setup_s": round(r["setup_s"], 3), "parallelism": "replicas" if world > 1 else "single",
                   "autotune": {"passes_tuned": r["tune"][0], "passes_changed": r["tune"][1]},
                   "extension": "along lines" if args.ext_mode == "lines" else "universal stencil"},
        "forms": {f: {"value": res[f]["tg"] * world / (res[f]["ms"] * 1e-3), "ms_per_step": res[f]["ms"],
                      "median_ms_per_step": statistics.median(res[f]["times"]) if res[f].get("times") else None,
                      "rel_err_vs_oracle": errs.get(f), "rel_err_end_to_end": errs_e2e.get(f),
                      "pass_ms": {k: round(x, 5) for k, x in res[f]["pass_ms"].items()}}
                  for f in forms},
        "rel_err_vs_oracle": errs.get(head),
        "rel_err_note": "rel_err_vs_oracle: the library's potential of the oracle's own extended source at the "
                        "sampled targets; rel_err_end_to_end: from the stencil data, including the difference of "
                        "the two sides' extension fits",
        "roofline": roof,
        "gpu_launches": r["graph_kernels"] * args.steps,
        "e2e": {"value": r["tg"] * world / r["e2e_s"], "unit": UNIT,
                "h2d_bytes_per_step": 8 * r["ns"] * args.nrhs,
                "d2h_bytes_per_step": 8 * (r["nt"] + r["nb"]) * args.nrhs},
        "clocks": r["clocks"],
        "latency_floor_us": latency_floor_us() if rank == 0 else None,
    }
    if batch is not None:
        out["batch"] = batch
    if ext_modes is not None:
        out["extension_modes"] = ext_modes
    if cpu is not None:
        out["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(out), flush=True)


def extension_modes(args):
    """Cost of the extension along lines (Section 6.4) beside the universal
    stencil's and a potential (VFMM) call, on the starfish (K = 16, the star
    of the lines through its centre): CUDA events around vpx_extend and
    vpx_potential on device-resident data, L2 flushed before each call, median
    of 20 calls, both forms of the mixed plan."""
    import torch
    import workloads as W
    from paper_2211_14537_gb300 import vpx as V
    wl = W.starfish_gaussian(K=16)
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {"workload": wl.name, "precision": "mixed"}

    def timed(call):
        ts = []
        for i in range(23):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            call()
            with torch.cuda.stream(stream):
                e1.record(stream)
            torch.cuda.synchronize(dev)
            if i >= 3:
                ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    for mode, code in (("stencil", 0), ("lines", 1)):
        o = V.vpx_default_options(K=wl.opts.K, min_level=wl.opts.min_level, max_level=wl.opts.max_level,
                                  refine_tol=wl.opts.refine_tol, f_scale=wl.opts.f_scale, p=args.p,
                                  precision=V.VPX_PREC_MIXED, ext_mode=code)
        plan = V.vpx_plan_create(o, wl.domain, wl.sources[0])
        _, nt, ns, nb = plan.sizes()
        f = torch.tensor(wl.sources[0](plan.stencil_points()), dtype=torch.float64, device=dev)
        fe = torch.empty(nt, dtype=torch.float64, device=dev)
        v = torch.empty(nt, dtype=torch.float64, device=dev)
        out[mode + "_extension_ms"] = timed(lambda: V.vpx_extend(plan, f, fe, stream=stream))
        if mode == "stencil":
            out["potential_ms"] = timed(lambda: V.vpx_potential(plan, fe, v, None, stream=stream))
        if V.vpx_sync_status(plan) != 0:
            raise RuntimeError("device status error in the extension timing")
        out[mode + "_stencil_points"] = ns
    out["lines_over_stencil"] = out["lines_extension_ms"] / out["stencil_extension_ms"]
    out["lines_over_potential"] = out["lines_extension_ms"] / out["potential_ms"]
    return out


def V_module():
    from paper_2211_14537_gb300 import vpx as V
    return V


def run_reference(args, world):
    """The oracle as the reference arm: each step = direct-quadrature V at a
    bounded seeded sample of the leaf nodes of the workload named by
    --workload (the first tree of the batch)."""
    from oracle import oracle as O
    import workloads as W
    # the same workload as the GPU arm's line (for the batch, its first tree)
    wl = W.star_batch(1)[0] if args.workload == "star-batch" else workload(args.workload)
    tree = O.build_tree(wl.domain, wl.opts, wl.sources[0])
    pts, meta = O.stencil_points(tree, wl.domain)
    vals, _ = O.leaf_values(tree, wl.domain, wl.sources[0](pts)[:, None], meta)
    nodes = O.all_leaf_nodes(tree)
    rng = np.random.Generator(np.random.PCG64(2214))
    # per-step sample sized so that warm-up + timed steps take about 150 s of
    # oracle work whatever --steps / --warmup are (calibrated on 64 targets),
    # but at least 64 targets: the oracle parallelises over targets, and a
    # target's singular quadrature alone takes a large part of a second
    t0 = time.perf_counter()
    O.volume_potential(tree, vals, nodes[rng.choice(len(nodes), 64, replace=False)])
    per_target = (time.perf_counter() - t0) / 64
    budget_s = 150.0
    n = int(budget_s / (max(args.steps + args.warmup, 1) * per_target))
    n = max(64, min(n, 2500, len(nodes)))
    for _ in range(args.warmup):
        O.volume_potential(tree, vals, nodes[rng.choice(len(nodes), n, replace=False)])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.volume_potential(tree, vals, nodes[rng.choice(len(nodes), n, replace=False)])
    dt = time.perf_counter() - t0
    thr = O.lib().orc_max_threads()
    val = n * args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "K": wl.opts.K, "sample_targets_per_step": n},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": thr, "kind": "oracle",
                         "sample": "%d seeded leaf nodes per step (sized for about %.0f s of oracle work over "
                                   "the run), direct quadrature" % (n, budget_s)},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


if __name__ == "__main__":
    main()
