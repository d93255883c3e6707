"""Host logic of the multi-rank benchmark, on CPU: the size-balanced share of
the batch's trees per rank, and the reduction of time (max) and work (sum)
over two gloo ranks."""
import os
import socket
import tempfile

import pytest

import bench


def test_shard_by_size_covers_every_tree_once_and_balances():
    sizes = [int(64 * 4 ** (2 + (7 * i) % 5)) for i in range(32)]   # uneven, like the star batch
    for world in (1, 2, 3, 4, 8):
        parts = bench.shard_by_size(sizes, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        # largest-first greedy: no rank exceeds the mean by more than one tree
        assert max(loads) <= sum(sizes) / world + max(sizes)
    assert bench.shard_by_size([5, 5, 5], 2) == [[0, 2], [1]]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, units = bench.reduce_over_ranks(1.5 + rank, 100 * (rank + 1), "cpu", world)
        with open(os.path.join(out_dir, "r%d" % rank), "w") as fh:
            fh.write("%r %r" % (ms, units))
    finally:
        dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(2, _free_port(), d), nprocs=2, join=True)
        for r in range(2):
            with open(os.path.join(d, "r%d" % r)) as fh:
                ms, units = fh.read().split()
            assert float(ms) == 2.5 and float(units) == 300.0


def test_reduce_on_one_rank_is_identity():
    assert bench.reduce_over_ranks(3.0, 7, "cpu", 1) == (3.0, 7.0)


@pytest.mark.parametrize("wl_name", ["lshape", "starfish", "exterior", "disk-multi-rhs", "doubly-connected"])
def test_bench_line_carries_the_contract_keys(monkeypatch, capsys, wl_name):
    """bench.main() on one rank, the GPU run and the oracle sample replaced by
    fixed results: one JSON line with the keys of the benchmark contract."""
    import json
    import sys
    import numpy as np

    def fake_run_gpu(args, rank, world, prec):
        return dict(plan=prec, wl=bench.workload(args.workload), ms=0.2 if prec == "mixed" else 1.5, setup_s=0.6,
                    tg=184832, nt=182272, nb=2560, ns=129619, n_leaves=712,
                    lc={"near": 4900, "m2l": 14104, "s2l": 822, "m2t": 1112, "n_levels": 7},
                    pass_ms={"near": 0.05}, near_flops=2.0 * 16 ** 4 * 4900, near_ms=0.05, clocks={"sm_mhz": 2070.0},
                    e2e_s=3e-4, v=np.ones(182272), K=16, graph_kernels=24, tune=(7, 0), times=[0.2, 0.21, 0.19])

    monkeypatch.setattr(bench, "run_gpu", fake_run_gpu)
    monkeypatch.setattr(bench, "oracle_sample",
                        lambda wl, n, **k: {"vals": None, "idx": np.arange(10), "V": np.ones(10), "seconds": 1.0,
                                            "threads": 16, "one_core": (4, 2.0), "n_leaves": 712})
    # the potential check of the oracle's own f^e: the FP64 form exact, the mixed form within 1e-10
    monkeypatch.setattr(bench, "potential_error", lambda V, plan, vals, idx, Vs: 3e-11 if plan == "mixed" else 1e-15)
    monkeypatch.setattr(bench, "V_module", lambda: None)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", wl_name, "--no-batch"])
    bench.main()
    d = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
              "gpu_launches", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["warmup"] >= 3 and d["config"]["workload"]
    assert d["config"]["extension"] == "universal stencil"
    assert d["value"] == pytest.approx(184832 / 0.2e-3)                      # the faster form that meets 1e-10
    assert set(d["roofline"]) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}
    assert d["roofline"]["frac"] == pytest.approx(d["roofline"]["achieved"] / d["roofline"]["peak"])
    # the method's own work, 2K^4 + 2K^2 per near pair, over the near pass time; the peak is the measured one
    assert d["roofline"]["achieved"] == pytest.approx(4900 * (2 * 16 ** 4 + 2 * 256) / 0.05e-3 / 1e12)
    assert d["roofline"]["peak"] == pytest.approx(bench.measured_peaks()["bf16_tflops"])
    # traffic only from a capture of this kernel source (and none for a source no capture covers)
    key = (d["config"]["workload"], 1, bench.kernel_source_key("gemm_ws.cu"))
    assert d["roofline"]["traffic"] == bench.NEAR_TRAFFIC.get(key)
    assert d["rel_err_vs_oracle"] == pytest.approx(3e-11)
    assert d["forms"]["mixed"]["rel_err_end_to_end"] == 0.0
    assert set(d["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert d["e2e"]["h2d_bytes_per_step"] == 8 * 129619 and d["gpu_launches"] == 24 * d["steps"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 16
    assert d["cpu_baseline"]["one_core"]["value"] == 2.0 and d["cpu_baseline"]["one_core"]["cores"] == 1
    assert d["cpu_baseline"]["extrapolated_full_s"] == pytest.approx(184832 / 10.0)
    fl = d["config"]["algorithmic_flops_per_rhs"]
    P = d["config"]["p"] + 1
    assert fl["near"] == 4900 * (2 * 16 ** 4 + 2 * 256) and fl["m2l"] == 8 * P ** 2 * 14104
    assert fl["total"] == sum(v for k, v in fl.items() if k != "total")
    assert d["forms"]["mixed"]["median_ms_per_step"] == pytest.approx(0.2)
    assert "latency_floor_us" in d                                             # None without a GPU
    assert d["config"]["workload"] == bench.workload(wl_name).name
    assert bench.DOMAIN_LABEL[wl_name] in d["data"]
    assert d["scaling"] == ("strong" if wl_name == "disk-multi-rhs" else "weak")


def test_plan_options_of_the_bench(monkeypatch):
    """The options bench.py builds its plans from: the default line keeps the
    universal-stencil extension; --ext-mode lines selects the line extension."""
    import sys
    from paper_2211_14537_gb300 import vpx as V
    for argv, mode in ((["bench.py"], 0), (["bench.py", "--ext-mode", "lines"], 1)):
        monkeypatch.setattr(sys, "argv", argv)
        args = bench.parse()
        wl = bench.workload(args.workload)
        for prec, code in (("mixed", V.VPX_PREC_MIXED), ("fp64", V.VPX_PREC_FP64)):
            o = bench.plan_options(V, wl, args, prec)
            assert (o.K, o.p, o.precision, o.max_rhs, o.ext_mode, o.rbf_eps) == (16, args.p, code, 1, mode, 0.0)
            assert o.refine_tol == wl.opts.refine_tol and o.max_level == wl.opts.max_level


@pytest.mark.parametrize("world", [1, 2, 3, 5, 8])
def test_rhs_blocks_cover_every_column_once(world):
    """The 64 right-hand sides of the multi-RHS workload split into
    contiguous blocks whose sizes differ by at most one."""
    blocks = [bench.rhs_block(64, r, world) for r in range(world)]
    assert sum(blocks, []) == list(range(64))
    sizes = [len(b) for b in blocks]
    assert max(sizes) - min(sizes) <= 1


def test_reference_arm_follows_the_workload(monkeypatch, capsys):
    """bench.py --impl reference times the oracle on the workload the GPU arm
    names (here the multi-RHS disk, with the oracle's potential replaced by a
    fast stand-in), and prints the reference line's keys."""
    import json
    import sys
    import numpy as np
    from oracle import oracle as O
    monkeypatch.setattr(O, "volume_potential", lambda tree, vals, pts, *a: np.zeros((len(pts), 1)))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "disk-multi-rhs",
                                      "--steps", "2", "--warmup", "1"])
    bench.main()
    d = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["config"]["workload"] == bench.workload("disk-multi-rhs").name
    assert d["steps"] == 2 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_traffic_key_follows_the_kernel_and_its_headers(tmp_path, monkeypatch):
    """The near kernel's traffic figure is keyed on its source and the headers
    it compiles with: changing either leaves the bench line without one."""
    import shutil
    src = tmp_path / "paper_2211_14537_gb300" / "csrc"
    src.mkdir(parents=True)
    for name in ("gemm_ws.cu",) + bench.KERNEL_HEADERS:
        shutil.copy(os.path.join(bench.ROOT, "paper_2211_14537_gb300", "csrc", name), src / name)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    k0 = bench.kernel_source_key("gemm_ws.cu")
    with open(src / "slice_math.cuh", "a") as fh:
        fh.write("\n")
    k1 = bench.kernel_source_key("gemm_ws.cu")
    with open(src / "gemm_ws.cu", "a") as fh:
        fh.write("\n")
    k2 = bench.kernel_source_key("gemm_ws.cu")
    assert len({k0, k1, k2}) == 3
    assert all(k[2] != k1 and k[2] != k2 for k in bench.NEAR_TRAFFIC)
