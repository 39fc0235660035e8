"""Benchmark: sketch-based influence maximisation (HyperFuseR, arXiv 2105.04023) on one GB300.

One step = one full seed selection (Algorithm 1: initial build, K greedy steps, reachability searches and the
error-adaptive rebuilds) with inputs resident in HBM.  Workloads (``--workload``):
  chunglu22_ic (default): directed Chung-Lu graph, n = 2^22, mean degree 16, degree exponent 2.1 (m = 56,688,349
      after merging duplicates), independent cascade p = 0.01, R = 512 uint8 registers, K = 100, eps_g = 0.02;
  rmat20_wc: R-MAT scale 20, edge factor 16 (m = 16,085,964), weighted cascade, R = 256, K = 50, eps_g = 0.01.

metric: sampled edge-simulation visits per second = (sum over every diffusion sweep of the step of
|{(u,v): v in L}| * R) / step time.  This counts the work of the paper's Jacobi sweeps; the kernels skip the
(edge, simulation) pairs that are not live, so the executed live pairs per second and the modelled bytes per second
of the sweep kernels are reported beside it.  The end-to-end seconds per K-seed selection are reported too.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
Under torchrun every rank runs its own replica (the workload does not shard: replicas only) and rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sampled edge-sim visits/sec"
UNIT = "edge-sim visits/s"
WORKLOADS = {
    "chunglu22_ic": "Chung-Lu n=2^22, mean degree 16, degree exponent 2.1, independent cascade p=0.01",
    "rmat20_wc": "R-MAT scale 20, edge factor 16 (a,b,c,d = .57,.19,.19,.05), weighted cascade",
    "chunglu20_ic": "Chung-Lu n=2^20, mean degree 16, degree exponent 2.1, independent cascade p=0.01 (profiling case)",
}
# the oracle sample of one step: the first Jacobi sweep over every ORACLE_STRIDE-th row
ORACLE_STRIDE = {"chunglu22_ic": 32, "rmat20_wc": 1, "chunglu20_ic": 8}


def load_workload(name: str):
    from synth import workloads

    return getattr(workloads, name)(cache=True)


def golden_record(name: str) -> dict | None:
    """The oracle's recorded whole-run times for this workload (written with its golden file, see tests/golden)."""
    path = os.path.join(ROOT, "tests", "golden", f"{name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        g = json.load(f)
    return {"build_s": g["build"].get("seconds"), "select_s": g["select"].get("seconds"),
            "select_visits": g["select"]["visits"], "host": g.get("host", "recorded when the golden file was written")}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) < 9:
                continue
            for name, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def aggregate(seconds: float, units: float, world: int) -> tuple[float, float]:
    """Replica timing: the job takes as long as the slowest rank and processes the units of all ranks."""
    if world == 1:
        return seconds, units
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def max_over_ranks(x: float, world: int) -> float:
    return aggregate(x, 0.0, world)[0]


def oracle_sample(prob, stride: int = 1) -> tuple[float, int, float, int]:
    """The CPU oracle as it stands on a bounded sample: the first Jacobi sweep of the workload's build over every
    `stride`-th row (rows u with u mod stride = 0 keep their out-edges, the others have none in the sample;
    thresholds are those of the whole graph), so that the sample has the graph's degree mix.  Returns
    (visits/s, visits, seconds, rows sampled)."""
    import oracle

    g = prob.graph
    T, ok = oracle.edge_thresholds(g.n, g.xadj, g.adj, prob.model, p=prob.p)
    keep_row = (np.arange(g.n) % stride) == 0
    deg = np.diff(g.xadj)
    keep_edge = np.repeat(keep_row, deg)
    xadj = np.zeros(g.n + 1, np.int64)
    np.cumsum(np.where(keep_row, deg, 0), out=xadj[1:])
    adj = np.ascontiguousarray(g.adj[keep_edge])
    X, Y = oracle.sim_words(prob.seed, prob.R)
    M = oracle.init_registers(g.n, prob.R, Y)
    t = time.perf_counter()
    _, visits, _ = oracle.simulate(g.n, xadj, adj, T[keep_edge], ok[keep_edge], prob.R, X, M, max_sweeps=1)
    dt = time.perf_counter() - t
    return visits / dt, visits, dt, int(keep_row.sum())


def run_reference(args, world, rank):
    if rank != 0:
        return
    prob = load_workload(args.workload)
    stride = ORACLE_STRIDE[args.workload]
    vals = []
    visits = rows = 0
    for i in range(args.warmup + args.steps):
        v, visits, dt, rows = oracle_sample(prob, stride)
        if i >= args.warmup:
            vals.append(dt)
    total = sum(vals)
    value = visits * len(vals) / total
    sample = (f"per step: the first Jacobi sweep of the build over every {stride}-th row of the full graph "
              f"({rows} rows, {visits} edge-simulation visits)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": config(prob, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "recorded_whole_run": golden_record(args.workload)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config(prob, args):
    g = prob.graph
    return {"workload": WORKLOADS[args.workload], "name": args.workload,
            "n": g.n, "m": g.m, "R": prob.R, "K": prob.K, "eps_g": prob.eps_g, "eps_l": prob.eps_l,
            "eps_c": prob.eps_c, "seed": prob.seed, "parallelism": f"replicas{args.gpus}",
            "l2": f"flushed between steps (256 MiB write); registers 3 x {g.n * prob.R >> 20} MiB exceed L2"}


def run_ours(args, world, rank, local):
    import torch

    import paper_2105_04023_gb300 as im

    torch.cuda.set_device(local)
    from paper_2105_04023_gb300 import build as b

    b.build()
    prob = load_workload(args.workload)
    if args.k:
        prob.K = args.k
    g = prob.graph
    prm = im.params(R=prob.R, K=prob.K, eps_g=prob.eps_g, eps_l=prob.eps_l, eps_c=prob.eps_c, seed=prob.seed)
    dev_graph = im.Graph.from_synth(g, prob.model, prob.p, device=f"cuda:{local}")
    # pinned host copies for the end-to-end leg
    hx = torch.from_numpy(np.ascontiguousarray(g.xadj)).pin_memory()
    ha = torch.from_numpy(np.ascontiguousarray(g.adj)).pin_memory()
    host_graph = im.Graph(g.n, hx.numpy(), ha.numpy(), prob.model, prob.p)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")
    ctx = im.Context(local)
    # set-up (untimed): the autotuner picks this graph class's launch shapes (results do not depend on them)
    tuning = ctx.im_autotune(dev_graph, prm) if not args.no_autotune else None

    seeds_ref = None
    for _ in range(args.warmup):
        out = ctx.im_select_seeds(dev_graph, prm, trace=False)
        seeds_ref = out["seeds"]
    torch.cuda.synchronize()

    # timed region: device-resident inputs
    ctx.set_timing(True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    dev_ms, visits, launches, prop_ms, prop_bytes, prop_launches, wall = [], 0, 0, 0.0, 0, 0, []
    pairs = first_bytes = first_launches = 0
    first_ms = 0.0
    phases = {"sweep_ms": 0.0, "scan_ms": 0.0, "bfs_ms": 0.0, "init_ms": 0.0}
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = ctx.im_select_seeds(dev_graph, prm, trace=False)
        wall.append(time.perf_counter() - t)
        st = ctx.stats()
        dev_ms.append(st["total_ms"])
        visits += st["visits"]
        launches += st["kernel_launches"]
        prop_ms += st["prop_ms"]
        prop_bytes += st["prop_bytes"]
        prop_launches += st["prop_launches"]
        pairs += st["live_pairs"]
        first_bytes += st["first_bytes"]
        first_ms += st["first_ms"]
        first_launches += st["first_launches"]
        for k in phases:
            phases[k] += st[k]
        if seeds_ref is not None:
            assert out["seeds"].tolist() == seeds_ref.tolist(), "seed sets differ between steps"
        seeds_ref = out["seeds"]
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ctx.set_timing(False)
    total_s, all_visits = aggregate(sum(dev_ms) / 1000.0, float(visits), world)
    value = all_visits / total_s

    # end-to-end through the public API with host inputs (copies inside the timed call)
    e2e_ms = []
    e2e_visits = 0
    for _ in range(max(1, args.steps)):
        flush.fill_(1)
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = ctx.im_select_seeds(host_graph, prm, trace=False)
        e2e_ms.append(1000 * (time.perf_counter() - t))
        e2e_visits += ctx.stats()["visits"]
    e2e_s, e2e_all = aggregate(sum(e2e_ms) / 1000.0, float(e2e_visits), world)

    hbm, peak_kind = peaks()
    # the dominant kernel: the first sweep of every diffusion (k_first), timed by CUDA events around its launches
    achieved = first_bytes / (first_ms / 1000.0) / 1e9 if first_ms > 0 else None
    sweeps_achieved = prop_bytes / (prop_ms / 1000.0) / 1e9 if prop_ms > 0 else None
    traffic = None
    tpath = os.path.join(ROOT, "profiles", f"k_first_{args.workload}_traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            traffic = json.load(f).get("dram_bytes_per_launch")
    if rank == 0:
        stride = ORACLE_STRIDE[args.workload]
        cpu_v, cpu_visits, cpu_dt, cpu_rows = oracle_sample(prob, stride)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": config(prob, args),
            "im_seconds_per_K_seeds": total_s / args.steps,
            "step_ms": {"p50": float(np.percentile(dev_ms, 50)), "p99": float(np.percentile(dev_ms, 99))},
            "visits_per_step": visits // args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
                         "peak_kind": f"{peak_kind} copy bandwidth (sustained copy; of measured)",
                         "kernel": "k_first: the first sweep of every diffusion (initial registers read from the "
                                   "problem's table, every sparse pair merged, every row written to both buffers "
                                   "with its change mask and register sum)",
                         "bytes_per_launch": first_bytes / max(first_launches, 1),
                         "launches": first_launches, "ms": first_ms,
                         "all_sweep_kernels": {"achieved": sweeps_achieved,
                                               "frac": (sweeps_achieved / hbm) if sweeps_achieved else None,
                                               "bytes": prop_bytes, "ms": prop_ms, "launches": prop_launches}},
            "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first Jacobi sweep of the build over every {stride}-th row of the full "
                                       f"graph ({cpu_rows} rows, {cpu_visits} visits, {cpu_dt:.1f} s)",
                             "recorded_whole_run": golden_record(args.workload)},
            "e2e": {"value": e2e_all / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(g.xadj.nbytes + g.adj.nbytes), "d2h_bytes_per_step": 4 * prob.K + 8,
                    "ms_per_step": 1000 * e2e_s / max(1, args.steps)},
            "gpu_launches": launches,
            "clocks": clk,
            "tuning": tuning,
            "executed": {"live_pairs_per_step": pairs // args.steps,
                         "live_pairs_per_s": pairs / (sum(dev_ms) / 1000.0),
                         "modelled_sweep_bytes_per_s": achieved * 1e9 if achieved else None,
                         "note": "value counts the Jacobi edge-simulation visits of Algorithm 2 (every edge into L "
                                 "times R); the kernels touch only the live (edge, simulation) pairs, counted here, "
                                 "and move the modelled bytes of roofline.achieved"},
            "wall_ms_per_step": 1000 * sum(wall) / len(wall),
            "phase_ms_per_step": {k: v / args.steps for k, v in phases.items()},
        }
        print(json.dumps(line), flush=True)
    ctx.close()


def run_build(args, local):
    """Sketch builds of the workload (initial registers + diffusion to the fixpoint), one per step."""
    import torch

    import paper_2105_04023_gb300 as im
    from paper_2105_04023_gb300 import build as b

    torch.cuda.set_device(local)
    b.build()
    prob = load_workload(args.workload)
    g = prob.graph
    graph = im.Graph.from_synth(g, prob.model, prob.p, device=f"cuda:{local}")
    prm = im.params(R=prob.R, seed=prob.seed)
    ctx = im.Context(local)
    for _ in range(args.warmup):
        ctx.im_build_sketches(graph, prm).close()
    ctx.set_timing(True)
    rows = []
    for _ in range(args.steps):
        sk = ctx.im_build_sketches(graph, prm)
        st = ctx.stats()
        sk.close()
        rows.append(st)
    hbm, _ = peaks()
    prop_ms = sum(r["prop_ms"] for r in rows)
    prop_bytes = sum(r["prop_bytes"] for r in rows)
    visits = sum(r["visits"] for r in rows)
    total_ms = sum(r["total_ms"] for r in rows)
    first_ms = sum(r["first_ms"] for r in rows)
    first_bytes = sum(r["first_bytes"] for r in rows)
    out = {"mode": "build", "workload": WORKLOADS[args.workload], "variant": os.environ.get("IM_PROP_VARIANT", "0"),
           "steps": args.steps, "first_ms": first_ms / args.steps, "first_bytes": first_bytes // args.steps,
           "first_GBps": first_bytes / first_ms / 1e6 if first_ms > 0 else None,
           "build_ms": total_ms / args.steps, "prop_ms": prop_ms / args.steps, "sweeps": rows[0]["sweeps"],
           "visits": visits // args.steps, "prop_GBps": prop_bytes / prop_ms / 1e6,
           "frac": prop_bytes / prop_ms / 1e6 / hbm, "visits_per_s": visits / (total_ms / 1000),
           "launches": rows[0]["kernel_launches"]}
    print(json.dumps(out), flush=True)
    ctx.close()


def run_mc(args, local):
    """The influence scorer on the bench workload: the 50 seeds the select picks, scored by sample-then-diffuse
    Monte Carlo over --mc-samples mt19937-sampled graphs (Section 4's way of scoring seed sets), timed with CUDA
    events; the oracle scores one sample on one core for comparison."""
    import torch

    import paper_2105_04023_gb300 as im
    from paper_2105_04023_gb300 import build as b

    torch.cuda.set_device(local)
    b.build()
    prob = load_workload(args.workload)
    g = prob.graph
    graph = im.Graph.from_synth(g, prob.model, prob.p, device=f"cuda:{local}")
    ctx = im.Context(local)
    sel = ctx.im_select_seeds(graph, im.params(R=prob.R, K=prob.K, eps_g=prob.eps_g, eps_l=prob.eps_l,
                                               eps_c=prob.eps_c, seed=prob.seed), trace=False)
    seeds = sel["seeds"]
    N = args.mc_samples
    for _ in range(args.warmup):
        ctx.im_influence_mc(graph, seeds, N, 77)
    ctx.set_timing(True)
    times, sig = [], None
    clocks = ClockSampler(local)
    clocks.start()
    for i in range(args.steps):
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        sig, reach = ctx.im_influence_mc(graph, seeds, N, 77)
        c.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(c) / 1000.0)
    clk = clocks.stop()
    st = ctx.stats()
    t = sum(times) / len(times)
    import oracle

    t0 = time.perf_counter()
    _, one = oracle.influence_mc(g.n, g.xadj, g.adj, prob.model, prob.p, seeds, 1, 77)
    t_cpu = time.perf_counter() - t0
    out = {"mode": "mc", "workload": f"{WORKLOADS[args.workload]} (the {prob.K} seeds of the select)", "clocks": clk,
           "samples": N, "steps": args.steps, "s_per_call": t, "samples_per_s": N / t,
           "edge_draws_per_s": g.m * N / t, "sigma_mc": sig, "sigma_sketch_samples": sel["sigma_final"],
           "mc_stderr": float(np.std(reach.astype(np.float64), ddof=1) / np.sqrt(N)),
           "sample_phase_ms": st["init_ms"], "search_phase_ms": st["bfs_ms"], "search_levels": st["bfs_levels"],
           "cpu_baseline": {"samples_per_s": 1.0 / t_cpu, "cores": 1, "kind": "oracle",
                            "sample": "sample 0 of the same scoring, drawn and searched on one core"},
           "oracle_sample0_matches": int(one[0]) == int(reach[0])}
    print(json.dumps(out), flush=True)
    ctx.close()


def run_batch(args, local):
    """The batched workload: many R-MAT graphs of uneven sizes, models and R, all selected together (one launch per
    phase for all of them) versus one graph per call on the same GPU, with identical seed sets required."""
    import torch

    import paper_2105_04023_gb300 as im
    from paper_2105_04023_gb300 import build as b
    from synth import graphs, workloads

    torch.cuda.set_device(local)
    b.build()
    probs = []
    for i in range(args.batch_graphs):
        scale, ef, model, p, R = workloads.batch_spec(i)
        scale = min(scale, args.batch_max_scale)
        g = graphs.cached(lambda: graphs.rmat(scale, ef, seed=1000 + i), f"rmat_s{scale}_ef{ef}_seed{1000 + i}")
        probs.append(workloads.Problem(g, model, p, R=R, K=20, eps_g=0.01, seed=1000 + i))
    gs = [im.Graph.from_synth(p.graph, p.model, p.p, device=f"cuda:{local}") for p in probs]
    prms = [im.params(R=p.R, K=p.K, eps_g=p.eps_g, eps_l=p.eps_l, seed=p.seed) for p in probs]
    ctx = im.Context(local)
    # autotuning: one graph of every (R, degree class) times the candidate launch shapes (untimed set-up)
    t_tune = time.perf_counter()
    classes = {}
    for p, g, prm in zip(probs, gs, prms):
        dc = 0 if p.graph.m < p.graph.n else int(np.log2(p.graph.m // p.graph.n)) + 1
        classes.setdefault((p.R, dc), (g, prm))
    tuning = {f"R{k[0]}_d{k[1]}": ctx.im_autotune(g, prm) for k, (g, prm) in sorted(classes.items())}
    t_tune = time.perf_counter() - t_tune
    ctx.im_select_seeds_batch(gs[:8], prms[:8])  # warm-up
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t = time.perf_counter()
    batch = ctx.im_select_seeds_batch(gs, prms)
    t_batch = time.perf_counter() - t
    st_b = ctx.stats()
    t = time.perf_counter()
    plain = []
    visits_plain = 0
    for g, prm in zip(gs, prms):
        plain.append(ctx.im_select_seeds(g, prm, trace=False))
        visits_plain += ctx.stats()["visits"]
    t_plain = time.perf_counter() - t
    clk = clocks.stop()
    same = all(a["seeds"].tolist() == c["seeds"].tolist() and a["sigma_final"] == c["sigma_final"]
               for a, c in zip(batch, plain))
    m_total = sum(p.graph.m for p in probs)
    out = {"mode": "batch", "graphs": len(probs), "edges_total": m_total, "max_scale": args.batch_max_scale,
           "batched_s": t_batch, "plain_s": t_plain, "speedup": t_plain / t_batch,
           "batched_graphs_per_s": len(probs) / t_batch, "plain_graphs_per_s": len(probs) / t_plain,
           "batched_visits_per_s": st_b["visits"] / t_batch, "plain_visits_per_s": visits_plain / t_plain,
           "identical_seed_sets": same, "batched_kernel_launches": st_b["kernel_launches"], "clocks": clk,
           "autotune_s": t_tune, "tuning": {k: (v["first_sweep_blocks"], v["stream_push"]) for k, v in tuning.items()}}
    print(json.dumps(out), flush=True)
    ctx.close()


def run_serve(args, local):
    """The served workload: a resident pool of 64 R-MAT graphs (scale 12 + i mod 9, edge factor 16, weighted
    cascade) and a Poisson stream of queries (K uniform in 5..100, R in {64, 256}, graph uniform over the pool, each
    query with its own run seed unless --serve-shared-seed); admission by a 120 GB HBM budget; continuous batching.
    The arrival rate is 0.8 x the saturation rate measured by a closed-loop pre-run.  Reported with the clocks of
    the timed stream: p50/p99 latency, queries/s, the share of queries started from a kept first diffusion, and, on
    a sample of the same queries answered one at a time through im_select_seeds, the sequential queries/s and
    whether every sampled result is identical."""
    import torch

    import paper_2105_04023_gb300 as im
    from paper_2105_04023_gb300 import build as b
    from synth import graphs, workloads

    torch.cuda.set_device(local)
    b.build()
    pool = []
    for i in range(64):
        scale = min(12 + (i % 9), args.serve_max_scale)
        pool.append(graphs.cached(lambda: graphs.rmat(scale, 16, seed=2000 + i), f"rmat_s{scale}_ef16_seed{2000 + i}"))
    Q = workloads.serve_queries(count=args.serve_queries + args.serve_saturation, pool=64, seed=5)
    ctx = im.Context(local)
    srv = im.Server(ctx, hbm_budget_bytes=120 << 30, max_active=256)
    gdev = [im.Graph.from_synth(g, im.IM_WC, device=f"cuda:{local}") for g in pool]
    gids = [srv.im_server_add_graph(g) for g in gdev]

    def prm(k):
        q = Q[k]
        seed = 7 if args.serve_shared_seed else 100000 + k
        return im.params(R=int(q[2]), K=int(q[1]), eps_g=0.01, eps_l=0.3, seed=seed)

    def drain(tickets):
        while tickets:
            srv.im_server_step()
            for tk in list(tickets):
                if srv.im_server_poll(tk) is not None:
                    tickets.discard(tk)

    # closed loop: the first queries submitted at once give the saturation rate
    n_sat = args.serve_saturation
    t0 = time.perf_counter()
    drain({srv.im_server_submit(gids[int(Q[k, 0])], prm(k)) for k in range(n_sat)})
    qps_sat = n_sat / (time.perf_counter() - t0)
    hits0 = srv.im_server_info()["build_hits"]
    lam = 0.8 * qps_sat
    # open loop: Poisson arrivals at lam
    ks = list(range(n_sat, len(Q)))
    arrive = np.cumsum(Q[n_sat:, 3]) / lam
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    pending, arrivals, results, lat = set(), {}, {}, []
    i = 0
    while i < len(ks) or pending:
        now = time.perf_counter() - t0
        while i < len(ks) and arrive[i] <= now:
            t = srv.im_server_submit(gids[int(Q[ks[i], 0])], prm(ks[i]))
            arrivals[t] = t0 + arrive[i]
            pending.add(t)
            results[t] = ks[i]
            i += 1
        if pending:
            srv.im_server_step()
            now2 = time.perf_counter()
            for t in list(pending):
                r = srv.im_server_poll(t)
                if r is not None:
                    lat.append(now2 - arrivals[t])
                    results[t] = (results[t], r)
                    pending.discard(t)
        elif i < len(ks):
            time.sleep(max(0.0, min(0.001, arrive[i] - (time.perf_counter() - t0))))
    span = time.perf_counter() - t0
    clk = clocks.stop()
    hits = srv.im_server_info()["build_hits"] - hits0
    # a sample of the same queries one at a time through the plain call
    sample = list(results.items())[: args.serve_sequential]
    t1 = time.perf_counter()
    same = True
    for t, (k, r) in sample:
        alone = ctx.im_select_seeds(gdev[int(Q[k, 0])], prm(k), trace=False)
        same = same and alone["seeds"].tolist() == r["seeds"].tolist() and alone["sigma_final"] == r["sigma_final"]
    t_seq = time.perf_counter() - t1
    lat_ms = np.array(lat) * 1000
    out = {"mode": "serve", "queries": len(ks), "pool_graphs": 64, "pool_max_scale": args.serve_max_scale,
           "seeds": "shared (one run seed)" if args.serve_shared_seed else "one run seed per query",
           "saturation_queries": n_sat, "saturation_qps": qps_sat, "lambda_qps": lam, "served_qps": len(ks) / span,
           "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
           "kept_diffusion_hit_rate": hits / len(ks),
           "sequential_sample": len(sample), "sequential_qps": len(sample) / t_seq,
           "identical_seed_sets": same, "hbm_budget_gb": 120, "clocks": clk}
    print(json.dumps(out), flush=True)
    srv.close()
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="chunglu22_ic", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="select", choices=["select", "build", "batch", "serve", "mc"],
                    help="build: sketch builds only (for profiling); batch: the 256-graph batched workload; "
                         "serve: the query stream on a resident graph pool; mc: the Monte-Carlo influence scorer")
    ap.add_argument("--mc-samples", type=int, default=1024)
    ap.add_argument("--k", type=int, default=0, help="override the workload's K (profiling runs)")
    ap.add_argument("--no-autotune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--batch-graphs", type=int, default=256)
    ap.add_argument("--batch-max-scale", type=int, default=18)
    ap.add_argument("--serve-queries", type=int, default=10000)
    ap.add_argument("--serve-saturation", type=int, default=200, help="queries of the closed-loop pre-run")
    ap.add_argument("--serve-sequential", type=int, default=200, help="queries re-run one at a time")
    ap.add_argument("--serve-max-scale", type=int, default=20)
    ap.add_argument("--serve-shared-seed", action="store_true", help="one run seed for every query")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.mode == "build":
        run_build(args, local)
    elif args.mode == "batch":
        run_batch(args, local)
    elif args.mode == "serve":
        run_serve(args, local)
    elif args.mode == "mc":
        run_mc(args, local)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
