#!/usr/bin/env python3
"""Benchmark of the BigGraphVis hot path on one GB300 (or N replicas).

A step is one pass of the whole hot path over the workload with its inputs
resident in HBM: degree sketch -> community rounds -> supergraph -> initial
positions -> ForceAtlas2 iterations.  Each step is timed on the device with
CUDA events on the launching stream; L2 is flushed (a 256 MiB write) before
every timed step.  `value` is edges per second of whole steps (m * N / the
slowest rank's mean step time).  `e2e` repeats the step through
bgv_layout_host from pinned host memory (host-to-device copy of the edges and
device-to-host copy of the layout inside the timed region), after one untimed
call of its own; its timed calls alternate with the first timed steps, so both
run under the same clocks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rmat22x]
    python bench.py --impl reference ...   # the CPU oracle, bounded sample

Under torchrun (N > 1) every rank lays out its own replica of the workload on
its own GPU (the path needs no exchange between GPUs); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import graphgen  # noqa: E402

METRIC = "edges/s streamed (sketch+community), FA2 iters/s, % of HBM/FP32 peak"
FALLBACK_HBM_GBS = 6800.0      # the profiling recipe's fallback when no measured peak is on file
FALLBACK_SM_MAX_MHZ = 2070.0
FP32_LANES_PER_SM = 128
FLOPS_PER_INTERACTION = 12     # dx, dy, d2 (3), division, k*m*M (2), two FMAs (4)


def hbm_peak():
    """(GB/s, source) of the HBM roofline: the measured copy bandwidth of
    MEASURED_PEAKS.json at the repository root, else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def fp32_peak_tflops(sms, mhz):
    """FP32 FMA peak: SMs x 128 lanes x 2 flops x clock."""
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


WORKLOADS = {
    "rmat20": dict(desc="R-MAT scale 20 (1,048,576 node ids), 10,000,000 unique edges, a,b,c,d=.57,.19,.19,.05, "
                        "shuffled int32 edge list", rows=4, width=65536, passes=3, threshold=0, growth=2,
                   iterations=500),
    "sbm16": dict(desc="planted partition, 10,000 nodes in 16 communities, p_in=0.01, p_out=0.0002, seed 1",
                  rows=4, width=4096, passes=3, threshold=64, growth=2, iterations=200),
    "rmat22x": dict(desc="R-MAT scale 22 restricted to 3,200,000 nodes, 34,000,000 unique edges, "
                         "a,b,c,d=.45,.22,.22,.11", rows=4, width=65536, passes=3, threshold=0, growth=2,
                    iterations=500),
    "lnpp1m": dict(desc="precision form: ForceAtlas2 on the whole 1,000,000-node, 8,000,000-edge planted "
                        "partition (256 communities of lognormal(8, 1) size), nodes coloured by their streamed "
                        "community", rows=4, width=65536, passes=3, threshold=0, growth=2, iterations=500,
                   whole=True),
    "batch512": dict(desc="batching form: 512 independent planted-partition graphs, node counts log-uniform in "
                          "[1,000, 200,000], 4 to 64 communities of lognormal(0, 0.5) size, average degree 10, "
                          "80% of edges inside communities", rows=4, width=4096, passes=3, threshold=0, growth=2,
                     iterations=300, batched=True),
}


# ---------------------------------------------------------------- helpers
def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def aggregate_throughput(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput of `world` replicas that each process
    `units_per_rank` units per step, at the slowest rank's step time."""
    return units_per_rank * world / (ms_max * 1e-3)


class Dist:
    def __init__(self):
        self.rank, self.world, self.local = dist_env()
        self.pg = None
        if self.world > 1:
            import torch.distributed as td
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            td.init_process_group("gloo", rank=self.rank, world_size=self.world)
            self.pg = td

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed
    region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpus):
        self.gpus = gpus
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            out = self.summarise(f, self.gpus)
        os.unlink(self.path)
        return out

    @staticmethod
    def summarise(lines, gpus):
        """Median SM clock, maximum clock and the throttle reasons seen active,
        from nvidia-smi CSV rows (index, clocks.sm, clocks.max.sm, power,
        active mask, then the four reason columns); rows of other GPUs and
        malformed rows are skipped.  None when no row counts."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                idx = int(parts[0])
            except ValueError:
                continue
            if gpus is not None and idx not in gpus:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle
def oracle_edge_stages(n, edges, cfg):
    """The oracle's sketch, community rounds and supergraph on the whole
    graph (single-threaded C); returns the supergraph and the seconds taken."""
    import oracle
    m = edges.shape[0]
    thr = cfg["threshold"] or (2 * m) // n
    t0 = time.perf_counter()
    _, dh = oracle.sketch_degrees(edges, n, cfg["rows"], cfg["width"], 1)
    lab, _ = oracle.communities(edges, n, dh, cfg["passes"], thr, cfg["growth"], 0)
    sg = oracle.supergraph(edges, n, lab, dh, cfg["rows"], cfg["width"], 1)
    return sg, time.perf_counter() - t0


def oracle_sample(n, edges, cfg, fa2_iters_sample=1):
    """Time the oracle on a bounded sample of one step: the three edge stages
    on the full graph plus `fa2_iters_sample` FA2 iterations on the resulting
    supergraph.  Returns a dict with the extrapolated step time (edge stages
    + iterations x FA2 iteration)."""
    import oracle
    sg, edge_s = oracle_edge_stages(n, edges, cfg)
    t1 = time.perf_counter()
    st = oracle.FA2State(oracle.fa2_init(sg["K"], 1))
    p = oracle.FA2Params()
    for _ in range(fa2_iters_sample):
        oracle.fa2_step(st, sg["csr_off"], sg["csr_adj"], sg["csr_w"], sg["mass"], p)
    t2 = time.perf_counter()
    t_fa2 = (t2 - t1) / max(fa2_iters_sample, 1)
    step = edge_s + cfg["iterations"] * t_fa2
    return dict(edge_s=edge_s, fa2_iter_s=t_fa2, step_s=step, wall_s=edge_s + (t2 - t1), K=sg["K"], Es=sg["Es"])


def cpu_info():
    model = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return model, os.cpu_count()


# ------------------------------------------------------- shared reporting
def workload_config(workload, n, m, world):
    """The config dict of a single-graph workload, the same in both arms."""
    cfg = WORKLOADS[workload]
    thr = cfg["threshold"] or (2 * m) // n
    return {"workload": f"{workload}: {cfg['desc']}", "n": n, "m": m, "sketch": f"{cfg['rows']}x{cfg['width']}",
            "passes": cfg["passes"], "threshold": thr, "growth": cfg["growth"], "fa2_iterations": cfg["iterations"],
            "theta": 1.2, "kr": 2.0, "kg": 1.0, "l2": "flushed before every timed step (256 MiB write)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def repulse_roofline(inter_per_launch, launch_ms, dev, clk):
    """FP32 roofline of the Barnes-Hut traversal: interactions x 12 flops per
    launch over the launch's event-timed duration, against the FMA peak of
    this GPU's SM count at its maximum SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clk or {}).get("sm_max_mhz") or FALLBACK_SM_MAX_MHZ
    peak = fp32_peak_tflops(sms, mhz)
    achieved = inter_per_launch * FLOPS_PER_INTERACTION / (launch_ms * 1e-3) / 1e12
    return {"kernel": "k_repulse (Barnes-Hut traversal)", "bound": "alu", "achieved": round(achieved, 3),
            "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
            "interactions_per_launch": int(inter_per_launch), "launch_ms": round(launch_ms, 4),
            "peak_note": f"FP32 FMA peak = {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {mhz:.0f} MHz "
                         "(unit counts of this GPU, maximum SM clock)",
            "traffic_note": "DRAM bytes per launch come from an ncu capture of the current kernel, not from this run"}


# --------------------------------------------------------------- GPU arm
def gpu_arm(args, dist: Dist):
    import torch

    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    if dist.rank == 0:
        from paper_2108_00529_gb300 import build
        build.build()
        graphgen.load(args.workload)
    dist.barrier()
    from paper_2108_00529_gb300 import load
    B = load()

    cfg = WORKLOADS[args.workload]
    n, edges_np, _ = graphgen.load(args.workload)
    m = edges_np.shape[0]
    thr = cfg["threshold"] or (2 * m) // n
    rows, width, passes, growth = cfg["rows"], cfg["width"], cfg["passes"], cfg["growth"]
    iters = args.fa2_iterations or cfg["iterations"]

    s = torch.cuda.Stream(device=dev)
    i32 = dict(dtype=torch.int32, device=dev)
    E = torch.from_numpy(edges_np).to(dev)
    S = torch.zeros(rows * width, **i32)
    dh = torch.zeros(n, **i32)
    labels = torch.zeros(n, **i32)
    node_map = torch.zeros(n, **i32)
    Kd = torch.zeros(1, dtype=torch.int64, device=dev)
    Esd = torch.zeros(1, dtype=torch.int64, device=dev)
    ssrc, sdst, sw = (torch.zeros(m, **i32) for _ in range(3))
    mass = torch.zeros(n, **i32)
    off = torch.zeros(n + 1, **i32)
    adj, cw = torch.zeros(2 * m, **i32), torch.zeros(2 * m, **i32)
    pos = torch.zeros((n, 2), dtype=torch.float32, device=dev)
    F, Fprev = torch.zeros_like(pos), torch.zeros_like(pos)
    speed = torch.zeros(1, dtype=torch.float64, device=dev)
    ws_sk = B.alloc_ws(B.bgv_sketch_degrees_ws_size(m, n, rows, width), dev)
    ws_cm = B.alloc_ws(B.bgv_communities_ws_size(m, n), dev)
    ws_sg = B.alloc_ws(B.bgv_supergraph_ws_size(m, n, rows, width), dev)
    ws_fa = B.alloc_ws(B.bgv_fa2_ws_size(n, 2 * m), dev)
    fp = B.bgv_fa2_default_params()
    K_host = torch.zeros(2, dtype=torch.int64).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sampled = max(1, min(args.stage_iterations, iters))

    def step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        with torch.cuda.stream(s):
            ev[0].record(s)
            B.bgv_sketch_degrees(E, m, n, rows, width, 1, S, dh, ws_sk, stream=s)
            ev[1].record(s)
            B.bgv_communities(E, m, n, dh, passes, thr, growth, 0, labels, None, ws_cm, stream=s)
            ev[2].record(s)
            B.bgv_supergraph(E, m, n, labels, dh, rows, width, 1, node_map, Kd, ssrc, sdst, sw, Esd, mass, off, adj,
                             cw, None, None, None, ws_sg, stream=s)
            ev[3].record(s)
            K_host[0:1].copy_(Kd, non_blocking=True)
            K_host[1:2].copy_(Esd, non_blocking=True)
        s.synchronize()
        K = int(K_host[0].item())
        nnz = 2 * int(K_host[1].item())
        with torch.cuda.stream(s):
            ev[4].record(s)  # the gap before it is the host reading K and Es
            B.bgv_fa2_init(K, fp, pos, Fprev, speed, stream=s)
            # the iterations run as replays of one captured step, as in
            # bgv_layout; the last `sampled` run launch by launch with events
            # at the stage boundaries, which time the kernels inside the step
            B.bgv_fa2_run(K, nnz, off, adj, cw, mass, fp, iters - sampled, 1, pos, F, Fprev, speed, ws_fa, stream=s)
            stages = B.bgv_fa2_run_timed(K, nnz, off, adj, cw, mass, fp, sampled, pos, F, Fprev, speed, ws_fa,
                                         stream=s)
            ev[5].record(s)
        s.synchronize()
        t = [ev[0].elapsed_time(ev[i]) for i in range(1, 6)]
        return dict(total=t[4], sketch=t[0], communities=t[1] - t[0], supergraph=t[2] - t[1], host_k=t[3] - t[2],
                    fa2=t[4] - t[3], fa2_stages=[x / sampled for x in stages], K=K)

    def flush_l2():
        flush.zero_()
        torch.cuda.synchronize(dev)

    # end to end through the host-buffer entry point: its timed calls alternate
    # with the first timed steps, so both legs run under the same clocks
    lp = B.bgv_layout_default_params()
    lp.rows, lp.width, lp.passes, lp.threshold, lp.growth, lp.iterations = rows, width, passes, thr, growth, iters
    n_e2e = 0 if args.no_e2e else max(1, min(args.steps, 3))
    if n_e2e:
        ws_e2e = B.alloc_ws(B.bgv_layout_host_ws_size(m, n, lp), dev)
        he = torch.from_numpy(edges_np).pin_memory()
        hmap = torch.zeros(n, dtype=torch.int32).pin_memory()
        hxy = torch.zeros((n, 2), dtype=torch.float32).pin_memory()
        hrad = torch.zeros(n, dtype=torch.float32).pin_memory()

    def e2e_call():
        with torch.cuda.stream(s):
            return B.bgv_layout_host(he, m, n, lp, hmap, hxy, hrad, ws_e2e, stream=s)

    for _ in range(args.warmup):
        flush_l2()
        step()
    if n_e2e:  # one untimed call first: the first host-buffer call of a process pays one-time costs
        e2e_call()
        s.synchronize()
        se0 = B.bgv_fa2_read_stats(ws_e2e, s)
    st0 = B.bgv_fa2_read_stats(ws_fa, s)
    launches = 0
    clocks = ClockSampler([dist.local] if dist.world == 1 else None)
    clocks.start()
    results, e2e = [], []
    K2 = None
    for k in range(args.steps):
        flush_l2()
        dist.barrier()
        torch.cuda.synchronize(dev)
        l0 = B.bgv_launch_count()
        results.append(step())
        torch.cuda.synchronize(dev)
        launches += B.bgv_launch_count() - l0  # the device-timed steps only
        dist.barrier()
        if k < n_e2e:
            flush_l2()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            K2, _ = e2e_call()
            e1.record(s)
            s.synchronize()
            e2e.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    st1 = B.bgv_fa2_read_stats(ws_fa, s)
    if st1.status:
        raise RuntimeError(f"device status {st1.status}")
    if n_e2e:  # the host-buffer calls' own Barnes-Hut work, beside the device-timed steps'
        se1 = B.bgv_fa2_read_stats(ws_e2e, s)
        e2e_inter = (se1.interactions_total - se0.interactions_total) / max(se1.steps_total - se0.steps_total, 1)

    ms = float(np.mean([r["total"] for r in results]))
    ms_max = dist.max(ms)
    K = results[-1]["K"]
    Es = int(Esd.item())
    m_cut = int(sw[:Es].to(torch.int64).sum().item())
    stage_ms = {k: float(np.mean([r[k] for r in results]))
                for k in ("sketch", "communities", "supergraph", "host_k", "fa2")}
    fa2_stage_ms = {nm: float(np.mean([r["fa2_stages"][i] for r in results]))
                    for i, nm in enumerate(B.FA2_STAGE_NAMES)}

    # dominant kernel: Barnes-Hut repulsion (one launch per FA2 iteration)
    steps_run = st1.steps_total - st0.steps_total
    inter_per_launch = (st1.interactions_total - st0.interactions_total) / max(steps_run, 1)
    rep_launch_ms = fa2_stage_ms["repulsion"]  # per iteration = per launch
    roofline = repulse_roofline(inter_per_launch, rep_launch_ms, dev, clk)

    # edge stages against HBM
    sort_passes = math.ceil(2 * max(1, math.ceil(math.log2(max(n, 2)))) / 8)
    edge_bytes = (passes + 2) * 8 * m + sort_passes * 16 * m_cut
    edge_ms = stage_ms["sketch"] + stage_ms["communities"] + stage_ms["supergraph"]
    edge_gbs = edge_bytes / (edge_ms * 1e-3) / 1e9
    hbm, hbm_src = hbm_peak()
    edge_roofline = {"bound": "hbm", "achieved": round(edge_gbs, 1), "peak": hbm, "peak_source": hbm_src,
                     "unit": "GB/s", "frac": round(edge_gbs / hbm, 4), "algorithmic_bytes": int(edge_bytes),
                     "edges_per_s": round(m / (edge_ms * 1e-3), 1), "ms": round(edge_ms, 4)}

    # what the community stage made of the graph (outside the timed region)
    ws_q = B.alloc_ws(B.bgv_modularity_ws_size(n), dev)
    q = B.bgv_modularity(E, m, n, labels, ws_q, stream=s)
    compression = {"isolated_ids": int(np.count_nonzero(np.bincount(edges_np.ravel(), minlength=n) == 0)),
                   "K_over_n": round(K / n, 4), "m_cut_over_m": round(m_cut / max(m, 1), 4),
                   "modularity_of_labels": round(q, 4)}

    e2e_ms = dist.max(float(np.mean(e2e))) if e2e else float("nan")
    K2 = K2 if e2e else K

    out = {
        "metric": METRIC,
        "value": round(aggregate_throughput(m, dist.world, ms_max), 1),
        "unit": "edges/s",
        "n_gpus": dist.world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_max, 3),
        "ms_each": [round(r["total"], 3) for r in results],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "i32+f32",
        "data": "synthetic",
        "config": workload_config(args.workload, n, m, dist.world),
        "K": K, "Es": Es, "m_cut": m_cut, "compression": compression,
        "fa2_iters_per_s": round(iters / (stage_ms["fa2"] * 1e-3), 2),
        "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "fa2_stage_us_per_iteration": {k: round(1000 * v, 2) for k, v in fa2_stage_ms.items()},
        "fa2_stage_note": f"CUDA events at the stage boundaries of the last {sampled} iterations of every timed step "
                          "(launched one by one; the others replay a captured step); the first of them sorts the "
                          "bodies with the radix sort, the rest with the hinted sort, as every run's steps after "
                          "its first do",
        "roofline": roofline,
        "edge_roofline": edge_roofline,
        "e2e": ({"value": round(aggregate_throughput(m, dist.world, e2e_ms), 1), "unit": "edges/s",
                 "ms_per_step": round(e2e_ms, 3), "h2d_bytes_per_step": int(8 * m),
                 "d2h_bytes_per_step": int(4 * n + 12 * K2), "entry": "bgv_layout_host",
                 "ms_each": [round(x, 3) for x in e2e], "interactions_per_iteration": int(e2e_inter)}
                if e2e else None),
        "gpu_launches": int(launches),
        "gpu_launches_per_step": int(launches // max(args.steps, 1)),
        "clocks": clk,
    }
    if dist.world == 1 and dist.rank == 0 and not args.no_cpu_baseline:
        r = oracle_sample(n, edges_np, cfg)
        model, ncpu = cpu_info()
        out["cpu_baseline"] = {"value": round(m / r["step_s"], 1), "unit": "edges/s", "cores": 1, "kind": "oracle",
                               "sample": (f"oracle (single-threaded C) on {args.workload}: the three edge stages on "
                                          f"the full graph ({r['edge_s']:.2f} s) plus 1 FA2 iteration on its "
                                          f"{r['K']}-node supergraph ({r['fa2_iter_s']:.2f} s); step time = edge "
                                          f"stages + {iters} x FA2 iteration = {r['step_s']:.1f} s"),
                               "cpu": model, "host_cpus": ncpu}
    return out


def gpu_arm_whole(args, dist: Dist):
    """Precision form: ForceAtlas2 directly on the whole graph (mass = degree
    + 1, unit weights), nodes coloured by their streamed community.  A step
    is sketch + community rounds + colour groups + whole-graph CSR + initial
    positions + the FA2 iterations."""
    import torch

    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    if dist.rank == 0:
        from paper_2108_00529_gb300 import build
        build.build()
        graphgen.load(args.workload)
    dist.barrier()
    from paper_2108_00529_gb300 import load
    B = load()
    cfg = WORKLOADS[args.workload]
    n, edges_np, _ = graphgen.load(args.workload)
    m = edges_np.shape[0]
    thr = cfg["threshold"] or (2 * m) // n
    rows, width, passes, growth = cfg["rows"], cfg["width"], cfg["passes"], cfg["growth"]
    iters = args.fa2_iterations or cfg["iterations"]
    s = torch.cuda.Stream(device=dev)
    i32 = dict(dtype=torch.int32, device=dev)
    E = torch.from_numpy(edges_np).to(dev)
    S, dh, labels = torch.zeros(rows * width, **i32), torch.zeros(n, **i32), torch.zeros(n, **i32)
    node_map, Kd, Esd = torch.zeros(n, **i32), torch.zeros(1, dtype=torch.int64, device=dev), \
        torch.zeros(1, dtype=torch.int64, device=dev)
    ssrc, sdst, sw = (torch.zeros(m, **i32) for _ in range(3))
    smass, soff = torch.zeros(n, **i32), torch.zeros(n + 1, **i32)
    sadj, scw = torch.zeros(2 * m, **i32), torch.zeros(2 * m, **i32)
    group = torch.zeros(n, dtype=torch.uint8, device=dev)
    colour = torch.zeros(n, dtype=torch.uint8, device=dev)
    off, adj, cw = torch.zeros(n + 1, **i32), torch.zeros(2 * m, **i32), torch.zeros(2 * m, **i32)
    mass, nnz_d = torch.zeros(n, **i32), torch.zeros(1, dtype=torch.int64, device=dev)
    pos = torch.zeros((n, 2), dtype=torch.float32, device=dev)
    F, Fprev = torch.zeros_like(pos), torch.zeros_like(pos)
    speed = torch.zeros(1, dtype=torch.float64, device=dev)
    ws_sk = B.alloc_ws(B.bgv_sketch_degrees_ws_size(m, n, rows, width), dev)
    ws_cm = B.alloc_ws(B.bgv_communities_ws_size(m, n), dev)
    ws_cs = B.alloc_ws(B.bgv_graph_csr_ws_size(m, n), dev)
    ws_sg = B.alloc_ws(B.bgv_supergraph_ws_size(m, n, rows, width), dev)
    ws_cg = B.alloc_ws(B.bgv_colour_groups_ws_size(n), dev)
    ws_fa = B.alloc_ws(B.bgv_fa2_ws_size(n, 2 * m), dev)
    fp = B.bgv_fa2_default_params()
    nnz_h = torch.zeros(1, dtype=torch.int64).pin_memory()
    K_h = torch.zeros(1, dtype=torch.int64).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sampled = max(1, min(args.stage_iterations, iters))

    def step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with torch.cuda.stream(s):
            ev[0].record(s)
            B.bgv_sketch_degrees(E, m, n, rows, width, 1, S, dh, ws_sk, stream=s)
            B.bgv_communities(E, m, n, dh, passes, thr, growth, 0, labels, None, ws_cm, stream=s)
            # each node takes the colour of its community's supernode
            B.bgv_supergraph(E, m, n, labels, dh, rows, width, 1, node_map, Kd, ssrc, sdst, sw, Esd, smass, soff,
                             sadj, scw, None, None, None, ws_sg, stream=s)
            K_h.copy_(Kd, non_blocking=True)
        s.synchronize()
        K = int(K_h.item())
        with torch.cuda.stream(s):
            B.bgv_colour_groups(K, smass, group, ws_cg, n=n, node_map=node_map, node_colour=colour, stream=s)
            ev[1].record(s)
            B.bgv_graph_csr(E, m, n, off, adj, cw, mass, nnz_d, ws_cs, stream=s)
            ev[2].record(s)
            nnz_h.copy_(nnz_d, non_blocking=True)
        s.synchronize()
        nnz = int(nnz_h.item())
        with torch.cuda.stream(s):
            B.bgv_fa2_init(n, fp, pos, Fprev, speed, stream=s)
            B.bgv_fa2_run(n, nnz, off, adj, cw, mass, fp, iters - sampled, 1, pos, F, Fprev, speed, ws_fa, stream=s)
            stages = B.bgv_fa2_run_timed(n, nnz, off, adj, cw, mass, fp, sampled, pos, F, Fprev, speed, ws_fa,
                                         stream=s)
            ev[3].record(s)
        s.synchronize()
        t = [ev[0].elapsed_time(ev[i]) for i in range(1, 4)]
        return dict(total=t[2], communities=t[0], graph_csr=t[1] - t[0], fa2=t[2] - t[1],
                    fa2_stages=[x / sampled for x in stages], nnz=nnz)

    for _ in range(args.warmup):
        flush.zero_()
        torch.cuda.synchronize(dev)
        step()
    st0 = B.bgv_fa2_read_stats(ws_fa, s)
    launches0 = B.bgv_launch_count()
    clocks = ClockSampler([dist.local] if dist.world == 1 else None)
    clocks.start()
    results = []
    for _ in range(args.steps):
        flush.zero_()
        dist.barrier()
        torch.cuda.synchronize(dev)
        results.append(step())
        torch.cuda.synchronize(dev)
    clk = clocks.stop()
    launches = B.bgv_launch_count() - launches0
    st1 = B.bgv_fa2_read_stats(ws_fa, s)
    ms = dist.max(float(np.mean([r["total"] for r in results])))
    fa2_ms = float(np.mean([r["fa2"] for r in results]))
    stage = {nm: float(np.mean([r["fa2_stages"][i] for r in results])) for i, nm in enumerate(B.FA2_STAGE_NAMES)}
    inter = (st1.interactions_total - st0.interactions_total) / max(st1.steps_total - st0.steps_total, 1)
    rep_ms = stage["repulsion"]  # per iteration = per launch
    out = {
        "metric": METRIC, "value": round(aggregate_throughput(m, dist.world, ms), 1), "unit": "edges/s",
        "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32+f32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {cfg['desc']}", "n": n, "m": m, "fa2_iterations": iters,
                   "theta": 1.2, "kr": 2.0, "kg": 1.0, "mass": "degree + 1",
                   "l2": "flushed before every timed step (256 MiB write)"},
        "fa2_iters_per_s": round(iters / (fa2_ms * 1e-3), 2),
        "stage_ms": {k: round(float(np.mean([r[k] for r in results])), 4)
                     for k in ("communities", "graph_csr", "fa2")},
        "fa2_stage_us_per_iteration": {k: round(1000 * v, 2) for k, v in stage.items()},
        "roofline": repulse_roofline(inter, rep_ms, dev, clk),
        "gpu_launches": int(launches), "clocks": clk,
    }
    if args.precision_sample:
        import oracle
        # per-step error of the FP32 forces against the FP64 oracle on a
        # sample of nodes, same tree and theta
        off_h, adj_h = off.cpu().numpy(), adj.cpu().numpy()
        cw_h, mass_h = cw.cpu().numpy().view(np.uint32), mass.cpu().numpy().view(np.uint32)
        nnz = results[-1]["nnz"]
        adj_h, cw_h = adj_h[:nnz], cw_h[:nnz]
        which = np.random.default_rng(4).choice(n, size=min(args.precision_sample, n), replace=False)
        p = oracle.FA2Params()
        Fr, Fa, Fg = (torch.zeros_like(pos) for _ in range(3))
        ws_f = B.alloc_ws(B.bgv_fa2_ws_size(n, nnz), dev)
        B.bgv_fa2_init(n, fp, pos, Fprev, speed, stream=s)
        log = {}
        done = 0
        for t in sorted({0, iters // 4, iters // 2, iters}):
            if t > done:
                B.bgv_fa2_run(n, nnz, off, adj, cw, mass, fp, t - done, 1, pos, F, Fprev, speed, ws_fa, stream=s)
                done = t
            B.bgv_fa2_forces(n, nnz, off, adj, cw, mass, fp, pos, Fr, Fa, Fg, ws_f, stream=s)
            s.synchronize()
            ph = pos.cpu().numpy()
            F32 = (Fr + Fa + Fg).cpu().numpy().astype(np.float64)[which]
            F64 = (oracle.bh_repulsion(ph, mass_h, p, which=which)[0]
                   + oracle.attraction(off_h, adj_h, cw_h, ph)[which]
                   + oracle.gravity(mass_h, ph, p.kg, p.strong_gravity)[which])
            nrm = np.linalg.norm(F64, axis=1)
            rel = np.linalg.norm(F32 - F64, axis=1) / np.maximum(nrm, 1e-3 * np.sqrt(np.mean(nrm ** 2)))
            log[str(t)] = {"max": float(rel.max()), "p99": float(np.percentile(rel, 99)),
                           "median": float(np.median(rel))}
        out["precision"] = {"sample": int(which.shape[0]), "reference": "FP64 oracle, same tree and theta",
                            "rel_err_by_step": log}
    return out


def gpu_arm_batched(args, dist: Dist):
    """Batching form: all 512 graphs through one bgv_layout_batched call per
    step (sketch, rounds, supergraph, 300 FA2 iterations for every graph),
    compared with the same graphs laid out one bgv_layout call at a time."""
    import torch

    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    if dist.rank == 0:
        from paper_2108_00529_gb300 import build
        build.build()
        graphgen.load_batch(args.workload)
    dist.barrier()
    from paper_2108_00529_gb300 import load
    B = load()
    cfg = WORKLOADS[args.workload]
    edges_np, eo, no = graphgen.load_batch(args.workload)
    Gn, m, N = eo.shape[0] - 1, int(eo[-1]), int(no[-1])
    iters = args.fa2_iterations or cfg["iterations"]
    p = B.bgv_layout_default_params()
    p.rows, p.width, p.passes, p.threshold, p.growth = cfg["rows"], cfg["width"], cfg["passes"], 0, cfg["growth"]
    p.iterations, p.use_graph = iters, 1
    s = torch.cuda.Stream(device=dev)
    E = torch.from_numpy(edges_np).to(dev)
    node_map = torch.zeros(N, dtype=torch.int32, device=dev)
    xy = torch.zeros((N, 2), dtype=torch.float32, device=dev)
    rad = torch.zeros(N, dtype=torch.float32, device=dev)
    ws = B.alloc_ws(B.bgv_layout_batched_ws_size(Gn, eo, no, p), dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def batched_step():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            e0.record(s)
            K_off, Es_off = B.bgv_layout_batched(E, Gn, eo, no, p, node_map, xy, rad, ws, stream=s)
            e1.record(s)
        s.synchronize()
        return e0.elapsed_time(e1), K_off, Es_off

    for _ in range(args.warmup):
        flush.zero_()
        torch.cuda.synchronize(dev)
        batched_step()
    st0 = B.bgv_fa2_read_stats(ws, s)
    launches0 = B.bgv_launch_count()
    clocks = ClockSampler([dist.local] if dist.world == 1 else None)
    clocks.start()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        dist.barrier()
        torch.cuda.synchronize(dev)
        t, K_off, Es_off = batched_step()
        times.append(t)
        torch.cuda.synchronize(dev)
    clk = clocks.stop()
    launches = B.bgv_launch_count() - launches0
    st1 = B.bgv_fa2_read_stats(ws, s)
    ms = dist.max(float(np.mean(times)))

    # the same graphs, one bgv_layout call each (own copy of its edges, so
    # every list starts 16-byte aligned); one warm-up pass, one timed pass
    per_graph = None
    if not args.no_per_graph:
        Eg = [torch.from_numpy(np.ascontiguousarray(edges_np[eo[g]:eo[g + 1]])).to(dev) for g in range(Gn)]
        nmax, mmax = int(np.max(np.diff(no))), int(np.max(np.diff(eo)))
        ws1 = B.alloc_ws(max(B.bgv_layout_ws_size(int(eo[g + 1] - eo[g]), int(no[g + 1] - no[g]), p)
                             for g in range(Gn)), dev)
        nm1 = torch.zeros(nmax, dtype=torch.int32, device=dev)
        xy1 = torch.zeros((nmax, 2), dtype=torch.float32, device=dev)
        r1 = torch.zeros(nmax, dtype=torch.float32, device=dev)
        same = True
        pg_ms = 0.0
        for rep in range(2):
            flush.zero_()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(s):
                e0.record(s)
                for g in range(Gn):
                    K, Es = B.bgv_layout(Eg[g], int(eo[g + 1] - eo[g]), int(no[g + 1] - no[g]), p, nm1, xy1, r1,
                                         ws1, stream=s)
                    if rep == 1:
                        same &= (K, Es) == (int(K_off[g + 1] - K_off[g]), int(Es_off[g + 1] - Es_off[g]))
                e1.record(s)
            s.synchronize()
            pg_ms = e0.elapsed_time(e1)
        per_graph = {"graphs_per_s": round(Gn / (pg_ms * 1e-3), 2), "ms": round(pg_ms, 1),
                     "entry": "bgv_layout, one call per graph", "counts_equal_batched": bool(same)}
    inter = (st1.interactions_total - st0.interactions_total) / max(st1.steps_total - st0.steps_total, 1)
    return {
        "metric": "graphs/s laid out (sketch, communities, supergraph, FA2)",
        "value": round(aggregate_throughput(Gn, dist.world, ms), 3),
        "unit": "graphs/s", "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "i32+f32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {cfg['desc']}", "graphs": Gn, "n": N, "m": m,
                   "sketch": f"{cfg['rows']}x{cfg['width']} per graph", "passes": cfg["passes"],
                   "fa2_iterations": iters, "K": int(K_off[-1]), "Es": int(Es_off[-1]),
                   "l2": "flushed before every timed step (256 MiB write)", "parallelism": "single GPU"},
        "edges_per_s": round(aggregate_throughput(m, dist.world, ms), 1),
        "interactions_per_iteration": int(inter),
        "per_graph_launches": per_graph,
        "gpu_launches": int(launches), "gpu_launches_per_step": int(launches // max(args.steps, 1)), "clocks": clk,
    }


def gpu_sweep(args, dist: Dist):
    """Parameter sweep of the edge stages on the workload (the paper's Tables
    2 and 3: sketch rows and community rounds; and the community variants):
    per setting, the time of sketch + rounds + supergraph, the supernode and
    superedge counts, and the modularity of the labels."""
    import torch

    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    from paper_2108_00529_gb300 import build
    build.build()
    from paper_2108_00529_gb300 import load
    B = load()
    cfg = WORKLOADS[args.workload]
    n, edges_np, _ = graphgen.load(args.workload)
    m = edges_np.shape[0]
    width = cfg["width"]
    s = torch.cuda.Stream(device=dev)
    i32 = dict(dtype=torch.int32, device=dev)
    E = torch.from_numpy(edges_np).to(dev)
    S = torch.zeros(16 * width, **i32)
    dh, labels, node_map = torch.zeros(n, **i32), torch.zeros(n, **i32), torch.zeros(n, **i32)
    Kd, Esd = torch.zeros(1, dtype=torch.int64, device=dev), torch.zeros(1, dtype=torch.int64, device=dev)
    ssrc, sdst, sw = (torch.zeros(m, **i32) for _ in range(3))
    mass, off = torch.zeros(n, **i32), torch.zeros(n + 1, **i32)
    adj, cw = torch.zeros(2 * m, **i32), torch.zeros(2 * m, **i32)
    ws_sk = B.alloc_ws(B.bgv_sketch_degrees_ws_size(m, n, 4, width), dev)
    ws_cm = B.alloc_ws(B.bgv_communities_ex_ws_size(m, n), dev)
    ws_sg = B.alloc_ws(B.bgv_supergraph_ws_size(m, n, 4, width), dev)
    ws_q = B.alloc_ws(B.bgv_modularity_ws_size(n), dev)
    settings = [dict(rows=r, passes=3, growth=2, tmode=0, jumps=0) for r in (1, 2, 3, 4)]
    settings += [dict(rows=4, passes=p, growth=2, tmode=0, jumps=0) for p in (2, 4)]
    settings += [dict(rows=4, passes=3, growth=2, tmode=1, jumps=0), dict(rows=4, passes=3, growth=0, tmode=1, jumps=0),
                 dict(rows=4, passes=3, growth=2, tmode=0, jumps=2)]
    out = []
    for st in settings:
        times = []
        for rep in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(s):
                e0.record(s)
                B.bgv_sketch_degrees(E, m, n, st["rows"], width, 1, S, dh, ws_sk, stream=s)
                D = B.bgv_communities_ex(E, m, n, dh, st["passes"], 0, st["growth"], 0, st["tmode"], st["jumps"],
                                         labels, None, ws_cm, stream=s)
                B.bgv_supergraph(E, m, n, labels, dh, st["rows"], width, 1, node_map, Kd, ssrc, sdst, sw, Esd, mass,
                                 off, adj, cw, None, None, None, ws_sg, stream=s)
                e1.record(s)
            s.synchronize()
            if rep:
                times.append(e0.elapsed_time(e1))
        q = B.bgv_modularity(E, m, n, labels, ws_q, stream=s)
        out.append({**st, "threshold": D, "edge_stage_ms": round(float(np.median(times)), 3), "K": int(Kd.item()),
                    "Es": int(Esd.item()), "modularity": round(q, 4)})
    return {"sweep": f"{args.workload}: {cfg['desc']}", "sketch_width": width, "n": n, "m": m,
            "note": "tmode 1 = mode-degree threshold; growth 0 = delta^i schedule; jumps = pointer-jumping steps "
                    "per round; the time of a mode-degree setting includes the read-back of the mode",
            "settings": out}


def reference_arm_batched(args, dist: Dist):
    """The oracle on the batching workload: graphs taken in a fixed strided
    order (every 32nd, so small and large ones alike) until about 10 s of
    oracle time; each graph's step time is its edge stages plus the
    workload's iterations x one timed FA2 iteration."""
    cfg = WORKLOADS[args.workload]
    edges_np, eo, no = graphgen.load_batch(args.workload)
    Gn = eo.shape[0] - 1
    order = [g for r in range(32) for g in range(r, Gn, 32)]
    steps = []
    for i in range(args.warmup + args.steps):
        spent, total, used = 0.0, 0.0, 0
        for g in order:
            if spent > 10.0:
                break
            e = edges_np[eo[g]:eo[g + 1]]
            r = oracle_sample(int(no[g + 1] - no[g]), e, cfg)
            spent += r["wall_s"]
            total += r["step_s"]
            used += 1
        if i >= args.warmup:
            steps.append((used, total))
    used = steps[-1][0]
    per_graph_s = float(np.mean([t / u for u, t in steps]))
    model, ncpu = cpu_info()
    value = round(1.0 / per_graph_s, 4)
    sample = (f"each step: the first {used} graphs of a stride-32 order over the {Gn}; per graph the three edge "
              f"stages plus 1 timed FA2 iteration, step time = edge stages + {cfg['iterations']} x FA2 iteration")
    return {"impl": "reference", "metric": "graphs/s laid out (sketch, communities, supergraph, FA2)",
            "value": value, "unit": "graphs/s", "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(per_graph_s * Gn * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "i32+f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {cfg['desc']}", "graphs": Gn,
                       "fa2_iterations": cfg["iterations"]},
            "cpu_baseline": {"value": value, "unit": "graphs/s", "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu": model, "host_cpus": ncpu},
            "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def reference_arm(args, dist: Dist):
    """The oracle as the reference implementation, on the host cores.  Its
    edge stages run once on the full graph (timed), then every warm-up and
    timed step is one oracle FA2 iteration on the resulting supergraph; a
    step's time is the edge stages plus the workload's iterations x the
    iteration time, so the run stays within a few minutes at full size."""
    if dist.rank != 0:
        return None
    if WORKLOADS[args.workload].get("batched"):
        return reference_arm_batched(args, dist)
    import oracle
    cfg = WORKLOADS[args.workload]
    n, edges_np, _ = graphgen.load(args.workload)
    m = edges_np.shape[0]
    sg, edge_s = oracle_edge_stages(n, edges_np, cfg)
    st = oracle.FA2State(oracle.fa2_init(sg["K"], 1))
    p = oracle.FA2Params()
    iters = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.fa2_step(st, sg["csr_off"], sg["csr_adj"], sg["csr_w"], sg["mass"], p)
        if i >= args.warmup:
            iters.append(time.perf_counter() - t0)
    fa2_iter_s = float(np.mean(iters))
    step_s = edge_s + cfg["iterations"] * fa2_iter_s
    model, ncpu = cpu_info()
    value = round(m / step_s, 1)
    sample = (f"the three edge stages once on the full {args.workload} graph ({edge_s:.2f} s), then per step one "
              f"FA2 iteration on its {sg['K']}-node supergraph (mean {fa2_iter_s:.2f} s); step time = edge stages "
              f"+ {cfg['iterations']} x FA2 iteration = {step_s:.1f} s")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32+f64",
            "data": "synthetic", "config": workload_config(args.workload, n, m, dist.world),
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu": model, "host_cpus": ncpu},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def finite(x):
    """The line as strict JSON: a number that is not finite (a leg that did
    not run) becomes null."""
    if isinstance(x, dict):
        return {k: finite(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [finite(v) for v in x]
    if isinstance(x, float) and not math.isfinite(x):
        return None
    return x


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="rmat22x", choices=sorted(WORKLOADS))
    ap.add_argument("--fa2-iterations", type=int, default=0,
                    help="override the workload's FA2 iteration count (short profiling runs only)")
    ap.add_argument("--stage-iterations", type=int, default=10,
                    help="FA2 iterations per timed step launched one by one with events at the stage boundaries "
                         "(the per-stage times and the roofline's kernel duration); the others replay a graph")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg (profiling runs)")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the timed step: sketch rows, rounds and community variants on the workload")
    ap.add_argument("--no-per-graph", action="store_true",
                    help="batched workload: skip the one-call-per-graph comparison")
    ap.add_argument("--precision-sample", type=int, default=0,
                    help="whole-graph workloads: nodes sampled for the FP64 force-error report")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    dist = Dist()
    try:
        if args.impl == "reference":
            out = reference_arm(args, dist)
        elif args.sweep:
            out = gpu_sweep(args, dist)
        elif WORKLOADS[args.workload].get("whole"):
            out = gpu_arm_whole(args, dist)
        elif WORKLOADS[args.workload].get("batched"):
            out = gpu_arm_batched(args, dist)
        else:
            out = gpu_arm(args, dist)
    finally:
        dist.close()
    if out is not None and dist.rank == 0:
        print(json.dumps(finite(out), allow_nan=False))


if __name__ == "__main__":
    main()
