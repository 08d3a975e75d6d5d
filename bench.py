"""Benchmark: exact FRNN self-query (grid build + query) on the tracking-event
shaped workload: N=300,000 points, D=8, 8,000 clusters x 30 (sigma 0.02) + 60,000
uniform background in [-1,1]^8, r=0.1, K=64.

One step = the whole hot path on one event: frnn_build_grid (cell ids, counting
sort, prefix scan, scatter, tasks) + frnn_query (TMA-staged candidate scan,
exact FP32 screen, warp top-K).  The metric is queries/s (value) and
neighbour-pairs/s; the dominant kernel's achieved algorithmic bandwidth is
reported against the measured HBM peak.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU brute-force oracle on a bounded sample of the
same workload (the paper publishes no GB300 number; the oracle is the baseline).
Under torchrun (N > 1) every rank runs its own replica of the event (queries are
independent: no collective on the data path) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "FRNN queries/s & neighbor-pairs/s at N=300k D=8; batched vs plain; % HBM peak"
L2_BYTES = 129 * 2 ** 20


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(name="event300k"):
    from paper_2609_31980_gb300 import synth
    return synth.config3() if name == "event500k" else synth.config2()


def profile_summary(path: str, wl: str):
    """Counters of the dominant kernel from its committed ncu summary of the
    same workload: DRAM bytes per launch ("traffic") and executed warp
    instructions per launch ("warp_instructions"); None when there is no
    summary or the kernel's sources changed since the capture."""
    import hashlib
    key = (path, wl)
    known = {("grid", "event300k"): ("grid_query_event300k_x8.md", ["query.cu", "frnn_internal.cuh"]),
             ("rows", "event500k"): ("row_query_event500k_x12.md", ["query_rows.cu", "frnn_internal.cuh"]),
             ("tc", "event500k"): ("tc_query_event500k_x12.md", ["tc.cu", "frnn_internal.cuh"])}
    if key not in known:
        return None
    name, srcs = known[key]
    f = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(f):
        return None
    h = hashlib.sha256()
    for s_ in srcs:
        with open(os.path.join(ROOT, "paper_2609_31980_gb300", "csrc", s_), "rb") as fh:
            h.update(fh.read())
    out, sha = {"traffic": None, "warp_instructions": None, "tensor_pipe_pct": None}, None
    with open(f) as fh:
        for line in fh:
            if line.startswith("traffic_bytes_per_launch:"):
                out["traffic"] = int(line.split(":")[1])
            elif line.startswith("source_sha256_16"):
                sha = line.split(":")[-1].strip()
            elif line.startswith("tensor_pipe_active_pct:"):
                out["tensor_pipe_pct"] = float(line.split(":")[1])
            elif line.startswith("| smsp__inst_executed.sum |"):
                # "| smsp__inst_executed.sum | 195.3 M warp instructions |"
                out["warp_instructions"] = float(line.split("|")[2].split()[0]) * 1e6
    return out if sha == h.hexdigest()[:16] else None


def profiled_traffic(path: str, wl: str):
    """DRAM bytes per launch of the dominant kernel (see profile_summary)."""
    p = profile_summary(path, wl)
    return p["traffic"] if p else None


def issue_roofline(warp_instructions, kernel_ms: float, sms: int, sm_mhz: float):
    """Instruction issue of the dominant kernel against the issue ceiling:
    every SM has four schedulers, each issuing at most one warp instruction
    per clock.  Rates in tera warp instructions per second."""
    if not warp_instructions or kernel_ms <= 0 or sms <= 0 or sm_mhz <= 0:
        return None
    achieved = warp_instructions / (kernel_ms / 1e3) / 1e12
    peak = sms * 4 * sm_mhz * 1e6 / 1e12
    return {"warp_instructions": warp_instructions, "achieved": achieved, "peak": peak,
            "unit": "T warp instructions/s", "frac": achieved / peak, "sms": sms,
            "sm_mhz": sm_mhz, "source": "instruction count of the committed ncu summary, "
            "time of this run"}


def link_bandwidth(dev, stream, nbytes: int = 64 << 20, reps: int = 5) -> dict:
    """Page-locked host <-> device copy bandwidth of this GPU's host link
    (GB/s each way; best of reps after one untimed copy, CUDA events on the
    copy's stream).  Copies from the SMs (loads and stores to page-locked
    memory) reach the same rates as the copy engines on this link."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    out = {"bytes": nbytes}
    for name, dst, src in (("h2d_gbs", d, h), ("d2h_gbs", h, d)):
        best = float("inf")
        for k in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                dst.copy_(src, non_blocking=True)
                e1.record(stream)
            e1.synchronize()
            if k:
                best = min(best, e0.elapsed_time(e1))
        out[name] = nbytes / (best / 1e3) / 1e9
    return out


def link_roofline(link: dict, h2d_bytes: int, d2h_bytes: int, step_ms: float) -> dict:
    """The part of an end-to-end step the host transfers alone take at the
    measured link rates (a lower bound on the step were nothing else in it)."""
    t = (h2d_bytes / (link["h2d_gbs"] * 1e9) + d2h_bytes / (link["d2h_gbs"] * 1e9)) * 1e3
    return {"h2d_gbs": link["h2d_gbs"], "d2h_gbs": link["d2h_gbs"], "transfer_ms": t,
            "frac": t / step_ms if step_ms > 0 else None}


def algorithmic_query_bytes(N: int, D: int, K: int) -> int:
    """Bytes the query step must move at least once: the cell-sorted padded
    rows read as queries and once as candidates, the slot->index map, and the
    dense outputs (counts + K indices + K distances per query)."""
    DP = (D + 3) // 4 * 4
    return N * DP * 4 * 2 + N * 4 + N * 4 + N * K * 8


def _cell_cap(N: int, naxes: int) -> int:
    """Cells the library allows an N-point grid requested with naxes axes
    (mirrors cell_cap_for in build.cu: 18 N for five, 2 N for four)."""
    c = 18 * N if naxes >= 5 else (2 * N if naxes == 4 else N // 2 + 1)
    return min(max(16384, c), (1 << 27) if naxes >= 5 else (1 << 24))


def _scan_launches(L: int) -> int:
    """Launches of one exclusive scan of L entries (blocks of 2048): one for
    a single block, else the reduce pass, a scan of the block sums beyond
    4096 blocks, the down pass."""
    nb = (L + 2047) // 2048
    return 1 if nb == 1 else (2 if nb <= 4096 else 3)


def launches_per_step(N: int, D: int, path: str = "grid", naxes_requested: int = 0) -> int:
    """Kernels one build + query launches (mirrors the library's host code):
    requested axes 0 (automatic, up to D = 8) or 5 take the chunk scan,
    1..4 the row-task scan, whose query call first makes the pair copy and
    the task list."""
    if naxes_requested == 0 and path != "tc":
        naxes_requested = 0 if D <= 8 else 4
    cap_axes = naxes_requested or min(D, 5)
    L = _cell_cap(N, cap_axes) + 1
    build = 4 + _scan_launches(L)          # init bbox cellid scan(s) scatter
    if path == "tc":
        # operand preparation + 128-query tasks (rowtasks scan emit), tc query, selection pass
        return build + 1 + (1 + _scan_launches(L) + 1) + 2
    if 1 <= naxes_requested <= 4:
        # pair copy + 16-query tasks (rowtasks scan emit), row-task query, selection pass
        return build + 1 + (1 + _scan_launches(L) + 1) + 2
    return build + 2                       # chunk query + selection pass


def max_over_ranks(x: float, device) -> float:
    """The largest x over all ranks of the default process group (x itself
    without one): the job takes as long as its slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, steps: int, ws: int, total_ms: float) -> float:
    """Units all ranks processed over the slowest rank's time (weak scaling:
    every rank runs its own replica of the workload)."""
    return units_per_rank * ws * steps / (total_ms / 1e3)


def time_config(frnn, pts_np, r, K, path, dev, steps=20, warmup=3, opts=None, tc_stats=False):
    """Build + query of one event in one configuration (a fresh context with
    the given options): median step and build ms (CUDA events on the
    context's stream, L2 flushed between steps), mean main-kernel ms, and
    for the tensor-core path the pre-filter's false-candidate rate."""
    import torch
    stream = torch.cuda.Stream()
    ctx = frnn.Context(stream=stream)
    for k, v in (opts or {}).items():
        ctx.set_option(k, v)
    N = pts_np.shape[0]
    with torch.cuda.stream(stream):
        pts = torch.from_numpy(pts_np).to(dev)
        out = (torch.empty(N, dtype=torch.int32, device=dev),
               torch.empty((N, K), dtype=torch.int32, device=dev),
               torch.empty((N, K), dtype=torch.float32, device=dev))
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    grid = ctx.build_grid(pts, r)
    for _ in range(warmup):
        ctx.build_grid(pts, r, grid=grid)
        ctx.query(grid, pts, r, K, True, path, out)
    ctx.sync()
    if tc_stats:
        ctx.set_option(frnn.FRNN_OPT_TC_SURVIVORS, 0)   # reset the pre-filter counters
    mk = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed_pass(split: bool):
        # split: events at the build/query boundary and around the main query
        # kernel too (those records cost the step a few microseconds, so the
        # step time comes from a pass without them)
        ctx.set_option(frnn.FRNN_OPT_KERNEL_TIMING, 1 if split else 0)
        evs = [(mk(), mk(), mk()) for _ in range(steps)]
        for k in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
            evs[k][0].record(stream)
            ctx.build_grid(pts, r, grid=grid)
            if split:
                evs[k][1].record(stream)
            ctx.query(grid, pts, r, K, True, path, out)
            evs[k][2].record(stream)
        ctx.sync()
        kern = ctx.kernel_times() if split else []
        ctx.set_option(frnn.FRNN_OPT_KERNEL_TIMING, 0)
        return evs, kern

    evs, _ = timed_pass(False)
    step_med = statistics.median(e[0].elapsed_time(e[2]) for e in evs)
    evs2, kern = timed_pass(True)
    res = {"step_ms_median": step_med,
           "build_ms_median": statistics.median(e[0].elapsed_time(e[1]) for e in evs2),
           "kernel_ms_mean": sum(kern) / max(len(kern), 1),
           "queries_per_s": N / (step_med / 1e3),
           "neighbor_pairs": int(out[0].sum().item())}
    if tc_stats:
        surv = ctx.get_option(frnn.FRNN_OPT_TC_SURVIVORS)
        acc = ctx.get_option(frnn.FRNN_OPT_TC_ACCEPTED)
        res["prefilter_survivors"] = surv
        res["exact_accepted"] = acc
        res["false_candidate_rate"] = (surv - acc) / surv if surv else None
    gp = grid.params()
    res["gridded_axes"] = gp["naxes"]
    res["cell_mult"] = gp["cell_mult"]
    res["grid_kernel"] = gp["kernel"]
    ctx.close()
    del out, pts, flush
    return res


def run_design_points(args, dev):
    """Other configurations of the same path, each timed on its own:
    the 300k x 8 event on grids over three coordinates (cell multiple 1 and 2;
    the library's default grids five up to D = 8), the uniform 4096 x 3 set, and the
    500k x 12 event on the grid scan against the tensor-core pre-filter
    (false-candidate rate of the pre-filter; tensor-pipe activity from the
    committed ncu summary of that kernel)."""
    from paper_2609_31980_gb300 import frnn, synth
    out = {}
    w2 = synth.config2()
    for m in (1, 2):
        out[f"event300k_3axes_m{m}"] = time_config(
            frnn, w2.points, w2.r, w2.K, "grid", dev,
            opts={frnn.FRNN_OPT_GRID_NAXES: 3, frnn.FRNN_OPT_CELL_MULT: m})
    w1 = synth.config1()
    out["uniform4096x3"] = time_config(frnn, w1.points, w1.r, w1.K, "grid", dev)
    w3 = synth.config3()
    g3 = time_config(frnn, w3.points, w3.r, w3.K, "grid", dev)
    t3 = time_config(frnn, w3.points, w3.r, w3.K, "tc", dev,
                     opts={frnn.FRNN_OPT_GRID_NAXES: 3}, tc_stats=True)
    prof = profile_summary("tc", "event500k") or {}
    t3["tensor_pipe_active_pct"] = prof.get("tensor_pipe_pct")
    out["event500k_x12"] = {"workload": w3.name, "grid": g3, "tc": t3,
                            "tc_kernel_over_grid_kernel": t3["kernel_ms_mean"] / g3["kernel_ms_mean"]}
    return out


def run_ours(args):
    import torch
    from paper_2609_31980_gb300 import frnn

    ws, rank, local = _dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    w = workload(args.workload)
    pts_np = w.points
    N, D, r, K = pts_np.shape[0], w.D, w.r, w.K
    path = args.path
    stream = torch.cuda.Stream()
    ctx = frnn.Context(stream=stream)
    if args.cell_mult:
        ctx.set_option(frnn.FRNN_OPT_CELL_MULT, args.cell_mult)
    if args.exit_dims:
        ctx.set_option(frnn.FRNN_OPT_EXIT_DIMS, args.exit_dims)
    if args.grid_axes:
        ctx.set_option(frnn.FRNN_OPT_GRID_AXES, args.grid_axes)
    if args.grid_naxes:
        ctx.set_option(frnn.FRNN_OPT_GRID_NAXES, args.grid_naxes)
    elif path == "tc":
        # the tensor-core path's 128-query tasks want the longer rows of a
        # three-axis grid (the library's five- and four-axis defaults suit the scans)
        ctx.set_option(frnn.FRNN_OPT_GRID_NAXES, 3)
    with torch.cuda.stream(stream):
        pts = torch.from_numpy(pts_np).to(dev)
        counts = torch.empty(N, dtype=torch.int32, device=dev)
        idx = torch.empty((N, K), dtype=torch.int32, device=dev)
        d2 = torch.empty((N, K), dtype=torch.float32, device=dev)
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    grid = ctx.build_grid(pts, r)
    ctx.query(grid, pts, r, K, True, path, (counts, idx, d2))
    ctx.sync()
    gparams = grid.params()

    def step(ev=None, split=False):
        # split: an event at the build/query boundary as well (the attribution
        # pass, which also brackets the main query kernel with events)
        if ev is not None:
            ev[0].record(stream)
        ctx.build_grid(pts, r, grid=grid)
        if ev is not None and split:
            ev[1].record(stream)
        ctx.query(grid, pts, r, K, True, path, (counts, idx, d2))
        if ev is not None:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    ctx.sync()
    pairs = int(counts.sum().item())
    mk = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    evs = [(mk(), mk(), mk()) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(dev.index)
    sampler.start()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))          # evict L2 between timed steps (not timed)
        step(evs[k])
    ctx.sync()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    kern_is_tc = path == "tc"   # auto: a grid scan (five gridded axes up to D = 8, four above)
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    # attribution pass: the same K steps with events at the build/query
    # boundary and around the main query kernel (CUDA events on the launching
    # stream); kept out of the headline pass, where those records added about
    # 9 us to a 0.25 ms step by breaking the kernels' programmatic overlap
    ctx.set_option(frnn.FRNN_OPT_KERNEL_TIMING, 1)
    ctx.kernel_times()
    evs2 = [(mk(), mk(), mk()) for _ in range(args.steps)]
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        step(evs2[k], split=True)
    ctx.sync()
    kern_ms = ctx.kernel_times()           # one per step of the pass, same stream
    ctx.set_option(frnn.FRNN_OPT_KERNEL_TIMING, 0)
    build_ms = [e[0].elapsed_time(e[1]) for e in evs2]
    query_ms = [e[1].elapsed_time(e[2]) for e in evs2]
    total_ms = max_over_ranks(sum(step_ms), dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(N, args.steps, ws, total_ms)

    # end to end through the public host-buffer call: H2D in, build, query, D2H out
    h_pts = torch.from_numpy(pts_np).pin_memory()
    h_c = torch.empty(N, dtype=torch.int32).pin_memory()
    h_i = torch.empty((N, K), dtype=torch.int32).pin_memory()
    h_d = torch.empty((N, K), dtype=torch.float32).pin_memory()
    e2e_args = (h_pts.numpy(), r, K, path, (h_c.numpy(), h_i.numpy(), h_d.numpy()))
    for _ in range(max(1, args.warmup)):
        ctx.self_query_host(*e2e_args)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.self_query_host(*e2e_args)
    e2e_s = (time.perf_counter() - t0) / args.steps
    ok_e2e = np.array_equal(h_c.numpy(), counts.cpu().numpy())
    # the same with compact host output (the paper's NumPy-binding interface)
    cap = N * K
    h_off = torch.empty(N + 1, dtype=torch.int64).pin_memory()
    h_ci = torch.empty(cap, dtype=torch.int32).pin_memory()
    h_cd = torch.empty(cap, dtype=torch.float32).pin_memory()
    c_out = (h_off.numpy(), h_ci.numpy(), h_cd.numpy())
    for _ in range(max(1, args.warmup)):
        ctx.self_query_host_csr(h_pts.numpy(), r, K, path, c_out)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        off_np, ci_np, _ = ctx.self_query_host_csr(h_pts.numpy(), r, K, path, c_out)
    e2e_c_s = (time.perf_counter() - t0) / args.steps
    n_edges = int(off_np[-1])
    link = link_bandwidth(dev, stream)
    e2e_s = max_over_ranks(e2e_s, dev)
    e2e_c_s = max_over_ranks(e2e_c_s, dev)
    if ws > 1:
        # what follows needs no collective (the single-GPU legs run at N = 1 only)
        torch.distributed.destroy_process_group()
    keep = np.arange(K)[None, :] < h_c.numpy()[:, None]
    ok_c = bool(np.array_equal(np.diff(off_np), h_c.numpy()) and
                np.array_equal(ci_np, h_i.numpy()[keep]))

    hbm_peak, peak_kind = _peaks()
    qbytes = algorithmic_query_bytes(N, D, K)
    q_med = statistics.median(query_ms)
    k_mean = sum(kern_ms) / len(kern_ms)
    achieved = qbytes / (k_mean / 1e3) / 1e9
    prof = profile_summary("tc" if kern_is_tc else ("rows" if gparams["kernel"] == "rows" else "grid"),
                           args.workload)
    sm_count = int(getattr(torch.cuda.get_device_properties(dev), "multi_processor_count", 0))
    res = {
        "metric": METRIC,
        "value": value,
        "unit": "queries/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded clusters + background shaped like a tracking event)",
        "config": {"workload": w.name, "N": N, "D": D, "r": r, "K": K, "path": path,
                   "grid_naxes_option": ctx.get_option(frnn.FRNN_OPT_GRID_NAXES),
                   "gridded_axes": gparams["naxes"], "cell_mult": gparams["cell_mult"],
                   "grid_dims": gparams["dims"], "grid_cells": gparams["cells"],
                   "grid_kernel": gparams["kernel"],
                   "staging": ctx.get_option(frnn.FRNN_OPT_STAGING),
                   "self_query": True, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "pairs_per_s": whole_job_rate(pairs, args.steps, ws, total_ms),
        "neighbor_pairs": pairs,
        "build_ms_median": statistics.median(build_ms),
        "query_ms_median": q_med,
        "roofline": {"bound": "hbm",
                     "kernel": "k_tc_query" if kern_is_tc else
                               ("k_row_query" if gparams["kernel"] == "rows" else "k_grid_query"),
                     "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "kernel_ms_mean": k_mean,
                     "kernel_timing": "CUDA events around each launch of the kernel, on its stream, "
                                      "over a second pass of the same timed steps",
                     "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                     "algorithmic_bytes": qbytes,
                     "traffic": (prof or {}).get("traffic"),
                     # the kernel is bound by instruction issue, not HBM
                     "issue": issue_roofline((prof or {}).get("warp_instructions"), k_mean,
                                             sm_count, (clocks or {}).get("sm_max_mhz") or 2070.0)},
        "e2e": {"value": N * ws / e2e_c_s, "unit": "queries/s",
                "h2d_bytes_per_step": N * D * 4,
                "d2h_bytes_per_step": (N + 1) * 8 + 2 * n_edges * 4,
                "ms_per_step": e2e_c_s * 1e3, "output": "compact rows (frnn_self_query_host_csr)",
                "matches_device_path": ok_c,
                "link": link_roofline(link, N * D * 4, (N + 1) * 8 + 2 * n_edges * 4, e2e_c_s * 1e3)},
        "e2e_dense": {"value": N * ws / e2e_s, "unit": "queries/s",
                      "h2d_bytes_per_step": N * D * 4,
                      "d2h_bytes_per_step": N * 4 + 2 * N * K * 4,
                      "ms_per_step": e2e_s * 1e3, "output": "dense rows (frnn_self_query_host)",
                      "matches_device_path": bool(ok_e2e),
                      "link": link_roofline(link, N * D * 4, N * 4 + 2 * N * K * 4, e2e_s * 1e3)},
        "gpu_launches": launches_per_step(N, D, "tc" if kern_is_tc else "grid",
                                          ctx.get_option(frnn.FRNN_OPT_GRID_NAXES)) * args.steps,
        "wall_s": wall,
    }
    if clocks:
        res["clocks"] = clocks
    # the single-GPU legs: reported by the N = 1 run only, so that a run on
    # N GPUs holds them for the replicated headline step alone
    extras = rank == 0 and ws == 1
    if extras and not args.no_compact:
        res["compact_rows"] = run_compact(ctx, grid, pts, r, K, path, stream)
    if extras and not args.no_batched:
        res["batched_vs_plain"] = run_batched(ctx, args, dev, args.batch_path)
        if not args.no_tuned_batch:
            res["batched_vs_plain_tuned"] = run_batched_tuned(args, dev)
    if extras and not args.no_design_points:
        res["design_points"] = run_design_points(args, dev)
    if extras and not args.no_serving:
        res["serving"] = run_serving(ctx, args)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(pts_np, r, K, args.cpu_rows,
                                           gpu=(h_c.numpy(), h_i.numpy(), h_d.numpy()))
    ctx.close()
    return res if rank == 0 else None


def median_ci(xs, resamples=10000, seed=0):
    """Median of xs with a percentile-bootstrap 95% interval."""
    x = np.asarray(xs, dtype=np.float64)
    g = np.random.default_rng(seed)
    meds = np.median(x[g.integers(0, len(x), size=(resamples, len(x)))], axis=1)
    return float(np.median(x)), float(np.percentile(meds, 2.5)), float(np.percentile(meds, 97.5))


def sign_test(a, b):
    """Exact two-sided sign test of paired samples a, b (ties dropped):
    (wins of a < b, losses, p-value)."""
    from math import comb
    wins = sum(1 for x, y in zip(a, b) if x < y)
    losses = sum(1 for x, y in zip(a, b) if x > y)
    n = wins + losses
    if n == 0:
        return 0, 0, 1.0
    k = min(wins, losses)
    p = 2.0 * sum(comb(n, i) for i in range(k + 1)) / 2.0 ** n
    return wins, losses, min(1.0, p)


def run_batched_tuned(args, dev):
    """The batched leg with the autotuner's choices: one representative event
    per size class of the batch (power-of-two bucket of N) is tuned with
    frnn_autotune, then batched and plain calls take FRNN_PATH_AUTO."""
    import torch
    from paper_2609_31980_gb300 import frnn, synth
    w = synth.config4(n_events=args.batch_events)
    stream = torch.cuda.Stream()
    ctx = frnn.Context(stream=stream)
    classes = {}
    for p in w.events:
        classes.setdefault(int(np.log2(max(len(p), 1))), p)
    tuned = {}
    for b, p in sorted(classes.items()):
        with torch.cuda.stream(stream):
            t = torch.from_numpy(p).to(dev)
        tuned[f"N in [2^{b}, 2^{b + 1})"] = dict(ctx.autotune(t, w.r, w.K), representative_N=len(p))
        del t
    res = run_batched(ctx, args, dev, "auto")
    res["tuned_classes"] = tuned
    ctx.close()
    return res


def run_batched(ctx, args, dev, path):
    """64 uneven events (N ~ U[50k, 350k], D=8, the event mix): one batched
    call (segmented build + persistent query launch, replayed from its CUDA
    graph) against the same events one by one through the plain path.
    Rounds of the two are interleaved in a seeded random order, each round
    bracketed by synchronisation; medians with bootstrap intervals and an
    exact sign test over the paired rounds."""
    import torch
    from paper_2609_31980_gb300 import synth
    w = synth.config4(n_events=args.batch_events)
    K, r = w.K, w.r
    evs = [torch.from_numpy(p).to(dev) for p in w.events]
    total = sum(len(p) for p in w.events)
    outs = [(torch.empty(len(p), dtype=torch.int32, device=dev),
             torch.empty((len(p), K), dtype=torch.int32, device=dev),
             torch.empty((len(p), K), dtype=torch.float32, device=dev)) for p in w.events]
    torch.cuda.synchronize()   # the copies above ran on torch's stream, not the context's
    stream = ctx.stream
    mk = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    # plain: every event built and queried on its own
    grids = [None] * len(evs)

    def plain():
        for e, p in enumerate(evs):
            grids[e] = ctx.build_grid(p, r, grid=grids[e])
            ctx.query(grids[e], p, r, K, True, path, outs[e])

    def batched():
        ctx.query_batched(evs, r, K, path=path, outs=outs)

    fns = {"plain": plain, "batched": batched}
    for _ in range(args.batch_warmup):
        plain()
        batched()
    ctx.sync()
    order = np.random.default_rng(7)
    times = {"plain": [], "batched": []}
    for _ in range(args.batch_reps):
        for name in (("plain", "batched") if order.random() < 0.5 else ("batched", "plain")):
            torch.cuda.synchronize()
            a, b = mk(), mk()
            a.record(stream)
            fns[name]()
            b.record(stream)
            ctx.sync()
            times[name].append(a.elapsed_time(b))
    res = {}
    for name, t in times.items():
        med, lo, hi = median_ci(t)
        res[name] = {"ms_median": med, "ms_ci95": [lo, hi], "queries_per_s": total / (med / 1e3)}
    wins, losses, p = sign_test(times["batched"], times["plain"])
    pairs = int(sum(int(c.sum().item()) for c, _, _ in outs))
    return {"workload": w.name, "events": len(evs), "queries": total, "neighbor_pairs": pairs,
            "path": path, "rounds": args.batch_reps, "warmup": args.batch_warmup,
            "plain": res["plain"], "batched": res["batched"],
            "batched_over_plain": res["plain"]["ms_median"] / res["batched"]["ms_median"],
            "sign_test": {"batched_faster": wins, "plain_faster": losses, "p_two_sided": p}}


def run_compact(ctx, grid, pts, r, K, path, stream, reps=20):
    """Count-first compact rows (frnn_query_csr_count + frnn_query_csr_fill)
    against the dense rows on the same grid, at the workload's K and at
    K = 1000 (the paper's real-event setting, where dense rows are mostly
    padding).  Device time per query (grid built once, outside)."""
    import torch
    N = pts.shape[0]
    mk = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    out = {}
    for k in sorted({K, 1000}):
        with torch.cuda.stream(stream):
            dense = (torch.empty(N, dtype=torch.int32, device=pts.device),
                     torch.empty((N, k), dtype=torch.int32, device=pts.device),
                     torch.empty((N, k), dtype=torch.float32, device=pts.device))
        res = {}
        for name in ("dense", "compact"):
            ts = []
            for i in range(3 + reps):
                a, b = mk(), mk()
                a.record(stream)
                if name == "dense":
                    ctx.query(grid, pts, r, k, True, path, dense)
                else:
                    with torch.cuda.stream(stream):
                        off, idx, d2, _ = ctx.query_csr(grid, pts, r, k, True, path)
                b.record(stream)
                ctx.sync()
                if i >= 3:
                    ts.append(a.elapsed_time(b))
            res[name] = statistics.median(ts)
        E = int(off[-1].item())
        dense_bytes = N * 4 + 2 * N * k * 4
        csr_bytes = (N + 1) * 8 + 2 * E * 4
        out[f"K{k}"] = {"dense_ms": res["dense"], "compact_ms": res["compact"],
                        "edges": E, "dense_output_bytes": dense_bytes,
                        "compact_output_bytes": csr_bytes,
                        "compact_matches_dense": bool(torch.equal(
                            torch.diff(off).to(torch.int32), dense[0]))}
        del dense
    return out


def _serving_inputs(n_ev, sizes, D):
    """All events of the serving stream in one page-locked host buffer
    (drawn by a pool of spawned processes: about 250 M points in total)."""
    import multiprocessing as mp
    import torch
    from paper_2609_31980_gb300 import synth
    offs = np.zeros(n_ev + 1, np.int64)
    offs[1:] = np.cumsum(sizes[:n_ev])
    flat = torch.empty(int(offs[-1]) * D, dtype=torch.float32, pin_memory=True)
    fv = flat.numpy()
    workers = max(1, min(16, len(os.sched_getaffinity(0))))
    with mp.get_context("spawn").Pool(workers) as pool:
        for e, p in enumerate(pool.imap(synth.config5_event_args, [(e, sizes) for e in range(n_ev)],
                                        chunksize=4)):
            fv[offs[e] * D:offs[e + 1] * D] = p.reshape(-1)
    return [fv[offs[e] * D:offs[e + 1] * D].reshape(-1, D) for e in range(n_ev)], flat


def run_serving(ctx, args):
    """The serving workload: a Poisson stream of 2,000 events (N log-uniform
    on [20k, 400k], D=8, the event mix, r=0.1, K=64) through the
    continuous-batching loop under a 40 GB budget, against the same stream
    served one event at a time (1 slot, batch of 1), at several offered loads
    (multiples of the measured one-at-a-time capacity).

    Inputs are page-locked host buffers.  Results go to a pool of
    page-locked output buffers: request e writes buffer e mod P (P > the
    requests one batch round can hold), so host memory stays bounded; two
    requests far apart in arrival order may share a buffer, which is harmless
    here because this leg only times the loop (served results are compared
    with the oracle and the single-event path by the tests)."""
    import torch
    from paper_2609_31980_gb300 import synth
    n_ev = args.serve_events
    sizes = synth.serving_sizes(2000)[:n_ev]
    K, r, D = 64, 0.1, 8
    t0 = time.perf_counter()
    events, _flat = _serving_inputs(n_ev, sizes, D)
    gen_s = time.perf_counter() - t0
    P = min(n_ev, max(args.serve_pool, args.serve_slots * args.serve_batch + 2))
    pool_n = [int(sizes[j::P].max()) for j in range(P)]
    pool = [(torch.empty(n, dtype=torch.int32, pin_memory=True).numpy(),
             torch.empty((n, K), dtype=torch.int32, pin_memory=True).numpy(),
             torch.empty((n, K), dtype=torch.float32, pin_memory=True).numpy()) for n in pool_n]
    outs = [tuple(a[:len(events[e])] for a in pool[e % P]) for e in range(n_ev)]
    budget = 40 * 10 ** 9
    # warm-up (module loading, first launches, slot workspaces), not measured
    ctx.serve(events[:8], np.zeros(8), r, K, budget, slots=args.serve_slots,
              max_batch=args.serve_batch, outs=outs[:8])
    # sequential capacity: everything queued at t = 0, one event at a time
    # (the better of two runs)
    cap = 0.0
    for _ in range(2):
        _, _, seq0 = ctx.serve(events, np.zeros(n_ev), r, K, budget, slots=1, max_batch=1,
                               outs=outs)
        cap = max(cap, seq0["events_per_s"])
    out = {"workload": f"serving-{n_ev}ev-logU20k-400k-x8-r0.1-k64", "events": n_ev,
           "mean_N": float(np.mean(sizes)), "points": int(np.sum(sizes)),
           "budget_bytes": budget, "slots": args.serve_slots, "max_batch": args.serve_batch,
           "output_pool_buffers": P, "input_generation_s": gen_s,
           "sequential_capacity_events_per_s": cap, "loads": []}
    for load in args.serve_loads:
        arr = synth.poisson_arrivals(n_ev, load * cap)
        _, _, cb = ctx.serve(events, arr, r, K, budget, slots=args.serve_slots,
                             max_batch=args.serve_batch, outs=outs)
        _, _, sq = ctx.serve(events, arr, r, K, budget, slots=1, max_batch=1, outs=outs)
        out["loads"].append({
            "rate_x_sequential_capacity": load, "rate_hz": load * cap,
            "continuous": {k: cb[k] for k in ("p50_ms", "p99_ms", "events_per_s", "completed",
                                               "peak_inflight_batches", "peak_inflight_bytes")},
            "sequential": {k: sq[k] for k in ("p50_ms", "p99_ms", "events_per_s", "completed")}})
    del pool, outs, events, _flat
    return out


def cpu_baseline(pts_np, r, K, rows, gpu=None):
    """The oracle (brute force, FP32 contract) on a bounded sample of queries;
    with ``gpu`` = the library's dense result (counts, idx, dist2) of the same
    event, the sampled rows are also compared with it element by element."""
    from oracle import oracle
    g = np.random.default_rng(0)
    sel = np.sort(g.choice(len(pts_np), size=min(rows, len(pts_np)), replace=False))
    oracle.self_query(pts_np, r, K, rows=sel[:64])     # warm (page-in, thread pool)
    t0 = time.perf_counter()
    want = oracle.self_query(pts_np, r, K, rows=sel)
    dt = time.perf_counter() - t0
    out = {"value": len(sel) / dt, "unit": "queries/s", "cores": oracle.num_threads(),
           "kind": "oracle",
           "sample": f"{len(sel)} of {len(pts_np)} query rows, each brute-forced against all "
                     f"{len(pts_np)} points ({dt:.1f} s)"}
    if gpu is not None:
        try:
            gc, gi, gd = gpu
            same = (np.array_equal(gc[sel], want[0]) and np.array_equal(gi[sel], want[1]) and
                    np.array_equal(np.ascontiguousarray(gd[sel]).view(np.uint32),
                                   want[2].view(np.uint32)))
            out["gpu_rows_equal"] = {"rows": int(len(sel)), "equal": bool(same),
                                     "compared": "counts, indices, distance bits"}
        except Exception as e:   # noqa: BLE001 - a report, never fatal
            out["gpu_rows_equal"] = {"error": str(e)[:100]}
    # the 4096 x 3 uniform set on one core and on all (a separate process, so
    # that the OpenMP thread count can be fixed)
    code = ("import sys, time; sys.path.insert(0, %r); from oracle import oracle; "
            "from paper_2609_31980_gb300 import synth; w = synth.config1(); "
            "oracle.self_query(w.points, w.r, w.K); t = time.perf_counter(); "
            "oracle.self_query(w.points, w.r, w.K); "
            "print(len(w.points) / (time.perf_counter() - t), oracle.num_threads())" % ROOT)
    for tag, env in (("uniform4096x3_1core", {"OMP_NUM_THREADS": "1"}), ("uniform4096x3_all_cores", {})):
        try:
            pr = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                                timeout=120, env={**os.environ, **env})
            v, c = pr.stdout.split()
            out[tag] = {"queries_per_s": float(v), "cores": int(c)}
        except Exception as e:   # noqa: BLE001 - a baseline detail, never fatal
            out[tag] = {"error": str(e)[:100]}
    return out


def run_reference(args):
    """--impl reference: the CPU oracle as it stands, on bounded samples."""
    ws, rank, _ = _dist_env()
    if rank != 0:
        return None
    from oracle import oracle
    w = workload(args.workload)
    pts_np = w.points
    N, D, r, K = pts_np.shape[0], w.D, w.r, w.K
    rows = args.ref_rows
    g = np.random.default_rng(1)
    for _ in range(args.warmup):
        oracle.self_query(pts_np, r, K, rows=g.choice(N, size=16, replace=False))
    times = []
    for _ in range(args.steps):
        sel = np.sort(g.choice(N, size=rows, replace=False))
        t0 = time.perf_counter()
        oracle.self_query(pts_np, r, K, rows=sel)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = rows * args.steps / tot
    cores = oracle.num_threads()
    sample = f"{rows} query rows per step of {N}, each brute-forced against all {N} points"
    return {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded clusters + background shaped like a tracking event)",
            "config": {"workload": w.name, "N": N, "D": D, "r": r, "K": K, "self_query": True},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-rows", type=int, default=300000, help="oracle query rows (all: ~20 s on 16 cores)")
    ap.add_argument("--ref-rows", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cell-mult", type=int, default=0, help="grid cell multiple m (0: library default)")
    ap.add_argument("--exit-dims", type=int, default=0, help="dims before the warp vote (0: default)")
    ap.add_argument("--grid-axes", type=int, default=0, help="0: last axes, 1: widest axes")
    ap.add_argument("--grid-naxes", type=int, default=0, help="gridded axes (0: library default)")
    ap.add_argument("--path", default="grid", choices=["grid", "tc", "auto"])
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-compact", action="store_true")
    ap.add_argument("--batch-events", type=int, default=64)
    ap.add_argument("--batch-reps", type=int, default=30, help="timed rounds of each")
    ap.add_argument("--batch-warmup", type=int, default=10)
    ap.add_argument("--batch-path", default="grid", choices=["grid", "tc", "auto"])
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-design-points", action="store_true")
    ap.add_argument("--no-tuned-batch", action="store_true")
    ap.add_argument("--serve-events", type=int, default=2000)
    ap.add_argument("--serve-pool", type=int, default=48, help="page-locked output buffers")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-batch", type=int, default=8)
    ap.add_argument("--serve-loads", type=float, nargs="*", default=[0.9, 1.5, 3.0])
    ap.add_argument("--workload", default="event300k", choices=["event300k", "event500k"])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
