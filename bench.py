"""Benchmark: edges/s to a full MIS on one GB300 (and N replicas under torchrun).

A step is one full solve of the hot path -- Eq. 1 priorities, then every
round of Algorithm 2 (selection test, exclusion test, state update,
compaction) until the alive set is empty -- on a graph already resident in
HBM.  value = arcs solved / device time of the K timed steps (CUDA events on
the launching stream; a 256 MB write between steps flushes L2).  The timed
graph is created with no create-time decisions (order_rows = 0), so each
solve starts from the CSR; the same solve on a graph whose create-time
structures decide the seed-independent round-0 vertices is reported beside
it as `amortized`, with create times and create + first solve.

Workloads (synthetic, seeded; stand-ins for the paper's SuiteSparse graphs):
  rmat22     R-MAT scale 22, edge factor 16, (0.57, 0.19, 0.19, 0.05), permuted (default;
             its line also carries the batch4096 and serve legs below)
  er10k      Erdos-Renyi G(10,000, 40,000)
  grid       2048 x 2048 grid + 5% random diagonals, natural ids
  grid_perm  the same grid, permuted ids
  stencil    160^3 lattice, 27-point stencil, natural ids (dense 16 x 16 tiles)
  rgg4m      random geometric graph, 2^22 vertices, average degree 10, cell-sorted ids
             (the geometric family of batch4096 as one graph; dense 16 x 16 tiles)
  batch4096  4096 graphs (log-uniform 64..65,536 vertices, ER / random geometric)
             packed as one block-diagonal union and solved in one launch
  serve      Poisson arrivals of solve requests over a resident pool of 512 graphs
             (continuous batching), graphs/s and p50/p99 vs sequential solves
  dynamic    batches of edge insertions/deletions on the resident R-MAT scale 22
             graph, each applied and the MIS repaired (H1 priority), vs a full solve

`--impl reference` times the CPU oracle (a plain sequential restatement of
the same computation) on the host cores instead.

Run: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]
"""
from __future__ import annotations

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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "edges/s to full MIS on 1 GB300"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
PATH_NAMES = {1: "csr", 2: "tile", 3: "tile_tc", 4: "push", 5: "cluster", 6: "rows_tc"}
PAYLOADS = {"bits": 0, "b1": 1, "int8": 2, "fp16": 3}  # mis_set_tile_payload forms


def _peak_hbm():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def profiled_traffic(kernel_files, summary):
    """DRAM bytes per launch from a committed ncu summary, if the kernel
    sources still hash to the digest recorded there (else None)."""
    import hashlib
    import re
    try:
        h = hashlib.sha256()
        for f in kernel_files:
            with open(os.path.join(ROOT, "paper_2605_29604_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
        text = open(os.path.join(ROOT, "profiles", summary)).read()
        digest = re.search(r"first 16 hex\): `([0-9a-f]{16})`", text).group(1)
        traffic = int(re.search(r"traffic_bytes_per_launch: (\d+)", text).group(1))
        return traffic if h.hexdigest()[:16] == digest else None
    except Exception:
        return None


def make_workload(name):
    from paper_2605_29604_gb300 import graphgen as gg
    if name == "rmat22":
        return gg.rmat22(seed=22), "R-MAT scale 22, edge factor 16, (0.57,0.19,0.19,0.05), permuted"
    if name == "rmat18":
        return gg.rmat22(seed=22, scale=18), "R-MAT scale 18, edge factor 16, permuted"
    if name == "er10k":
        return gg.er_10k_deg8(1), "Erdos-Renyi G(n=10,000, m=40,000), avg degree 8"
    if name == "grid":
        return gg.grid2048(seed=3), "2048x2048 grid + 5% random diagonals, natural ids"
    if name == "grid_perm":
        return gg.grid2048(seed=3, permute_ids=True), "2048x2048 grid + 5% diagonals, permuted ids"
    if name == "stencil":
        return gg.stencil160(), "160x160x160 lattice, 27-point stencil, natural ids"
    if name == "rgg4m":
        return (gg.rgg(1 << 22, 10.0, 7),
                "random geometric graph, 4,194,304 vertices in the unit square, average degree 10, "
                "cell-sorted ids")
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_rate(g, min_seconds=0.0, max_repeats=1):
    """CPU oracle (keys + round simulation), sequential C on one host core:
    edges/s over `repeats` full solves of g (repeated until min_seconds)."""
    import oracle
    n, rp, col = g
    t0 = time.perf_counter()
    reps = 0
    while True:
        res = oracle.solve(n, rp, col, 1)
        reps += 1
        if reps >= max_repeats and time.perf_counter() - t0 >= min_seconds:
            break
    dt = (time.perf_counter() - t0) / reps
    return int(rp[-1]) / dt, dt, res, reps


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    name = {"rmat22": "rmat18", "batch4096": "er10k", "serve": "er10k",
            "dynamic": "rmat18"}.get(args.workload, args.workload)
    g, desc = make_workload(name)
    n, rp, col = g
    for _ in range(args.warmup):
        oracle_rate(g)
    times = []
    for _ in range(args.steps):
        _, dt, res, _ = oracle_rate(g)
        times.append(dt)
    total = sum(times)
    value = args.steps * int(rp[-1]) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload, "sample": desc, "n": n, "arcs": int(rp[-1]),
                   "rounds": res.rounds},
        "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                         "sample": f"one full oracle solve of {desc} per step"},
        "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _dist_setup():
    """World size, rank and local rank from the torchrun environment: one
    process per GPU over NCCL, or gloo on a host without a GPU."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    return world, rank, local


def _reduce_over_ranks(x, world, op):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=op)
    return float(t.item())


def _max_over_ranks(x, world):
    import torch.distributed as dist
    return _reduce_over_ranks(x, world, dist.ReduceOp.MAX)


def _sum_over_ranks(x, world):
    import torch.distributed as dist
    return _reduce_over_ranks(x, world, dist.ReduceOp.SUM)


def replica_throughput(world, steps, units_per_step, max_total_ms):
    """Whole-job throughput of `world` independent replicas (weak scaling):
    every rank processes steps * units_per_step, the job takes the slowest
    rank's time."""
    return world * steps * units_per_step / (max_total_ms / 1e3)


def time_device_steps(native, h, seeds, out_ptr, stream, steps, warmup, local, world,
                      replay=None):
    """Per-step CUDA-event times (L2 flushed between steps), clocks sampled.
    With `replay` (from mis_capture) each step replays the captured solve."""
    import torch
    import torch.distributed as dist
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device="cuda")

    def step():
        if replay is not None:
            native.mis_replay_launch(replay, stream)
        else:
            native.mis_solve_ex(h, seeds, out_ptr, stream)

    for _ in range(max(warmup, 3)):
        step()
    native.mis_get_stats(h)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(steps):
            flush.add_(1.0)  # write 256 MB: evicts the previous step from L2
            starts[i].record()
            step()
            ends[i].record()
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    return step_ms, clk.summary()


def create_timings(native, n, drp, dcol, stream, local, variants, reps=2):
    """Create from a device-resident CSR, then the first solve, per option set:
    the best of `reps` of create alone (host wall clock; mis_create_ex returns
    once the graph is resident) and of create + first solve between CUDA
    events on the solve stream."""
    import torch
    out = {}
    res = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    for name, opt in variants:
        best_c, best_cs = float("inf"), float("inf")
        for _ in range(reps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record()
            h = native.mis_create_ex(n, drp, dcol, 1, opt, stream)
            t1 = time.perf_counter()
            native.mis_solve_ex(h, [1], res.data_ptr(), stream)
            e1.record()
            torch.cuda.synchronize()
            native.mis_destroy(h)
            best_c = min(best_c, t1 - t0)
            best_cs = min(best_cs, e0.elapsed_time(e1))
        out[name] = {"create_s": best_c, "create_plus_first_solve_ms": best_cs}
    return out


def tuned_handle(native, n, drp, dcol, stream, local, order_rows, args):
    """A resident graph with the given create-time row ordering, on the launch
    configuration the flags force or the autotuner picks."""
    opt = native.options(device=local, check_symmetry=1, order_rows=order_rows)
    h = native.mis_create_ex(n, drp, dcol, 1, opt, stream)
    tuning, tune_s = None, 0.0
    if args.tpr is not None:
        native.mis_set_path(h, native.MIS_PATH_CSR, args.tpr)
        if args.csr_pending is not None:
            native.mis_set_csr_pending(h, args.csr_pending)
        if args.bins:
            native.mis_set_csr_bins(h, [int(x) for x in args.bins.split(",")])
        if args.grid:
            native.mis_set_grid(h, args.grid)
    elif args.path:
        if args.path == "tile_tc":
            native.mis_set_tile_payload(h, PAYLOADS[args.payload])
        native.mis_set_path(h, {"tile": 2, "tile_tc": 3, "push": 4, "cluster": 5}[args.path],
                            args.tile if args.path in ("tile", "tile_tc") else 0)
    else:
        t0 = time.perf_counter()
        tuning = native.mis_autotune(h, 3)
        tune_s = time.perf_counter() - t0
    return h, tuning, tune_s


def tuning_dict(tuning, tune_s):
    if tuning is None:
        return None
    return {"path": PATH_NAMES.get(tuning.path), "param": tuning.param,
            "bounds": list(tuning.bounds), "grid": tuning.grid, "candidates": tuning.candidates,
            "seconds": tune_s, "csr_pending": tuning.csr_pending,
            "arcs_per_tile": tuning.arcs_per_tile}


def phase_us(st):
    r = min(st.rounds, 64)
    return {"init": st.init_ns / 1e3, "select": [st.select_ns[i] / 1e3 for i in range(r)],
            "exclude": [st.exclude_ns[i] / 1e3 for i in range(r)]}


def run_single(args):
    import torch

    from paper_2605_29604_gb300 import native
    world, rank, local = _dist_setup()
    g, desc = make_workload(args.workload)
    n, rp, col = g
    arcs = int(rp[-1])
    stream = torch.cuda.current_stream().cuda_stream
    # the CSR resident in HBM before anything is timed
    drp_t = torch.from_numpy(rp).cuda()
    dcol_t = torch.from_numpy(col if arcs else np.zeros(1, np.int32)).cuda()
    drp, dcol = drp_t.data_ptr(), dcol_t.data_ptr()

    # create, and create + first solve, per create-time option set
    creates = create_timings(native, n, drp, dcol, stream, local, [
        ("default", native.options(device=local)),
        ("full_rows", native.options(device=local, check_symmetry=1, order_rows=0)),
        ("round0_structures", native.options(device=local, check_symmetry=1, order_rows=2)),
    ])

    # ---- the headline: Algorithm 2 from the CSR.  A graph created with
    # order_rows = 0 keeps no create-time decision (no degree-ordered rows,
    # round-0 classes, tested subgraph or keyed list): every solve computes
    # every key and tests every undecided vertex over its full row.
    h, tuning, tune_s = tuned_handle(native, n, drp, dcol, stream, local, 0, args)
    out = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    seeds = np.array([1], dtype=np.uint64)
    step_ms, clocks = time_device_steps(native, h, seeds, out.data_ptr(), stream, args.steps,
                                        args.warmup, local, world)
    total_ms = _max_over_ranks(sum(step_ms), world)
    st = native.mis_get_stats(h)
    value = replica_throughput(world, args.steps, arcs, total_ms)
    launch_s = (total_ms / 1e3) / args.steps
    full_result = out[:n].cpu().numpy()
    # with a pinned tile path: several seeds of the same graph per launch on it
    path_multi = None
    if (args.path in ("tile", "tile_tc") or args.multi_form) and args.multi > 0:
        kk = min(args.multi, 8)
        if args.multi_form == "auto":
            native.mis_autotune_multi(h, kk, 3)
        elif args.multi_form:
            native.mis_set_multi_form(h, {"rows": native.MIS_MULTI_ROWS,
                                          "rows_tc": native.MIS_MULTI_ROWS_TC}[args.multi_form])
        mout = torch.empty(max(kk * n, 1), dtype=torch.uint8, device="cuda")
        mseeds = np.arange(1, kk + 1, dtype=np.uint64)
        flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device="cuda")
        for _ in range(max(args.warmup, 3)):
            native.mis_solve_multi_ex(h, mseeds, mout.data_ptr(), stream)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for e0, e1 in ev:
            flush.add_(1.0)
            e0.record()
            native.mis_solve_multi_ex(h, mseeds, mout.data_ptr(), stream)
            e1.record()
        torch.cuda.synchronize()
        mst = native.mis_get_stats(h)
        mt = float(np.median([e0.elapsed_time(e1) for e0, e1 in ev]))
        path_multi = {"k": kk, "launch_ms_p50": mt, "per_solve_ms": mt / kk,
                      "path": PATH_NAMES.get(mst.path), "rounds": mst.rounds,
                      "phase_us": phase_us(mst)}
    native.mis_destroy(h)

    # ---- amortised: the same solve on a graph whose create-time structures
    # (degree-sorted rows, round-0 classes, tested subgraph, keyed list) have
    # already decided every seed-independent round-0 vertex
    amort = None
    multi = None
    if args.amortized and args.path is None:
        ha, atuning, atune_s = tuned_handle(native, n, drp, dcol, stream, local, 2, args)
        aout = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
        a_ms, a_clocks = time_device_steps(native, ha, seeds, aout.data_ptr(), stream,
                                           args.steps, args.warmup, local, world)
        ast = native.mis_get_stats(ha)
        a_solve = float(np.median(a_ms))
        f_solve = float(np.median(step_ms))
        dc = creates["round0_structures"]["create_s"] - creates["full_rows"]["create_s"]
        gain_s = (f_solve - a_solve) / 1e3
        amort = {
            "per_solve_ms_p50": a_solve, "edges_per_s": arcs / (a_solve / 1e3),
            "create_s": creates["round0_structures"]["create_s"],
            "break_even_seeds": (dc / gain_s) if gain_s > 0 else None,
            "rounds": ast.rounds, "sure_in": ast.sure_in, "sure_out": ast.sure_out,
            "tested_rows": ast.tested_rows, "tested_arcs": ast.tested_arcs,
            "keyed": ast.keyed, "phase_us": phase_us(ast), "autotune": tuning_dict(atuning, atune_s),
            "same_result": bool(np.array_equal(aout[:n].cpu().numpy(), full_result)),
            "what": "mis_create_ex with order_rows=2: seed-independent round-0 decisions made at "
                    "create time, so a solve tests only the tested subgraph; valid for repeated "
                    "seeds of one resident graph"}
        # several seeds of the same resident graph per launch (mis_solve_multi_ex)
        if args.multi > 0:
            kk = min(args.multi, 8)
            mout = torch.empty(max(kk * n, 1), dtype=torch.uint8, device="cuda")
            mseeds = np.arange(1, kk + 1, dtype=np.uint64)
            flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device="cuda")
            for _ in range(max(args.warmup, 3)):
                native.mis_solve_multi_ex(ha, mseeds, mout.data_ptr(), stream)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            for e0, e1 in ev:
                flush.add_(1.0)  # L2 flushed between launches, as for the single solves
                e0.record()
                native.mis_solve_multi_ex(ha, mseeds, mout.data_ptr(), stream)
                e1.record()
            torch.cuda.synchronize()
            mst = native.mis_get_stats(ha)
            mt = float(np.median([e0.elapsed_time(e1) for e0, e1 in ev]))
            multi = {"k": kk, "launch_ms_p50": mt, "per_solve_ms": mt / kk,
                     "edges_per_s_aggregate": kk * arcs / (mt / 1e3), "rounds": mst.rounds,
                     "kernel": "multi_solve_kernel (k seeds of the amortised graph per "
                               "persistent launch)"}
        native.mis_destroy(ha)
    del drp_t, dcol_t

    # end to end through the C ABI with host buffers: pinned CSR in, result out
    e2e = None
    if args.e2e_steps > 0:
        prp = torch.from_numpy(rp).pin_memory().numpy()
        pcol = torch.from_numpy(col).pin_memory().numpy()
        hout = torch.empty(max(n, 1), dtype=torch.uint8).pin_memory().numpy()
        # one create + one solve per step: no create-time row ordering (for a
        # single solve it costs more than it saves), input symmetry trusted (it
        # was checked when the graph was made); the upload overlaps its checks
        e2e_opt = native.options(device=local, check_symmetry=0, order_rows=0)
        times = []
        for i in range(args.e2e_steps + 1):
            t0 = time.perf_counter()
            h2 = native.mis_create_ex(n, prp, pcol, 0, e2e_opt, None)
            native.mis_solve(h2, 1, hout)
            native.mis_destroy(h2)
            if i:
                times.append(time.perf_counter() - t0)
        e2e_s = _max_over_ranks(sum(times), world)
        e2e = {"value": world * arcs * len(times) / e2e_s, "unit": "edges/s",
               "h2d_bytes_per_step": 4 * (n + 1) + 4 * arcs, "d2h_bytes_per_step": n,
               "same_result": bool(np.array_equal(hout[:n], full_result)),
               "path": "mis_create_ex(host CSR from pinned memory, uploaded in pieces with "
                       "row-pointer/range/order validation overlapped; degree binning included; "
                       "no row ordering; symmetry check off) + mis_solve(host result) + "
                       "mis_destroy"}

    peak, peak_kind = _peak_hbm()
    # the one-read volume of the CSR (B0): every arc and row pointer once
    b0 = 4 * arcs + 4 * (n + 1)
    achieved = b0 / launch_s / 1e9
    traffic = args.traffic
    if traffic is None and args.workload == "rmat22" and st.path == 1:
        traffic = profiled_traffic(["kernels_csr.cu", "common.cuh", "init.cuh", "worklist.cuh"],
                                   "csr_solve_full_rmat22.md")
    path = PATH_NAMES.get(st.path, str(st.path))
    line = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload, "graph": desc, "n": n, "arcs": arcs,
                   "solve": "Algorithm 2 from the CSR: graph created with order_rows=0, no "
                            "create-time decisions; every key computed and every undecided "
                            "vertex tested over its full row in every solve",
                   "rounds": st.rounds, "path": path, "threads_per_row": st.threads_per_row,
                   "tile": st.tile, "mis_size": st.mis_size,
                   "l2": "flushed between steps (256 MB write); graph (513 MB col_idx for rmat22) "
                         "also exceeds L2",
                   "parallelism": f"replicas{world}", "create": creates,
                   "step_ms_p10_p50_p90": [float(np.percentile(step_ms, q)) for q in (10, 50, 90)],
                   "phase_us": phase_us(st), "autotune": tuning_dict(tuning, tune_s)},
        "gpu_launches": args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": f"{peak_kind} burst copy bandwidth (of {peak_kind})",
                     "alg_bytes_per_launch": b0,
                     "alg_bytes_def": "B0 = 4*arcs + 4*(n+1): one read of col_idx and row_ptr",
                     "kernel": f"{path} persistent round kernel (one launch per solve), full rows"},
        "clocks": clocks,
        "e2e": e2e,
    }
    if amort is not None:
        line["config"]["amortized"] = amort
    if path_multi is not None:
        line["config"]["multi_seed_on_path"] = path_multi
    if args.path == "tile_tc":
        line["config"]["tile_payload"] = args.payload
    if multi is not None:
        line["config"]["multi_seed"] = multi
    legs = [x for x in (args.legs or "").split(",") if x]
    if "batch" in legs:
        line["batch4096"] = batch_leg(args, native, local, world)
    if "serve" in legs:
        line["serve"] = serve_leg(args, native, local, world, rank)
    if "tc" in legs:
        line["tiles_tc"] = tc_leg(args, native, local, world, "grid")
        line["tiles_tc_stencil"] = tc_leg(args, native, local, world, "stencil")
        line["tiles_tc_rgg"] = tc_leg(args, native, local, world, "rgg4m")
    if rank == 0 and args.cpu_baseline:
        import oracle
        rate, dt, res, reps = oracle_rate(g, min_seconds=args.cpu_seconds)
        mdg, _ = oracle.min_degree_greedy(*g)
        line["cpu_baseline"] = {"value": rate, "unit": "edges/s", "cores": 1, "kind": "oracle",
                                "sample": f"{reps} full oracle solve(s) of the same graph "
                                          f"({dt:.2f} s each)",
                                "quality": {"mis_size": int(res.status.sum()),
                                            "min_degree_greedy": mdg},
                                "gpu_result_equals_oracle": bool(np.array_equal(
                                    full_result, res.status))}
        # work bytes of the pull rounds (each undecided row read in full, each
        # round's alive set listed and read back), from the oracle's counts
        wb = 4 * int(res.work) + 8 * int(res.alive_sum) + 4 * n + n
        line["roofline"]["work_bytes"] = wb
        line["roofline"]["work_def"] = ("B_csr = 4*W + 8*sum_r |und_r| + 4*n + n, W = sum over "
                                        "rounds of the degrees of the undecided vertices "
                                        f"(oracle: W = {int(res.work)}, sum |und_r| = "
                                        f"{int(res.alive_sum)})")
        line["roofline"]["work_frac"] = wb / launch_s / 1e9 / peak
        # the second CPU baseline: the same rounds on all host cores (OpenMP)
        pn, prp, pcol = g
        pkeys = oracle.keys(pn, prp, 1)
        oracle.rounds_parallel(pn, prp, pcol, pkeys)  # warm-up (threads, pages)
        t0 = time.perf_counter()
        preps = 0
        while True:
            pres = oracle.rounds_parallel(pn, prp, pcol, pkeys)
            preps += 1
            if preps >= 3 and time.perf_counter() - t0 >= min(args.cpu_seconds, 5.0):
                break
        pdt = (time.perf_counter() - t0) / preps
        line["cpu_parallel"] = {
            "value": int(prp[-1]) / pdt, "unit": "edges/s", "cores": oracle.parallel_threads(),
            "kind": "Algorithm 2's rounds over worklists, OpenMP (oracle/cpu_parallel.c); "
                    "keys precomputed, not timed",
            "sample": f"{preps} full solves of the same graph ({pdt * 1e3:.1f} ms each)",
            "result_equals_oracle": bool(np.array_equal(pres.status, res.status))}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def batch_leg(args, native, local, world):
    """Config 4: the 4096-graph union, one captured persistent launch per step."""
    import torch

    from paper_2605_29604_gb300 import graphgen as gg
    t0 = time.perf_counter()
    parts = gg.batch_mixed(args.batch_count, seed=4096, nmin=64, nmax=65536)
    t_gen = time.perf_counter() - t0
    arcs = int(sum(int(p[1][-1]) for p in parts))
    nsum = int(sum(p[0] for p in parts))
    t0 = time.perf_counter()
    h = native.mis_create_batch(parts, native.options(device=local, check_symmetry=1,
                                                      order_rows=args.batch_order))
    t_create = time.perf_counter() - t0
    tuning = native.mis_autotune(h, 3)
    size = native.lib().mis_result_size(h)
    out = torch.empty(max(size, 1), dtype=torch.uint8, device="cuda")
    seeds = np.arange(1, len(parts) + 1, dtype=np.uint64)
    stream = torch.cuda.current_stream().cuda_stream
    # one persistent launch per step, replayed from a captured CUDA graph
    replay = native.mis_capture(h, seeds, out.data_ptr())
    step_ms, clocks = time_device_steps(native, h, seeds, out.data_ptr(), stream, args.steps,
                                        args.warmup, local, world, replay=replay)
    total_ms = _max_over_ranks(sum(step_ms), world)
    st = native.mis_get_stats(h)
    native.mis_replay_destroy(replay)
    # the union's result against standalone solves of a sample of its graphs
    got = out[:size].cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([p[0] for p in parts])])
    checked, same = 0, True
    for i in range(0, len(parts), max(1, len(parts) // 64)):
        pn, prp, pcol = parts[i]
        h1 = native.mis_create_ex(pn, prp, pcol, 0, native.options(device=local,
                                                                    check_symmetry=0), None)
        want = native.mis_solve(h1, int(seeds[i]))
        native.mis_destroy(h1)
        same &= bool(np.array_equal(got[offs[i]:offs[i + 1]], want[:pn]))
        checked += 1
    native.mis_destroy(h)
    peak, peak_kind = _peak_hbm()
    launch_s = (total_ms / 1e3) / args.steps
    b0 = 4 * arcs + 4 * (nsum + len(parts))
    return {
        "graphs": len(parts), "n_total": nsum, "arcs": arcs, "steps": args.steps,
        "ms_per_launch": total_ms / args.steps,
        "graphs_per_s": world * args.steps * len(parts) / (total_ms / 1e3),
        "edges_per_s": replica_throughput(world, args.steps, arcs, total_ms),
        "rounds": st.rounds, "path": PATH_NAMES.get(st.path), "gen_s": t_gen,
        "create_s": t_create, "create_order_rows": args.batch_order,
        "create_note": ("order_rows=2: the union's round-0 classes are made at create time "
                        "(seed-independent), so each replayed solve tests only the rest"
                        if args.batch_order else "no create-time decisions"),
        "autotune": {"path": PATH_NAMES.get(tuning.path), "bounds": list(tuning.bounds),
                     "grid": tuning.grid, "csr_pending": tuning.csr_pending},
        "launch": "captured CUDA graph replay (mis_capture, mis_replay_launch)",
        "phase_us": phase_us(st), "l2": "flushed between steps (256 MB write)",
        "roofline": {"b0_bytes": b0, "b0_frac": b0 / launch_s / 1e9 / peak, "peak": peak,
                     "b0_def": "4*arcs + 4*(n+1) per graph"},
        "standalone_check": {"graphs_checked": checked, "all_equal": same},
        "clocks": clocks,
    }


def tc_leg(args, native, local, world, workload="grid"):
    """The tile paths on a graph with dense 16 x 16 tiles (the grid with
    natural ids, 13 arcs per tile; the 27-point stencil, 16): one solve per
    path and tile payload, and 8 seeds per launch on the CSR rows (CUDA
    cores) against the forms with the exclusion product A x [C_1 .. C_8] on
    tensor cores: the selection on the CSR rows with the product over the
    bitmask tiles (rows_tc_b1), and the tile kernel per payload form."""
    import torch
    (n, rp, col), desc = make_workload(workload)
    stream = torch.cuda.current_stream().cuda_stream
    drp = torch.from_numpy(rp).cuda()
    dcol = torch.from_numpy(col).cuda()
    h = native.mis_create_ex(n, drp.data_ptr(), dcol.data_ptr(), 1,
                             native.options(device=local, order_rows=0), stream)
    out = torch.empty(8 * n, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device="cuda")

    def timeit(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(max(5, args.steps // 2)):
            flush.add_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    seeds8 = np.arange(1, 9, dtype=np.uint64)
    one = lambda: native.mis_solve_ex(h, [1], out.data_ptr(), stream)  # noqa: E731
    eight = lambda: native.mis_solve_multi_ex(h, seeds8, out.data_ptr(), stream)  # noqa: E731
    native.mis_autotune(h, 3)
    res = {"graph": desc, "n": n, "arcs": int(rp[-1]), "single_ms": {}, "multi8_ms": {}}
    res["single_ms"]["csr"] = timeit(one)
    res["multi8_ms"]["csr"] = timeit(eight)
    ref8 = out.clone()
    exclude_us = {}
    select_us = {}

    def phases(nm):
        st = native.mis_get_stats(h)
        exclude_us[nm] = [round(st.exclude_ns[r] / 1e3, 1) for r in range(min(st.rounds, 64))]
        select_us[nm] = [round(st.select_ns[r] / 1e3, 1) for r in range(min(st.rounds, 64))]

    phases("csr")
    # selection on the CSR rows, exclusion as the single-bit MMA over the tiles
    native.mis_set_multi_form(h, native.MIS_MULTI_ROWS_TC)
    res["multi8_ms"]["rows_tc_b1"] = timeit(eight)
    phases("rows_tc_b1")
    same_rows_tc = bool(torch.equal(out, ref8))
    native.mis_set_multi_form(h, native.MIS_MULTI_ROWS)
    for T in (8, 16):
        native.mis_set_path(h, native.MIS_PATH_TILE, T)
        res["single_ms"][f"tile{T}_popc"] = timeit(one)
    res["tiles16"] = native.mis_get_stats(h).ntiles
    names = {native.MIS_TILE_BITS: "bits_fp16", native.MIS_TILE_BITS_B1: "b1",
             native.MIS_TILE_INT8: "int8", native.MIS_TILE_FP16: "fp16"}
    same = same_rows_tc
    res["autotune_multi_form"] = {native.MIS_MULTI_ROWS: "csr",
                                  native.MIS_MULTI_ROWS_TC: "rows_tc_b1"}[
        native.mis_autotune_multi(h, 8, 3)]
    res["autotuned_multi8_ms"] = timeit(eight)  # the form and switch point it kept
    same &= bool(torch.equal(out, ref8))
    native.mis_set_multi_form(h, native.MIS_MULTI_ROWS)
    for p, nm in names.items():
        native.mis_set_tile_payload(h, p)
        native.mis_set_path(h, native.MIS_PATH_TILE_TC, 16)
        res["single_ms"][f"tc_{nm}"] = timeit(one)
        res["multi8_ms"][f"tc_{nm}"] = timeit(eight)
        st = native.mis_get_stats(h)
        exclude_us[nm] = [round(st.exclude_ns[r] / 1e3, 1) for r in range(min(st.rounds, 64))]
        select_us[nm] = [round(st.select_ns[r] / 1e3, 1) for r in range(min(st.rounds, 64))]
        same &= bool(torch.equal(out, ref8))
    native.mis_destroy(h)
    best = min((k for k in res["multi8_ms"] if k != "csr"), key=lambda k: res["multi8_ms"][k])
    res["multi_seed_tc"] = {
        "k": 8, "best_form": best, "tc_launch_ms": res["multi8_ms"][best],
        "csr_launch_ms": res["multi8_ms"]["csr"],
        "tc_over_csr_speed": res["multi8_ms"]["csr"] / res["multi8_ms"][best],
        "exclude_phase_us_per_round": exclude_us,
        "select_phase_us_per_round": select_us,
        "results_equal_csr": same}
    res["arcs_per_tile16"] = res["arcs"] / max(res["tiles16"], 1)
    return res


def run_batch(args):
    from paper_2605_29604_gb300 import native
    world, rank, local = _dist_setup()
    leg = batch_leg(args, native, local, world)
    line = {
        "metric": METRIC, "value": leg["edges_per_s"], "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": leg["ms_per_launch"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": {"workload": "batch4096", **leg},
        "gpu_launches": args.steps, "clocks": leg["clocks"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0 if leg["standalone_check"]["all_equal"] else 1


def run_dynamic(args):
    """Dynamic graphs: batches of edge insertions and deletions on the
    resident R-MAT scale 22 graph, each applied (mis_update_edges) and the
    MIS repaired (mis_repair, H1 priority), against a full solve."""
    import torch

    from paper_2605_29604_gb300 import native
    world, rank, local = _dist_setup()
    (n, rp, col), desc = make_workload("rmat22")
    arcs = int(rp[-1])
    stream = torch.cuda.current_stream().cuda_stream
    h = native.mis_create_ex(n, rp, col, 0, native.options(device=local, check_symmetry=0,
                                                           priority=native.MIS_PRIORITY_HASH),
                             stream)
    native.mis_set_path(h, native.MIS_PATH_CSR, 0)
    seed = 1
    out = torch.empty(n, dtype=torch.uint8, device="cuda")
    seeds = np.array([seed], dtype=np.uint64)
    step_ms, clocks = time_device_steps(native, h, seeds, out.data_ptr(), stream, args.steps,
                                        args.warmup, local, world)
    solve_ms = float(np.median(step_ms))
    native.mis_solve_ex(h, seeds, out.data_ptr(), stream)
    rng = np.random.default_rng(2605)
    src = np.repeat(np.arange(n, dtype=np.int32), np.diff(rp))
    half = args.dyn_edges // 2
    upd, rep, sizes, rounds = [], [], [], []
    for _ in range(args.dyn_steps):
        pick = rng.integers(0, arcs, size=half)  # existing arcs (either direction)
        dels = np.stack([src[pick], col[pick]], axis=1).astype(np.int32)
        u = rng.integers(0, n, size=half)
        ins = np.stack([u, (u + rng.integers(1, n, size=half)) % n], axis=1).astype(np.int32)
        t0 = time.perf_counter()
        native.mis_update_edges(h, ins, dels, stream)
        t1 = time.perf_counter()
        size, r = native.mis_repair(h, seed, np.concatenate([ins, dels]), out.data_ptr(), stream)
        t2 = time.perf_counter()
        upd.append(t1 - t0)
        rep.append(t2 - t1)
        sizes.append(size)
        rounds.append(r)
    # the repaired result against a full solve of the updated graph
    full = torch.empty(n, dtype=torch.uint8, device="cuda")
    native.mis_solve_ex(h, seeds, full.data_ptr(), stream)
    torch.cuda.synchronize()
    same = bool(torch.equal(full, out))
    rep_ms = 1e3 * float(np.median(rep))
    upd_ms = 1e3 * float(np.median(upd))
    line = {
        "metric": "edge changes applied and repaired per second", "impl": "ours",
        "value": args.dyn_edges / ((rep_ms + upd_ms) / 1e3), "unit": "edge changes/s",
        "n_gpus": world, "steps": args.dyn_steps, "warmup": max(args.warmup, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": "dynamic", "graph": desc + ", H1 priority", "n": n, "arcs": arcs,
                   "edges_per_batch": args.dyn_edges, "insert_delete_split": "half and half",
                   "full_solve_ms": solve_ms, "repair_ms_p50": rep_ms, "update_ms_p50": upd_ms,
                   "repair_rounds": rounds, "mis_sizes": sizes,
                   "repair_equals_full_solve": same,
                   "timing": "full solve: CUDA events, L2 flushed; update and repair: host "
                             "wall clock (both synchronise their stream)"},
        "clocks": clocks,
    }
    native.mis_destroy(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0 if same else 1


def serve_pool_specs(pool, seed=5):
    """Config 5's pool: sizes log-uniform in [1K, 2M] vertices, even entries
    R-MAT (edge factor 8..32, permuted, size rounded up to a power of two),
    odd entries Erdos-Renyi (average degree 4..64)."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(pool):
        n = int(round(math.exp(math.log(1000) + rng.random() * (math.log(2_000_000) - math.log(1000)))))
        if i % 2 == 0:
            scale = max(10, int(math.ceil(math.log2(n))))
            specs.append(("rmat", scale, int(rng.integers(8, 33)), 100 + i))
        else:
            specs.append(("er", n, float(rng.uniform(4, 64)), 100 + i))
    return specs


def serve_leg(args, native, local, world, rank):
    """Config 5: continuous batching over a resident pool -- saturated
    throughput, then Poisson arrivals at fractions of it (p50/p99) -- against
    sequential plain solves of the same request list; a sample of the served
    results is checked against standalone solves."""
    import torch

    from paper_2605_29604_gb300 import graphgen as gg
    specs = serve_pool_specs(args.pool)

    def gen(spec):
        if spec[0] == "rmat":
            return gg.rmat(spec[1], spec[2], 0.57, 0.19, 0.19, spec[3])
        n, d, s = spec[1], spec[2], spec[3]
        return gg.er_gnm(n, int(n * d / 2), s)

    from concurrent.futures import ThreadPoolExecutor
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=max(4, os.cpu_count() or 4)) as ex:
        graphs = list(ex.map(gen, specs))
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    handles = [native.mis_create_ex(g[0], g[1], g[2], 0, native.options(device=local,
                                                                          check_symmetry=0), None)
               for g in graphs]
    t_create = time.perf_counter() - t0
    native.mis_serve_shutdown()
    native.mis_serve_configure(native.options(device=local, serve_blocks=args.serve_blocks))
    for h in handles:
        native.mis_set_path(h, native.MIS_PATH_CSR, 0)
    rng = np.random.default_rng(7)
    reqs = rng.integers(0, len(graphs), size=args.requests)
    arcs = np.array([int(g[1][-1]) for g in graphs])
    nmax = max(g[0] for g in graphs)
    # every request writes a host buffer; a sample of requests gets its own,
    # checked afterwards, the rest share one buffer per graph
    sample = set(rng.choice(len(reqs), size=min(args.serve_check, len(reqs)),
                            replace=False).tolist())
    shared = [np.empty(g[0], dtype=np.uint8) for g in graphs]

    # sequential plain solves of the same request list, one after another on
    # one stream, results in device memory (the fastest plain form)
    stream = torch.cuda.current_stream().cuda_stream
    dout = torch.empty(nmax, dtype=torch.uint8, device="cuda")
    for k in range(min(16, len(reqs))):  # warm-up
        native.mis_solve_ex(handles[reqs[k]], [1000 + k], dout.data_ptr(), stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, i in enumerate(reqs):
        native.mis_solve_ex(handles[i], [1000 + k], dout.data_ptr(), stream)
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    seq_rate = len(reqs) / seq_s

    def run(arrival_rate, base_seed, keep):
        """Submit the request list (all at once if rate is None, else with
        Poisson arrivals); returns (graphs/s, latencies in ms).  Latency is
        measured by the library, from mis_submit to the result in the host
        buffer (mis_poll_ex)."""
        n_req = len(reqs)
        lat = np.zeros(n_req)

        def buf(k):
            if k in keep:
                return keep[k]
            return shared[reqs[k]]

        if arrival_rate is None:
            # everything at once; collect in submission order (one poll at a
            # time keeps the library's lock free for its scheduler)
            t_start = time.perf_counter()
            tickets = [native.mis_submit(handles[i], base_seed + k, buf(k))
                       for k, i in enumerate(reqs)]
            for kk, t in enumerate(tickets):
                while True:
                    rc, ns = native.mis_poll_ex(t)
                    if rc != native.MIS_ENOTREADY:
                        break
                    time.sleep(20e-6)
                if rc != native.MIS_OK:
                    raise RuntimeError(f"served request failed: {rc}")
                lat[kk] = ns / 1e6
            return n_req / (time.perf_counter() - t_start), lat
        gaps = rng.exponential(1.0 / arrival_rate, size=n_req)
        arrive = np.cumsum(gaps)
        outstanding = []
        k = done = 0
        t_start = time.perf_counter()
        t_end = t_start
        while done < n_req:
            now = time.perf_counter() - t_start
            while k < n_req and arrive[k] <= now:
                i = reqs[k]
                outstanding.append((k, native.mis_submit(handles[i], base_seed + k, buf(k))))
                k += 1
            still = []
            for kk, t in outstanding:
                rc, ns = native.mis_poll_ex(t)
                if rc == native.MIS_ENOTREADY:
                    still.append((kk, t))
                    continue
                if rc != native.MIS_OK:
                    raise RuntimeError(f"served request failed: {rc}")
                lat[kk] = ns / 1e6
                done += 1
                t_end = time.perf_counter()
            outstanding = still
            if k < n_req and not outstanding:
                wait = arrive[k] - (time.perf_counter() - t_start)
                if wait > 200e-6:
                    time.sleep(wait - 100e-6)
        return n_req / (t_end - t_start), lat

    keep = {k: np.empty(graphs[reqs[k]][0], dtype=np.uint8) for k in sample}
    cap, lat_sat = run(None, 2000, keep)
    results = {"saturated": {"graphs_per_s": cap, "p50_ms": float(np.percentile(lat_sat, 50)),
                             "p99_ms": float(np.percentile(lat_sat, 99))}}
    for frac in (0.5, 0.8, 1.0):
        rate, lat = run(frac * cap, 50000, {})
        results[f"poisson_{frac}"] = {"offered_per_s": frac * cap, "graphs_per_s": rate,
                                      "p50_ms": float(np.percentile(lat, 50)),
                                      "p99_ms": float(np.percentile(lat, 99))}
    native.mis_serve_shutdown()
    # each sampled served result against a standalone solve with its seed
    same = True
    for k, got in keep.items():
        h = handles[reqs[k]]
        native.mis_solve_ex(h, [2000 + k], dout.data_ptr(), stream)
        torch.cuda.synchronize()
        same &= bool(np.array_equal(got, dout[:len(got)].cpu().numpy()))
    for h in handles:
        native.mis_destroy(h)
    per_graph = np.bincount(reqs, minlength=len(graphs))
    return {
        "metric": "served graphs/s (continuous batching) vs sequential plain solves",
        "pool": len(graphs), "pool_vertices_mean": float(np.mean([g[0] for g in graphs])),
        "pool_arcs_mean": float(arcs.mean()), "pool_arcs_total": int(arcs.sum()),
        "requests": len(reqs), "requests_per_graph_max": int(per_graph.max()),
        "gen_s": t_gen, "create_s": t_create,
        "sequential_graphs_per_s": seq_rate,
        "sequential": "the same request list as mis_solve_ex calls back to back on one stream, "
                      "results in device memory",
        "served_graphs_per_s": cap, "speedup_vs_sequential": cap / seq_rate,
        "serve_blocks": args.serve_blocks or "default (half the SMs)",
        "latency": "library-measured, mis_submit to result in host buffer",
        **results,
        "standalone_check": {"requests_checked": len(keep), "all_equal": same},
    }


def run_serve(args):
    from paper_2605_29604_gb300 import native
    world, rank, local = _dist_setup()
    leg = serve_leg(args, native, local, world, rank)
    line = {
        "metric": leg["metric"], "value": leg["served_graphs_per_s"], "unit": "graphs/s",
        "n_gpus": world, "steps": leg["requests"], "warmup": 0, "higher_is_better": True,
        "data": "synthetic", "dtype": "u32", "config": {"workload": "serve", **leg},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0 if leg["standalone_check"]["all_equal"] else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rmat22")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tpr", type=int, default=None, help="force the CSR path with these lanes")
    ap.add_argument("--csr-pending", type=int, default=None, choices=[0, 1],
                    help="with --tpr: Phase 2 over Phase 1's pending list (1) or a triage (0)")
    ap.add_argument("--bins", default=None,
                    help="with --tpr 0: the CSR kernel's four degree-bin bounds, comma separated")
    ap.add_argument("--grid", type=int, default=0,
                    help="with --tpr: blocks of the persistent CSR launch (0 = all co-resident)")
    ap.add_argument("--path", default=None, choices=["tile", "tile_tc", "push", "cluster"])
    ap.add_argument("--payload", default="b1", choices=sorted(PAYLOADS),
                    help="with --path tile_tc: the tile payload form of the tensor-core exclusion")
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch from an ncu capture of this kernel")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--batch-order", type=int, default=2, choices=[0, 1, 2],
                    help="create-time row ordering of the batched union (mis_options.order_rows)")
    ap.add_argument("--pool", type=int, default=512)
    ap.add_argument("--requests", type=int, default=20000)
    ap.add_argument("--serve-check", type=int, default=256,
                    help="served results checked against standalone solves")
    ap.add_argument("--serve-blocks", type=int, default=0)
    ap.add_argument("--dyn-edges", type=int, default=1000,
                    help="dynamic workload: edge changes per batch (half inserted, half deleted)")
    ap.add_argument("--dyn-steps", type=int, default=5)
    ap.add_argument("--legs", default=None,
                    help="extra legs of the single-graph run, comma separated: batch (the "
                         "4096-graph union), serve (the served pool), tc (tile and tensor-core "
                         "paths on the grid, the stencil lattice and the geometric graph); "
                         "default all for rmat22, none otherwise")
    ap.add_argument("--no-amortized", dest="amortized", action="store_false",
                    help="skip the solve on a graph with create-time round-0 structures")
    ap.add_argument("--multi", type=int, default=8,
                    help="also time this many seeds of the graph per launch (0 = off)")
    ap.add_argument("--multi-form", choices=["rows", "rows_tc", "auto"], default=None,
                    help="with --multi: also time that many seeds per launch on the full-row "
                         "graph in this multi-seed form (rows: CUDA cores; rows_tc: the "
                         "exclusion on tensor cores over 16 x 16 bitmask tiles; auto: "
                         "mis_autotune_multi's choice)")
    args = ap.parse_args()
    if args.legs is None:
        args.legs = "batch,serve,tc" if args.workload == "rmat22" else ""
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch4096":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "dynamic":
        return run_dynamic(args)
    return run_single(args)


if __name__ == "__main__":
    sys.exit(main())
