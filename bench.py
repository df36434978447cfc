"""Benchmark: edges/s to a full MIS on one GB300 (and N replicas under torchrun).

A step is one full solve of the hot path -- Eq. 1 priorities, then every
round of Algorithm 2 (selection test, exclusion test, state update,
compaction) until the alive set is empty -- on a graph already resident in
HBM.  value = arcs solved / device time of the K timed steps (CUDA events on
the launching stream, L2 flushed between steps).

Workloads (synthetic, seeded; stand-ins for the paper's SuiteSparse graphs):
  rmat22     R-MAT scale 22, edge factor 16, (0.57, 0.19, 0.19, 0.05), permuted (default)
  er10k      Erdos-Renyi G(10,000, 40,000)
  grid       2048 x 2048 grid + 5% random diagonals, natural ids
  grid_perm  the same grid, permuted ids
  batch4096  4096 graphs (log-uniform 64..65,536 vertices, ER / random geometric) in one launch

`--impl reference` times the CPU oracle (a plain sequential restatement of
the same computation) on the host cores instead.

Run: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "edges/s to full MIS on 1 GB300"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def _peak_hbm():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


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


def oracle_rate(g, repeats=1):
    """CPU oracle (keys + round simulation), sequential C on one host core."""
    import oracle
    n, rp, col = g
    t0 = time.perf_counter()
    for _ in range(repeats):
        res = oracle.solve(n, rp, col, 1)
    dt = (time.perf_counter() - t0) / repeats
    return int(rp[-1]) / dt, dt, res


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    name = args.workload if args.workload != "rmat22" else "rmat18"
    g, desc = make_workload(name)
    n, rp, col = g
    for _ in range(args.warmup):
        oracle_rate(g)
    times = []
    for _ in range(args.steps):
        _, dt, res = oracle_rate(g)
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


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2605_29604_gb300 import native
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    g, desc = make_workload(args.workload)
    n, rp, col = g
    arcs = int(rp[-1])
    stream = torch.cuda.current_stream().cuda_stream
    opt = native.options(device=local, check_symmetry=1)
    t_create = time.perf_counter()
    h = native.mis_create_ex(n, rp, col, 0, opt, stream)
    t_create = time.perf_counter() - t_create
    if args.tpr:
        native.mis_set_path(h, native.MIS_PATH_CSR, args.tpr)
    out = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
    seeds = np.array([1], dtype=np.uint64)
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device=dev)

    def step():
        native.mis_solve_ex(h, seeds, out.data_ptr(), stream)

    for _ in range(max(args.warmup, 3)):
        step()
    st = native.mis_get_stats(h)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.add_(1.0)  # write 256 MB: evicts the previous step from L2
            starts[i].record()
            step()
            ends[i].record()
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    st = native.mis_get_stats(h)
    value = world * args.steps * arcs / (total_ms / 1e3)

    # end to end through the C ABI with host buffers: pinned CSR in, result out
    e2e = None
    if args.e2e_steps > 0:
        prp = torch.from_numpy(rp).pin_memory().numpy()
        pcol = torch.from_numpy(col).pin_memory().numpy()
        hout = torch.empty(max(n, 1), dtype=torch.uint8).pin_memory().numpy()
        e2e_opt = native.options(device=local, check_symmetry=0)
        times = []
        for i in range(args.e2e_steps + 1):
            t0 = time.perf_counter()
            h2 = native.mis_create_ex(n, prp, pcol, 0, e2e_opt, None)
            native.mis_solve(h2, 1, hout)
            native.mis_destroy(h2)
            if i:
                times.append(time.perf_counter() - t0)
        e2e = {"value": world * arcs * len(times) / sum(times), "unit": "edges/s",
               "h2d_bytes_per_step": 4 * (n + 1) + 4 * arcs, "d2h_bytes_per_step": n,
               "path": "mis_create_ex(host CSR, pinned) + mis_solve(host result) + mis_destroy"}

    peak, peak_kind = _peak_hbm()
    alg_bytes = 4 * arcs + 4 * (n + 1) + 4 * n + n
    launch_s = (total_ms / 1e3) / args.steps
    achieved = alg_bytes / launch_s / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload, "graph": desc, "n": n, "arcs": arcs,
                   "rounds": st.rounds, "path": "csr", "threads_per_row": st.threads_per_row,
                   "mis_size": st.mis_size, "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas{world}", "create_s": t_create,
                   "step_ms_p10_p50_p90": [float(np.percentile(step_ms, q)) for q in (10, 50, 90)]},
        "gpu_launches": args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_kind": f"{peak_kind} burst copy bandwidth",
                     "alg_bytes_per_launch": alg_bytes,
                     "kernel": "csr_solve_kernel (one persistent launch per solve)"},
        "clocks": clk.summary(),
        "e2e": e2e,
    }
    if rank == 0 and args.cpu_baseline:
        import oracle
        sample_name = "rmat18" if args.workload == "rmat22" else args.workload
        gs, sdesc = make_workload(sample_name) if sample_name != args.workload else (g, desc)
        rate, dt, res = oracle_rate(gs)
        mdg, _ = oracle.min_degree_greedy(*gs)
        line["cpu_baseline"] = {"value": rate, "unit": "edges/s", "cores": 1, "kind": "oracle",
                                "sample": f"one oracle solve of {sdesc} ({dt:.2f} s)",
                                "quality": {"mis_size": int(res.status.sum()),
                                            "min_degree_greedy": mdg}}
    native.mis_destroy(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rmat22")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tpr", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
