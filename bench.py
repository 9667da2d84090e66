#!/usr/bin/env python
"""Benchmark of the TPC sector tracker on B300: TPC clusters/s tracked.

Default workload: the full TPC (36 sectors x 152 rows) with one central
Pb-Pb-like event of 6000 primary helices (~0.9M clusters) plus 5% noise,
synthetic (seeded), plain mode (one launch per step over all 36 sectors).
A "step" is one tpc_track() over the resident batch (every step of the path).

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload instead.
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

# algorithmic bytes per input cluster of each step (minimum traffic the step must
# move) and the dominant step's unit
ALGO_BYTES = {"quantise+row_stats": 16 + 12, "row_setup": 0, "group_scatter": 12 + 12, "row_sort": 12 + 16,
              "links": 12 + 8, "clean+starts": 8 + 8, "tracklets": 28, "selection": 20, "output": 8}

WORKLOADS = {
    "c1": "1 sector x 152 rows, 200 helices pT 0.1-10 GeV |eta|<0.9, sigma 0.1 cm, 5% noise, seed 1",
    "c2": "36 sectors x 152 rows, 6000 helices (central Pb-Pb-like), sigma 0.1 cm, 5% noise, seed 1",
}


def make_workload(name: str, rank: int):
    from paper_1910_12214_b300 import synth
    seed = 1 + rank  # each rank tracks its own events (weak scaling)
    if name == "c1":
        return synth.make_config1(seed=seed)
    if name == "c2":
        return synth.make_config2(seed=seed)
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def cpu_baseline(name: str, budget_s: float = 12.0):
    """The FP64 oracle as it stands, single-threaded on the host, over whole
    events of the same workload until about budget_s of CPU work."""
    import oracle
    cl = make_workload(name, 0)
    n, t = 0, 0.0
    runs = 0
    while t < budget_s and runs < 50:
        t0 = time.perf_counter()
        oracle.run(cl, what=["trk_i"])
        t += time.perf_counter() - t0
        n += cl.n
        runs += 1
    return {"value": n / t, "unit": "clusters/s", "cores": 1, "kind": "oracle",
            "sample": f"{runs} full events of workload {name} ({cl.n} clusters each), single-threaded FP64"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    cb = cpu_baseline(args.workload, budget_s=max(3.0, min(60.0, 6.0 * args.steps)))
    line = {"impl": "reference", "metric": "TPC clusters/s tracked", "value": cb["value"], "unit": "clusters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]}, "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "clusters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    from paper_1910_12214_b300 import tpc

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cl = make_workload(args.workload, rank)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    # resident inputs
    d = type("D", (), {})()
    d.x, d.y, d.z = (torch.from_numpy(a).to(dev) for a in (cl.x, cl.y, cl.z))
    d.row = torch.from_numpy(cl.row).to(dev)
    d.item_off, d.item_sector, d.item_event = cl.item_off, cl.item_sector, cl.item_event
    d.item_core = None
    t = tpc.Tracker(device=local, stream=stream, profile=True)
    t.load(d, on_device=True)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (126 MB)
    for _ in range(args.warmup):
        t.track()
        flush.zero_()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stage_acc = {}
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        starts[k].record(stream)
        t.track()
        ends[k].record(stream)
        st = t.stage_times()  # syncs; events recorded on the tracker's stream
        for kk, v in st.items():
            stage_acc[kk] = stage_acc.get(kk, 0.0) + v
        flush.zero_()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = float(np.mean(step_ms))
    if dist:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    n_tr, n_ids = t.counts()

    # end to end through the public API with host buffers (H2D + track + D2H per step)
    e2e_times = []
    h2d = 16 * cl.n + 8 * (cl.n_items + 1) + 8 * cl.n_items
    for k in range(max(3, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t.load(cl)
        t.track()
        trk, ids = t.get_tracks()
        e2e_times.append(time.perf_counter() - t0)
    d2h = trk.nbytes + ids.nbytes + 32
    e2e_s = float(np.median(e2e_times[1:]))

    if rank == 0:
        stage_us = {k: v / args.steps for k, v in stage_acc.items()}
        dom = max(stage_us, key=stage_us.get)
        peak, peak_kind = measured_peak_hbm()
        algo = ALGO_BYTES[dom] * cl.n
        achieved = algo / (stage_us[dom] * 1e-6) / 1e9
        value = cl.n * world / (ms * 1e-3)
        line = {
            "metric": "TPC clusters/s tracked (plain sector tracker)",
            "value": value, "unit": "clusters/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "clusters_per_step": cl.n, "items": cl.n_items,
                       "tracks": n_tr, "l2": "flushed between steps (256 MB write)", "mode": "plain"},
            "e2e": {"value": cl.n * world / e2e_s, "unit": "clusters/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": 18 * args.steps,
            "stage_us": {k: round(v, 2) for k, v in stage_us.items()},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "algo_bytes_per_cluster": ALGO_BYTES[dom]},
            "clocks": clk, "wall_s_timed_region": wall,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(line), flush=True)
    t.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
