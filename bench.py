#!/usr/bin/env python
"""Benchmark of the TPC sector tracker on B300: TPC clusters/s tracked.

Headline workload: the full TPC (36 sectors x 152 rows), one central Pb-Pb-like
event of 6000 primary helices (~0.9M clusters, 5% noise), synthetic and seeded;
one step = one tpc_track() over the resident batch (every step of the path),
launch shapes chosen by the library's autotuner, replayed as a CUDA graph.
Further forms (rank 0, N=1): 64 uneven events (plain vs the batched form's
persistent tracklet kernels), a 50 kHz continuous-readout time frame (128
collisions, sliced on the device inside the timed step), and
the same 64 events distorted by a space-charge field, corrected by the grid or
by the trained BF16 network, the cluster codec (float to integer with dynamic
precision) over the 64 events' clusters, the cluster removal masks
(attachment, adjacency, protection, strategies A and B) of the 64 events,
their compression (delta and track-model coding, rANS), the merger of their
sector tracks with refit and looper legs, and the whole reduction chain (legs
and their join, masks, removal, compression) on an event whose low-pT helices
loop.  Every batch form checks its tracks against the oracle on a sample of its
items in the same run.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic bytes per input cluster of each step: the minimum HBM traffic the
# step must move (cluster SoA 16 B, quantised (qy,qz) 8 B, sorted hit 16 B, link
# words 4 B each; the tracklets read about two passes of 8 B of coordinates and
# 4 B of bin lookup per hit and write a 4 B hit slot).
ALGO_BYTES = {"quantise+row_stats": 16 + 12, "row_setup": 0, "group_scatter": 12 + 12, "row_sort": 12 + 16 + 8,
              "links": 16 + 8, "clean+starts": 8 + 8 + 4, "tracklets": 28, "selection": 20, "output": 8}
# DRAM bytes (read + write) of the dominant step per tracking step, as one ncu
# capture of the current kernels measured them (dram__bytes_read.sum +
# dram__bytes_write.sum of k_tracklets_up<1> and k_tracklets_down<1> on the
# full TPC event: 21.52 + 18.60 MB read, writes kept in L2); they cannot be
# measured inside this run.  To be emptied whenever those kernels change.
TRAFFIC = {("c2", "tracklets"): 40.12e6}
TRAFFIC_SOURCE = ("ncu --set full capture of the same kernels on the same workload, per step "
                  "(dram__bytes_read.sum + dram__bytes_write.sum); not measurable in this run")
KERNELS_PER_STEP = {"plain": 20, "batched": 23}  # kernels per tracking step of an event batch (the
# launch sequence of launch_stages: 19 and 22 before the warp-per-row sort, as the launch lists show)

METRIC = "TPC clusters/s tracked (sector tracker, full TPC event)"
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


# ------------------------------------------------------------ input generation (CPU, before CUDA)
def _gen_batched(n_events=64):
    from paper_1910_12214_b300 import synth
    return synth.make_batched(seed=1, n_events=n_events)


def _gen_frame():
    from paper_1910_12214_b300 import synth
    fr = synth.make_timeframe(seed=1)
    fr.truth = None
    return fr


def _gen_loopers():
    from paper_1910_12214_b300 import synth
    cl = synth.make_event(42, 6000, second_leg=True)
    return cl, synth.cluster_props(cl, seed=42)


def _gen_grid():
    from paper_1910_12214_b300 import synth
    d = synth.make_distortion(seed=1, n_sectors=36)
    g, b = synth.correction_grid(d)
    return d, g, b


def generate_forms(forms, batch_events=64):
    """Generate the form workloads in spawned worker processes (no CUDA yet)."""
    out = {}
    jobs = {}
    ctx = mp.get_context("spawn")
    with ctx.Pool(3) as pool:
        if "c10" in forms:
            jobs["c10"] = pool.apply_async(_gen_loopers)
        if any(f in forms for f in ("c3", "c5", "c6", "c7", "c8", "c9")):
            jobs["c3"] = pool.apply_async(_gen_batched, (batch_events,))
        if "c4" in forms:
            jobs["c4"] = pool.apply_async(_gen_frame)
        if "c5" in forms:
            jobs["grid"] = pool.apply_async(_gen_grid)
        for k, j in jobs.items():
            out[k] = j.get()
    if "c6" in forms:
        from paper_1910_12214_b300 import synth
        out["c6"] = synth.cluster_props(out["c3"], seed=1)
    if "c7" in forms:
        out["c7"] = out["c3"]
    if "c9" in forms:
        out["c9"] = out["c3"]
    if "c8" in forms:
        from paper_1910_12214_b300 import synth
        out["c8"] = (out["c3"], out["c6"] if "c6" in out else synth.cluster_props(out["c3"], seed=1))
    if "c5" in forms:
        from paper_1910_12214_b300 import synth
        d, g, b = out["grid"]
        out["c5"] = (synth.distort(out["c3"], d), g, b)
    if "c3" not in forms:
        out.pop("c3", None)  # generated only as the input of another form
    return out


# ------------------------------------------------------------ measurement helpers
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


def _parity(cl, trk, ids, ref):
    """Track parity of the GPU's tracks with the oracle's on the same clusters:
    >= 99.5% of oracle tracks matched with >= 90% shared clusters, and >= 99.5%
    of the matched ones with parameters within 1e-3 relative."""
    import contextlib
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from gpu_helpers import compare_tracks
    with contextlib.redirect_stdout(sys.stderr):  # one JSON line on stdout
        r = compare_tracks(cl, trk, ids, ref)
    return {k: (round(v, 6) if isinstance(v, float) else v) for k, v in r.items() if k != "bad_by_param"}


def cpu_baseline(name: str, budget_s: float = 12.0, gpu=None):
    """The FP64 oracle as it stands, single-threaded on the host, over whole
    events of the same workload until about budget_s of CPU work.  With the
    GPU's tracks of the same event (gpu = (tracks, ids)), the oracle's first run
    also gives the parity check of this run."""
    import oracle
    cl = make_workload(name, 0)
    n, t = 0, 0.0
    runs = 0
    parity = None
    while t < budget_s and runs < 50:
        t0 = time.perf_counter()
        ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"] if runs == 0 else ["trk_i"])
        t += time.perf_counter() - t0
        if runs == 0 and gpu is not None:
            parity = _parity(cl, gpu[0], gpu[1], ref)
        n += cl.n
        runs += 1
    out = {"value": n / t, "unit": "clusters/s", "cores": 1, "kind": "oracle",
           "sample": f"{runs} full events of workload {name} ({cl.n} clusters each), single-threaded FP64"}
    if parity is not None:
        out["parity"] = parity
    return out


def sample_items(cl, k, seed):
    """k items of a batch for the oracle: the 4 largest and k - 4 at random."""
    from paper_1910_12214_b300 import shard
    costs = shard.item_costs(cl)
    k = min(k, cl.n_items)
    largest = np.argsort(-costs, kind="stable")[:min(4, k)]
    rng = np.random.default_rng(seed)
    rest = rng.choice(np.setdiff1d(np.arange(cl.n_items), largest), size=k - largest.shape[0], replace=False)
    return np.sort(np.concatenate([largest, rest]))


def tracks_of_items(trk, ids, items, index, key="item"):
    """GPU tracks of the given items, renumbered for the sub-batch that
    shard.take_items(cl, items) makes (item numbers and cluster ids).  key:
    the track field that names the item ("sector" for the tracks of a sliced
    frame, whose items are the frame's sectors)."""
    pos_of_item = {int(it): j for j, it in enumerate(items)}
    inv = np.full(max(int(ids.max()) + 1 if ids.size else 1, int(np.max(index)) + 1 if len(index) else 1), -1,
                  np.int64)
    inv[np.asarray(index, np.int64)] = np.arange(len(index))
    keep = np.array([i for i in range(len(trk)) if int(trk[key][i]) in pos_of_item], np.int64)
    sub = trk[keep].copy()
    out_ids, base = [], 0
    for j, i in enumerate(keep):
        f, n = int(trk["first_cluster"][i]), int(trk["n_clusters"][i])
        out_ids.append(inv[ids[f:f + n].astype(np.int64)])
        sub["item"][j] = pos_of_item[int(trk[key][i])]
        sub["first_cluster"][j] = base
        base += n
    return sub, (np.concatenate(out_ids) if out_ids else np.zeros(0, np.int64)).astype(np.uint32)


def form_baseline(cl, trk, ids, k, seed, correct=None, key="item"):
    """CPU-baseline leg of a form: the oracle on a seeded sample of k items
    (timed, single-threaded FP64) and the parity of the GPU's tracks of those
    items with the oracle's.  correct = (grid, bounds): the oracle corrects the
    sampled clusters with its own trilinear grid first (grid-corrected form).
    key = "sector": cl is a frame tracked through tpc_load_frame, sampled by
    whole (unsliced) sectors."""
    import oracle
    from paper_1910_12214_b300 import shard
    items = sample_items(cl, k, seed)
    sub, index = shard.take_items(cl, items)
    t0 = time.perf_counter()
    if correct is not None:
        oy, oz = oracle.correct_clusters(sub, *correct)
        sub.y, sub.z = oy.astype(np.float32), oz.astype(np.float32)
    ref = oracle.run(sub, what=["trk_f", "trk_i", "trk_ids"])
    dt = time.perf_counter() - t0
    g_trk, g_ids = tracks_of_items(trk, ids, items, index, key=key)
    return ({"value": sub.n / dt, "unit": "clusters/s", "cores": 1, "kind": "oracle",
             "sample": f"{len(items)} items of the form (4 largest, the rest seeded at random; {sub.n} clusters)"
                       + (", corrected by the oracle's grid" if correct is not None else "")},
            _parity(sub, g_trk, g_ids, ref))


def _oracle_share(args):
    """Worker of the all-cores baseline: the oracle on one share of the items."""
    name, items, reps = args
    import oracle
    from paper_1910_12214_b300 import shard
    cl = make_workload(name, 0)
    sub, _ = shard.take_items(cl, items)
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.run(sub, what=["trk_i"])
        best = min(best, time.perf_counter() - t0)
    return best, sub.n


def cpu_baseline_all_cores(name: str, reps: int = 2):
    """The same oracle, one single-threaded instance per host core, each on an
    LPT share of the event's items (spawned processes; each times its own run;
    the event takes as long as the slowest share)."""
    from paper_1910_12214_b300 import shard, synth
    cl = make_workload(name, 0)
    cores = os.cpu_count() or 1
    parts = [p for p in shard.lpt_partition(shard.item_costs(cl), min(cores, cl.n_items)) if p.size]
    with mp.get_context("spawn").Pool(len(parts)) as pool:
        res = pool.map(_oracle_share, [(name, p, reps) for p in parts])
    t = max(r[0] for r in res)
    return {"value": cl.n / t, "unit": "clusters/s", "cores": len(parts), "kind": "oracle",
            "sample": f"one event of workload {name} ({cl.n} clusters, {cl.n_items} items) split over "
                      f"{len(parts)} single-threaded oracle processes, best of {reps}"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    cb = cpu_baseline(args.workload, budget_s=max(3.0, min(60.0, 6.0 * args.steps)))
    cl = make_workload(args.workload, 0)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "clusters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded helices, ALICE simulation not available)",
            "config": {"workload": WORKLOADS[args.workload], "clusters_per_step": cl.n, "items": cl.n_items},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "clusters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def to_device(cl, dev):
    import torch
    d = type("D", (), {})()
    d.x, d.y, d.z = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (cl.x, cl.y, cl.z))
    d.row = torch.from_numpy(np.ascontiguousarray(cl.row)).to(dev)
    d.item_off, d.item_sector, d.item_event = cl.item_off, cl.item_sector, cl.item_event
    d.item_core = getattr(cl, "item_core", None)
    return d


def pinned_clusters(cl, torch):
    """The cluster arrays in pinned (page-locked) host memory."""
    d = type("P", (), {})()
    d.keep = []  # the pinned tensors behind the numpy views
    for name, dt in (("x", torch.float32), ("y", torch.float32), ("z", torch.float32), ("row", torch.int32)):
        a = getattr(cl, name)
        buf = torch.empty(a.shape[0], dtype=dt, pin_memory=True)
        buf.numpy()[:] = a
        d.keep.append(buf)
        setattr(d, name, buf.numpy())
    d.item_off, d.item_sector, d.item_event = cl.item_off, cl.item_sector, cl.item_event
    d.item_core = getattr(cl, "item_core", None)
    return d


def e2e_pipelined(hcl, tuning, tpc, torch, dev, local, steps):
    """Seconds per step end to end through the public API, double-buffered.
    A step is tpc_load_clusters of the step's clusters from pinned host memory
    (H2D; the call returns when its copies are done), tpc_track, and
    tpc_get_tracks of the tracks and ids into pinned host memory (D2H).  Two
    contexts on two streams take alternate steps: while one tracks, the other
    loads the next step and reads its previous result; a stream wait keeps the
    tracking of consecutive steps in order, one event at a time on the GPU."""
    ss = [torch.cuda.Stream(dev) for _ in range(2)]
    ts = [tpc.Tracker(device=local, stream=s) for s in ss]
    outs = []
    for t in ts:
        t.set_tuning(**{**tuning, "use_graph": 2})
        t.load(hcl)
        t.track()
        t.sync()
        nt, ni = t.counts()
        ot = torch.empty((nt + 64) * tpc.TRACK_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
        oi = torch.empty(ni + 4096, dtype=torch.int32, pin_memory=True)
        outs.append((ot.numpy().view(tpc.TRACK_DTYPE), oi.numpy().view(np.uint32), ot, oi))
    done = [torch.cuda.Event(), torch.cuda.Event()]

    def run(k_steps):
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        ts[0].load(hcl)
        ts[0].track()
        done[0].record(ss[0])
        for k in range(k_steps):
            cur, nxt = k % 2, (k + 1) % 2
            if k + 1 < k_steps:
                ts[nxt].load(hcl)
                ss[nxt].wait_event(done[cur])
                ts[nxt].track()
                done[nxt].record(ss[nxt])
            ts[cur].get_tracks(out=outs[cur][:2])
        return (time.perf_counter() - w0) / k_steps

    run(4)
    per = [run(steps) for _ in range(3)]
    res = [t.get_tracks(out=o[:2]) for t, o in zip(ts, outs)]
    for t in ts:
        t.close()
    return float(np.median(per)), res[0]


def time_steps(t, stream, steps, flush):
    """Device time of `steps` tpc_track() calls, L2 flushed between them."""
    import torch
    ms = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t.track()
        e1.record(stream)
        with torch.cuda.stream(stream):  # on the timed stream: between steps, not beside the next one
            flush.zero_()
        ms.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ms]


def stage_profile(t, stream, steps=3):
    """Per-step device times from the library's events (direct launches).  A
    bounded spin kernel ahead of each step keeps the GPU busy while the host
    enqueues the step, so that the events time the kernels, not the host."""
    import torch
    tun = t.get_tuning()
    t.set_tuning(use_graph=1)
    acc = {}
    for _ in range(steps):
        with torch.cuda.stream(stream):
            torch.cuda._sleep(2_000_000)  # about 1 ms of clock cycles
        t.track()
        for k, v in t.stage_times().items():
            acc[k] = acc.get(k, 0.0) + v / steps
    t.set_tuning(use_graph=tun["use_graph"])
    return acc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--forms", default="c3,c4,c5,c6,c7,c8,c9,c10", help="extra forms at N=1: c3,...,c10 or none")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-events", type=int, default=64, help="events of the batch forms (c3, c5-c9)")
    ap.add_argument("--train-samples", type=int, default=40_000_000,
                    help="surrogate training samples per sector (c5)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    forms = [] if args.forms == "none" or world > 1 or rank != 0 else [f for f in args.forms.split(",") if f]
    gen = generate_forms(forms, args.batch_events) if forms else {}  # CPU work before CUDA is touched

    import torch
    from paper_1910_12214_b300 import shard, tpc

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (126 MB)
    cl = make_workload(args.workload, rank)
    with torch.cuda.stream(stream):
        d = to_device(cl, dev)
    stream.synchronize()
    t = tpc.Tracker(device=local, stream=stream, profile=True)
    t.load(d, on_device=True)
    tuning, tune_us = t.autotune(iters=3)
    t.set_tuning(use_graph=2)
    for _ in range(args.warmup):
        t.track()
        with torch.cuda.stream(stream):
            flush.zero_()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("tpc_timed")  # lets a profiler select the timed launches
    step_ms = time_steps(t, stream, args.steps, flush)
    torch.cuda.nvtx.range_pop()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = shard.max_over_ranks(float(np.mean(step_ms)), dist, device=dev)
    n_all = shard.sum_over_ranks(cl.n, dist, device=dev)  # clusters of all ranks' events
    n_tr, n_ids = t.counts()
    stages = stage_profile(t, stream)

    # end to end through the public API with host buffers: H2D of the step's
    # clusters from pinned host memory, tracking, D2H of the tracks and their
    # cluster ids into pinned host memory
    e2e = []
    h2d = 16 * cl.n + 8 * (cl.n_items + 1) + 8 * cl.n_items
    hcl = pinned_clusters(cl, torch)
    nt0, ni0 = t.counts()
    out_t = torch.empty((nt0 + 64) * tpc.TRACK_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
    out_i = torch.empty(ni0 + 4096, dtype=torch.int32, pin_memory=True)
    out = (out_t.numpy().view(tpc.TRACK_DTYPE), out_i.numpy().view(np.uint32))
    trk = ids = None
    for _ in range(max(4, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t.load(hcl)
        t.track()
        trk, ids = t.get_tracks(out=out)
        e2e.append(time.perf_counter() - t0)
    d2h = trk.nbytes + ids.nbytes + 32
    e2e_serial = shard.max_over_ranks(float(np.median(e2e[1:])), dist, device=dev)
    t.close()
    e2e_s, (trk_p, ids_p) = e2e_pipelined(hcl, tuning, tpc, torch, dev, local, max(8, args.steps))
    same_tracks = bool(np.array_equal(trk_p, trk) and np.array_equal(ids_p, ids))  # as the serial calls
    e2e_s = shard.max_over_ranks(e2e_s, dist, device=dev)

    form_out = {}
    if rank == 0 and forms:
        form_out = run_forms(gen, dev, stream, flush, tpc, torch, args.train_samples, args.batch_events)

    if rank == 0:
        dom = max(stages, key=stages.get)
        peak, peak_kind = measured_peak_hbm()
        algo = ALGO_BYTES.get(dom, 0) * cl.n
        achieved = algo / (stages[dom] * 1e-6) / 1e9
        value = n_all / (ms * 1e-3)
        line = {
            "metric": METRIC,
            "value": value, "unit": "clusters/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded helices, ALICE simulation not available)",
            "config": {"workload": WORKLOADS[args.workload], "clusters_per_step": cl.n, "items": cl.n_items,
                       "tracks": n_tr, "l2": "flushed between steps (256 MB write)", "tuning": tuning,
                       "autotune_best_us": tune_us},
            "e2e": {"value": n_all / e2e_s, "unit": "clusters/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "pipeline": "two contexts, each step's H2D and D2H "
                    "overlapping the other context's tracking; tracking serialised",
                    "serial_value": n_all / e2e_serial, "tracks_equal_serial": same_tracks},
            "gpu_launches": KERNELS_PER_STEP["batched" if tuning["mode"] == 2 else "plain"] * args.steps,
            "stage_us": {k: round(v, 2) for k, v in stages.items()},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": TRAFFIC.get((args.workload, dom)),
                         "traffic_source": TRAFFIC_SOURCE
                         if TRAFFIC.get((args.workload, dom)) else "null: no ncu capture of the current kernels",
                         "peak_kind": peak_kind,
                         "algo_bytes_per_cluster": ALGO_BYTES.get(dom)},
            "clocks": clk, "wall_s_timed_region": wall,
            "forms": form_out,
        }
        if not args.no_cpu_baseline:
            cb = cpu_baseline(args.workload, gpu=(trk, ids))
            line["parity"] = cb.pop("parity")
            line["cpu_baseline"] = cb
            line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args.workload)
            if not line["parity"]["ok"]:  # a number is reported only with its parity check passed
                line["invalid"] = "parity check against the oracle failed on this run"
                line["value"] = None
        else:
            line["parity"] = "not checked (--no-cpu-baseline)"
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_forms(gen, dev, stream, flush, tpc, torch, train_samples=40_000_000, batch_events=64):
    """clusters/s of the other forms (device time of tpc_track, L2 flushed)."""
    res = {}

    def bench_batch(cl, label, n_clusters, modes=("plain", "batched"), setup=None, steps=5, sample=40, seed=11):
        with torch.cuda.stream(stream):
            d = to_device(cl, dev)
        stream.synchronize()
        out = {}
        first = None
        with tpc.Tracker(stream=stream, profile=True) as t:
            if setup:
                setup(t)
            t.load(d, on_device=True)
            for mode in modes:
                tun, _ = t.autotune(iters=2, mode=1 if mode == "plain" else 2)  # best shapes of this mode
                t.set_tuning(use_graph=2)
                for _ in range(2):
                    t.track()
                ms = float(np.median(time_steps(t, stream, steps, flush)))
                trk, ids = t.get_tracks()
                out[mode] = {"clusters_per_s": n_clusters / (ms * 1e-3), "ms": ms, "tracks": t.counts()[0],
                             "tuning": tun, "stage_us": {k: round(v, 2) for k, v in stage_profile(t, stream).items()}}
                if first is None:
                    first = (trk, ids)
                else:  # every mode must give the first mode's tracks byte for byte
                    out[mode]["identical_to_" + modes[0]] = bool(trk.tobytes() == first[0].tobytes() and
                                                                 np.array_equal(ids, first[1]))
        del d
        torch.cuda.empty_cache()
        cb, par = form_baseline(cl, first[0], first[1], sample, seed)
        out["parity"] = par
        out["cpu_baseline"] = cb
        return out

    if "c3" in gen:
        c3 = gen["c3"]
        res[f"batched_{batch_events}_events"] = {"clusters": c3.n, "items": c3.n_items, **bench_batch(c3, "c3", c3.n)}
    if "c4" in gen:
        res["timeframe_50khz_128_collisions"] = bench_frame(gen["c4"], dev, stream, flush, tpc, torch)
    if "c5" in gen:
        c5, grid, bounds = gen["c5"]
        info = {}

        def setup(t):
            t.set_grid_correction(grid, bounds)
            t0 = time.perf_counter()
            mx, rms = t.surrogate_train(train_samples, seed=1)
            info.update(train_s=time.perf_counter() - t0, resid_max_cm=mx, resid_rms_cm=rms)

        out = {}
        with torch.cuda.stream(stream):
            d = to_device(c5, dev)
        stream.synchronize()
        with tpc.Tracker(stream=stream, profile=True) as t:
            setup(t)
            t.load(d, on_device=True)
            grid_tracks = None
            for corr in ("mlp", "grid", "none"):
                t.set_correction(corr)
                t.autotune(iters=2, mode=1)
                t.set_tuning(use_graph=2)
                for _ in range(2):
                    t.track()
                ms = float(np.median(time_steps(t, stream, 5, flush)))
                if corr == "grid":
                    grid_tracks = t.get_tracks()
                t.set_tuning(use_graph=1)
                t.track()
                st = t.stage_times()
                out[corr] = {"clusters_per_s": c5.n / (ms * 1e-3), "ms": ms, "tracks": t.counts()[0],
                             "correction_us": round(st.get("correction", 0.0), 2)}
        cb, par = form_baseline(c5, grid_tracks[0], grid_tracks[1], 40, 13, correct=(grid, bounds))
        out["grid"]["parity"] = par
        out["grid"]["cpu_baseline"] = cb
        out["mlp"]["parity"] = ("by the GPU tests: the network here is trained on the GPU, and the oracle takes "
                                "no input from the CUDA path")
        res[f"distorted_{batch_events}_events"] = {"clusters": c5.n, "surrogate": info, **out}
    if "c6" in gen:
        res[f"codec_{batch_events}_events"] = bench_codec(gen["c6"], dev, stream, flush, tpc, torch)
    if "c7" in gen:
        res[f"masks_{batch_events}_events"] = bench_masks(gen["c7"], dev, stream, flush, tpc, torch)
    if "c8" in gen:
        res[f"compress_{batch_events}_events"] = bench_compress(*gen["c8"], dev, stream, flush, tpc, torch)
    if "c9" in gen:
        res[f"merge_{batch_events}_events"] = bench_merge(gen["c9"], dev, stream, flush, tpc, torch)
    if "c10" in gen:
        res["removal_chain_loopers"] = bench_removal_chain(*gen["c10"], dev, stream, tpc, torch)
    return res


def bench_frame(fr, dev, stream, flush, tpc, torch, steps=5):
    """The continuous read-out frame resident on the device: every step cuts it
    into slices on the device (tpc_load_frame: 1000 cm cores, 300 cm overlaps;
    the call waits for the slice sizes) and tracks them (tpc_track); the time
    runs from before the slicing to the end of the tracking."""
    with torch.cuda.stream(stream):
        d = to_device(fr, dev)
    d.item_core = None
    stream.synchronize()
    out = {"clusters": fr.n, "items": fr.n_items,
           "note": "clusters/s counts the frame's clusters; slicing on the device is inside the timed step"}
    first = None
    with tpc.Tracker(stream=stream, profile=True) as t:
        t.load_frame(d, 1000.0, 300.0, on_device=True)
        t.track()
        out["slices"] = int(t.debug_dump(1).shape[0] // (7 * t.n_rows))
        for mode in ("plain", "batched"):
            tun, _ = t.autotune(iters=2, mode=1 if mode == "plain" else 2)
            t.set_tuning(use_graph=2)
            ms = []
            for k in range(steps + 2):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                t.load_frame(d, 1000.0, 300.0, on_device=True)
                t.track()
                e1.record(stream)
                with torch.cuda.stream(stream):
                    flush.zero_()
                torch.cuda.synchronize()
                if k >= 2:
                    ms.append(e0.elapsed_time(e1))
            m = float(np.median(ms))
            trk, ids = t.get_tracks()
            out[mode] = {"clusters_per_s": fr.n / (m * 1e-3), "ms": m, "tracks": int(trk.shape[0]), "tuning": tun}
            if first is None:
                first = (trk, ids)
            else:
                out[mode]["identical_to_plain"] = bool(trk.tobytes() == first[0].tobytes() and
                                                       np.array_equal(ids, first[1]))
    del d
    torch.cuda.empty_cache()
    cb, par = form_baseline(fr, first[0], first[1], 3, 12, key="sector")
    cb["sample"] += " (whole, unsliced sectors of the frame)"
    out["parity"] = par
    out["cpu_baseline"] = cb
    return out


def bench_removal_chain(cl, props, dev, stream, tpc, torch):
    """The paper's data-reduction chain (Sec. 4) on one central event whose
    low-pT helices also leave their returning legs: tracking, merger with
    looper legs, the legs joined into one refitted track, masks with the legs,
    compression without removal and with strategies A and B (the form of
    Fig. 6 on synthetic data)."""
    with torch.cuda.stream(stream):
        d = to_device(cl, dev)
        ch = {k: torch.from_numpy(np.ascontiguousarray(props[k])).to(dev)
              for k in ("q_tot", "q_max", "sigma_y", "sigma_z")}
    stream.synchronize()
    res = {"clusters": cl.n, "returning_leg_clusters": int((cl.leg == 1).sum())}
    with tpc.Tracker(stream=stream) as t:
        t.load(d, on_device=True)
        for _ in range(2):  # the second pass is timed (the first allocates the buffers)
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            t.track()
            n_trk = t.counts()[0]
            link, group, fit, partner, leg = t.merge_tracks(n_tracks=n_trk, legs=True, on_device=True)
            joined, jfit, n_joined = t.join_loopers(link, group, partner, leg, n_tracks=n_trk, on_device=True)
            m, _ = t.cluster_masks(on_device=True, with_owner=False, leg=leg, n_tracks=n_trk)
            sizes = {}
            for name, bit in (("none", 0), ("A", 4), ("B", 8)):
                keep = None if bit == 0 else ((m & bit) == 0).to(torch.uint8)
                sizes[name] = int(t.compress(ch, on_device=True, keep=keep).shape[0])
            torch.cuda.synchronize()
            wall = time.perf_counter() - w0
        jw = []  # the join on its own (the call waits for its end)
        for _ in range(5):
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            t.join_loopers(link, group, partner, leg, n_tracks=n_trk, on_device=True)
            jw.append(time.perf_counter() - w0)
    mh = m.cpu().numpy()
    partner = partner.cpu().numpy()
    sec = cl.leg == 1
    # the form of Fig. 6: per bin of the particle's pT, the fractions of its clusters that are
    # associated to a track (attached or in the 1.5 cm tube), protected, and removed by A and by B
    # (below 0.375 GeV/c a helix from the vertex turns inside the chamber, R < 250 cm at 0.5 T; below
    # about 64 MeV/c it does not reach the inner radius of 85 cm, so no cluster has so low a pT here)
    pt = np.where(cl.mc >= 0, cl.tracks["pt"][np.maximum(cl.mc, 0)], -1.0)
    edges = [0.0, 0.15, 0.2, 0.3, 0.375, 0.5, 1.0, 2.0, 1e9]
    by_pt = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (pt >= lo) & (pt < hi)
        if sel.any():
            mm = mh[sel]
            by_pt.append({"pt_gev": [lo, hi if hi < 1e9 else None], "clusters": int(sel.sum()),
                          "associated": float(((mm & 1) != 0).mean()), "protected": float(((mm & 2) != 0).mean()),
                          "removed_by_a": float(((mm & 4) != 0).mean()), "removed_by_b": float(((mm & 8) != 0).mean())})
    noise = cl.mc < 0
    res["by_pt"] = by_pt
    res["noise_clusters"] = {"clusters": int(noise.sum()), "removed_by_b": float(((mh[noise] & 8) != 0).mean())}
    res.update(tracks=n_trk, leg_pairs=int((partner >= 0).sum() // 2), joined_loopers=n_joined,
               join_ms=1e3 * float(np.median(jw)), chain_wall_ms=1e3 * wall,
               removed_by_a=float(((mh & 4) != 0).mean()), removed_by_b=float(((mh & 8) != 0).mean()),
               returning_leg_removed_by_a=float(((mh & 4) != 0)[sec].mean()),
               bytes_per_cluster={k: v / cl.n for k, v in sizes.items()},
               reduction_vs_float_clusters={k: 28.0 * cl.n / v for k, v in sizes.items()})
    del d, ch
    torch.cuda.empty_cache()
    return res


def bench_merge(cl, dev, stream, flush, tpc, torch, steps=10):
    """Sector-track merger with refit and looper legs over the 64 events' own tracks, outputs
    on the device.  The call waits for its end, so it is timed by the host
    clock and, on its stream, by CUDA events around it; the same call with
    host outputs (12 MB of links, groups and refits copied back) beside it.
    L2 flushed between calls."""
    with torch.cuda.stream(stream):
        d = to_device(cl, dev)
    stream.synchronize()
    res = {"clusters": cl.n}
    with tpc.Tracker(stream=stream) as t:
        t.load(d, on_device=True)
        t.track()
        n_trk = t.counts()[0]
        def timed(on_device):
            for _ in range(3):
                t.merge_tracks(n_tracks=n_trk, legs=True, on_device=on_device)
            wall, dev_ms = [], []
            for _ in range(steps):
                with torch.cuda.stream(stream):
                    flush.zero_()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                w0 = time.perf_counter()
                e0.record(stream)
                out = t.merge_tracks(n_tracks=n_trk, legs=True, on_device=on_device)
                e1.record(stream)
                wall.append(time.perf_counter() - w0)
                torch.cuda.synchronize()
                dev_ms.append(e0.elapsed_time(e1))
            return out, 1e3 * float(np.median(wall)), float(np.median(dev_ms))

        (link, group, fit, partner, leg), ms, dms = timed(True)
        link, group, partner = link.cpu().numpy(), group.cpu().numpy(), partner.cpu().numpy()
        _, ms_host, _ = timed(False)
    res.update(tracks=n_trk, tracks_per_s=n_trk / (ms * 1e-3), clusters_per_s=cl.n / (ms * 1e-3), ms=ms,
               device_ms=dms, ms_host_outputs=ms_host, links=int((link >= 0).sum() // 2),
               groups=int(np.unique(group).size), leg_pairs=int((partner >= 0).sum() // 2))
    del d
    torch.cuda.empty_cache()
    return res


def bench_compress(cl, props, dev, stream, flush, tpc, torch, steps=10):
    """Compression of the 64-event batch (Sec. 4, steps 3-4) with the tracker's
    own tracks, charges and output on the device.  The call waits for its
    result (it reads the sizes it needs), so it is timed by the host clock; the
    phases by the library's events.  L2 flushed between calls."""
    with torch.cuda.stream(stream):
        d = to_device(cl, dev)
        ch = {k: torch.from_numpy(np.ascontiguousarray(props[k])).to(dev)
              for k in ("q_tot", "q_max", "sigma_y", "sigma_z")}
    stream.synchronize()
    res = {"clusters": cl.n}
    with tpc.Tracker(stream=stream, profile=True) as t:
        t.load(d, on_device=True)
        t.track()
        blob = t.compress(ch, on_device=True)
        out = torch.empty(blob.shape[0] + (1 << 20), dtype=torch.uint8, device=dev)
        for _ in range(3):
            t.compress(ch, on_device=True, out=out)
        wall, ph = [], {}
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            b = t.compress(ch, on_device=True, out=out)
            wall.append(time.perf_counter() - w0)
            for k, v in t.stage_times().items():
                if k.startswith("compress"):
                    ph.setdefault(k, []).append(v)
        size = int(b.shape[0])
        # the form of the paper's Fig. 6 on synthetic data: stored volume without removal and with the
        # removal of strategies A and B (masks of the tracker's own tracks)
        m, _ = t.cluster_masks(on_device=True, with_owner=False)
        strategies = {}
        for name, bit in (("A", 4), ("B", 8)):
            keep = ((m & bit) == 0).to(torch.uint8)
            bs = t.compress(ch, on_device=True, out=out, keep=keep).shape[0]
            strategies[name] = {"blob_bytes": int(bs), "bytes_per_cluster": bs / cl.n,
                                "kept_clusters": int(keep.sum().item()), "reduction_vs_float_clusters": 28.0 * cl.n / bs}
    ms = 1e3 * float(np.median(wall))
    phases = {k: float(np.median(v)) for k, v in ph.items()}
    # algorithmic bytes of a call: every input read once (positions, row and charges 28 B, the
    # grid order 16 B per cluster, track cluster ids 4 B per cluster at most) and the blob written
    algo = (28 + 16 + 4) * cl.n + size
    peak, kind = measured_peak_hbm()
    dev_us = sum(phases.values())
    achieved = algo / (dev_us * 1e-6) / 1e9
    res.update(clusters_per_s=cl.n / (ms * 1e-3), ms=ms, phase_us=phases, blob_bytes=size,
               bytes_per_cluster=size / cl.n, ratio_vs_integer_codes=13.0 * cl.n / size,
               ratio_vs_float_clusters=28.0 * cl.n / size, removal=strategies,
               roofline={"bound": "hbm", "kernel": "all phases (device time)", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_kind": kind, "algo_bytes": algo})
    del d, ch
    torch.cuda.empty_cache()
    return res


def time_masks(t, stream, flush, steps=10):
    """Device time of tpc_cluster_masks on the tracker's own tracks (device
    buffers, L2 flushed between calls) and of its two kernels."""
    import torch
    for _ in range(3):
        t.cluster_masks(on_device=True)
    ev, st = [], {"mask_assoc": [], "mask_final": []}
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mask, owner = t.cluster_masks(on_device=True)
        e1.record(stream)
        for k, v in t.stage_times().items():  # waits for the stream
            if k in st:
                st[k].append(v)
        with torch.cuda.stream(stream):
            flush.zero_()
        ev.append((e0, e1))
    torch.cuda.synchronize()
    ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
    m = mask.cpu().numpy()
    counts = {"protected": int((m == 3).sum()), "removed_by_a": int(((m & 4) != 0).sum()),
              "removed_by_b": int(((m & 8) != 0).sum())}
    return ms, {k: float(np.median(v)) for k, v in st.items()}, counts


def bench_masks(cl, dev, stream, flush, tpc, torch, steps=10):
    """Cluster association, protection and strategy A/B masks (Sec. 4) over
    the 64-event batch with the tracker's own tracks (graph-replayed
    tracking first, then the masks, device resident)."""
    with torch.cuda.stream(stream):
        d = to_device(cl, dev)
    stream.synchronize()
    res = {"clusters": cl.n}
    with tpc.Tracker(stream=stream, profile=True) as t:
        t.load(d, on_device=True)
        t.track()
        n_trk, n_ids = t.counts()
        ms, kern, counts = time_masks(t, stream, flush, steps)
    peak, kind = measured_peak_hbm()
    n_assoc = counts["protected"] + counts["removed_by_a"]  # associated = protected or removed by A
    # algorithmic bytes: pass 1 reads every sorted hit (16 B) and the tracks' cluster ids (4 B), and
    # reads and writes the association word of every associated cluster (16 B); pass 2 reads the word
    # and the row (12 B), clears the associated words (8 B), writes mask and owner (5 B)
    algo = {"mask_assoc": 16 * cl.n + 4 * n_ids + 16 * n_assoc, "mask_final": 17 * cl.n + 8 * n_assoc}
    dom = max(kern, key=kern.get)
    achieved = algo[dom] / (kern[dom] * 1e-6) / 1e9
    res.update(tracks=n_trk, clusters_per_s=cl.n / (ms * 1e-3), ms=ms, kernel_us=kern, **counts,
               roofline={"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": kind, "algo_bytes": algo[dom]})
    del d
    torch.cuda.empty_cache()
    return res


CODEC_BYTES = 28 + 13  # per cluster: 7 float/int32 properties in, 13 bytes of codes out


def bench_codec(props, dev, stream, flush, tpc, torch, steps=10):
    """Cluster codec (Sec. 4, step 2) on the 64-event batch: device-resident
    properties (L2 flushed between calls), then end to end with pinned host
    buffers; the oracle on a bounded sample for the CPU baseline."""
    n = int(props["y"].shape[0])
    d = {k: torch.from_numpy(np.ascontiguousarray(props[k], dt)).to(dev) for k, dt in tpc.PROP_FIELDS}
    tdt = {np.int16: torch.int16, np.int32: torch.int32, np.uint8: torch.uint8, np.uint16: torch.uint16}
    out = {k: torch.empty(n, dtype=tdt[dt], device=dev) for k, dt in tpc.CODE_FIELDS}
    torch.cuda.synchronize()
    res = {"clusters": n}
    with tpc.Tracker(stream=stream) as t:
        for _ in range(3):
            t.encode_clusters(d, out=out, report_bad=False)
        ev = []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t.encode_clusters(d, out=out, report_bad=False)
            e1.record(stream)
            with torch.cuda.stream(stream):
                flush.zero_()
            ev.append((e0, e1))
        torch.cuda.synchronize()
        ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
        _, bad = t.encode_clusters(d, out=out)
        peak, kind = measured_peak_hbm()
        gbs = CODEC_BYTES * n / (ms * 1e-3) / 1e9
        res.update(clusters_per_s=n / (ms * 1e-3), ms=ms, bad=bad,
                   roofline={"bound": "hbm", "kernel": "k_encode_vec", "achieved": gbs, "peak": peak, "unit": "GB/s",
                             "frac": gbs / peak, "peak_kind": kind, "algo_bytes_per_cluster": CODEC_BYTES})
        # end to end: pinned host properties in, pinned host codes out, copies inside the timed region
        hp = {}
        keep = []
        for k, dt in tpc.PROP_FIELDS:
            buf = torch.empty(n, dtype=torch.from_numpy(np.zeros(1, dt)).dtype, pin_memory=True)
            buf.numpy()[:] = props[k]
            keep.append(buf)
            hp[k] = buf.numpy()
        ho = {}
        for k, dt in tpc.CODE_FIELDS:
            buf = torch.empty(n, dtype=tdt[dt], pin_memory=True)
            keep.append(buf)
            ho[k] = buf.numpy()
        wall = []
        for _ in range(5):
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            t.encode_clusters(hp, out=ho)
            wall.append(time.perf_counter() - w0)
        e2e = float(np.median(wall[1:]))
        res["e2e"] = {"value": n / e2e, "unit": "clusters/s", "h2d_bytes_per_step": 28 * n,
                      "d2h_bytes_per_step": 13 * n}
    del d, out
    torch.cuda.empty_cache()
    # the oracle on a bounded sample, one host core
    import oracle
    m = min(n, 4_000_000)
    sample = {k: np.ascontiguousarray(props[k][:m]) for k, _ in tpc.PROP_FIELDS}
    t0 = time.perf_counter()
    oracle.encode_clusters(sample)
    dt = time.perf_counter() - t0
    res["cpu_baseline"] = {"value": m / dt, "unit": "clusters/s", "cores": 1, "kind": "oracle",
                           "sample": f"first {m} clusters of the 64-event batch"}
    return res


if __name__ == "__main__":
    main()
