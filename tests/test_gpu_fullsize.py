"""Parity at the full sizes of the benchmark workloads, in the launch shapes the
benchmark times (autotuned): every item of a batch is independent, so the oracle
runs on a seeded sample of items (the largest ones included) and the GPU tracks
of those items are compared with it; the rest is checked by properties that hold
at any size (plain and batched forms give identical bytes)."""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import compare_tracks
from paper_1910_12214_b300 import shard, synth

pytestmark = pytest.mark.gpu


def _tracks_of_items(trk, ids, items, index):
    """GPU tracks of the given items, renumbered for the sub-batch made by
    shard.take_items(cl, items) (item numbers and cluster ids)."""
    pos_of_item = {int(it): j for j, it in enumerate(items)}
    inv = {int(g): k for k, g in enumerate(index)}
    keep = [i for i in range(len(trk)) if int(trk["item"][i]) in pos_of_item]
    sub = trk[keep].copy()
    out_ids = []
    base = 0
    for j, i in enumerate(keep):
        f, n = int(trk["first_cluster"][i]), int(trk["n_clusters"][i])
        out_ids.extend(inv[int(c)] for c in ids[f:f + n])
        sub["item"][j] = pos_of_item[int(trk["item"][i])]
        sub["first_cluster"][j] = base
        base += n
    return sub, np.asarray(out_ids, dtype=np.uint32)


def _sample_items(cl, k, seed):
    costs = shard.item_costs(cl)
    rng = np.random.default_rng(seed)
    largest = np.argsort(-costs, kind="stable")[:4]
    rest = rng.choice(np.setdiff1d(np.arange(cl.n_items), largest), size=k - 4, replace=False)
    return np.sort(np.concatenate([largest, rest]))


@pytest.fixture(scope="module")
def batch64():
    return synth.make_batched(seed=1, n_events=64)


def _run(cl, mode, tracker_kw=None):
    from paper_1910_12214_b300 import tpc
    with tpc.Tracker(**(tracker_kw or {})) as t:
        t.load(cl)
        tun, _ = t.autotune(iters=1, mode=mode)
        t.track()
        trk, ids = t.get_tracks()
    return trk, ids, tun


def test_64_events_plain_and_batched_at_autotuned_shapes(batch64):
    cl = batch64
    trk_p, ids_p, tun_p = _run(cl, 1)
    trk_b, ids_b, tun_b = _run(cl, 2)
    assert tun_p["mode"] == 1 and tun_b["mode"] == 2
    assert trk_p.tobytes() == trk_b.tobytes() and np.array_equal(ids_p, ids_b)
    items = _sample_items(cl, 40, seed=11)
    sub, index = shard.take_items(cl, items)
    ref = oracle.run(sub)
    trk_s, ids_s = _tracks_of_items(trk_p, ids_p, items, index)
    r = compare_tracks(sub, trk_s, ids_s, ref)
    print("PARITY 64 events, 40 sampled items", r)
    assert r["ok"], r


def test_time_frame_sampled_slices_at_autotuned_shape():
    fr = synth.make_timeframe(seed=1)
    sl = synth.slice_frame(fr)
    trk, ids, _ = _run(sl, 1)
    items = _sample_items(sl, 24, seed=12)
    sub, index = shard.take_items(sl, items)
    ref = oracle.run(sub)
    trk_s, ids_s = _tracks_of_items(trk, ids, items, index)
    r = compare_tracks(sub, trk_s, ids_s, ref)
    print("PARITY time frame, 24 sampled slices", r)
    assert r["ok"], r


def test_full_tpc_event_at_autotuned_shape():
    cl = synth.make_config2()
    trk, ids, tun = _run(cl, 0)
    ref = oracle.run(cl)
    r = compare_tracks(cl, trk, ids, ref)
    print("PARITY full TPC event, autotuned", tun, r)
    assert r["ok"], r


def test_corrections_of_the_distorted_64_events_sampled(batch64):
    """Grid and network corrections of every cluster of the distorted 64-event
    batch, checked against the FP64 oracle on a sample of 200,000 clusters."""
    from paper_1910_12214_b300 import tpc
    d = synth.make_distortion(seed=1, n_sectors=36)
    grid, bounds = synth.correction_grid(d)
    dcl = synth.distort(batch64, d)
    P = oracle.mlp_init(5, 0)
    P[-3:] = [0.0, 0.2, -0.1]
    with tpc.Tracker() as t:
        t.set_grid_correction(grid, bounds)
        for s in range(36):
            t.surrogate_set_params(s, P)
        t.load(dcl)
        t.set_correction("grid")
        t.track()
        gy, gz = t.corrected()
        t.set_correction("mlp")
        t.track()
        my, mz = t.corrected()
    rng = np.random.default_rng(13)
    pick = np.sort(rng.choice(dcl.n, size=200_000, replace=False))
    off = dcl.item_off.astype(np.int64)
    item = np.searchsorted(off, pick, side="right") - 1
    sec = dcl.item_sector[item].astype(np.int64)
    xr = np.rint((85.0 + np.arange(152) * (161.0 / 151.0)) * 1024.0) / 1024.0
    x = xr[dcl.row[pick]]
    y = dcl.y[pick].astype(np.float64)
    z = dcl.z[pick].astype(np.float64)
    # grid: FP64 trilinear oracle at the quantised pad-row x (FP32 on the GPU)
    dy, dz = oracle.trilinear(grid, bounds, sec, x, y, z)
    ey = float(np.max(np.abs(gy[pick] - (y + dy).astype(np.float32))))
    ez = float(np.max(np.abs(gz[pick] - (z + dz).astype(np.float32))))
    assert ey < 2e-4 and ez < 2e-4, (ey, ez)
    # network: FP64 forward of the same parameters
    x0, x1, v0, v1, z0, z1 = (bounds[sec, k].astype(np.float64) for k in range(6))
    v = y / (x * math.tan(math.radians(10.0)))
    inp = np.stack([(x - x0) * (2 / (x1 - x0)) - 1, (v - v0) * (2 / (v1 - v0)) - 1, (z - z0) * (2 / (z1 - z0)) - 1], 1)
    out = oracle.mlp_forward(P, inp)
    scale = 10.0 * np.abs(out[:, 1:]).max()
    assert np.max(np.abs(my[pick] - (y + 10.0 * out[:, 1]))) <= 1e-2 * scale
    assert np.max(np.abs(mz[pick] - (z + 10.0 * out[:, 2]))) <= 1e-2 * scale
