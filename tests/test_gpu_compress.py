"""Parity of the CUDA compression (Sec. 4, steps 3 to 5) with the oracle,
through the C ABI: given the same tracks (the oracle tracker's), the GPU's blob
equals the oracle's byte for byte; with the GPU's own tracks the oracle's
decoder restores every stored cluster exactly."""
import numpy as np
import pytest

import oracle
from test_gpu_masks import to_records

pytestmark = pytest.mark.gpu


def tracked(cl):
    from paper_1910_12214_b300 import tpc
    t = tpc.Tracker(device=0)
    t.load(cl).track()
    t.sync()
    return t


def oracle_blob(cl, props):
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids", "sorted_id", "rows"])
    tf, ti, ids = oracle.oracle_tracks(ref)
    order, seg = oracle.grid_order(ref)
    return oracle.compress(cl, props, order, seg, tf, ti, ids), (tf, ti, ids), (order, seg)


def first_difference(a, b):
    n = min(a.size, b.size)
    d = np.flatnonzero(a[:n] != b[:n])
    return int(d[0]) if d.size else n


@pytest.mark.parametrize("cfg", ["c1", "c2"])
def test_blob_equals_the_oracle_blob(cfg):
    from paper_1910_12214_b300 import synth
    cl = synth.make_config1(seed=12) if cfg == "c1" else synth.make_config2(seed=12)
    props = synth.cluster_props(cl, seed=12)
    want, (tf, ti, ids), _ = oracle_blob(cl, props)
    with tracked(cl) as t:
        got = t.compress(props, to_records(tf, ti), ids)
        again = t.compress(props, to_records(tf, ti), ids, out=np.empty(got.size + 100, np.uint8))
    assert got.size == want.size, (got.size, want.size, first_difference(got, want))
    assert np.array_equal(got, want), first_difference(got, want)
    assert np.array_equal(again, want)


def test_own_tracks_device_call_round_trips_through_the_oracle_decoder():
    """The product path: the GPU's own tracks and device buffers; the blob
    decodes (oracle decoder) to exactly the codes of the stored clusters."""
    import torch
    from paper_1910_12214_b300 import synth
    cl = synth.make_config2(seed=13)
    props = synth.cluster_props(cl, seed=13)
    with tracked(cl) as t:
        trk, tids = t.get_tracks()
        dprops = {k: torch.from_numpy(props[k]).cuda() for k in ("q_tot", "q_max", "sigma_y", "sigma_z")}
        blob = t.compress(dprops, on_device=True).cpu().numpy()
        order = t.debug_dump(0).reshape(-1, 3)[:, 2]  # canonical order of the binned clusters
    d = oracle.decompress(blob)
    codes, _ = oracle.encode_clusters(props)
    attached = np.zeros(cl.n, bool)
    attached[tids] = True
    seq = np.concatenate([order[~attached[order]], tids.astype(np.int64)])
    for k in ("y", "z", "q_tot", "q_max", "sigma_y", "sigma_z"):
        assert np.array_equal(d[k], codes[k][seq].astype(np.int32)), k
    assert np.array_equal(d["row"], cl.row[seq])
    trk_of = np.repeat(np.arange(trk.shape[0]), trk["n_clusters"].astype(np.int64))
    assert np.array_equal(d["track"][-trk_of.size:], trk_of)
    raw = 13 * seq.size  # the integer codes of the stored clusters
    assert blob.size < raw / 1.3


def test_full_size_64_events_device_call():
    """The benchmark's 64-event batch (16.1M clusters): device buffers, oracle
    tracks; the blob equals the oracle's byte for byte."""
    import torch
    from paper_1910_12214_b300 import synth
    cl = synth.make_batched(seed=1)
    props = synth.cluster_props(cl, seed=1)
    want, (tf, ti, ids), _ = oracle_blob(cl, props)
    rec = to_records(tf, ti)
    with tracked(cl) as t:
        dprops = {k: torch.from_numpy(props[k]).cuda() for k in ("q_tot", "q_max", "sigma_y", "sigma_z")}
        d_rec = torch.from_numpy(rec.view(np.uint8).reshape(-1, rec.dtype.itemsize)).cuda()
        d_ids = torch.from_numpy(ids.view(np.int32)).cuda()
        got = t.compress(dprops, d_rec, d_ids, on_device=True).cpu().numpy()
    assert got.size == want.size, (got.size, want.size, first_difference(got, want))
    assert np.array_equal(got, want), first_difference(got, want)


def test_edge_cases():
    from paper_1910_12214_b300 import synth, tpc
    cl = synth.make_config1(seed=14)
    props = synth.cluster_props(cl, seed=14)
    t = tpc.Tracker(device=0)
    t.load(cl)
    with pytest.raises(tpc.TpcError) as e:
        t.compress(props)
    assert e.value.status == 2
    t.track()
    # no tracks: every binned cluster is stored as unattached; equal to the oracle's blob
    empty = np.zeros(0, dtype=tpc.TRACK_DTYPE)
    ref = oracle.run(cl, what=["sorted_id", "rows"])
    order, seg = oracle.grid_order(ref)
    want = oracle.compress(cl, props, order, seg, np.zeros((0, 6)), np.zeros((0, 3)), np.zeros(0, np.uint32))
    got = t.compress(props, empty, np.zeros(0, np.uint32))
    assert np.array_equal(got, want)
    # a buffer too small: the size is reported, nothing is written
    import ctypes as C
    ch = tpc.tpc_cluster_charges(*[props[k].ctypes.data for k in ("q_tot", "q_max", "sigma_y", "sigma_z")])
    size = C.c_uint64()
    small = np.zeros(16, np.uint8)
    st = tpc._lib.tpc_compress(t._h, C.byref(ch), empty.ctypes.data, 0, None, 0, None, 0, small.ctypes.data, 16,
                               C.byref(size))
    assert st == 5 and size.value == want.size and not small.any()
    # a track outside the batch
    rtf, rti, rids = oracle.oracle_tracks(oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"]))
    rec = to_records(rtf, rti)
    rec["item"][1] = 7
    with pytest.raises(tpc.TpcError) as e:
        t.compress(props, rec, rids)
    assert e.value.status == 7
    t.close()


def test_removal_by_strategy_a_b_and_random():
    """Sec. 4, step 5: with the keep masks of strategies A and B (from the
    oracle's masks) and a random one, the blob equals the oracle's byte for
    byte, and the stored volume shrinks in the order none > A > B."""
    from paper_1910_12214_b300 import synth
    cl = synth.make_config2(seed=15)
    props = synth.cluster_props(cl, seed=15)
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids", "sorted_id", "rows"])
    tf, ti, ids = oracle.oracle_tracks(ref)
    order, seg = oracle.grid_order(ref)
    wm, _, _ = oracle.cluster_masks(cl, tf, ti, ids)
    keeps = {"A": ((wm & 4) == 0).astype(np.uint8), "B": ((wm & 8) == 0).astype(np.uint8),
             "random": (np.random.default_rng(1).uniform(size=cl.n) < 0.7).astype(np.uint8)}
    sizes = {}
    with tracked(cl) as t:
        full = t.compress(props, to_records(tf, ti), ids)
        for name, keep in keeps.items():
            want = oracle.compress(cl, props, order, seg, tf, ti, ids, keep=keep)
            got = t.compress(props, to_records(tf, ti), ids, keep=keep)
            assert got.size == want.size and np.array_equal(got, want), (name, first_difference(got, want))
            sizes[name] = got.size
    assert full.size > sizes["A"] > sizes["B"]
