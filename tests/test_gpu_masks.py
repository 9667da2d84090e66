"""Parity of the CUDA cluster masks (Sec. 4: attachment, adjacency, protection,
strategies A and B) with the oracle, through the C ABI.

Both sides get the same tracks (the oracle tracker's, never the GPU's), so
every cluster's mask and owner must agree exactly, except clusters the oracle
flags as rounding-sensitive (a tube distance within 1e-3 cm of the radius, an
inclination within 1e-5 of a limit): there only validity is checked."""
import numpy as np
import pytest

import oracle
from test_oracle_masks_pins import golden_case

pytestmark = pytest.mark.gpu


def to_records(tf, ti):
    from paper_1910_12214_b300 import tpc
    r = np.zeros(tf.shape[0], dtype=tpc.TRACK_DTYPE)
    for k, name in enumerate(("x_ref", "y", "z", "snp", "tgl", "qpt")):
        r[name] = tf[:, k]
    r["item"], r["first_cluster"], r["n_clusters"] = ti[:, 0], ti[:, 1], ti[:, 2]
    return r


def compare(mask, owner, want_mask, want_owner, amb, max_amb=1e-3):
    ok = amb == 0
    assert ok.mean() >= 1.0 - max_amb
    bad = np.flatnonzero(ok & ((mask != want_mask) | (owner != want_owner)))
    assert bad.size == 0, (bad[:10], mask[bad[:10]], want_mask[bad[:10]], owner[bad[:10]], want_owner[bad[:10]])
    # rounding-sensitive clusters: a valid outcome all the same
    assert np.all(np.isin(mask[~ok], [3, 13, 8]))
    assert np.all((owner[~ok] >= 0) == (mask[~ok] != 8))


def tracked(cl, bz=0.5):
    from paper_1910_12214_b300 import tpc
    t = tpc.Tracker(device=0, bz_tesla=bz)
    t.load(cl).track()
    t.sync()
    return t


def test_hand_worked_fixture_on_the_gpu():
    g, cl, tf, ti, ids, leg, names, own, extra = golden_case()
    with tracked(cl, bz=g["bz"]) as t:
        mask, owner = t.cluster_masks(to_records(tf, ti), ids, leg, tube=g["tube"], min_pt=g["min_pt"],
                                      max_incl_deg=g["max_incl_deg"])
    wm, wo, amb = oracle.cluster_masks(cl, tf, ti, ids, leg, tube=g["tube"], bz=g["bz"])
    for c, (who, m) in enumerate(own):
        assert names[owner[c]] == who and mask[c] == m
    for k, e in enumerate(extra):
        c = len(own) + k
        if e["ambiguous"]:
            continue
        want = -1 if e["owner"] is None else names.index(e["owner"])
        assert (owner[c], mask[c]) == (want, e["mask"]), e["name"]
    compare(mask, owner, wm, wo, amb, max_amb=0.05)


@pytest.mark.parametrize("cfg,tube", [("c1", 1.5), ("c1", 4.0), ("c2", 1.5)])
def test_oracle_tracks_host_call(cfg, tube):
    from paper_1910_12214_b300 import synth
    cl = synth.make_config1(seed=5) if cfg == "c1" else synth.make_config2(seed=5)
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.oracle_tracks(ref)
    leg = (np.arange(tf.shape[0]) % 7 == 2).astype(np.uint8)
    wm, wo, amb = oracle.cluster_masks(cl, tf, ti, ids, leg, tube=tube)
    with tracked(cl) as t:
        mask, owner = t.cluster_masks(to_records(tf, ti), ids, leg, tube=tube)
        # a second call gives the same (the association words are cleared between calls)
        mask2, owner2 = t.cluster_masks(to_records(tf, ti), ids, leg, tube=tube)
    compare(mask, owner, wm, wo, amb)
    assert np.array_equal(mask, mask2) and np.array_equal(owner, owner2)


def test_own_tracks_device_call_agrees_with_the_oracle_chain():
    """The product path: the GPU tracker's own tracks, masks on the device.
    The two tracker outputs differ slightly, so the masks are compared as
    fractions; the relations between the masks hold exactly."""
    import torch
    from paper_1910_12214_b300 import synth
    cl = synth.make_config2(seed=6)
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.oracle_tracks(ref)
    wm, _, _ = oracle.cluster_masks(cl, tf, ti, ids)
    with tracked(cl) as t:
        trk, tids = t.get_tracks()
        m, o = t.cluster_masks(on_device=True)
        torch.cuda.synchronize()
        mask, owner = m.cpu().numpy(), o.cpu().numpy()
    assert (mask == wm).mean() > 0.995
    keep_a, keep_b = (mask & 4) == 0, (mask & 8) == 0
    assert np.all(keep_a[keep_b])
    assert np.all((owner >= 0) == ((mask & 1) != 0))
    tr = np.repeat(np.arange(trk.shape[0]), trk["n_clusters"].astype(np.int64))
    w = owner[tids]
    assert np.all(w >= 0)
    assert np.all(np.abs(trk["qpt"][w]) <= np.abs(trk["qpt"][tr]))


def test_full_size_64_events_device_call():
    """The benchmark's 64-event batch (16.1M clusters), tracks of the oracle
    tracker given as device arrays, masks compared for every cluster."""
    import torch
    from paper_1910_12214_b300 import synth
    cl = synth.make_batched(seed=1)
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.oracle_tracks(ref)
    wm, wo, amb = oracle.cluster_masks(cl, tf, ti, ids)
    rec = to_records(tf, ti)
    with tracked(cl) as t:
        d_rec = torch.from_numpy(rec.view(np.uint8).reshape(-1, rec.dtype.itemsize)).cuda()
        d_ids = torch.from_numpy(ids.view(np.int32)).cuda()
        m, o = t.cluster_masks(d_rec, d_ids, on_device=True)
        torch.cuda.synchronize()
        t.sync()
        mask, owner = m.cpu().numpy(), o.cpu().numpy()
    compare(mask, owner, wm, wo, amb)


def test_edge_cases():
    from paper_1910_12214_b300 import synth, tpc
    cl = synth.make_config1(seed=7)
    t = tpc.Tracker(device=0)
    t.load(cl)
    with pytest.raises(tpc.TpcError) as e:  # no bins before tpc_track
        t.cluster_masks()
    assert e.value.status == 2
    t.track()
    empty = np.zeros(0, dtype=tpc.TRACK_DTYPE)
    mask, owner = t.cluster_masks(empty, np.zeros(0, np.uint32))
    assert np.all(mask == 8) and np.all(owner == -1)
    # a track pointing outside the batch is skipped and reported; the others still count
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.oracle_tracks(ref)
    rec = to_records(tf, ti)
    rec["item"][0] = 99
    with pytest.raises(tpc.TpcError) as e:
        t.cluster_masks(rec, ids)
    assert e.value.status == 7
    t.close()


def test_unaligned_buffers_take_the_scalar_final_pass():
    """Cluster arrays and outputs off their vector alignment: the scalar form of
    the final pass gives the same masks and owners as the vector form."""
    import torch
    from paper_1910_12214_b300 import synth, tpc
    cl = synth.make_config1(seed=8)
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.oracle_tracks(ref)
    rec = to_records(tf, ti)
    with tracked(cl) as t:
        want_m, want_o = t.cluster_masks(rec, ids)
    d = type("D", (), {})()
    for name in ("x", "y", "z", "row"):
        a = torch.from_numpy(np.ascontiguousarray(getattr(cl, name)))
        buf = torch.empty(a.shape[0] + 1, dtype=a.dtype, device="cuda")
        buf[1:].copy_(a)
        setattr(d, name, buf[1:])  # 4 bytes past a 16-byte boundary
    d.item_off, d.item_sector, d.item_event, d.item_core = cl.item_off, cl.item_sector, cl.item_event, None
    with tpc.Tracker(device=0) as t:
        t.load(d, on_device=True).track()
        t.sync()
        mask, owner = t.cluster_masks(rec, ids)
    assert np.array_equal(mask, want_m) and np.array_equal(owner, want_o)
