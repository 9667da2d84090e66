"""Continuous-readout time frames (Abstract: 50 kHz continuous read-out, no a
priori vertex).  Collisions overlap in the drift volume; cluster z carries the
drift-time offset.  tpc_load_frame cuts each sector's frame into slices on the
device (1000 cm core, 300 cm overlap each side); a track is reported by the
slice whose core holds its innermost cluster.  Slicing must be invisible: the
CUDA result equals the oracle on the whole, unsliced frame."""
import numpy as np
import pytest

import oracle
import trackeval
from paper_1910_12214_b300 import synth
from gpu_helpers import FLOORS, compare_stages, compare_tracks, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def frame():
    fr = synth.make_timeframe(n_coll=8, seed=3)
    sl = synth.slice_frame(fr)
    return fr, sl


def _frame_run(fr, on_device=False, **kw):
    import torch
    from paper_1910_12214_b300 import tpc
    src = fr
    if on_device:
        dev = torch.device("cuda", 0)
        src = type("F", (), {})()
        for k in ("x", "y", "z", "row"):
            setattr(src, k, torch.from_numpy(np.ascontiguousarray(getattr(fr, k))).to(dev))
        src.item_off, src.item_sector, src.item_event = fr.item_off, fr.item_sector, fr.item_event
    with tpc.Tracker(**kw) as t:
        t.load_frame(src, 1000.0, 300.0)
        t.track()
        trk, ids = t.get_tracks()
        dumps = {s: t.debug_dump(s) for s in (0, 1)}
    return trk, ids, dumps


def test_sliced_frame_bit_exact_on_its_own_input(frame):
    fr, sl = frame
    assert sl.n_items > fr.n_items  # several slices per sector
    ref = oracle.run(sl)
    trk, ids, d = run_gpu(sl)
    compare_stages(d, ref)
    r = compare_tracks(sl, trk, ids, ref)
    assert r["ok"], r


def test_device_slicing_equals_the_generator_slicing(frame):
    """The slices built on the device are the generator's (same items, same
    clusters in the same order); the tracks are the same, with frame indices."""
    fr, sl = frame
    trk_f, ids_f, d_f = _frame_run(fr)
    trk_s, ids_s, d_s = run_gpu(sl)
    assert np.array_equal(d_f[0], d_s[0]) and np.array_equal(d_f[1], d_s[1])
    assert np.array_equal(trk_f["item"], trk_s["item"]) and np.array_equal(trk_f["sector"], trk_s["sector"])
    assert trk_f.tobytes() == trk_s.tobytes()
    assert np.array_equal(ids_f, sl.src_index[ids_s.astype(np.int64)])


def test_device_input_frame_equals_host_input_frame(frame):
    fr, _ = frame
    trk_h, ids_h, _ = _frame_run(fr)
    trk_d, ids_d, _ = _frame_run(fr, on_device=True)
    assert trk_h.tobytes() == trk_d.tobytes() and np.array_equal(ids_h, ids_d)


def test_slicing_is_invisible_against_the_unsliced_oracle(frame):
    fr, _ = frame
    ref = oracle.run(fr)  # one item per sector, whole frame
    trk, ids, _ = _frame_run(fr)
    gsets = [(int(sec), np.sort(ids[f:f + n].astype(np.int64)))
             for sec, f, n in zip(trk["sector"], trk["first_cluster"], trk["n_clusters"])]
    rsets = [(int(fr.item_sector[it]), s_) for it, s_ in trackeval.track_sets(ref["trk_i"], ref["trk_ids"])]
    pairs = trackeval.match_tracks(rsets, gsets)
    matched = len(pairs) / len(rsets)
    assert matched >= 0.995, (matched, len(rsets), len(gsets))
    assert abs(len(gsets) - len(rsets)) <= 0.005 * len(rsets)  # no duplicates from the overlaps
    good = 0
    for i, j in pairs.items():
        fr_ = ref["trk_f"][i]
        pg = np.array([trk["y"][j], trk["z"][j], trk["snp"][j], trk["tgl"][j], trk["qpt"][j]], np.float64)
        if abs(float(trk["x_ref"][j]) - fr_[0]) > 1e-4:
            out = oracle.propagate(pg, float(trk["x_ref"][j]), fr_[0])
            if out is None:
                continue
            pg = out[0]
        rel = np.abs(pg - fr_[1:6]) / np.maximum(np.abs(fr_[1:6]), FLOORS)
        good += bool(np.all(rel <= 1e-3))
    assert good / len(pairs) >= 0.995


def test_frame_tracking_efficiency_without_vertex(frame):
    fr, _ = frame
    trk, ids, _ = _frame_run(fr)
    # efficiency against MC truth per sector (sanity, not a parity gate)
    trk_i = np.stack([trk["sector"].astype(np.int64), trk["first_cluster"].astype(np.int64),
                      trk["n_clusters"].astype(np.int64), np.arange(trk.shape[0])], axis=1)
    e = trackeval.efficiency(fr, trk_i, ids.astype(np.int64))
    assert e["eff"] > 0.95 and e["fake_rate"] < 0.01, e


def test_frame_errors_leave_the_context_usable(frame):
    from paper_1910_12214_b300 import tpc
    fr, _ = frame
    with tpc.Tracker() as t:
        with pytest.raises(tpc.TpcError) as ex:
            t.load_frame(fr, 1000.0, 3500.0)  # overlap above 3 cores
        assert ex.value.status == 1
        bad = type("F", (), {})()
        bad.x, bad.y, bad.row = fr.x, fr.y, fr.row
        bad.z = fr.z.copy()
        bad.z[7] = np.nan
        bad.item_off, bad.item_sector, bad.item_event = fr.item_off, fr.item_sector, fr.item_event
        with pytest.raises(tpc.TpcError) as ex:
            t.load_frame(bad)
        assert ex.value.status == 7
        t.load_frame(fr).track()  # still usable
        n_trk, _ = t.counts()
        assert n_trk > 0
        with pytest.raises(tpc.TpcError) as ex:  # the reduction calls take tpc_load_clusters batches
            t.merge_tracks()
        assert ex.value.status == 2
