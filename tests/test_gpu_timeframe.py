"""Continuous-readout time frames (Abstract: 50 kHz continuous read-out, no a
priori vertex).  Collisions overlap in the drift volume; cluster z carries the
drift-time offset.  Each sector's frame is cut into slices (1000 cm core,
300 cm overlap each side); a track is reported by the slice whose core holds its
innermost cluster.  Slicing must be invisible: the sliced CUDA result equals
the oracle on the whole, unsliced frame."""
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


def test_sliced_frame_bit_exact_on_its_own_input(frame):
    fr, sl = frame
    assert sl.n_items > fr.n_items  # several slices per sector
    ref = oracle.run(sl)
    trk, ids, d = run_gpu(sl)
    compare_stages(d, ref)
    r = compare_tracks(sl, trk, ids, ref)
    assert r["ok"], r


def test_slicing_is_invisible_against_the_unsliced_oracle(frame):
    from paper_1910_12214_b300 import tpc
    fr, sl = frame
    ref = oracle.run(fr)  # one item per sector, whole frame
    trk, ids, _ = run_gpu(sl)
    # GPU tracks in frame coordinates: cluster ids through the slice map, items as sectors
    ids_fr = sl.src_index[ids.astype(np.int64)]
    gsets = [(int(sl.item_sector[it]), np.sort(ids_fr[f:f + n]))
             for it, f, n in zip(trk["item"], trk["first_cluster"], trk["n_clusters"])]
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
    fr, sl = frame
    trk, ids, _ = run_gpu(sl)
    from paper_1910_12214_b300 import tpc
    ids_fr = sl.src_index[ids.astype(np.int64)]
    # efficiency against MC truth per sector (sanity, not a parity gate)
    sector_of = np.repeat(np.arange(fr.n_items), np.diff(fr.item_off.astype(np.int64)))
    trk_i = np.stack([sl.item_sector[trk["item"]].astype(np.int64), trk["first_cluster"].astype(np.int64),
                      trk["n_clusters"].astype(np.int64), np.arange(trk.shape[0])], axis=1)
    e = trackeval.efficiency(fr, trk_i, ids_fr)
    assert e["eff"] > 0.95 and e["fake_rate"] < 0.01, e
