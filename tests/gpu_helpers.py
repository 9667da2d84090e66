"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on the
same seeded input and compare (no tracker arithmetic here)."""
import numpy as np

import oracle
import trackeval

STAGE_KEYS = {3: "up_raw", 4: "dn_raw", 5: "up", 6: "dn", 7: "starts"}
FLOORS = np.array([1.0, 1.0, 1.0, 1.0, 0.1])  # y, z [cm]; sinphi, tanlambda; q/pT [c/GeV]


def run_gpu(cl, **kw):
    from paper_1910_12214_b300 import tpc
    with tpc.Tracker(**kw) as t:
        t.load(cl).track()
        trk, ids = t.get_tracks()
        dumps = {s: t.debug_dump(s) for s in range(11)}
    return trk, ids, dumps


def compare_stages(dumps, ref):
    s0 = dumps[0].reshape(-1, 3)
    assert np.array_equal(s0[:, 0], ref["sorted_qy"])
    assert np.array_equal(s0[:, 1], ref["sorted_qz"])
    assert np.array_equal(s0[:, 2], ref["sorted_id"])
    assert np.array_equal(dumps[1].reshape(-1, 7), ref["rows"])
    assert np.array_equal(dumps[2], ref["first"])
    for s, k in STAGE_KEYS.items():
        assert np.array_equal(dumps[s], ref[k]), k


def compare_tracks(cl, trk, ids, ref, min_match=0.995, min_param=0.995):
    """Oracle track A matches GPU track B if |A & B| >= 0.9|A| (one-to-one, greedy);
    matched parameters agree within 1e-3 * max(|oracle|, floor) at the oracle's x_ref
    (GPU parameters propagated in FP64 if the reference rows differ)."""
    from paper_1910_12214_b300 import tpc
    ref_sets = trackeval.track_sets(ref["trk_i"], ref["trk_ids"])
    gpu_sets = trackeval.track_sets(tpc.tracks_to_trk_i(trk), ids.astype(np.int64))
    pairs = trackeval.match_tracks(ref_sets, gpu_sets)
    n_ref = len(ref_sets)
    frac = len(pairs) / max(1, n_ref)
    good = 0
    worst = 0.0
    same_sets = same_good = 0
    bad_params = np.zeros(5, int)
    worst_same = 0.0
    for i, j in pairs.items():
        same = np.array_equal(ref_sets[i][1], gpu_sets[j][1])
        fr = ref["trk_f"][i]
        pg = np.array([trk["y"][j], trk["z"][j], trk["snp"][j], trk["tgl"][j], trk["qpt"][j]], np.float64)
        if abs(float(trk["x_ref"][j]) - fr[0]) > 1e-4:
            out = oracle.propagate(pg, float(trk["x_ref"][j]), fr[0])
            if out is None:
                continue
            pg = out[0]
        rel = np.abs(pg - fr[1:6]) / np.maximum(np.abs(fr[1:6]), FLOORS)
        worst = max(worst, float(rel.max()))
        ok = bool(np.all(rel <= 1e-3))
        good += ok
        bad_params += rel > 1e-3
        if same:
            same_sets += 1
            same_good += ok
            worst_same = max(worst_same, float(rel.max()))
    pfrac = good / max(1, len(pairs))
    res = dict(n_ref=n_ref, n_gpu=len(gpu_sets), matched=frac, param_ok=pfrac, worst_rel=worst,
                identical_sets=same_sets / max(1, len(pairs)), param_ok_identical=same_good / max(1, same_sets),
                worst_rel_identical=worst_same, bad_by_param=bad_params.tolist(),
                ok=frac >= min_match and pfrac >= min_param)
    print("PARITY", res)
    return res


def compare_tracklets_and_selection(trk, ids, dumps, ref, min_identical=0.995):
    """Element-wise comparison of the tracklets (S6) and of the selection (S7/S8).
    The start hits are bit-exact, so tracklet t is built from the same start on
    both sides: its hit count and hit list (outermost first) must be equal on
    >= min_identical of the tracklets (the hit choice is an FP32 vs FP64 chi2
    decision).  Selection is integer work: on every item whose tracklets are all
    identical, the output tracks (tracklet, owned cluster ids) must equal the
    oracle's bit for bit.  Returns the fractions compared."""
    n_g, n_o = dumps[8].astype(np.int64), ref["tl_n"].astype(np.int64)
    assert n_g.shape == n_o.shape
    off_g = np.concatenate([[0], np.cumsum(n_g)])
    off_o = np.concatenate([[0], np.cumsum(n_o)])
    hits_g, hits_o = dumps[9], ref["tl_hits"]
    meta = ref["tl_meta"].reshape(-1, 2)
    same = np.array([n_g[t] == n_o[t] and np.array_equal(hits_g[off_g[t]:off_g[t + 1]], hits_o[off_o[t]:off_o[t + 1]])
                     for t in range(n_g.shape[0])], bool)
    frac = float(same.mean()) if same.size else 1.0
    assert frac >= min_identical, frac
    items_all = np.unique(meta[:, 0])
    bad_items = set(meta[~same, 0].tolist())
    clean = [int(i) for i in items_all if int(i) not in bad_items]
    # GPU tracks per item: (item-local tracklet id, sorted owned cluster ids)
    tl_of_track = dumps[10]
    got, want = {}, {}
    for k in range(trk.shape[0]):
        it, loc = (int(v) for v in meta[tl_of_track[k]])
        assert it == int(trk["item"][k])
        f, n = int(trk["first_cluster"][k]), int(trk["n_clusters"][k])
        got.setdefault(it, []).append((loc, tuple(sorted(ids[f:f + n].tolist()))))
    ti, tids = ref["trk_i"].reshape(-1, 4), ref["trk_ids"]
    for it, f, n, loc in ti:
        want.setdefault(int(it), []).append((int(loc), tuple(sorted(tids[f:f + n].tolist()))))
    for it in clean:
        assert sorted(got.get(it, [])) == sorted(want.get(it, [])), it
    n_tracks_clean = sum(len(want.get(it, [])) for it in clean)
    res = dict(tracklets=int(n_g.shape[0]), identical=frac, items=int(items_all.shape[0]), items_all_identical=len(clean),
               tracks_compared_bitwise=n_tracks_clean, tracks=int(ti.shape[0]))
    print("TRACKLETS", res)
    return res
