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
        dumps = {s: t.debug_dump(s) for s in range(10)}
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
