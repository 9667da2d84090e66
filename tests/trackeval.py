"""Track-level evaluation helpers shared by the tests (no tracker arithmetic)."""
from __future__ import annotations

import numpy as np


def track_sets(trk_i: np.ndarray, ids: np.ndarray):
    """List of (item, sorted cluster-id array) per track from (item, first, count, ...) rows."""
    out = []
    for it, first, cnt in trk_i[:, :3]:
        out.append((int(it), np.sort(ids[int(first):int(first) + int(cnt)])))
    return out


def efficiency(cl, trk_i, ids, min_findable=20, purity=0.9, coverage=0.5, pt_min=0.0):
    """Findable = MC track with >= min_findable clusters in one item; found = a track of
    >= purity from it covering >= coverage of its clusters; fake = purity below threshold."""
    item_of = np.repeat(np.arange(cl.n_items), np.diff(cl.item_off.astype(np.int64)))
    mc = cl.mc
    sig = mc >= 0
    key = mc[sig].astype(np.int64) * (cl.n_items + 1) + item_of[sig]
    uk, cnt = np.unique(key, return_counts=True)
    pt = cl.tracks["pt"]
    findable = {int(k): int(c) for k, c in zip(uk, cnt) if c >= min_findable and pt[k // (cl.n_items + 1)] >= pt_min}
    found, fakes = set(), 0
    for it, s in track_sets(trk_i, ids):
        labels = mc[s]
        vals, c = np.unique(labels, return_counts=True)
        j = int(np.argmax(c))
        if vals[j] < 0 or c[j] < purity * s.shape[0]:
            fakes += 1
            continue
        k = int(vals[j]) * (cl.n_items + 1) + it
        if k in findable and c[j] >= coverage * findable[k]:
            found.add(k)
    n_f = max(1, len(findable))
    return dict(findable=len(findable), found=len(found), eff=len(found) / n_f,
                fake_rate=fakes / max(1, trk_i.shape[0]), n_tracks=int(trk_i.shape[0]))


def match_tracks(ref, test, min_shared=0.9):
    """Greedy one-to-one matching: ref track A matches test track B (same item) if
    |A & B| >= min_shared*|A|; greedy by descending overlap, ties by lower B index."""
    by_item = {}
    for j, (it, s) in enumerate(test):
        by_item.setdefault(it, []).append(j)
    cands = []
    for i, (it, a) in enumerate(ref):
        for j in by_item.get(it, []):
            ov = np.intersect1d(a, test[j][1], assume_unique=True).shape[0]
            if ov >= min_shared * a.shape[0]:
                cands.append((-ov, j, i))
    cands.sort()
    used_r, used_t, pairs = set(), set(), {}
    for nov, j, i in cands:
        if i in used_r or j in used_t:
            continue
        used_r.add(i)
        used_t.add(j)
        pairs[i] = j
    return pairs
