"""Pins of the removal-mask oracle (Sec. 4: attachment, adjacency, protection,
strategies A and B): a hand-worked fixture, an independent brute force that
places tracks by exact circle geometry, and the relations the paper states
between the two strategies."""
import json
import math
import os
import types

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "removal_masks.json")
N_ROWS, X_MIN, X_MAX = 152, 85.0, 246.0
KB = 0.299792458e-2
A_, P_, RA, RB = 1, 2, 4, 8


def row_x():
    r = np.arange(N_ROWS)
    return np.rint((X_MIN + r * ((X_MAX - X_MIN) / (N_ROWS - 1))) * 1024.0) / 1024.0


def clusters(y, z, row, item_off=None):
    y = np.asarray(y, np.float32)
    n = y.shape[0]
    off = np.array([0, n], np.uint64) if item_off is None else np.asarray(item_off, np.uint64)
    return types.SimpleNamespace(x=row_x()[np.asarray(row)].astype(np.float32), y=y,
                                 z=np.asarray(z, np.float32), row=np.asarray(row, np.int32), item_off=off)


def golden_case():
    g = json.load(open(GOLDEN))
    xr = row_x()
    ys, zs, rows, trk_f, trk_i, ids, legs, names = [], [], [], [], [], [], [], []
    own = []
    for t in g["tracks"]:
        first = len(ids)
        rr = list(range(10)) if "rows 0-9" in t["clusters"] else [0, 1]
        tan = t["snp"] / math.sqrt(1.0 - t["snp"] ** 2)
        for r in rr:
            ids.append(len(ys))
            own.append(t["own"])
            ys.append(t["y"] + (xr[r] - xr[0]) * tan)  # straight line (Bz = 0)
            zs.append(0.0)
            rows.append(r)
        trk_f.append([xr[0], t["y"], 0.0, t["snp"], 0.0, t["qpt"]])
        trk_i.append([0, first, len(rr)])
        legs.append(t["leg"])
        names.append(t["name"])
    extra = g["extra_clusters"]
    for e in extra:
        ys.append(e["y"])
        zs.append(e["z"])
        rows.append(e["row"])
    cl = clusters(ys, zs, rows)
    return g, cl, np.array(trk_f, np.float32), np.array(trk_i), np.array(ids, np.uint32), \
        np.array(legs, np.uint8), names, own, extra


def test_hand_worked_cases():
    g, cl, tf, ti, ids, leg, names, own, extra = golden_case()
    mask, owner, amb = oracle.cluster_masks(cl, tf, ti, ids, leg, tube=g["tube"], min_pt=g["min_pt"],
                                            max_incl_deg=g["max_incl_deg"], bz=g["bz"])
    n_own = len(own)
    for c, (who, m) in enumerate(own):
        assert names[owner[c]] == who and mask[c] == m, (c, who, m, owner[c], mask[c])
        assert amb[c] == 0
    for k, e in enumerate(extra):
        c = n_own + k
        want = -1 if e["owner"] is None else names.index(e["owner"])
        assert (owner[c], mask[c], amb[c]) == (want, e["mask"], e["ambiguous"]), e["name"]


def circle_position(state, x_ref, X, bz):
    """Crossing of the plane x = X by the helix with state (y, z, sinphi,
    tanlambda, q/pT) at x_ref, from its circle's centre and radius and the
    turning angle (an independent route from the tracker's chord formula).
    None if the circle does not reach X on the outgoing half-turn."""
    y, z, s, t, qpt = (float(v) for v in state)
    kappa = KB * bz * qpt  # d(sinphi)/dx = -kappa
    c = math.sqrt(1.0 - s * s)
    s2 = s - kappa * (X - x_ref)
    if abs(s2) >= 0.9999:
        return None
    if kappa == 0.0:
        return y + (X - x_ref) * s / c, z + t * (X - x_ref) / c
    xc, yc = x_ref + s / kappa, y - c / kappa
    R = 1.0 / abs(kappa)
    Y = yc + math.copysign(math.sqrt(max(R * R - (X - xc) ** 2, 0.0)), kappa)
    a0 = math.atan2(y - yc, x_ref - xc)
    a1 = math.atan2(Y - yc, X - xc)
    da = (a1 - a0 + math.pi) % (2.0 * math.pi) - math.pi
    return Y, z + t * R * abs(da) * math.copysign(1.0, X - x_ref)


def brute_force(cl, tf, ti, ids, leg, tube, bz):
    """The paper's rules written out per cluster over every track of its item."""
    xr = row_x()
    mq, ms = oracle.mask_thresholds()
    n = cl.y.shape[0]
    cand = [[] for _ in range(n)]
    for t in range(tf.shape[0]):
        for j in range(ti[t, 2]):
            cand[ids[ti[t, 1] + j]].append(t)
    item_of = np.repeat(np.arange(cl.item_off.shape[0] - 1), np.diff(cl.item_off.astype(np.int64)))
    qy = np.rint(cl.y.astype(np.float64) * 1024) / 1024
    qz = np.rint(cl.z.astype(np.float64) * 1024) / 1024
    for t in range(tf.shape[0]):
        rr = cl.row[ids[ti[t, 1]:ti[t, 1] + ti[t, 2]]]
        lo, hi = rr.min(), rr.max()
        members = np.flatnonzero((item_of == ti[t, 0]) & (cl.row >= lo) & (cl.row <= hi))
        for r in range(lo, hi + 1):
            P = circle_position(tf[t, 1:], float(tf[t, 0]), xr[r], bz)
            if P is None:
                continue
            on = members[cl.row[members] == r]
            d = np.hypot(qy[on] - P[0], qz[on] - P[1])
            for c in on[d <= tube]:
                cand[c].append(t)
    mask = np.zeros(n, np.uint8)
    owner = np.full(n, -1, np.int32)
    for c in range(n):
        if not cand[c]:
            mask[c] = RB
            continue
        w = min(cand[c], key=lambda t: (abs(np.float32(tf[t, 5])), t))
        s = abs(float(tf[w, 3]) - KB * bz * float(tf[w, 5]) * (xr[cl.row[c]] - float(tf[w, 0])))
        prot = abs(tf[w, 5]) < mq and leg[w] == 0 and s < ms
        owner[c] = w
        mask[c] = A_ | P_ if prot else A_ | RA | RB
    return mask, owner


@pytest.fixture(scope="module")
def config1_tracks():
    from paper_1910_12214_b300 import synth
    cl = synth.make_config1(seed=2)
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.oracle_tracks(ref)
    return cl, tf, ti, ids


@pytest.mark.parametrize("tube", [1.5, 4.0])
def test_equals_brute_force_by_circle_geometry(config1_tracks, tube):
    cl, tf, ti, ids = config1_tracks
    leg = (np.arange(tf.shape[0]) % 5 == 3).astype(np.uint8)  # some tracks declared secondary legs
    mask, owner, amb = oracle.cluster_masks(cl, tf, ti, ids, leg, tube=tube)
    bm, bo = brute_force(cl, tf, ti, ids, leg, tube, 0.5)
    ok = amb == 0
    assert ok.mean() > 0.999
    assert np.array_equal(mask[ok], bm[ok])
    assert np.array_equal(owner[ok], bo[ok])
    # the mix is not degenerate: every outcome occurs
    for m in (A_ | P_, A_ | RA | RB, RB):
        assert (mask == m).sum() > 10, m


def test_strategy_relations_on_a_full_event():
    """Strategy B keeps a subset of what A keeps; protection implies
    association; A removes only associated, unprotected clusters; every track's
    own cluster is associated to it or to a track of higher pT."""
    from paper_1910_12214_b300 import synth
    cl = synth.make_config2(seed=3)
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.oracle_tracks(ref)
    mask, owner, amb = oracle.cluster_masks(cl, tf, ti, ids)
    keep_a, keep_b = (mask & RA) == 0, (mask & RB) == 0
    assert np.all(keep_a[keep_b])
    assert np.all((mask & A_)[(mask & P_) != 0])
    ra = (mask & RA) != 0
    assert np.all((mask & A_)[ra]) and not np.any((mask & P_)[ra])
    assert np.all((owner >= 0) == ((mask & A_) != 0))
    tr = np.repeat(np.arange(tf.shape[0]), ti[:, 2])
    w = owner[ids]
    assert np.all(w >= 0)
    assert np.all(np.abs(tf[w, 5]) <= np.abs(tf[tr, 5]))
    # a central event keeps most clusters under A and removes the unassociated noise under B
    assert keep_a.mean() > 0.9 and 0.0 < (~keep_b).mean() < 0.5


def test_no_tracks_and_zero_tube():
    from paper_1910_12214_b300 import synth
    cl = synth.make_config1(seed=4)
    mask, owner, _ = oracle.cluster_masks(cl, np.zeros((0, 6)), np.zeros((0, 3)), np.zeros(0, np.uint32))
    assert np.all(mask == RB) and np.all(owner == -1)
    # a zero tube leaves attachment alone: exactly the tracks' clusters are associated
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.oracle_tracks(ref)
    mask, owner, _ = oracle.cluster_masks(cl, tf, ti, ids, tube=0.0)
    assoc = np.zeros(cl.n, bool)
    assoc[ids] = True
    assert np.array_equal((mask & A_) != 0, assoc)
