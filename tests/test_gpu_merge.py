"""Parity of the CUDA sector-track merger with the oracle, through the C ABI:
with the same tracks (the oracle tracker's), identical links and groups except
tracks the oracle flags as rounding-sensitive, and the same refitted helices;
with the GPU's own tracks, the merger's structure and MC-truth quality.

The refit tolerance follows from the arithmetic.  The GPU sums in float-float
(48-bit significands: cluster positions to a few 1e-12 cm), the oracle in FP64.
A short, nearly straight group determines its circle's radius only through its
sagitta (ten clusters of a 10 GeV/c track: about 1e-3 cm), so its radius and
centre can differ by a few 1e-9 relative while the two circles agree along the
clusters.  The test therefore requires the two fitted circles to agree at every
cluster of the group to 1e-8 cm, and every refit parameter to 1e-6 relative."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def to_records(tf7, ti):
    from paper_1910_12214_b300 import tpc
    r = np.zeros(tf7.shape[0], dtype=tpc.TRACK_DTYPE)
    for k, name in enumerate(("x_ref", "y", "z", "snp", "tgl", "qpt")):
        r[name] = tf7[:, k]
    r["cov"][:, 14] = tf7[:, 6]
    r["item"], r["first_cluster"], r["n_clusters"] = ti[:, 0], ti[:, 1], ti[:, 2]
    return r


def circle_disagreement(cl, ti, ids, group, roots, fit, wf, n_rows=152, x_min=85.0, x_max=246.0):
    """Largest difference, over the clusters of the given groups, between their
    distances to the GPU's and to the oracle's refitted circle [cm]."""
    xr = np.rint((x_min + np.arange(n_rows) * ((x_max - x_min) / (n_rows - 1))) * 1024.0) / 1024.0
    is_root = np.zeros(group.shape[0], bool)
    is_root[roots] = True
    trk = np.flatnonzero(is_root[group])
    if trk.size == 0:
        return 0.0
    cnt = ti[trk, 2].astype(np.int64)
    owner = np.repeat(trk, cnt)
    pos = np.repeat(ti[trk, 1].astype(np.int64) - np.cumsum(cnt) + cnt, cnt) + np.arange(cnt.sum())
    c = ids[pos].astype(np.int64)
    ang = (cl.item_sector[ti[owner, 0]].astype(np.int64) % 18) * (2.0 * np.pi / 18.0)
    lx, ly = xr[cl.row[c]], cl.y[c].astype(np.float64)
    X, Y = lx * np.cos(ang) - ly * np.sin(ang), lx * np.sin(ang) + ly * np.cos(ang)
    g = group[owner]
    d_gpu = np.hypot(X - fit[g, 0], Y - fit[g, 1]) - fit[g, 2]
    d_orc = np.hypot(X - wf[g, 0], Y - wf[g, 1]) - wf[g, 2]
    return float(np.max(np.abs(d_gpu - d_orc)))


def tracked(cl):
    from paper_1910_12214_b300 import tpc
    t = tpc.Tracker(device=0)
    t.load(cl).track()
    t.sync()
    return t


def compare(cl, tf, ti, ids, link, group, fit):
    wl, wg, amb, wf = oracle.merge(cl, tf, ti, ids)
    bad = amb.astype(bool)
    # groups touched by a rounding-sensitive track are compared for validity only
    touched = np.zeros(tf.shape[0], bool)
    touched[np.isin(wg, wg[bad])] = True
    touched[np.isin(group, group[bad])] = True
    ok = ~touched
    assert ok.mean() > 0.99
    assert np.array_equal(link[ok], wl[ok])
    assert np.array_equal(group[ok], wg[ok])
    roots = np.flatnonzero(ok & (wg == np.arange(tf.shape[0])))
    assert np.allclose(fit[roots], wf[roots], rtol=1e-6, atol=1e-6)
    assert circle_disagreement(cl, ti, ids, group, roots, fit, wf) < 1e-8
    for t in np.flatnonzero(~ok):  # validity: mutual links
        for d in range(2):
            b = link[t, d]
            if b >= 0:
                assert link[b, 1 - d] == t


@pytest.mark.parametrize("cfg", ["c2", "c3"])
def test_oracle_tracks(cfg):
    from paper_1910_12214_b300 import synth
    cl = synth.make_config2(seed=31) if cfg == "c2" else synth.make_batched(seed=1)
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.merge_tracks(ref)
    with tracked(cl) as t:
        link, group, fit = t.merge_tracks(to_records(tf, ti), ids)
    compare(cl, tf, ti, ids, link, group, fit)


def test_own_tracks_product_path():
    from paper_1910_12214_b300 import synth
    cl = synth.make_config2(seed=32)
    with tracked(cl) as t:
        trk, tids = t.get_tracks()
        link, group, fit = t.merge_tracks()
    n = trk.shape[0]
    first = trk["first_cluster"].astype(np.int64)
    cnt = trk["n_clusters"].astype(np.int64)
    labels = np.array([np.bincount(cl.mc[tids[f:f + k]][cl.mc[tids[f:f + k]] >= 0]).argmax()
                       if (cl.mc[tids[f:f + k]] >= 0).any() else -1 for f, k in zip(first, cnt)])
    a, d = np.nonzero(link >= 0)
    b = link[a, d]
    assert a.size > 1000
    assert np.all(link[b, 1 - d] == a)
    assert (labels[a] == labels[b]).mean() > 0.995
    sec = trk["sector"].astype(np.int64)
    assert np.all(((sec[b] % 18 - sec[a] % 18) % 18) == np.where(d == 0, 1, 17))
    for g in np.unique(group):
        members = np.flatnonzero(group == g)
        assert members.min() == g
        if fit[g, 2] > 0:
            assert fit[g, 6] == members.size and fit[g, 5] == cnt[members].sum()
    # the merged groups' refitted radius against the MC particle's
    R_true = cl.tracks["pt"] / (0.299792458e-2 * 0.5)
    roots = np.unique(group[a])
    rel = np.abs(fit[roots, 2] - R_true[labels[roots]]) / R_true[labels[roots]]
    assert np.median(rel) < 0.01


def test_errors():
    from paper_1910_12214_b300 import synth, tpc
    cl = synth.make_config1(seed=33)
    t = tpc.Tracker(device=0)
    t.load(cl)
    with pytest.raises(tpc.TpcError) as e:
        t.merge_tracks()
    assert e.value.status == 2
    t.track()
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.merge_tracks(ref)
    rec = to_records(tf, ti)
    rec["item"][0] = 5  # out of range and out of order
    with pytest.raises(tpc.TpcError) as e:
        t.merge_tracks(rec, ids)
    assert e.value.status == 7
    t.close()
    # a batch without item tables cannot be merged
    cl2 = synth.make_config1(seed=34)
    cl2.item_sector = None
    cl2.item_event = None
    with tpc.Tracker(device=0) as t2:
        t2.load(cl2).track()
        with pytest.raises(tpc.TpcError) as e:
            t2.merge_tracks()
        assert e.value.status == 2


def test_looper_legs_oracle_tracks():
    """An event whose low-pT helices also leave their returning leg: with the
    oracle tracker's tracks the leg pairs and secondary flags equal the
    oracle's, except tracks it flags as rounding-sensitive."""
    from paper_1910_12214_b300 import synth
    cl = synth.make_event(41, 6000, second_leg=True)
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.merge_tracks(ref)
    wl, wg, amb, wf, wp, wleg = oracle.merge(cl, tf, ti, ids, legs=True)
    with tracked(cl) as t:
        link, group, fit, partner, leg = t.merge_tracks(to_records(tf, ti), ids, legs=True)
    touched = amb.astype(bool)
    touched |= (wp >= 0) & touched[np.maximum(wp, 0)]
    touched |= (partner >= 0) & touched[np.maximum(partner, 0)]
    ok = ~touched
    assert ok.mean() > 0.99 and (wp[ok] >= 0).sum() > 1000
    assert np.array_equal(partner[ok], wp[ok])
    assert np.array_equal(leg[ok], wleg[ok])
    compare(cl, tf, ti, ids, link, group, fit)


def test_secondary_legs_removed_by_strategy_a():
    """The chain the paper describes: the merger marks the returning legs of
    loopers, and strategy A removes their clusters (they are no longer
    protected), while the primary legs stay protected."""
    from paper_1910_12214_b300 import synth
    cl = synth.make_event(42, 6000, second_leg=True)
    with tracked(cl) as t:
        trk, tids = t.get_tracks()
        link, group, fit, partner, leg = t.merge_tracks(legs=True)
        m0, _ = t.cluster_masks(leg=None, n_tracks=trk.shape[0])
        m1, _ = t.cluster_masks(leg=leg, n_tracks=trk.shape[0])
    sec_cl = cl.leg == 1
    prim_cl = cl.leg == 0
    removed0 = (m0 & 4) != 0
    removed1 = (m1 & 4) != 0
    assert leg.sum() > 500
    # clusters of returning legs: strategy A removes many more of them once the legs are known
    assert removed1[sec_cl].mean() > removed0[sec_cl].mean() + 0.3
    # clusters of first legs: essentially untouched
    assert removed1[prim_cl].mean() < removed0[prim_cl].mean() + 0.02


def test_device_outputs_equal_host_outputs():
    """The same call with device inputs and outputs (the oracle tracker's tracks
    uploaded) and with host arrays: identical links, groups, refits and legs."""
    import torch
    from paper_1910_12214_b300 import synth
    cl = synth.make_event(42, 3000, second_leg=True)
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.merge_tracks(ref)
    rec = to_records(tf, ti)
    with tracked(cl) as t:
        host = t.merge_tracks(rec, ids, legs=True)
        d_rec = torch.from_numpy(rec.view(np.uint8).reshape(-1, rec.dtype.itemsize)).cuda()
        d_ids = torch.from_numpy(ids.view(np.int32)).cuda()
        dev = t.merge_tracks(d_rec, d_ids, legs=True, on_device=True)
        own_host = t.merge_tracks(legs=True)
        own_dev = t.merge_tracks(legs=True, on_device=True)
    for h, d in zip(host + own_host, dev + own_dev):
        assert np.array_equal(h, d.cpu().numpy(), equal_nan=True)
    assert (host[0] >= 0).sum() > 100 and (host[3] >= 0).sum() > 10


def test_sorted_lists_and_item_scans_agree():
    """The candidate search through the tan(lambda)-sorted lists, through the
    item-by-item scans (merge_sort_cap = -1) and through a mix of both (a cap
    between the sizes of the 64 uneven events' lists) gives the same links,
    groups, refits and looper legs bit for bit."""
    import torch
    from paper_1910_12214_b300 import synth
    cl = synth.make_batched(seed=3)
    with tracked(cl) as t:
        n = t.counts()[0]
        outs = []
        for cap in (16384, -1, 1200):
            t.set_tuning(merge_sort_cap=cap)
            assert t.get_tuning()["merge_sort_cap"] == cap
            outs.append([x.cpu().numpy() for x in t.merge_tracks(n_tracks=n, legs=True, on_device=True)])
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert np.array_equal(a, b, equal_nan=True)
    assert (outs[0][0] >= 0).sum() > 10000


def test_joined_loopers_equal_the_oracle_on_oracle_merger_outputs():
    """The joining step on its own: given the oracle merger's links, groups and
    leg pairs of the oracle tracker's tracks, the GPU joins the same groups
    (labels exact) and its FP64 refit of every joined looper equals the
    oracle's (centre, radius, tan(lambda), z0 within 1e-9 relative, counts
    exact)."""
    from paper_1910_12214_b300 import synth
    cl = synth.make_event(41, 6000, second_leg=True)
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.merge_tracks(ref)
    link, group, amb, fit, partner, leg = oracle.merge(cl, tf, ti, ids, legs=True)
    wj, wf, wk = oracle.join_loopers(cl, tf, ti, ids, group, partner, leg)
    with tracked(cl) as t:
        joined, jfit, k = t.join_loopers(link, group, partner, leg, tracks=to_records(tf, ti), ids=ids)
    assert k == wk and wk > 500
    assert np.array_equal(joined, wj)
    roots = np.flatnonzero(wf[:, 5] > 0)
    assert np.array_equal(np.flatnonzero(jfit[:, 5] > 0), roots)
    assert np.array_equal(jfit[roots, 5:], wf[roots, 5:])
    scale = np.maximum(np.abs(wf[roots, :5]), np.array([1.0, 1.0, 1.0, 1e-3, 1.0]))
    assert np.max(np.abs(jfit[roots, :5] - wf[roots, :5]) / scale) < 1e-9


def test_joined_loopers_of_own_tracks_recover_the_particles():
    """The product path: the GPU's own tracks, merged with looper legs and
    joined: the joined tracks are the two legs of one particle (>= 95%) and
    their refitted radius and tan(lambda) are the particle's (median error
    below 1% and 0.01)."""
    from paper_1910_12214_b300 import synth
    cl = synth.make_event(41, 6000, second_leg=True)
    with tracked(cl) as t:
        trk, ids = t.get_tracks()
        n = trk.shape[0]
        link, group, fit, partner, leg = t.merge_tracks(None, None, n, legs=True)
        joined, jfit, k = t.join_loopers(link, group, partner, leg, n_tracks=n)
        dl, dg, _, dp, dleg = t.merge_tracks(None, None, n, legs=True, on_device=True)
        dj, df, dk = t.join_loopers(dl, dg, dp, dleg, n_tracks=n, on_device=True)
    assert k > 500
    # device buffers give the host call's outputs (members are summed in index order)
    assert dk == k and np.array_equal(dj.cpu().numpy(), joined) and np.array_equal(df.cpu().numpy(), jfit)
    kb = 0.299792458e-2 * 0.5
    roots = np.flatnonzero(jfit[:, 5] > 0)
    pure, dR, dT = 0, [], []
    for r in roots:
        members = np.flatnonzero(joined == r)
        cs = np.concatenate([ids[trk["first_cluster"][u]:trk["first_cluster"][u] + trk["n_clusters"][u]]
                             for u in members])
        mc = cl.mc[cs]
        lab = np.bincount(mc[mc >= 0]).argmax()
        if (mc == lab).mean() >= 0.9 and (cl.leg[cs[mc == lab]] == 1).any() and (cl.leg[cs[mc == lab]] == 0).any():
            pure += 1
            R = cl.tracks["pt"][lab] / kb
            dR.append(abs(jfit[r, 2] - R) / R)
            dT.append(abs(jfit[r, 3] - cl.tracks["tgl"][lab]))
    assert pure >= 0.95 * roots.size, (pure, roots.size)
    assert np.median(dR) < 0.01 and np.median(dT) < 0.01, (np.median(dR), np.median(dT))
