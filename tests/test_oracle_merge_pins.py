"""Pins of the sector-track merger oracle: a hand-built split helix, the
refit on exact helices, MC-truth purity and efficiency of the links, and the
structure of links and groups."""
import math

import numpy as np
import pytest

import oracle
from test_oracle_masks_pins import row_x

KB = 0.299792458e-2 * 0.5
WEDGE = 2.0 * math.pi / 18.0


def local_state(xc, yc, R, q, k, X, tgl, z):
    """Track state (x_ref, y, z, sinphi, tanlambda, q/pT) in sector k's frame at
    local x = X on the circle of global centre (xc, yc) and radius R; the sign q
    of the curvature picks the branch (centre = (x + sinphi/kappa, y - cosphi/kappa))."""
    a = k * WEDGE
    lx, ly = xc * math.cos(a) + yc * math.sin(a), -xc * math.sin(a) + yc * math.cos(a)
    kap = q / (R * 1.0)  # kappa = kB q/pT = q / R
    s = (lx - X) * kap  # from x_c = x + s / kappa
    y = ly + math.sqrt(1.0 - s * s) / kap
    return [X, y, z, s, tgl, q / (R * KB), 1e-6]


def test_hand_built_split_helix_is_linked_and_a_bent_copy_is_not():
    """One helix from the beam axis (R = 150 cm, centre at azimuth 75 degrees,
    q = -1: it bends from sector 0 into sector 1) seen as a sector-0 piece at
    x = 100 cm and a sector-1 piece at x = 150 cm: the two states describe the
    same circle, so they link; the same pair with tan(lambda) 0.03 apart does
    not."""
    R, q, tgl = 150.0, -1.0, 0.2
    xc, yc = R * math.cos(math.radians(75.0)), R * math.sin(math.radians(75.0))
    s0 = local_state(xc, yc, R, q, 0, 100.0, tgl, 10.0)
    s1 = local_state(xc, yc, R, q, 1, 150.0, tgl, 0.0)
    assert abs(s0[1]) < 100.0 * math.tan(math.radians(10)) and abs(s1[1]) < 150.0 * math.tan(math.radians(10))
    # z of the second piece from the chord-series arc between the two reference points
    a1 = WEDGE
    P0 = np.array([s0[0], s0[1]])
    P1 = np.array([s1[0] * math.cos(a1) - s1[1] * math.sin(a1), s1[0] * math.sin(a1) + s1[1] * math.cos(a1)])
    c = float(np.hypot(*(P1 - P0)))
    s1[2] = 10.0 + tgl * c * (1 + c * c / (24 * R * R))
    assert abs(s0[3]) < 0.9 and abs(s1[3]) < 0.9

    def run(tf):
        cl = type("C", (), {})()
        n_rows = 152
        # each track needs clusters for the refit: put 3 on each track's reference row
        cl.y = np.array([s0[1]] * 3 + [s1[1]] * 3, np.float32)
        cl.z = np.array([s0[2]] * 3 + [s1[2]] * 3, np.float32)
        cl.row = np.array([0] * 6, np.int32)
        cl.item_sector = np.array([0, 1], np.uint32)
        cl.item_event = np.array([0, 0], np.uint32)
        ti = np.array([[0, 0, 3], [1, 3, 3]])
        return oracle.merge(cl, tf, ti, np.arange(6, dtype=np.uint32), n_rows=n_rows)

    tf = np.array([s0, s1], np.float32)
    link, group, amb, _ = run(tf)
    assert link[0].tolist() == [1, -1] and link[1].tolist() == [-1, 0]
    assert group.tolist() == [0, 0] and not amb.any()
    tf2 = tf.copy()
    tf2[1, 4] += 0.03
    link, group, _, _ = run(tf2)
    assert (link == -1).all() and group.tolist() == [0, 1]
    # curvatures 5 sigma apart (chi2 = 25 > 16; the sector-0 piece's circle, which the
    # continuity test uses, is unchanged): no link; 3 sigma apart (chi2 = 9): linked
    sig = math.sqrt(float(tf[0, 6]) + float(tf[1, 6]))
    for k, want in ((5.0, [-1, -1]), (3.0, [1, -1])):
        tf3 = tf.copy()
        tf3[1, 5] += np.float32(k * sig)
        link, _, _, _ = run(tf3)
        assert link[0].tolist() == want, k


def test_refit_recovers_exact_helices():
    """Noise-free helices of one full event: every refitted group (one track or
    several) gives the true radius and tan(lambda) of its MC particle."""
    from paper_1910_12214_b300 import synth
    cl = synth.make_config2(seed=21, n_tracks=600, sigma_y=0.0, sigma_z=0.0, noise_frac=0.0, pt_range=(0.3, 3.0))
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.merge_tracks(ref)
    link, group, amb, fit = oracle.merge(cl, tf, ti, ids)
    roots = np.unique(group)
    R_true = cl.tracks["pt"] / KB
    checked = 0
    for g in roots:
        members = np.flatnonzero(group == g)
        mc = cl.mc[np.concatenate([ids[ti[t, 1]:ti[t, 1] + ti[t, 2]] for t in members])]
        if (mc < 0).any() or np.unique(mc).size != 1:
            continue
        m = mc[0]
        # the clusters are quantised to 2^-10 cm by nothing here: exact float32 positions
        assert abs(fit[g, 2] - R_true[m]) < 2e-4 * R_true[m] + 0.05, (g, fit[g, 2], R_true[m])
        assert abs(fit[g, 3] - cl.tracks["tgl"][m]) < 2e-3
        # the centre of the circle through the vertex: q R (sin phi0, -cos phi0)
        q, ph = cl.tracks["q"][m], cl.tracks["phi0"][m]
        xc, yc = q * R_true[m] * math.sin(ph), -q * R_true[m] * math.cos(ph)
        assert math.hypot(fit[g, 0] - xc, fit[g, 1] - yc) < 2e-4 * R_true[m] + 0.05
        checked += 1
    assert checked > 500


@pytest.fixture(scope="module")
def event_merge():
    from paper_1910_12214_b300 import synth
    cl = synth.make_config2(seed=22)
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.merge_tracks(ref)
    link, group, amb, fit = oracle.merge(cl, tf, ti, ids)
    labels = np.array([np.bincount(cl.mc[ids[f:f + n]][cl.mc[ids[f:f + n]] >= 0]).argmax()
                       if (cl.mc[ids[f:f + n]] >= 0).any() else -1 for _, f, n in ti])
    return cl, tf, ti, ids, link, group, amb, fit, labels


def test_links_are_pure_and_split_tracks_are_merged(event_merge):
    cl, tf, ti, ids, link, group, amb, fit, labels = event_merge
    a, d = np.nonzero(link >= 0)
    b = link[a, d]
    assert a.size > 500
    assert (labels[a] == labels[b]).mean() > 0.995
    # MC particles found as two or more tracks in neighbouring sectors of one side: merged into one group
    sec = cl.item_sector[ti[:, 0]].astype(np.int64)
    split, merged = 0, 0
    for m in np.unique(labels[labels >= 0]):
        tr = np.flatnonzero(labels == m)
        if tr.size < 2:
            continue
        ks = sec[tr] % 18
        if sec[tr].max() // 18 != sec[tr].min() // 18:
            continue
        if not any(((ks[i] - ks[j]) % 18) in (1, 17) for i in range(tr.size) for j in range(tr.size)):
            continue
        split += 1
        merged += np.unique(group[tr]).size == 1
    assert split > 200
    assert merged / split > 0.95


def test_link_and_group_structure(event_merge):
    cl, tf, ti, ids, link, group, amb, fit, labels = event_merge
    sec = cl.item_sector[ti[:, 0]].astype(np.int64)
    for t in range(tf.shape[0]):
        for d in range(2):
            b = link[t, d]
            if b < 0:
                continue
            assert link[b, 1 - d] == t
            assert sec[b] // 18 == sec[t] // 18
            assert (sec[b] % 18 - sec[t] % 18) % 18 == (1 if d == 0 else 17)
            assert group[b] == group[t]
    for g in np.unique(group):
        members = np.flatnonzero(group == g)
        assert members.min() == g
        assert fit[g, 6] == members.size
        assert fit[g, 5] == ti[members, 2].sum()


def test_hand_built_looper_legs_are_paired():
    """One looper (R = 100 cm through the beam axis, centre at azimuth 60 deg):
    its outgoing leg seen in sector 1 and its returning leg in sector 5, the
    latter fitted in the reversed direction (opposite q/pT and tan lambda
    signs) and farther along the helix (larger |z|).  They pair, the returning
    one is the secondary leg; with tan lambda no longer opposite they do not."""
    R = 100.0
    xc, yc = R * math.cos(math.radians(60.0)), R * math.sin(math.radians(60.0))
    prim = local_state(xc, yc, R, -1.0, 1, 150.0, 0.3, 20.0)
    secd = local_state(xc, yc, R, 1.0, 5, 150.0, -0.3, 60.0)
    assert abs(prim[1]) < 150 * math.tan(math.radians(10)) and abs(secd[1]) < 150 * math.tan(math.radians(10))

    def run(tf):
        cl = type("C", (), {})()
        cl.y = np.array([prim[1]] * 3 + [secd[1]] * 3, np.float32)
        cl.z = np.array([prim[2]] * 3 + [secd[2]] * 3, np.float32)
        cl.row = np.array([60] * 6, np.int32)
        cl.item_sector = np.array([1, 5], np.uint32)
        cl.item_event = np.array([0, 0], np.uint32)
        ti = np.array([[0, 0, 3], [1, 3, 3]])
        return oracle.merge(cl, tf, ti, np.arange(6, dtype=np.uint32), legs=True)

    tf = np.array([prim, secd], np.float32)
    link, group, amb, fit, partner, leg = run(tf)
    assert partner.tolist() == [1, 0] and leg.tolist() == [0, 1] and not amb.any()
    assert (link == -1).all()  # sectors 1 and 5 are not neighbours: no sector link
    tf2 = tf.copy()
    tf2[1, 4] = -0.33
    *_, partner, leg = run(tf2)
    assert partner.tolist() == [-1, -1] and leg.tolist() == [0, 0]


def test_looper_legs_on_an_event_with_secondary_legs():
    """Helices that turn inside the chamber also leave their returning leg: the
    pairs found are the two legs of one particle (>= 97%), most particles whose
    two legs were both tracked get paired (>= 70%), and the secondary one is the
    returning leg (>= 99%)."""
    from paper_1910_12214_b300 import synth
    cl = synth.make_event(41, 6000, second_leg=True)
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids"])
    tf, ti, ids = oracle.merge_tracks(ref)
    link, group, amb, fit, partner, leg = oracle.merge(cl, tf, ti, ids, legs=True)
    lab = np.full(tf.shape[0], -1)
    true_leg = np.full(tf.shape[0], -1)
    for t, (_, f, n) in enumerate(ti):
        m, lg = cl.mc[ids[f:f + n]], cl.leg[ids[f:f + n]]
        if (m >= 0).any():
            lab[t] = np.bincount(m[m >= 0]).argmax()
            true_leg[t] = int(np.round(lg[m == lab[t]].mean()))
    p = np.flatnonzero(partner >= 0)
    assert np.all(partner[partner[p]] == p)
    assert np.all(leg[p] + leg[partner[p]] == 1)
    assert np.all(np.sign(tf[p, 5]) != np.sign(tf[partner[p], 5]))
    assert p.size > 1000
    assert (lab[p] == lab[partner[p]]).mean() > 0.97
    both = [m for m in np.unique(lab[true_leg == 1]) if ((lab == m) & (true_leg == 0)).any()]
    paired = np.mean([((lab == m) & (partner >= 0)).any() for m in both])
    assert len(both) > 500 and paired > 0.70
    assert (leg[p] == true_leg[p]).mean() > 0.99


def _looper_pieces(seed=43):
    """A noise-free event whose low-pT helices leave both legs; for one particle
    with both legs in two or more sectors each, its pieces per (leg, sector) as
    tracks: primary pieces first (one group), then the secondary pieces (another
    group), the first pieces of the two legs paired."""
    from paper_1910_12214_b300 import synth
    cl = synth.make_event(seed, 400, sigma_y=0.0, sigma_z=0.0, noise_frac=0.0, pt_range=(0.15, 0.35),
                          second_leg=True)
    item_of = np.repeat(np.arange(cl.n_items), np.diff(cl.item_off.astype(np.int64)))
    for m in range(cl.tracks["pt"].shape[0]):
        pieces = []
        for lg in (0, 1):
            sel = (cl.mc == m) & (cl.leg == lg)
            its = [it for it in np.unique(item_of[sel]) if ((item_of == it) & sel).sum() >= 10]
            pieces.append([np.flatnonzero(sel & (item_of == it)) for it in its])
        if len(pieces[0]) >= 2 and len(pieces[1]) >= 1:
            break
    ids, ti = [], []
    for lg in (0, 1):
        for p in pieces[lg]:
            ti.append([item_of[p[0]], len(ids), p.shape[0]])
            ids.extend(p.tolist())
    n0, n = len(pieces[0]), len(ti)
    tf = np.zeros((n, 7), np.float32)
    q, pt = cl.tracks["q"][m], cl.tracks["pt"][m]
    tf[:n0, 5] = q / pt       # primary pieces move outward with the particle's charge
    tf[n0:, 5] = -q / pt      # the returning leg is fitted in the reversed direction
    group = np.array([0] * n0 + [n0] * (n - n0), np.int32)
    partner = np.full(n, -1, np.int32)
    partner[0], partner[n0] = n0, 0
    leg = np.array([0] * n0 + [1] * (n - n0), np.uint8)
    return cl, m, tf, np.array(ti, np.int64), np.array(ids, np.uint32), group, partner, leg


def test_joined_looper_refit_recovers_the_helix():
    """The two legs of a noise-free looper, joined: one component labelled by
    its smallest track, and its refit (circle over both legs, z against the arc
    R dtheta turned from the primary leg's innermost cluster) gives the true
    radius, centre and tan(lambda), and z0 = z of that cluster."""
    cl, m, tf, ti, ids, group, partner, leg = _looper_pieces()
    joined, jfit, k = oracle.join_loopers(cl, tf, ti, ids, group, partner, leg)
    assert k == 1 and (joined == 0).all()
    R = cl.tracks["pt"][m] / KB
    q, ph = cl.tracks["q"][m], cl.tracks["phi0"][m]
    xc, yc = q * R * math.sin(ph), -q * R * math.cos(ph)
    f = jfit[0]
    assert abs(f[2] - R) < 1e-4 * R, (f[2], R)
    assert math.hypot(f[0] - xc, f[1] - yc) < 1e-4 * R
    assert abs(f[3] - cl.tracks["tgl"][m]) < 1e-4, (f[3], cl.tracks["tgl"][m])
    prim = ids[:ti[group == 0][:, 2].sum()]
    xr = row_x()
    gx, gy = [], []
    for t in range(ti.shape[0]):
        if group[t] != 0:
            continue
        a = (int(cl.item_sector[ti[t, 0]]) % 18) * WEDGE
        c = ids[ti[t, 1]:ti[t, 1] + ti[t, 2]]
        gx.extend(xr[cl.row[c]] * math.cos(a) - cl.y[c] * math.sin(a))
        gy.extend(xr[cl.row[c]] * math.sin(a) + cl.y[c] * math.cos(a))
    ref = prim[int(np.argmin(np.hypot(gx, gy)))]
    assert abs(f[4] - cl.z[ref]) < 1e-3, (f[4], cl.z[ref])
    assert f[5] == ids.shape[0] and f[6] == ti.shape[0]


def test_unpaired_groups_are_not_joined():
    cl, m, tf, ti, ids, group, partner, leg = _looper_pieces()
    joined, jfit, k = oracle.join_loopers(cl, tf, ti, ids, group, np.full_like(partner, -1), np.zeros_like(leg))
    assert k == 0 and np.array_equal(joined, group) and not jfit.any()
