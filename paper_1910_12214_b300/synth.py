"""Seeded synthetic TPC inputs: helices from the vertex, crossed with pad-row planes.

This module is shared test/bench infrastructure.  It holds none of the tracker's
arithmetic: crossings are computed from exact circle geometry (centre + radius),
not from the tracker's propagation formula, so that a fit of these clusters is
an independent check of the tracker's track model.

Workloads follow the collision environment the paper describes (central Pb-Pb
events, Sec. 1; 50 kHz continuous read-out with overlapping collisions and an
unknown vertex, Abstract and Sec. 1).  The paper measures on ALICE simulation,
which is not available; these synthetic helices stand in for it.

Geometry (a reading; the paper gives none): 18 azimuthal wedges of 20 degrees per
side, centred at k*20 deg; sectors 0-17 are the z>=0 side, 18-35 the z<0 side.
Pad rows are planes at sector-local x_r = x_min + r*(x_max-x_min)/(n_rows-1).
Local frame: x along the wedge centre, y = r*sin(phi - phi_k), z global.
Field Bz along +z; a positive track bends clockwise seen from +z.
Units: cm, GeV/c, T.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# GeV/c -> curvature: kappa[1/cm] = C_LIGHT * B[T] * q / pT   (c = 0.299792458 GeV/(T m))
C_LIGHT_CM = 0.299792458e-2


@dataclasses.dataclass
class Geometry:
    n_rows: int = 152
    x_min: float = 85.0
    x_max: float = 246.0
    half_angle_deg: float = 10.0
    bz_tesla: float = 0.5
    z_max: float = 250.0

    def row_x(self) -> np.ndarray:
        r = np.arange(self.n_rows, dtype=np.float64)
        return self.x_min + r * ((self.x_max - self.x_min) / (self.n_rows - 1))


@dataclasses.dataclass
class Clusters:
    """Cluster SoA grouped by work item (event, sector[, slice]) with CSR offsets."""
    x: np.ndarray            # float32 [n]
    y: np.ndarray            # float32 [n]
    z: np.ndarray            # float32 [n]
    row: np.ndarray          # int32   [n]
    item_off: np.ndarray     # uint64  [n_items + 1]
    item_sector: np.ndarray  # uint32  [n_items]
    item_event: np.ndarray   # uint32  [n_items]
    item_core: Optional[np.ndarray] = None  # int32 [n_items, 2]: slice core [lo, hi) in z quanta
    mc: Optional[np.ndarray] = None         # int32 [n]: MC track index, -1 = noise
    truth: Optional[np.ndarray] = None      # float64 [n, 5]: (y, z, sinphi, tanlambda, q/pT) at the row
    leg: Optional[np.ndarray] = None        # int8 [n]: helix leg of the cluster (0 first, 1 second), -1 noise
    tracks: Optional[dict] = None           # per MC track arrays
    n_physical: int = 0                     # clusters before slice duplication

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_items(self) -> int:
        return int(self.item_off.shape[0] - 1)


def splitmix64(x: int) -> int:
    """splitmix64 finaliser (Steele, Lea, Flood 2014) used to derive sub-stream seeds."""
    m = (1 << 64) - 1
    x = (x + 0x9E3779B97F4A7C15) & m
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def rng_for(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[splitmix64(seed) ^ stream, splitmix64(seed + 7919 * (stream + 1))]))


def draw_tracks(rng: np.random.Generator, n: int, pt_range=(0.1, 10.0), eta_max=0.9) -> dict:
    """pT log-uniform, eta uniform, q = +-1, phi0 uniform in [0, 2pi)."""
    lo, hi = math.log(pt_range[0]), math.log(pt_range[1])
    pt = np.exp(rng.uniform(lo, hi, n))
    eta = rng.uniform(-eta_max, eta_max, n)
    q = np.where(rng.uniform(0.0, 1.0, n) < 0.5, -1.0, 1.0)
    phi0 = rng.uniform(0.0, 2.0 * math.pi, n)
    return dict(pt=pt, tgl=np.sinh(eta), q=q, phi0=phi0, z0=np.zeros(n), t0=np.zeros(n))


def _crossings(tr: dict, geom: Geometry, single_sector: bool, chunk: int = 4096, second_leg: bool = False):
    """Exact first-leg crossings of each helix with every pad-row plane it meets.

    Returns per-crossing arrays: track index, sector, row, y_loc, z, sin(phi_loc)
    and the leg (0 first, 1 second).  A crossing is kept if the track moves outward
    in local x there (cos phi_loc > 0), |sin phi_loc| < 0.999, it lies on the first
    leg (arc length <= pi*R from the vertex), inside the wedge |y| <= x tan(half
    angle) and inside |z| <= z_max on the sector's side.  At most one crossing
    exists per (track, sector, row).  second_leg: also the crossings of the second
    half-turn (pi*R < arc length <= 2*pi*R), where a helix that turns inside the
    chamber comes back inward (cos phi_loc < 0): the looper's secondary leg.
    """
    kB = C_LIGHT_CM * geom.bz_tesla
    xr = geom.row_x()
    tan_h = math.tan(math.radians(geom.half_angle_deg))
    wedge = math.radians(2.0 * geom.half_angle_deg)
    n_side = int(round(2 * math.pi / wedge))
    out = []
    nt = tr["pt"].shape[0]
    for c0 in range(0, nt, chunk):
        sl = slice(c0, min(nt, c0 + chunk))
        pt, q, phi0, tgl, z0 = (tr[k][sl] for k in ("pt", "q", "phi0", "tgl", "z0"))
        R = pt / kB
        Xc = q * R * np.sin(phi0)
        Yc = -q * R * np.cos(phi0)
        T = pt.shape[0]
        if single_sector:
            cand = np.zeros((T, geom.n_rows, 1), dtype=np.int64)
        else:
            # azimuth of the track at radius x_r on its first leg picks the wedge; keep neighbours too
            ratio = np.minimum(xr[None, :] / (2.0 * R[:, None]), 1.0)
            phipos = phi0[:, None] - q[:, None] * np.arcsin(ratio)
            k0 = np.floor(phipos / wedge + 0.5).astype(np.int64)
            cand = (k0[:, :, None] + np.array([-1, 0, 1])[None, None, :]) % n_side
        alpha = cand * wedge
        ca, sa = np.cos(alpha), np.sin(alpha)
        xc = Xc[:, None, None] * ca + Yc[:, None, None] * sa
        yc = -Xc[:, None, None] * sa + Yc[:, None, None] * ca
        qR = (q * R)[:, None, None]
        s = (xc - xr[None, :, None]) / qR
        ok = np.abs(s) < 0.999
        s = np.where(ok, s, 0.0)
        phil = np.arcsin(s)
        ell = R[:, None, None] * np.mod(q[:, None, None] * (phi0[:, None, None] - alpha - phil), 2.0 * math.pi)
        ok &= (ell > 0.0) & (ell <= math.pi * R[:, None, None])
        y = yc + qR * np.sqrt(1.0 - s * s)
        ok &= np.abs(y) <= xr[None, :, None] * tan_h
        z = z0[:, None, None] + tgl[:, None, None] * ell
        ok &= np.abs(z) <= geom.z_max
        if not single_sector:
            side_c = z < 0.0
            sector = np.where(side_c, cand + n_side, cand)
        else:
            sector = cand
        ti, ri, ci = np.nonzero(ok)
        out.append((ti + c0, sector[ti, ri, ci], ri, y[ti, ri, ci], z[ti, ri, ci], s[ti, ri, ci],
                    np.zeros(ti.shape[0], np.int64)))
        if second_leg:
            # the inward branch of the second half-turn: at radius r the helix is at azimuth
            # phi0 - q (pi - asin(r / 2R)), moving in direction pi - phil (local), on the
            # other side of the centre
            if single_sector:
                cand2 = cand
            else:
                phipos2 = phi0[:, None] - q[:, None] * (math.pi - np.arcsin(ratio))
                k2 = np.floor(phipos2 / wedge + 0.5).astype(np.int64)
                cand2 = (k2[:, :, None] + np.array([-1, 0, 1])[None, None, :]) % n_side
            alpha2 = cand2 * wedge
            ca2, sa2 = np.cos(alpha2), np.sin(alpha2)
            xc2 = Xc[:, None, None] * ca2 + Yc[:, None, None] * sa2
            yc2 = -Xc[:, None, None] * sa2 + Yc[:, None, None] * ca2
            s2 = (xc2 - xr[None, :, None]) / qR
            ok2 = np.abs(s2) < 0.999
            s2 = np.where(ok2, s2, 0.0)
            phil2 = math.pi - np.arcsin(s2)
            ell2 = R[:, None, None] * np.mod(q[:, None, None] * (phi0[:, None, None] - alpha2 - phil2), 2.0 * math.pi)
            ok2 &= (ell2 > math.pi * R[:, None, None]) & (ell2 <= 2.0 * math.pi * R[:, None, None])
            y2 = yc2 - qR * np.sqrt(1.0 - s2 * s2)
            ok2 &= np.abs(y2) <= xr[None, :, None] * tan_h
            z2 = z0[:, None, None] + tgl[:, None, None] * ell2
            ok2 &= np.abs(z2) <= geom.z_max
            sector2 = cand2 if single_sector else np.where(z2 < 0.0, cand2 + n_side, cand2)
            t2, r2, c2 = np.nonzero(ok2)
            out.append((t2 + c0, sector2[t2, r2, c2], r2, y2[t2, r2, c2], z2[t2, r2, c2], s2[t2, r2, c2],
                        np.ones(t2.shape[0], np.int64)))
    cat = [np.concatenate([o[i] for o in out]) if out else np.zeros(0) for i in range(7)]
    return cat


def _noise(rng, n_noise, geom: Geometry, single_sector: bool, z_lo=None, z_hi=None):
    """Uniform noise: uniform sector and row, y uniform across the row, z uniform on the side."""
    xr = geom.row_x()
    tan_h = math.tan(math.radians(geom.half_angle_deg))
    n_sec = 1 if single_sector else int(round(360.0 / geom.half_angle_deg))
    sector = rng.integers(0, n_sec, n_noise)
    row = rng.integers(0, geom.n_rows, n_noise)
    y = rng.uniform(-1.0, 1.0, n_noise) * xr[row] * tan_h
    u = rng.uniform(0.0, 1.0, n_noise)
    if z_lo is not None:
        z = z_lo[sector] + u * (z_hi[sector] - z_lo[sector])
    elif single_sector:
        z = -geom.z_max + u * 2.0 * geom.z_max
    else:
        half = n_sec // 2
        z = np.where(sector < half, u * geom.z_max, -u * geom.z_max)
    return sector, row, y, z


def make_event(seed: int, n_tracks: int, *, geom: Geometry = None, single_sector: bool = False,
               sigma_y: float = 0.1, sigma_z: float = 0.1, noise_frac: float = 0.05,
               pt_range=(0.1, 10.0), eta_max: float = 0.9, event_id: int = 0,
               shuffle: bool = True, second_leg: bool = False) -> Clusters:
    """One collision at the origin (config-1 and config-2 shapes).

    single_sector: one 152-row wedge (sector 0) spanning both z sides; each helix's
    phi0 is chosen so that its azimuth at r_ref = min(165, (x_min + 2R)/2) is uniform
    over the wedge, so that low-pT helices still cross it.
    """
    geom = geom or Geometry()
    rng = rng_for(seed)
    tr = draw_tracks(rng, n_tracks, pt_range, eta_max)
    if single_sector:
        kB = C_LIGHT_CM * geom.bz_tesla
        R = tr["pt"] / kB
        r_ref = np.minimum(165.0, (geom.x_min + 2.0 * R) / 2.0)
        target = np.radians(rng.uniform(-geom.half_angle_deg, geom.half_angle_deg, n_tracks))
        tr["phi0"] = target + tr["q"] * np.arcsin(np.minimum(r_ref / (2.0 * R), 1.0))
    return _assemble([tr], [event_id], rng, geom, single_sector, sigma_y, sigma_z, noise_frac, shuffle,
                     second_leg=second_leg)


def _assemble(track_sets, event_ids, rng, geom, single_sector, sigma_y, sigma_z, noise_frac, shuffle,
              drift=None, second_leg=False):
    n_sec = 1 if single_sector else int(round(360.0 / geom.half_angle_deg))
    xs, ys, zs, rows, secs, evs, mcs, truths, legs = [], [], [], [], [], [], [], [], []
    base = 0
    all_tracks = {k: [] for k in ("pt", "tgl", "q", "phi0", "z0", "t0")}
    for tr, ev in zip(track_sets, event_ids):
        ti, sec, row, y, z, s, lg = _crossings(tr, geom, single_sector, second_leg=second_leg)
        ti = ti.astype(np.int64)
        lg = lg.astype(np.int64)
        row = row.astype(np.int64)
        sec = sec.astype(np.int64)
        n_sig = ti.shape[0]
        truth = np.stack([y, z, s, tr["tgl"][ti], tr["q"][ti] / tr["pt"][ti]], axis=1)
        ym = y + (rng.normal(0.0, sigma_y, n_sig) if sigma_y > 0 else 0.0)
        zm = z + (rng.normal(0.0, sigma_z, n_sig) if sigma_z > 0 else 0.0)
        if drift is not None:
            # continuous read-out: z' = z - side * v_d * t_collision (vertex time unknown to tracking)
            side = np.where(sec < n_sec // 2, 1.0, -1.0)
            shift = side * drift * tr["t0"][ti]
            zm = zm - shift
            truth[:, 1] -= shift
        n_noise = int(round(noise_frac * n_sig))
        if n_noise:
            z_lo = z_hi = None
            if drift is not None:
                t_ev = tr["t0"][0] if tr["t0"].shape[0] else 0.0
                z_lo = np.where(np.arange(n_sec) < n_sec // 2, -drift * t_ev, -geom.z_max + drift * t_ev)
                z_hi = np.where(np.arange(n_sec) < n_sec // 2, geom.z_max - drift * t_ev, drift * t_ev)
            nsec, nrow, ny, nz = _noise(rng, n_noise, geom, single_sector, z_lo, z_hi)
            sec = np.concatenate([sec, nsec])
            row = np.concatenate([row, nrow])
            ym = np.concatenate([ym, ny])
            zm = np.concatenate([zm, nz])
            truth = np.concatenate([truth, np.full((n_noise, 5), np.nan)])
            ti = np.concatenate([ti, np.full(n_noise, -1 - base)])
            lg = np.concatenate([lg, np.full(n_noise, -1)])
        xs.append(geom.row_x()[row])
        ys.append(ym)
        zs.append(zm)
        rows.append(row)
        secs.append(sec)
        evs.append(np.full(sec.shape[0], ev, dtype=np.int64))
        mcs.append(np.where(ti >= 0, ti + base, -1))
        truths.append(truth)
        legs.append(lg)
        for k in all_tracks:
            all_tracks[k].append(tr[k])
        base += tr["pt"].shape[0]
    x = np.concatenate(xs)
    y = np.concatenate(ys)
    z = np.concatenate(zs)
    row = np.concatenate(rows)
    sec = np.concatenate(secs)
    ev = np.concatenate(evs)
    mc = np.concatenate(mcs)
    truth = np.concatenate(truths)
    leg = np.concatenate(legs)
    # group by item = (event, sector); shuffle inside each item
    ev_ids = np.asarray(event_ids, dtype=np.int64)
    ev_rank = np.searchsorted(np.sort(ev_ids), ev)
    item = ev_rank * n_sec + sec
    key = rng.permutation(x.shape[0]) if shuffle else np.arange(x.shape[0])
    order = np.lexsort((key, item))
    n_items = len(event_ids) * n_sec
    counts = np.bincount(item, minlength=n_items)
    item_off = np.zeros(n_items + 1, dtype=np.uint64)
    item_off[1:] = np.cumsum(counts)
    sorted_ev = np.sort(ev_ids)
    return Clusters(
        x=x[order].astype(np.float32), y=y[order].astype(np.float32), z=z[order].astype(np.float32),
        row=row[order].astype(np.int32), item_off=item_off,
        item_sector=np.tile(np.arange(n_sec, dtype=np.uint32), len(event_ids)),
        item_event=np.repeat(sorted_ev.astype(np.uint32), n_sec),
        mc=mc[order].astype(np.int32), truth=truth[order], leg=leg[order].astype(np.int8),
        tracks={k: np.concatenate(v) for k, v in all_tracks.items()}, n_physical=int(x.shape[0]))


def make_config1(seed: int = 1, **kw) -> Clusters:
    """One sector, 200 helices, pT log-uniform 0.1-10 GeV, |eta| < 0.9, sigma 0.1 cm, 5% noise."""
    return make_event(seed, kw.pop("n_tracks", 200), single_sector=True, **kw)


def make_config2(seed: int = 1, **kw) -> Clusters:
    """Full TPC (36 sectors), one central Pb-Pb-like event of 6000 helices, 5% noise."""
    return make_event(seed, kw.pop("n_tracks", 6000), single_sector=False, **kw)


def make_batched(seed: int = 1, n_events: int = 64, mult=(50, 8000), geom: Geometry = None,
                 sigma: float = 0.1, noise_frac: float = 0.05) -> Clusters:
    """Many independent events of uneven multiplicity (log-uniform tracks per event)."""
    geom = geom or Geometry()
    rng = rng_for(seed, stream=1)
    lo, hi = math.log(mult[0]), math.log(mult[1])
    counts = np.rint(np.exp(rng.uniform(lo, hi, n_events))).astype(np.int64)
    sets = [draw_tracks(rng_for(seed + 1 + k), int(c)) for k, c in enumerate(counts)]
    return _assemble(sets, list(range(n_events)), rng, geom, False, sigma, sigma, noise_frac, True)


def make_timeframe(seed: int = 1, n_coll: int = 128, rate_khz: float = 50.0, mean_mult: float = 1500.0,
                   vz_sigma: float = 5.0, drift_cm_per_us: float = 2.58, geom: Geometry = None,
                   sigma: float = 0.1, noise_frac: float = 0.05) -> Clusters:
    """Continuous read-out frame: Poisson arrivals, exponential multiplicity, vertex z unknown.

    All collisions go into one frame (event id 0); cluster z carries the drift-time
    offset z' = z - side * v_d * t.  Items are whole sectors (36); see slice_frame().
    """
    geom = geom or Geometry()
    rng_t = rng_for(seed, stream=2)
    gaps = rng_t.exponential(1e3 / rate_khz, n_coll)  # microseconds
    t = np.cumsum(gaps) - gaps[0]
    mult = np.maximum(1, np.rint(rng_t.exponential(mean_mult, n_coll))).astype(np.int64)
    sets = []
    for k in range(n_coll):
        r = rng_for(seed + 1 + k, stream=3)
        tr = draw_tracks(r, int(mult[k]))
        tr["z0"] = r.normal(0.0, vz_sigma, int(mult[k]))
        tr["t0"] = np.full(int(mult[k]), t[k])
        sets.append(tr)
    rng = rng_for(seed, stream=4)
    # assemble each collision as its own "event" then merge into one frame
    cl = _assemble(sets, list(range(n_coll)), rng, geom, False, sigma, sigma, noise_frac, True,
                   drift=drift_cm_per_us)
    n_sec = 36
    sec = np.repeat(cl.item_sector, np.diff(cl.item_off).astype(np.int64))
    order = np.argsort(sec, kind="stable")
    counts = np.bincount(sec, minlength=n_sec)
    item_off = np.zeros(n_sec + 1, dtype=np.uint64)
    item_off[1:] = np.cumsum(counts)
    perm = rng.permutation(order.shape[0])
    order = order[np.lexsort((perm, sec[order]))]
    frame = Clusters(x=cl.x[order], y=cl.y[order], z=cl.z[order], row=cl.row[order], item_off=item_off,
                     item_sector=np.arange(n_sec, dtype=np.uint32), item_event=np.zeros(n_sec, np.uint32),
                     mc=cl.mc[order], truth=cl.truth[order], tracks=cl.tracks, n_physical=int(order.shape[0]))
    frame.tracks["t_coll"] = t
    return frame


def slice_frame(frame: Clusters, core_cm: float = 1000.0, overlap_cm: float = 300.0) -> Clusters:
    """Cut each sector's z' axis into slices: core of core_cm, plus overlap_cm on each side.

    A cluster is copied into every slice whose [core_lo - overlap, core_hi + overlap)
    contains it.  item_core holds the core range in z quanta (2^-10 cm); a track is
    reported by the slice whose core contains its innermost cluster.
    """
    Q = 1024.0
    xs, ys, zs, rows, mcs, truths, ids = [], [], [], [], [], [], []
    off = [0]
    secs, cores = [], []
    for s in range(frame.n_items):
        a, b = int(frame.item_off[s]), int(frame.item_off[s + 1])
        if b == a:
            continue
        z = frame.z[a:b].astype(np.float64)
        lo = math.floor(z.min() / core_cm) * core_cm
        hi = z.max()
        c = lo
        while c <= hi:
            m = (z >= c - overlap_cm) & (z < c + core_cm + overlap_cm)
            idx = np.nonzero(m)[0] + a
            xs.append(frame.x[idx]); ys.append(frame.y[idx]); zs.append(frame.z[idx])
            rows.append(frame.row[idx]); mcs.append(frame.mc[idx]); truths.append(frame.truth[idx])
            ids.append(idx)
            off.append(off[-1] + idx.shape[0])
            secs.append(frame.item_sector[s])
            cores.append((int(round(c * Q)), int(round((c + core_cm) * Q))))
            c += core_cm
    out = Clusters(x=np.concatenate(xs), y=np.concatenate(ys), z=np.concatenate(zs), row=np.concatenate(rows),
                   item_off=np.asarray(off, dtype=np.uint64), item_sector=np.asarray(secs, dtype=np.uint32),
                   item_event=np.zeros(len(secs), np.uint32), item_core=np.asarray(cores, dtype=np.int32),
                   mc=np.concatenate(mcs), truth=np.concatenate(truths), tracks=frame.tracks,
                   n_physical=frame.n_physical)
    out.src_index = np.concatenate(ids)
    return out


# ---------------------------------------------------------------- distortions
@dataclasses.dataclass
class Distortion:
    """Per-sector smooth space-charge distortion of the measured (y, z).

    d_s(x, y, z) = sum_k A_k exp(-|p - c_k|^2 / (2 w_k^2)), k < 32, with (y, z)
    components (the pad row fixes x, so a radial shift is not measurable on it);
    centres uniform in the sector volume, widths uniform in [30, 80] cm,
    amplitudes in the unit disc, the field rescaled so that max |d| = max_d on a
    probe grid.  Measured = true + d(true).
    """
    centres: np.ndarray   # [S, K, 3]
    widths: np.ndarray    # [S, K]
    amps: np.ndarray      # [S, K, 2]
    z_side: np.ndarray    # [S] +1 (z >= 0) or -1; 0 = both sides (single-sector config)
    geom: Geometry

    def field(self, s: int, x, y, z):
        c, w, a = self.centres[s], self.widths[s], self.amps[s]
        d2 = ((x[..., None] - c[:, 0]) ** 2 + (y[..., None] - c[:, 1]) ** 2 + (z[..., None] - c[:, 2]) ** 2)
        g = np.exp(-d2 / (2.0 * w ** 2))
        return g @ a[:, 0], g @ a[:, 1]

    def field_jac(self, s: int, x, y, z):
        """Field and its derivatives d(dy, dz)/d(y, z)."""
        c, w, a = self.centres[s], self.widths[s], self.amps[s]
        ry, rz = y[..., None] - c[:, 1], z[..., None] - c[:, 2]
        g = np.exp(-((x[..., None] - c[:, 0]) ** 2 + ry * ry + rz * rz) / (2.0 * w ** 2))
        gy, gz = -g * ry / w ** 2, -g * rz / w ** 2
        return g @ a[:, 0], g @ a[:, 1], gy @ a[:, 0], gz @ a[:, 0], gy @ a[:, 1], gz @ a[:, 1]

    def invert(self, s: int, x, ym, zm, tol: float = 1e-10, max_iter: int = 50):
        """True (y, z) with measured = true + d(true): Newton's method on the 2x2
        system (the field gradient is well below 1, so the root is unique)."""
        yt, zt = np.array(ym, np.float64, copy=True), np.array(zm, np.float64, copy=True)
        for _ in range(max_iter):
            dy, dz, dyy, dyz, dzy, dzz = self.field_jac(s, x, yt, zt)
            fy, fz = yt + dy - ym, zt + dz - zm
            a11, a12, a21, a22 = 1.0 + dyy, dyz, dzy, 1.0 + dzz
            det = a11 * a22 - a12 * a21
            sy = (a22 * fy - a12 * fz) / det
            sz = (a11 * fz - a21 * fy) / det
            yt -= sy
            zt -= sz
            if max(np.abs(sy).max(initial=0.0), np.abs(sz).max(initial=0.0)) < tol:
                break
        return yt, zt

    def z_range(self, s: int):
        zm = self.geom.z_max
        return {1: (0.0, zm), -1: (-zm, 0.0), 0: (-zm, zm)}[int(self.z_side[s])]


def make_distortion(seed: int = 1, n_sectors: int = 36, n_gauss: int = 32, max_d: float = 10.0,
                    geom: Geometry = None, single_sector: bool = False) -> Distortion:
    geom = geom or Geometry()
    rng = rng_for(seed, stream=5)
    tan_h = math.tan(math.radians(geom.half_angle_deg))
    side = np.zeros(n_sectors) if single_sector else np.where(np.arange(n_sectors) < n_sectors // 2, 1.0, -1.0)
    cen = np.zeros((n_sectors, n_gauss, 3))
    wid = rng.uniform(30.0, 80.0, (n_sectors, n_gauss))
    amp = np.zeros((n_sectors, n_gauss, 2))
    for s in range(n_sectors):
        x = rng.uniform(geom.x_min, geom.x_max, n_gauss)
        cen[s, :, 0] = x
        cen[s, :, 1] = rng.uniform(-1.0, 1.0, n_gauss) * x * tan_h
        lo, hi = {1: (0.0, geom.z_max), -1: (-geom.z_max, 0.0), 0: (-geom.z_max, geom.z_max)}[int(side[s])]
        cen[s, :, 2] = rng.uniform(lo, hi, n_gauss)
        r = np.sqrt(rng.uniform(0.0, 1.0, n_gauss))
        ph = rng.uniform(0.0, 2.0 * math.pi, n_gauss)
        amp[s, :, 0] = r * np.cos(ph)
        amp[s, :, 1] = r * np.sin(ph)
    d = Distortion(cen, wid, amp, side, geom)
    # rescale each sector so that max |d| = max_d over a probe grid of its volume
    for s in range(n_sectors):
        lo, hi = d.z_range(s)
        xs = np.linspace(geom.x_min, geom.x_max, 24)
        vs = np.linspace(-1.0, 1.0, 24)
        zs = np.linspace(lo, hi, 48)
        X, V, Z = np.meshgrid(xs, vs, zs, indexing="ij")
        dy, dz = d.field(s, X, V * X * tan_h, Z)
        m = max(np.abs(dy).max(), np.abs(dz).max())
        d.amps[s] *= max_d / m
    return d


def distort(cl: Clusters, dist: Distortion) -> Clusters:
    """Measured clusters: y, z shifted by the field at the true position (x, row kept)."""
    out = dataclasses.replace(cl)
    y = cl.y.astype(np.float64).copy()
    z = cl.z.astype(np.float64).copy()
    x = cl.x.astype(np.float64)
    sec = np.repeat(cl.item_sector.astype(np.int64), np.diff(cl.item_off.astype(np.int64)))
    for s in np.unique(sec):
        m = sec == s
        dy, dz = dist.field(int(s), x[m], y[m], z[m])
        y[m] += dy
        z[m] += dz
    out.y = y.astype(np.float32)
    out.z = z.astype(np.float32)
    return out


def correction_grid(dist: Distortion, n: int = 64, margin: float = 12.0, tol: float = 1e-9):
    """Per sector n^3 grid over the distorted volume (x, v = y / (x tan), z) with
    margins; node value = (0, dy, dz) such that true = measured + value, found by
    Newton's method on measured = true + d(true) to tol (FP64).
    Returns grid float32 [S, n, n, n, 3] (axes x, v, z) and bounds float32
    [S, 6] = (x0, x1, v0, v1, z0, z1)."""
    g = dist.geom
    tan_h = math.tan(math.radians(g.half_angle_deg))
    S = dist.centres.shape[0]
    grid = np.zeros((S, n, n, n, 3), np.float32)
    bounds = np.zeros((S, 6), np.float32)
    for s in range(S):
        lo, hi = dist.z_range(s)
        x0, x1 = g.x_min - margin, g.x_max + margin
        v0, v1 = -1.3, 1.3
        z0, z1 = lo - margin, hi + margin
        bounds[s] = (x0, x1, v0, v1, z0, z1)
        X, V, Z = np.meshgrid(np.linspace(x0, x1, n), np.linspace(v0, v1, n), np.linspace(z0, z1, n), indexing="ij")
        ym = V * X * tan_h
        yt, zt = dist.invert(s, X, ym, Z, tol=tol)
        grid[s, ..., 1] = (yt - ym).astype(np.float32)
        grid[s, ..., 2] = (zt - Z).astype(np.float32)
    return grid, bounds


def exact_correction(dist: Distortion, sector: int, x, ym, zm, tol: float = 1e-10):
    """True (y, z) of measured points (FP64 inversion of the field)."""
    return dist.invert(sector, np.asarray(x, np.float64), np.asarray(ym, np.float64), np.asarray(zm, np.float64), tol)


def cluster_props(cl: Clusters, seed: int = 1, geom: Geometry = None) -> dict:
    """Charge and size of every cluster, for the cluster codec (float32 arrays).

    Shapes follow a TPC's physics (a reading; the paper gives no distributions):
    q_tot [ADC counts] is a Moyal (Landau-like) energy loss, MPV 60 with a
    scale of 12, times the path length through the pad row (1 / (cos phi * cos
    lambda)); q_max is 25-45 % of q_tot and saturates at the 10-bit ADC limit
    1023; sigma_y and sigma_z [cm] grow with the drift length L = z_max - |z|
    (diffusion 0.021 cm/sqrt(cm)) on top of an intrinsic 0.06 cm, and with the
    track's crossing angles, with 10 % log-normal spread.  Noise clusters
    (no truth) take phi = lambda = 0.  A Moyal variate is -ln(Z^2), Z ~ N(0,1).
    Also returns y, z, row of the clusters, so that the dict is a codec input.
    """
    geom = geom or Geometry()
    rng = rng_for(seed, stream=7)
    n = cl.n
    snp = np.zeros(n)
    tgl = np.zeros(n)
    if cl.truth is not None:
        ok = np.isfinite(cl.truth[:, 2])
        snp[ok] = np.clip(cl.truth[ok, 2], -0.99, 0.99)
        tgl[ok] = cl.truth[ok, 3]
    cos_phi = np.sqrt(1.0 - snp * snp)
    path = np.sqrt(1.0 + tgl * tgl) / cos_phi
    zeta = rng.standard_normal(n)
    moyal = -np.log(np.maximum(zeta * zeta, 1e-300))
    q_tot = np.maximum(60.0 + 12.0 * moyal, 5.0) * path
    q_max = np.minimum(q_tot * rng.uniform(0.25, 0.45, n), 1023.0)
    drift = np.clip(geom.z_max - np.abs(cl.z.astype(np.float64)), 0.0, None)
    diff2 = 0.021 ** 2 * drift
    tan_phi = snp / cos_phi
    sy = np.sqrt(0.06 ** 2 + diff2 + (0.2 * tan_phi) ** 2) * np.exp(0.1 * rng.standard_normal(n))
    sz = np.sqrt(0.06 ** 2 + diff2 + (0.2 * tgl) ** 2) * np.exp(0.1 * rng.standard_normal(n))
    return {"y": cl.y, "z": cl.z, "row": cl.row, "q_tot": q_tot.astype(np.float32),
            "q_max": q_max.astype(np.float32), "sigma_y": sy.astype(np.float32), "sigma_z": sz.astype(np.float32)}
