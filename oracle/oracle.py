"""ctypes binding of liboracle.so (FP64 CPU oracle, test infrastructure only)."""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SRC = [os.path.join(HERE, f) for f in ("tpc_oracle.cpp", "corr_oracle.cpp", "mlp_oracle.cpp", "codec_oracle.cpp",
                                                        "masks_oracle.cpp", "entropy_oracle.cpp",
                                                        "merge_oracle.cpp")
       if os.path.exists(os.path.join(HERE, f))]


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, no fast-math) if missing or stale."""
    deps = SRC + [os.path.join(HERE, "tpc_oracle.h")]
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in deps):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
           "-o", tmp] + SRC
    subprocess.check_call(cmd, cwd=HERE)
    os.replace(tmp, LIB)
    return LIB


class _Cfg(C.Structure):
    _fields_ = [("n_rows", C.c_int), ("x_min", C.c_double), ("x_max", C.c_double),
                ("half_angle_deg", C.c_double), ("bz_tesla", C.c_double),
                ("sigma_y", C.c_double), ("sigma_z", C.c_double), ("brute", C.c_int)]


@dataclasses.dataclass
class OracleConfig:
    n_rows: int = 152
    x_min: float = 85.0
    x_max: float = 246.0
    half_angle_deg: float = 10.0
    bz_tesla: float = 0.5
    sigma_y: float = 0.1
    sigma_z: float = 0.1
    brute: bool = False


_lib = None


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        lib = C.CDLL(LIB)
        lib.orc_run.restype = C.c_int
        lib.orc_run.argtypes = [C.POINTER(_Cfg), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64,
                                C.c_void_p, C.c_uint32, C.c_void_p, C.POINTER(C.c_void_p)]
        lib.orc_free.argtypes = [C.c_void_p]
        lib.orc_get.restype = C.c_int64
        lib.orc_get.argtypes = [C.c_void_p, C.c_char_p, C.c_void_p, C.c_int64]
        lib.orc_propagate.restype = C.c_int
        lib.orc_propagate.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_void_p, C.c_void_p]
        lib.orc_fit_hits.restype = C.c_int
        lib.orc_fit_hits.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_double, C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.orc_trilinear.restype = None
        lib.orc_trilinear.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        if hasattr(lib, "orc_mlp_forward"):
            lib.orc_counter_uniform.restype = C.c_double
            lib.orc_counter_uniform.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64]
            lib.orc_bf16.restype = C.c_float
            lib.orc_bf16.argtypes = [C.c_float]
            lib.orc_mlp_forward.restype = None
            lib.orc_mlp_forward.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]
            lib.orc_mlp_grad.restype = C.c_double
            lib.orc_mlp_grad.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
            lib.orc_adam.restype = None
            lib.orc_adam.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                     C.c_double, C.c_double, C.c_double, C.c_double]
            lib.orc_mlp_init.restype = None
            lib.orc_mlp_init.argtypes = [C.c_uint64, C.c_int, C.c_void_p]
            lib.orc_mlp_batch.restype = None
            lib.orc_mlp_batch.argtypes = [C.c_uint64, C.c_int, C.c_uint64, C.c_int, C.c_void_p, C.c_int, C.c_int,
                                          C.c_int, C.c_void_p, C.c_void_p]
        lib.orc_dyn_round.restype = C.c_uint32
        lib.orc_dyn_round.argtypes = [C.c_uint32, C.c_int, C.c_int]
        lib.orc_encode_clusters.restype = C.c_int64
        lib.orc_encode_clusters.argtypes = [C.c_int64, C.c_int] + [C.c_void_p] * 14
        lib.orc_cluster_masks.restype = C.c_int64
        lib.orc_cluster_masks.argtypes = ([C.c_int, C.c_double, C.c_double, C.c_double, C.c_int64] + [C.c_void_p] * 4 +
                                          [C.c_int64, C.c_int64] + [C.c_void_p] * 4 + [C.c_double, C.c_float,
                                                                                     C.c_float] + [C.c_void_p] * 3)
        lib.orc_compress.restype = C.c_int64
        lib.orc_compress.argtypes = ([C.c_int, C.c_double, C.c_double, C.c_float, C.c_int64] + [C.c_void_p] * 7 +
                                     [C.c_int64, C.c_void_p, C.c_void_p, C.c_int64] + [C.c_void_p] * 5 + [C.c_int64])
        lib.orc_decompress.restype = C.c_int64
        lib.orc_decompress.argtypes = [C.c_void_p, C.c_int64, C.c_int64] + [C.c_void_p] * 9
        lib.orc_code_stream.restype = C.c_int64
        lib.orc_code_stream.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64]
        lib.orc_decode_stream.restype = C.c_int64
        lib.orc_decode_stream.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64]
        lib.orc_predict.restype = None
        lib.orc_predict.argtypes = [C.c_void_p, C.c_float, C.c_float, C.c_void_p, C.c_void_p]
        lib.orc_merge.restype = C.c_int64
        lib.orc_merge.argtypes = ([C.c_int, C.c_double, C.c_double, C.c_double, C.c_int64] + [C.c_void_p] * 3 +
                                  [C.c_int64, C.c_void_p, C.c_void_p, C.c_int64] + [C.c_void_p] * 9)
        lib.orc_join_loopers.restype = C.c_int64
        lib.orc_join_loopers.argtypes = ([C.c_int, C.c_double, C.c_double, C.c_double, C.c_int64] + [C.c_void_p] * 3 +
                                         [C.c_int64, C.c_void_p, C.c_int64] + [C.c_void_p] * 8)
        lib.orc_chi2.restype = C.c_double
        lib.orc_chi2.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double]
        _lib = lib
    return _lib


_DT = {"sorted_qy": np.int32, "sorted_qz": np.int32, "sorted_id": np.int32, "rows": np.int32,
       "first": np.int32, "up_raw": np.int32, "dn_raw": np.int32, "up": np.int32, "dn": np.int32,
       "starts": np.int32, "trk_f": np.float64, "trk_i": np.int64, "trk_ids": np.int32,
       "tl_n": np.int32, "tl_hits": np.int32, "tl_meta": np.int32}


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def run(cl, cfg: OracleConfig = None, what=None) -> dict:
    """Run every step on a synth.Clusters-like object; returns the requested arrays."""
    lib = _load()
    cfg = cfg or OracleConfig()
    c = _Cfg(cfg.n_rows, cfg.x_min, cfg.x_max, cfg.half_angle_deg, cfg.bz_tesla, cfg.sigma_y, cfg.sigma_z,
             int(cfg.brute))
    x = np.ascontiguousarray(cl.x, np.float32)
    y = np.ascontiguousarray(cl.y, np.float32)
    z = np.ascontiguousarray(cl.z, np.float32)
    row = np.ascontiguousarray(cl.row, np.int32)
    off = np.ascontiguousarray(cl.item_off, np.uint64)
    core = None if getattr(cl, "item_core", None) is None else np.ascontiguousarray(cl.item_core, np.int32)
    h = C.c_void_p()
    st = lib.orc_run(C.byref(c), _p(x), _p(y), _p(z), _p(row), x.shape[0], _p(off), off.shape[0] - 1,
                     _p(core), C.byref(h))
    if st != 0:
        raise ValueError(f"oracle rejected the input (status {st})")
    out = {"status": st}
    try:
        for k in (what or _DT.keys()):
            n = lib.orc_get(h, k.encode(), None, 0)
            a = np.empty(n, dtype=_DT[k])
            lib.orc_get(h, k.encode(), _p(a), n)
            out[k] = a
    finally:
        lib.orc_free(h)
    if "trk_f" in out:
        out["trk_f"] = out["trk_f"].reshape(-1, 24)
    if "trk_i" in out:
        out["trk_i"] = out["trk_i"].reshape(-1, 4)
    if "tl_meta" in out:
        out["tl_meta"] = out["tl_meta"].reshape(-1, 2)
    if "rows" in out:
        out["rows"] = out["rows"].reshape(-1, 7)
    return out


def propagate(p, x1, x2, bz=0.5):
    lib = _load()
    p = np.ascontiguousarray(p, np.float64)
    q = np.empty(5)
    F = np.empty((5, 5))
    ok = lib.orc_propagate(_p(p), x1, x2, bz, _p(q), _p(F))
    return (q, F) if ok else None


def fit_hits(x, y, z, p0, C0, sigma_y=0.1, sigma_z=0.1, bz=0.5):
    lib = _load()
    x, y, z = (np.ascontiguousarray(a, np.float64) for a in (x, y, z))
    p0 = np.ascontiguousarray(p0, np.float64)
    C0 = np.ascontiguousarray(C0, np.float64)
    p = np.empty(5)
    Cm = np.empty((5, 5))
    chi2 = np.empty(1)
    ok = lib.orc_fit_hits(x.shape[0], _p(x), _p(y), _p(z), _p(p0), _p(C0), sigma_y, sigma_z, bz, _p(p), _p(Cm),
                          _p(chi2))
    return (p, Cm, float(chi2[0])) if ok else None


def chi2(p, Cm, my, mz, vy=0.01, vz=0.01):
    lib = _load()
    p = np.ascontiguousarray(p, np.float64)
    Cm = np.ascontiguousarray(Cm, np.float64)
    return float(lib.orc_chi2(_p(p), _p(Cm), my, mz, vy, vz))


def trilinear(grid, bounds, sector, x, y, z, tan_half=None):
    """(dy, dz) of the per-sector grid at points (x = pad-row radius), FP64."""
    import math
    lib = _load()
    tan_half = math.tan(math.radians(10.0)) if tan_half is None else tan_half
    grid = np.ascontiguousarray(grid, np.float32)
    bounds = np.ascontiguousarray(bounds, np.float32)
    S, nx, ny, nz, _ = grid.shape
    sector = np.ascontiguousarray(sector, np.int32)
    x, y, z = (np.ascontiguousarray(a, np.float64) for a in (x, y, z))
    n = x.shape[0]
    dy, dz = np.empty(n), np.empty(n)
    lib.orc_trilinear(_p(grid), _p(bounds), nx, ny, nz, tan_half, n, _p(sector), _p(x), _p(y), _p(z), _p(dy), _p(dz))
    return dy, dz


def correct_clusters(cl, grid, bounds, n_rows=152, x_min=85.0, x_max=246.0):
    """Corrected cluster y, z (float32) with the grid read at the quantised pad-row x."""
    xr = np.rint((x_min + np.arange(n_rows) * ((x_max - x_min) / (n_rows - 1))) * 1024.0) / 1024.0
    sec = np.repeat(cl.item_sector.astype(np.int64), np.diff(cl.item_off.astype(np.int64)))
    x = xr[cl.row]
    y = cl.y.astype(np.float64)
    z = cl.z.astype(np.float64)
    dy, dz = trilinear(grid, bounds, sec, x, y, z)
    return (y + dy).astype(np.float32), (z + dz).astype(np.float32)


MLP_NP = 4611


def counter_uniform(seed, a, b, k):
    return _load().orc_counter_uniform(seed, a, b, k)


def mlp_forward(P, inputs, exact=False):
    lib = _load()
    P = np.ascontiguousarray(P, np.float32)
    x = np.ascontiguousarray(inputs, np.float64).reshape(-1, 3)
    out = np.empty_like(x)
    lib.orc_mlp_forward(_p(P), x.shape[0], _p(x), int(exact), _p(out))
    return out


def mlp_grad(P, inputs, targets, exact=False):
    lib = _load()
    P = np.ascontiguousarray(P, np.float32)
    x = np.ascontiguousarray(inputs, np.float64).reshape(-1, 3)
    t = np.ascontiguousarray(targets, np.float64).reshape(-1, 3)
    g = np.empty(MLP_NP)
    loss = lib.orc_mlp_grad(_p(P), x.shape[0], _p(x), _p(t), int(exact), _p(g))
    return g, loss


def adam(w, m, v, g, t, T, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    lib = _load()
    w, m, v = (np.ascontiguousarray(a, np.float64).copy() for a in (w, m, v))
    g = np.ascontiguousarray(g, np.float64)
    lib.orc_adam(_p(w), _p(m), _p(v), _p(g), w.shape[0], t, T, lr, b1, b2, eps)
    return w, m, v


def mlp_init(seed, sector):
    P = np.empty(MLP_NP, np.float32)
    _load().orc_mlp_init(seed, sector, _p(P))
    return P


def mlp_batch(seed, sector, step, n, grid_sector):
    g = np.ascontiguousarray(grid_sector, np.float32)
    nx, ny, nz, _ = g.shape
    x, t = np.empty((n, 3)), np.empty((n, 3))
    _load().orc_mlp_batch(seed, sector, step, n, _p(g), nx, ny, nz, _p(x), _p(t))
    return x, t


def bf16(v):
    return _load().orc_bf16(float(v))


CODE_FIELDS = (("y", np.int16), ("z", np.int32), ("row", np.uint8), ("q_tot", np.uint16), ("q_max", np.uint16),
               ("sigma_y", np.uint8), ("sigma_z", np.uint8))


def dyn_round(v, n, width):
    """Dynamic precision of one non-negative integer (n bits after the leading one)."""
    return int(_load().orc_dyn_round(int(v), int(n), int(width)))


def encode_clusters(props, n_rows=152):
    """Integer codes of cluster properties (dict of y, z, row, q_tot, q_max, sigma_y,
    sigma_z arrays); returns (dict of code arrays, number of bad clusters)."""
    lib = _load()
    src = [np.ascontiguousarray(props[k], np.int32 if k == "row" else np.float32)
           for k in ("y", "z", "row", "q_tot", "q_max", "sigma_y", "sigma_z")]
    n = src[0].shape[0]
    out = {k: np.empty(n, dt) for k, dt in CODE_FIELDS}
    bad = lib.orc_encode_clusters(n, n_rows, *[_p(a) for a in src], *[_p(out[k]) for k, _ in CODE_FIELDS])
    return out, int(bad)


MASK_ASSOCIATED, MASK_PROTECTED, MASK_REMOVE_A, MASK_REMOVE_B = 1, 2, 4, 8


def mask_thresholds(min_pt=0.05, max_incl_deg=70.0):
    """The float32 thresholds of the protection test: |q/pT| < fl(1/min_pt) and
    |sin phi| < fl(sin max_incl), from the float32 parameters."""
    import math
    max_qpt = np.float32(1.0 / float(np.float32(min_pt)))
    max_snp = np.float32(math.sin(float(np.float32(max_incl_deg)) * math.pi / 180.0))
    return max_qpt, max_snp


def cluster_masks(cl, trk_f, trk_i, ids, leg=None, tube=1.5, min_pt=0.05, max_incl_deg=70.0, bz=0.5, n_rows=152,
                  x_min=85.0, x_max=246.0):
    """Association, protection and strategy A/B removal of every cluster.

    trk_f: [n, 6] float32 (x_ref, y, z, sinphi, tanlambda, q/pT); trk_i: [n, 3]
    int64 (item, first, count) into ids (cluster indices, innermost first);
    leg: uint8 per track (0 = primary) or None.  Returns (mask uint8, owner
    int32 (-1 = none), ambiguous uint8)."""
    lib = _load()
    y = np.ascontiguousarray(cl.y, np.float32)
    z = np.ascontiguousarray(cl.z, np.float32)
    row = np.ascontiguousarray(cl.row, np.int32)
    off = np.ascontiguousarray(cl.item_off, np.uint64)
    tf = np.ascontiguousarray(np.asarray(trk_f, np.float32).reshape(-1, 6))
    ti = np.ascontiguousarray(np.asarray(trk_i, np.int64).reshape(-1, 3))
    ids = np.ascontiguousarray(ids, np.uint32)
    lg = None if leg is None else np.ascontiguousarray(leg, np.uint8)
    n = y.shape[0]
    mask = np.empty(n, np.uint8)
    owner = np.empty(n, np.int32)
    amb = np.empty(n, np.uint8)
    mq, ms = mask_thresholds(min_pt, max_incl_deg)
    lib.orc_cluster_masks(n_rows, x_min, x_max, bz, n, _p(y), _p(z), _p(row), _p(off), off.shape[0] - 1,
                          tf.shape[0], _p(tf), _p(ti), _p(ids), _p(lg), float(tube), float(mq), float(ms),
                          _p(mask), _p(owner), _p(amb))
    return mask, owner, amb


def oracle_tracks(ref):
    """(trk_f [n,6] float32, trk_i [n,3] int64, ids uint32) of the oracle tracker's output."""
    tf = ref["trk_f"][:, :6].astype(np.float32)
    ti = ref["trk_i"][:, :3].astype(np.int64)
    return tf, ti, ref["trk_ids"].astype(np.uint32)


def compress(cl, props, order, seg_off, trk_f, trk_i, ids, bz=0.5, n_rows=152, x_min=85.0, x_max=246.0, keep=None):
    """Compressed blob (bytes) of a tracked batch: entropy reduction and rANS
    coding.  props: charges and sizes (q_tot, q_max, sigma_y, sigma_z);
    order / seg_off: canonical order of the binned clusters and its (item, row)
    segment offsets; tracks as for cluster_masks; keep: uint8 per cluster (0 =
    removed, not stored) or None."""
    lib = _load()
    f32 = lambda a: np.ascontiguousarray(a, np.float32)
    y, z = f32(cl.y), f32(cl.z)
    row = np.ascontiguousarray(cl.row, np.int32)
    pr = [f32(props[k]) for k in ("q_tot", "q_max", "sigma_y", "sigma_z")]
    order = np.ascontiguousarray(order, np.int32)
    seg_off = np.ascontiguousarray(seg_off, np.int64)
    tf = np.ascontiguousarray(np.asarray(trk_f, np.float32).reshape(-1, 6))
    ti = np.ascontiguousarray(np.asarray(trk_i, np.int64).reshape(-1, 3))
    ids = np.ascontiguousarray(ids, np.uint32)
    kB = np.float32(0.299792458e-2 * np.float32(bz))
    n_items = (seg_off.shape[0] - 1) // n_rows
    kp = None if keep is None else np.ascontiguousarray(keep, np.uint8)
    args = [n_rows, x_min, x_max, float(kB), y.shape[0], _p(y), _p(z), _p(row), *[_p(a) for a in pr], n_items,
            _p(order), _p(seg_off), tf.shape[0], _p(tf), _p(ti), _p(ids), _p(kp)]
    size = lib.orc_compress(*args, None, 0)
    if size < 0:
        raise ValueError("bad input")
    out = np.empty(size, np.uint8)
    lib.orc_compress(*args, _p(out), size)
    return out


def decompress(blob):
    """Stored clusters of a blob: dict of item, row, y, z, q_tot, q_max,
    sigma_y, sigma_z codes and track (-1 = unattached)."""
    lib = _load()
    blob = np.ascontiguousarray(blob, np.uint8)
    n = lib.orc_decompress(_p(blob), blob.shape[0], 0, *([None] * 9))
    if n < 0:
        raise ValueError("malformed blob")
    keys = ("item", "row", "y", "z", "q_tot", "q_max", "sigma_y", "sigma_z", "track")
    out = {k: np.empty(n, np.int32) for k in keys}
    if lib.orc_decompress(_p(blob), blob.shape[0], n, *[_p(out[k]) for k in keys]) != n:
        raise ValueError("malformed blob")
    return out


def grid_order(ref, n_rows=152):
    """(order, seg_off) of the oracle tracker's binning: canonical sorted ids and
    the offsets of its (item, row) segments."""
    rows = ref["rows"]
    seg_off = np.zeros(rows.shape[0] + 1, np.int64)
    seg_off[1:] = np.cumsum(rows[:, 1])
    return ref["sorted_id"].astype(np.int32), seg_off


def code_stream(values):
    """One symbol stream (uint64 values) coded by byte planes and rANS, as in a blob."""
    lib = _load()
    v = np.ascontiguousarray(values, np.uint64)
    n = lib.orc_code_stream(_p(v), v.shape[0], None, 0)
    out = np.empty(n, np.uint8)
    lib.orc_code_stream(_p(v), v.shape[0], _p(out), n)
    return out


def decode_stream(blob):
    lib = _load()
    b = np.ascontiguousarray(blob, np.uint8)
    n = lib.orc_decode_stream(_p(b), b.shape[0], None, 0)
    if n < 0:
        raise ValueError("malformed stream")
    v = np.empty(n, np.uint64)
    lib.orc_decode_stream(_p(b), b.shape[0], _p(v), n)
    return v


def predict_codes(state6, bz, X):
    """(y, z) codes of the track model at pad-row radius X (float32 arithmetic)."""
    lib = _load()
    st = np.ascontiguousarray(state6, np.float32)
    py, pz = C.c_int64(), C.c_int64()
    kB = np.float32(0.299792458e-2 * np.float32(bz))
    lib.orc_predict(_p(st), float(kB), float(np.float32(X)), C.byref(py), C.byref(pz))
    return int(py.value), int(pz.value)


def merge(cl, trk_f, trk_i, ids, bz=0.5, n_rows=152, x_min=85.0, x_max=246.0, legs=False):
    """Sector-track merger of tracks trk_f [n,7] (x_ref, y, z, sinphi, tanlambda,
    q/pT, variance of q/pT), trk_i [n,3] (item, first, count): (link [n,2] (partner in sector k+1, k-1; -1 none),
    group [n] (smallest index of the group), ambiguous [n], fit [n,7] (per group
    root: centre x, y, radius, tan lambda, z0, clusters, tracks)); with legs=True
    also (partner [n] (the other leg of a looper, -1), leg [n] (1 secondary))."""
    lib = _load()
    y = np.ascontiguousarray(cl.y, np.float32)
    z = np.ascontiguousarray(cl.z, np.float32)
    row = np.ascontiguousarray(cl.row, np.int32)
    sec = np.ascontiguousarray(cl.item_sector, np.uint32)
    ev = np.ascontiguousarray(cl.item_event, np.uint32)
    tf = np.ascontiguousarray(np.asarray(trk_f, np.float32).reshape(-1, 7))
    ti = np.ascontiguousarray(np.asarray(trk_i, np.int64).reshape(-1, 3))
    ids = np.ascontiguousarray(ids, np.uint32)
    n = tf.shape[0]
    link = np.empty((n, 2), np.int32)
    group = np.empty(n, np.int32)
    amb = np.empty(n, np.uint8)
    fit = np.empty((n, 7), np.float64)
    partner = np.empty(n, np.int32)
    leg = np.empty(n, np.uint8)
    st = lib.orc_merge(n_rows, x_min, x_max, bz, y.shape[0], _p(y), _p(z), _p(row), sec.shape[0], _p(sec), _p(ev),
                       n, _p(tf), _p(ti), _p(ids), _p(link), _p(group), _p(amb), _p(fit), _p(partner), _p(leg))
    if st < 0:
        raise ValueError("bad input")
    if legs:
        return link, group, amb, fit, partner, leg
    return link, group, amb, fit


def join_loopers(cl, trk_f, trk_i, ids, group, partner, leg, bz=0.5, n_rows=152, x_min=85.0, x_max=246.0):
    """The legs of every looper joined into one track (after merge(..., legs=True)):
    (joined [n] component label, jfit [n,7] per joined component (centre x, y,
    radius, tan lambda, z0 at the primary legs' innermost cluster, clusters,
    tracks)), and the number of joined components."""
    lib = _load()
    y = np.ascontiguousarray(cl.y, np.float32)
    z = np.ascontiguousarray(cl.z, np.float32)
    row = np.ascontiguousarray(cl.row, np.int32)
    sec = np.ascontiguousarray(cl.item_sector, np.uint32)
    tf = np.ascontiguousarray(np.asarray(trk_f, np.float32).reshape(-1, 7))
    ti = np.ascontiguousarray(np.asarray(trk_i, np.int64).reshape(-1, 3))
    ids = np.ascontiguousarray(ids, np.uint32)
    group = np.ascontiguousarray(group, np.int32)
    partner = np.ascontiguousarray(partner, np.int32)
    leg = np.ascontiguousarray(leg, np.uint8)
    n = tf.shape[0]
    joined = np.empty(n, np.int32)
    jfit = np.empty((n, 7), np.float64)
    k = lib.orc_join_loopers(n_rows, x_min, x_max, bz, y.shape[0], _p(y), _p(z), _p(row), sec.shape[0], _p(sec), n,
                             _p(tf), _p(ti), _p(ids), _p(group), _p(partner), _p(leg), _p(joined), _p(jfit))
    if k < 0:
        raise ValueError("bad input")
    return joined, jfit, int(k)


def merge_tracks(ref):
    """(trk_f [n,7] float32 with the q/pT variance, trk_i, ids) of the oracle tracker's output."""
    tf = np.concatenate([ref["trk_f"][:, :6], ref["trk_f"][:, 20:21]], axis=1).astype(np.float32)
    return tf, ref["trk_i"][:, :3].astype(np.int64), ref["trk_ids"].astype(np.uint32)
