"""Thin ctypes binding of libtpc.so (include/tpc.h).  Argument marshalling only:
every step of the tracker runs in the library's CUDA kernels.  torch supplies
device memory (its caching allocator, through the allocator callback) and the
stream.  There is no CPU fallback: without the built library this module fails
to import."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtpc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1910_12214_b300.build` "
                      "(nvcc, sm_103a); there is no CPU fallback")

_lib = C.CDLL(LIB_PATH)

TPC_OK = 0
STATUS = {0: "TPC_OK", 1: "TPC_ERR_INVALID_ARG", 2: "TPC_ERR_STATE", 3: "TPC_ERR_CUDA", 4: "TPC_ERR_OOM",
          5: "TPC_ERR_CAPACITY", 6: "TPC_ERR_TIMEOUT", 7: "TPC_ERR_BAD_INPUT"}
MODE = {"plain": 0, "batched": 1}
CORR = {"none": 0, "grid": 1, "mlp": 2}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class tpc_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class tpc_config(C.Structure):
    _fields_ = [("device", C.c_int), ("stream", C.c_void_p), ("bz_tesla", C.c_float), ("n_rows", C.c_int),
                ("row_x_min", C.c_float), ("row_x_max", C.c_float), ("sector_half_angle_deg", C.c_float),
                ("sigma_y", C.c_float), ("sigma_z", C.c_float), ("mode", C.c_int), ("correction", C.c_int),
                ("max_clusters", C.c_uint64), ("max_items", C.c_uint32), ("allocator", C.POINTER(tpc_allocator)),
                ("profile", C.c_int), ("tune_cache_path", C.c_char_p)]


class tpc_clusters(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("row", C.c_void_p), ("n", C.c_uint64),
                ("item_off", C.c_void_p), ("n_items", C.c_uint32), ("item_sector", C.c_void_p),
                ("item_event", C.c_void_p), ("item_core", C.c_void_p), ("on_device", C.c_int)]


class tpc_tuning(C.Structure):
    _fields_ = [("tracklet_lanes", C.c_int), ("tracklet_block", C.c_int), ("tracklet_blocks_per_sm", C.c_int),
                ("sort_smem", C.c_int), ("link_rows", C.c_int), ("mode", C.c_int),
                ("batch_lanes", C.c_int), ("use_graph", C.c_int), ("merge_sort_cap", C.c_int)]


class tpc_cluster_props(C.Structure):
    _fields_ = [("y", C.c_void_p), ("z", C.c_void_p), ("row", C.c_void_p), ("q_tot", C.c_void_p),
                ("q_max", C.c_void_p), ("sigma_y", C.c_void_p), ("sigma_z", C.c_void_p), ("n", C.c_uint64)]


class tpc_cluster_codes(C.Structure):
    _fields_ = [("y", C.c_void_p), ("z", C.c_void_p), ("row", C.c_void_p), ("q_tot", C.c_void_p),
                ("q_max", C.c_void_p), ("sigma_y", C.c_void_p), ("sigma_z", C.c_void_p)]


class tpc_mask_params(C.Structure):
    _fields_ = [("tube_cm", C.c_float), ("min_pt_gev", C.c_float), ("max_incl_deg", C.c_float)]


MASK_ASSOCIATED, MASK_PROTECTED, MASK_REMOVE_A, MASK_REMOVE_B = 1, 2, 4, 8


class tpc_cluster_charges(C.Structure):
    _fields_ = [("q_tot", C.c_void_p), ("q_max", C.c_void_p), ("sigma_y", C.c_void_p), ("sigma_z", C.c_void_p)]

PROP_FIELDS = (("y", np.float32), ("z", np.float32), ("row", np.int32), ("q_tot", np.float32),
               ("q_max", np.float32), ("sigma_y", np.float32), ("sigma_z", np.float32))
CODE_FIELDS = (("y", np.int16), ("z", np.int32), ("row", np.uint8), ("q_tot", np.uint16), ("q_max", np.uint16),
               ("sigma_y", np.uint8), ("sigma_z", np.uint8))

TRACK_DTYPE = np.dtype([("x_ref", "<f4"), ("y", "<f4"), ("z", "<f4"), ("snp", "<f4"), ("tgl", "<f4"),
                        ("qpt", "<f4"), ("cov", "<f4", (15,)), ("chi2", "<f4"), ("ndf", "<i4"), ("item", "<u4"),
                        ("sector", "<u4"), ("event", "<u4"), ("first_cluster", "<u4"), ("n_clusters", "<u4")])
assert TRACK_DTYPE.itemsize == 112

_P = C.c_void_p
_sig = {
    "tpc_init": ([C.POINTER(tpc_config), C.POINTER(_P)], C.c_int),
    "tpc_load_clusters": ([_P, C.POINTER(tpc_clusters)], C.c_int),
    "tpc_track": ([_P], C.c_int),
    "tpc_sync": ([_P], C.c_int),
    "tpc_get_tracks": ([_P, _P, C.c_uint64, _P, C.c_uint64, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)], C.c_int),
    "tpc_device_tracks": ([_P, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P)], C.c_int),
    "tpc_stage_times": ([_P, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int)], C.c_int),
    "tpc_stage_name": ([C.c_int], C.c_char_p),
    "tpc_debug_dump": ([_P, C.c_int, _P, C.c_uint64, C.POINTER(C.c_uint64)], C.c_int),
    "tpc_set_tuning": ([_P, C.POINTER(tpc_tuning)], C.c_int),
    "tpc_get_tuning": ([_P, C.POINTER(tpc_tuning)], C.c_int),
    "tpc_autotune": ([_P, C.c_int, C.POINTER(tpc_tuning), C.POINTER(C.c_float)], C.c_int),
    "tpc_autotune_mode": ([_P, C.c_int, C.c_int, C.POINTER(tpc_tuning), C.POINTER(C.c_float)], C.c_int),
    "tpc_set_grid_correction": ([_P, _P, _P, C.c_uint32, C.c_int, C.c_int, C.c_int], C.c_int),
    "tpc_set_correction": ([_P, C.c_int], C.c_int),
    "tpc_surrogate_train": ([_P, C.c_uint64, C.c_uint64, C.c_int, C.c_float, C.POINTER(C.c_float),
                             C.POINTER(C.c_float)], C.c_int),
    "tpc_surrogate_eval": ([_P, C.c_uint64, C.POINTER(C.c_float), C.POINTER(C.c_float)], C.c_int),
    "tpc_surrogate_params": ([_P, C.c_int, _P, C.c_int], C.c_int),
    "tpc_surrogate_set_params": ([_P, C.c_int, _P, C.c_int], C.c_int),
    "tpc_surrogate_grad": ([_P, C.c_int, C.c_uint64, C.c_uint64, C.c_int, _P, C.c_int, C.POINTER(C.c_float)], C.c_int),
    "tpc_surrogate_save": ([_P, C.c_char_p], C.c_int),
    "tpc_surrogate_load": ([_P, C.c_char_p], C.c_int),
    "tpc_bin_sector_noalloc": ([_P, _P, _P, C.c_uint32, C.c_int, _P, _P, _P, _P], C.c_int),
    "tpc_load_frame": ([_P, C.POINTER(tpc_clusters), C.c_float, C.c_float], C.c_int),
    "tpc_encode_clusters": ([_P, C.POINTER(tpc_cluster_props), C.POINTER(tpc_cluster_codes), C.c_int,
                             C.POINTER(C.c_uint64)], C.c_int),
    "tpc_cluster_masks": ([_P, C.POINTER(tpc_mask_params), _P, C.c_uint64, _P, C.c_uint64, _P, C.c_int, _P, _P],
                          C.c_int),
    "tpc_compress": ([_P, C.POINTER(tpc_cluster_charges), _P, C.c_uint64, _P, C.c_uint64, _P, C.c_int, _P,
                      C.c_uint64, C.POINTER(C.c_uint64)], C.c_int),
    "tpc_merge_tracks": ([_P, _P, C.c_uint64, _P, C.c_uint64, C.c_int, _P, _P, _P, _P, _P], C.c_int),
    "tpc_join_loopers": ([_P, _P, C.c_uint64, _P, C.c_uint64, C.c_int, _P, _P, _P, _P, _P, _P,
                          C.POINTER(C.c_uint64)], C.c_int),
    "tpc_destroy": ([_P], None),
    "tpc_last_error": ([_P], C.c_char_p),
}
for _name, (_a, _r) in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _a
    _f.restype = _r

EXPORTED = sorted(_sig)
NOALLOC_MAX_CLUSTERS = 65536


class TpcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _torch_allocator(device):
    import torch

    def alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, torch.cuda.current_stream(device))
        except Exception:
            return None

    def free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    fa, ff = ALLOC_FN(alloc), FREE_FN(free)
    return tpc_allocator(fa, ff, None), (fa, ff)


def _ptr(a):
    """Host numpy array -> address; torch tensor -> data_ptr (device or host)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


class Tracker:
    """One tpc_ctx.  Cluster input may be numpy (host) or CUDA torch tensors (device)."""

    def __init__(self, device: int = 0, stream=None, n_rows: int = 152, row_x_min: float = 85.0,
                 row_x_max: float = 246.0, half_angle_deg: float = 10.0, bz_tesla: float = 0.5,
                 sigma_y: float = 0.1, sigma_z: float = 0.1, mode: str = "plain", correction: str = "none",
                 max_clusters: int = 0, max_items: int = 0, torch_allocator: bool = True, profile: bool = False,
                 tune_cache_path: str = None):
        self._keep = []
        alloc_ptr = None
        if torch_allocator:
            al, keep = _torch_allocator(device)
            self._alloc = al
            self._keep.append(keep)
            alloc_ptr = C.pointer(self._alloc)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device)
        sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        if not sptr:
            sptr = 1  # cudaStreamLegacy: torch's default stream (a NULL handle would mean a library stream)
        self.cfg = tpc_config(device, sptr, bz_tesla, n_rows, row_x_min, row_x_max, half_angle_deg, sigma_y, sigma_z,
                              MODE[mode], CORR[correction], max_clusters, max_items, alloc_ptr, int(profile),
                              None if tune_cache_path is None else os.fsencode(tune_cache_path))
        self.n_rows = n_rows
        h = _P()
        st = _lib.tpc_init(C.byref(self.cfg), C.byref(h))
        if st != TPC_OK:
            raise TpcError(st, "tpc_init failed")
        self._h = h
        self._loaded = None

    def _check(self, st):
        if st != TPC_OK:
            raise TpcError(st, _lib.tpc_last_error(self._h).decode())

    def load(self, cl, on_device: bool = None):
        """cl: object with x, y, z, row (numpy or torch), item_off, optional item_sector,
        item_event, item_core (host numpy)."""
        return self._load(cl, on_device, None)

    def load_frame(self, fr, core_cm: float = 1000.0, overlap_cm: float = 300.0, on_device: bool = None):
        """A continuous read-out frame (items = sectors over their whole z axis),
        cut into overlapping slices on the device (tpc_load_frame); the tracks'
        cluster ids are frame indices."""
        return self._load(fr, on_device, (core_cm, overlap_cm))

    def _load(self, cl, on_device, frame):
        if on_device is None:
            on_device = hasattr(cl.x, "is_cuda") and cl.x.is_cuda
        keep = []

        def host(a, dt):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a

        if on_device:
            x, y, z, row = cl.x, cl.y, cl.z, cl.row
            n = int(x.shape[0])
        else:
            x, y, z = (host(a, np.float32) for a in (cl.x, cl.y, cl.z))
            row = host(cl.row, np.int32)
            n = int(x.shape[0])
        off = host(cl.item_off, np.uint64)
        sec = host(getattr(cl, "item_sector", None), np.uint32)
        ev = host(getattr(cl, "item_event", None), np.uint32)
        core = None if frame else host(getattr(cl, "item_core", None), np.int32)
        c = tpc_clusters(_ptr(x), _ptr(y), _ptr(z), _ptr(row), n, _ptr(off), int(off.shape[0] - 1), _ptr(sec),
                         _ptr(ev), _ptr(core), int(bool(on_device)))
        if frame:
            self._check(_lib.tpc_load_frame(self._h, C.byref(c), float(frame[0]), float(frame[1])))
        else:
            self._check(_lib.tpc_load_clusters(self._h, C.byref(c)))
        self._loaded = (cl, keep) if on_device else None
        self.n_loaded = n
        return self

    def track(self):
        self._check(_lib.tpc_track(self._h))
        return self

    def sync(self):
        self._check(_lib.tpc_sync(self._h))

    def counts(self):
        nt, ni = C.c_uint64(), C.c_uint64()
        st = _lib.tpc_get_tracks(self._h, None, 0, None, 0, C.byref(nt), C.byref(ni))
        if st not in (TPC_OK, 5):
            self._check(st)
        return int(nt.value), int(ni.value)

    def get_tracks(self, out=None):
        """Tracks (TRACK_DTYPE records) and their cluster ids.  out = (tracks,
        ids): caller-owned arrays (e.g. views of pinned host memory) reused if
        large enough; the returned arrays are then views of them."""
        nt, ni = self.counts()
        if out is not None and out[0].shape[0] >= nt and out[1].shape[0] >= ni:
            trk, ids = out[0][:nt], out[1][:ni]
        else:
            trk = np.zeros(nt, dtype=TRACK_DTYPE)
            ids = np.zeros(ni, dtype=np.uint32)
        a, b = C.c_uint64(), C.c_uint64()
        self._check(_lib.tpc_get_tracks(self._h, _ptr(trk) if nt else None, nt, _ptr(ids) if ni else None, ni,
                                        C.byref(a), C.byref(b)))
        return trk, ids

    def device_tracks(self):
        t, i, cnt = _P(), _P(), _P()
        self._check(_lib.tpc_device_tracks(self._h, C.byref(t), C.byref(i), C.byref(cnt)))
        return t.value, i.value, cnt.value

    def stage_times(self):
        us = (C.c_float * 32)()
        n = C.c_int()
        self._check(_lib.tpc_stage_times(self._h, us, 32, C.byref(n)))
        return {_lib.tpc_stage_name(i).decode(): float(us[i]) for i in range(n.value) if us[i] > 0}

    def debug_dump(self, stage: int) -> np.ndarray:
        n = C.c_uint64()
        st = _lib.tpc_debug_dump(self._h, stage, None, 0, C.byref(n))
        if st not in (TPC_OK, 5):
            self._check(st)
        buf = np.zeros(int(n.value), dtype=np.int32)
        self._check(_lib.tpc_debug_dump(self._h, stage, _ptr(buf) if n.value else None, n.value, C.byref(n)))
        return buf

    def set_tuning(self, **kw):
        t = tpc_tuning(**kw)
        self._check(_lib.tpc_set_tuning(self._h, C.byref(t)))

    def get_tuning(self) -> dict:
        t = tpc_tuning()
        self._check(_lib.tpc_get_tuning(self._h, C.byref(t)))
        return {f: getattr(t, f) for f, _ in tpc_tuning._fields_}

    def autotune(self, iters: int = 3, mode: int = 0):
        """Fastest launch shapes for the loaded batch (mode 1 = plain only,
        2 = batched only, 0 = both); returns (tuning dict, microseconds)."""
        t = tpc_tuning()
        us = C.c_float()
        self._check(_lib.tpc_autotune_mode(self._h, iters, mode, C.byref(t), C.byref(us)))
        return {f: getattr(t, f) for f, _ in tpc_tuning._fields_}, float(us.value)

    def set_grid_correction(self, grid, bounds):
        grid = np.ascontiguousarray(grid, np.float32)
        bounds = np.ascontiguousarray(bounds, np.float32)
        S, nx, ny, nz, k = grid.shape
        assert k == 3 and bounds.shape == (S, 6)
        self._check(_lib.tpc_set_grid_correction(self._h, _ptr(grid), _ptr(bounds), S, nx, ny, nz))

    def set_correction(self, mode: str):
        self._check(_lib.tpc_set_correction(self._h, CORR[mode]))

    def corrected(self):
        """Corrected (y, z) of the last tpc_track() (debug stage 11)."""
        d = self.debug_dump(11).view(np.float32).reshape(-1, 2)
        return d[:, 0].copy(), d[:, 1].copy()

    MLP_NP = 4611

    def surrogate_train(self, n_samples, seed=1, max_steps=0, lr=0.0):
        mx, rms = C.c_float(), C.c_float()
        self._check(_lib.tpc_surrogate_train(self._h, n_samples, seed, max_steps, lr, C.byref(mx), C.byref(rms)))
        return float(mx.value), float(rms.value)

    def surrogate_eval(self, n_points=65536):
        mx, rms = C.c_float(), C.c_float()
        self._check(_lib.tpc_surrogate_eval(self._h, n_points, C.byref(mx), C.byref(rms)))
        return float(mx.value), float(rms.value)

    def surrogate_params(self, sector=0):
        out = np.zeros(self.MLP_NP, np.float32)
        self._check(_lib.tpc_surrogate_params(self._h, sector, _ptr(out), out.shape[0]))
        return out

    def surrogate_set_params(self, sector, params):
        p = np.ascontiguousarray(params, np.float32)
        self._check(_lib.tpc_surrogate_set_params(self._h, sector, _ptr(p), p.shape[0]))

    def surrogate_grad(self, sector, seed, step, batch):
        g = np.zeros(self.MLP_NP, np.float32)
        loss = C.c_float()
        self._check(_lib.tpc_surrogate_grad(self._h, sector, seed, step, batch, _ptr(g), g.shape[0], C.byref(loss)))
        return g, float(loss.value)

    def surrogate_save(self, path):
        self._check(_lib.tpc_surrogate_save(self._h, str(path).encode()))

    def surrogate_load(self, path):
        self._check(_lib.tpc_surrogate_load(self._h, str(path).encode()))

    def encode_clusters(self, props, out=None, report_bad=True):
        """Integer codes of cluster properties (Sec. 4, step 2; include/tpc_reduce.h).

        props: dict of y, z, row, q_tot, q_max, sigma_y, sigma_z -- numpy arrays
        (host call: copied, encoded, copied back, waited for) or CUDA torch
        tensors (device call on the tracker's stream).  out: dict of code arrays
        of the same kind (allocated if None).  Returns (codes, n_bad); with a
        device call and report_bad=False the call does not wait and n_bad is
        None."""
        on_device = hasattr(props["y"], "is_cuda") and props["y"].is_cuda
        n = int(props["y"].shape[0])
        keep = []
        if on_device:
            import torch
            src = [props[k] for k, _ in PROP_FIELDS]
            if out is None:
                tdt = {np.int16: torch.int16, np.int32: torch.int32, np.uint8: torch.uint8, np.uint16: torch.uint16}
                out = {k: torch.empty(n, dtype=tdt[dt], device=props["y"].device) for k, dt in CODE_FIELDS}
        else:
            src = [np.ascontiguousarray(props[k], dt) for k, dt in PROP_FIELDS]
            keep.append(src)
            if out is None:
                out = {k: np.empty(n, dt) for k, dt in CODE_FIELDS}
        pin = tpc_cluster_props(*[_ptr(a) for a in src], n)
        cod = tpc_cluster_codes(*[_ptr(out[k]) for k, _ in CODE_FIELDS])
        bad = C.c_uint64()
        want = report_bad or not on_device
        st = _lib.tpc_encode_clusters(self._h, C.byref(pin), C.byref(cod), int(on_device),
                                      C.byref(bad) if want else None)
        if st not in (TPC_OK, 7):
            self._check(st)
        return out, (int(bad.value) if want else None)

    def cluster_masks(self, tracks=None, ids=None, leg=None, tube=1.5, min_pt=0.05, max_incl_deg=70.0,
                      on_device=False, with_owner=True, n_tracks=None):
        """Association, protection and strategy A/B removal masks of the loaded
        clusters (Sec. 4; include/tpc_reduce.h).  tracks=None uses the last
        tpc_track() output on the device; else tracks (TRACK_DTYPE records, or
        with on_device a CUDA uint8 tensor [n, 112]) and ids (uint32).  leg: one
        byte per track (0 = primary) or None; with tracks=None pass n_tracks.
        Returns (mask uint8, owner int32 or None) per loaded cluster: numpy, or
        CUDA tensors with on_device (enqueued on the tracker's stream)."""
        prm = tpc_mask_params(tube, min_pt, max_incl_deg)
        n = self.n_loaded
        if on_device:
            import torch
            dev = torch.device("cuda", self.cfg.device)
            mask = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)[:n]
            owner = torch.empty(max(n, 1), dtype=torch.int32, device=dev)[:n] if with_owner else None
            nt = int(tracks.shape[0]) if tracks is not None else int(n_tracks or 0)
        else:
            mask = np.empty(n, np.uint8)
            owner = np.empty(n, np.int32) if with_owner else None
            if tracks is not None:
                tracks = np.ascontiguousarray(tracks, TRACK_DTYPE)
                ids = np.ascontiguousarray(ids, np.uint32)
            if leg is not None:
                leg = np.ascontiguousarray(leg, np.uint8)
            nt = int(tracks.shape[0]) if tracks is not None else int(n_tracks or 0)
        ni = int(ids.shape[0]) if ids is not None else 0
        self._check(_lib.tpc_cluster_masks(self._h, C.byref(prm), _ptr(tracks), nt, _ptr(ids), ni, _ptr(leg),
                                           int(on_device), _ptr(mask), _ptr(owner)))
        return mask, owner

    def compress(self, charges, tracks=None, ids=None, on_device=False, out=None, keep=None):
        """Compressed blob of the loaded, tracked clusters (Sec. 4, steps 3-5;
        include/tpc_reduce.h).  charges: dict of q_tot, q_max, sigma_y, sigma_z
        (numpy, or CUDA tensors with on_device).  tracks=None uses the last
        tpc_track() output; else TRACK_DTYPE records and uint32 ids (numpy), or
        a CUDA uint8 tensor [n, 112] and int32 ids with on_device.  keep: one
        byte per loaded cluster, 0 = removed and not stored (numpy, or a CUDA
        tensor with on_device), None = keep all.  out: a buffer to write into
        (numpy uint8, or a CUDA uint8 tensor with on_device); too small or None:
        sized by a first call.  Returns the blob (a view of out)."""
        hold = []  # host arrays that must outlive the call
        if on_device:
            arrs = [charges[k] for k in ("q_tot", "q_max", "sigma_y", "sigma_z")]
        else:
            arrs = [np.ascontiguousarray(charges[k], np.float32) for k in ("q_tot", "q_max", "sigma_y", "sigma_z")]
            if tracks is not None:
                tracks = np.ascontiguousarray(tracks, TRACK_DTYPE)
                ids = np.ascontiguousarray(ids, np.uint32)
            if keep is not None:
                keep = np.ascontiguousarray(keep, np.uint8)
        hold += arrs + [tracks, ids, keep]
        nt = int(tracks.shape[0]) if tracks is not None else 0
        ch = tpc_cluster_charges(*[_ptr(a) for a in arrs])
        ni = int(ids.shape[0]) if ids is not None else 0
        size = C.c_uint64()

        def call(buf):
            cap = int(buf.shape[0]) if buf is not None else 0
            return _lib.tpc_compress(self._h, C.byref(ch), _ptr(tracks), nt, _ptr(ids), ni, _ptr(keep),
                                     int(on_device), _ptr(buf) if cap else None, cap, C.byref(size))

        st = call(out)
        if st == 5:  # TPC_ERR_CAPACITY: size the buffer and run again
            n = int(size.value)
            if on_device:
                import torch
                out = torch.empty(n, dtype=torch.uint8, device=torch.device("cuda", self.cfg.device))
            else:
                out = np.empty(n, np.uint8)
            st = call(out)
        self._check(st)
        return out[:int(size.value)]

    def merge_tracks(self, tracks=None, ids=None, n_tracks=None, legs=False, on_device=False):
        """Sector-track merger (include/tpc_reduce.h): (link [n,2], group [n],
        fit [n,7]) as numpy arrays, or CUDA tensors with on_device; with
        legs=True also (leg_partner [n], leg [n]) of the looper legs.
        tracks=None merges the last tpc_track() output (n_tracks = its count,
        read here if None); else TRACK_DTYPE records sorted by item and uint32
        ids (with on_device a CUDA uint8 tensor [n, 112] and int32 ids)."""
        if tracks is None:
            n = self.counts()[0] if n_tracks is None else int(n_tracks)
        elif on_device:
            n = int(tracks.shape[0])
        else:
            tracks = np.ascontiguousarray(tracks, TRACK_DTYPE)
            ids = np.ascontiguousarray(ids, np.uint32)
            n = int(tracks.shape[0])
        if on_device:
            import torch
            dev = torch.device("cuda", self.cfg.device)
            m = max(n, 1)
            link = torch.empty((m, 2), dtype=torch.int32, device=dev)[:n]
            group = torch.empty(m, dtype=torch.int32, device=dev)[:n]
            fit = torch.empty((m, 7), dtype=torch.float64, device=dev)[:n]
            partner = torch.empty(m, dtype=torch.int32, device=dev)[:n] if legs else None
            leg = torch.empty(m, dtype=torch.uint8, device=dev)[:n] if legs else None
        else:
            link = np.zeros((n, 2), np.int32)
            group = np.zeros(n, np.int32)
            fit = np.zeros((n, 7), np.float64)
            partner = np.zeros(n, np.int32) if legs else None
            leg = np.zeros(n, np.uint8) if legs else None
        ni = int(ids.shape[0]) if ids is not None else 0
        nz = lambda a: _ptr(a) if (a is not None and n) else None
        self._check(_lib.tpc_merge_tracks(self._h, _ptr(tracks), n, _ptr(ids), ni, int(bool(on_device)), nz(link),
                                          nz(group), nz(fit), nz(partner), nz(leg)))
        return (link, group, fit, partner, leg) if legs else (link, group, fit)

    def join_loopers(self, link, group, partner, leg, tracks=None, ids=None, n_tracks=None, on_device=False):
        """Looper legs joined into one track (include/tpc_reduce.h): (joined [n],
        jfit [n, 7], number of joined tracks) from the merger's outputs, as
        numpy arrays, or CUDA tensors with on_device (then link, group,
        partner, leg are the merger's CUDA tensors); tracks=None uses the last
        tpc_track() output."""
        if tracks is None:
            n = self.counts()[0] if n_tracks is None else int(n_tracks)
        elif on_device:
            n = int(tracks.shape[0])
        else:
            tracks = np.ascontiguousarray(tracks, TRACK_DTYPE)
            ids = np.ascontiguousarray(ids, np.uint32)
            n = int(tracks.shape[0])
        if on_device:
            import torch
            dev = torch.device("cuda", self.cfg.device)
            m = max(n, 1)
            joined = torch.empty(m, dtype=torch.int32, device=dev)[:n]
            jfit = torch.empty((m, 7), dtype=torch.float64, device=dev)[:n]
        else:
            link = np.ascontiguousarray(link, np.int32)
            group = np.ascontiguousarray(group, np.int32)
            partner = np.ascontiguousarray(partner, np.int32)
            leg = np.ascontiguousarray(leg, np.uint8)
            joined = np.zeros(n, np.int32)
            jfit = np.zeros((n, 7), np.float64)
        k = C.c_uint64()
        ni = int(ids.shape[0]) if ids is not None else 0
        nz = lambda a: _ptr(a) if n else None
        self._check(_lib.tpc_join_loopers(self._h, _ptr(tracks), n, _ptr(ids), ni, int(bool(on_device)), nz(link),
                                          nz(group), nz(partner), nz(leg), nz(joined), nz(jfit), C.byref(k)))
        return joined, jfit, int(k.value)

    def close(self):
        if getattr(self, "_h", None):
            _lib.tpc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def tracks_to_trk_i(trk: np.ndarray) -> np.ndarray:
    """(item, first_cluster, n_clusters, index) rows, the layout of the evaluation helpers."""
    return np.stack([trk["item"].astype(np.int64), trk["first_cluster"].astype(np.int64),
                     trk["n_clusters"].astype(np.int64), np.arange(trk.shape[0])], axis=1)
