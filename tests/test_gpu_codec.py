"""Parity of the CUDA cluster codec (Sec. 4, step 2) with the oracle: every
code bit-exact, the bad-cluster count equal, through the C ABI with host and
device buffers, on the aligned (vector) and unaligned (scalar) paths."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

FIELDS = ("y", "z", "row", "q_tot", "q_max", "sigma_y", "sigma_z")


def _same(got, want):
    for k in FIELDS:
        g = got[k].cpu().numpy() if hasattr(got[k], "cpu") else got[k]
        assert np.array_equal(g, want[k]), (k, np.flatnonzero(g != want[k])[:10])


def _to_dev(p, torch, offset=0):
    """Device copies of the property arrays; offset > 0 shifts them off 16-byte alignment."""
    out = {}
    for k in FIELDS:
        a = torch.from_numpy(np.ascontiguousarray(p[k]))
        buf = torch.empty(a.shape[0] + offset, dtype=a.dtype, device="cuda")
        buf[offset:].copy_(a)
        out[k] = buf[offset:]
    return out


@pytest.fixture(scope="module")
def tracker():
    from paper_1910_12214_b300 import tpc
    t = tpc.Tracker(device=0)
    yield t
    t.close()


def special_values():
    """Values on every rounding and saturation boundary of every field."""
    v = np.arange(65536, dtype=np.float64)
    q = np.concatenate([v, v + 0.5, v - 0.5, [-1.0, -0.49, 1e9, np.inf, -np.inf, np.nan, 65535.4, 65535.5]])
    n = q.shape[0]
    rng = np.random.default_rng(5)
    s = np.concatenate([np.arange(512) / 256.0, [-0.1, 1.99, 2.0, 1e6, np.nan, np.inf]])
    ys = np.concatenate([np.arange(-2048, 2048) / 128.0, [511.99, 512.0, -512.0, -600.0, np.nan, -np.inf]])
    zs = np.concatenate([np.arange(-2048, 2048) / 128.0 * 3, [3.4e7, -3.4e7, 33554431.0, np.nan, np.inf]])
    take = lambda a: a[rng.integers(0, a.shape[0], n)]
    props = {"y": take(ys).astype(np.float32), "z": take(zs).astype(np.float32),
             "row": rng.integers(-3, 156, n).astype(np.int32),
             "q_tot": q.astype(np.float32), "q_max": q[::-1].copy().astype(np.float32),
             "sigma_y": take(s).astype(np.float32), "sigma_z": take(s).astype(np.float32)}
    return props


def test_host_call_matches_oracle_on_a_full_tpc_event(tracker):
    from paper_1910_12214_b300 import synth
    cl = synth.make_config2(seed=4)
    p = synth.cluster_props(cl, seed=4)
    want, bad_w = oracle.encode_clusters(p)
    got, bad = tracker.encode_clusters(p)
    assert bad == bad_w == 0
    _same(got, want)


def test_special_values_every_boundary(tracker):
    p = special_values()
    want, bad_w = oracle.encode_clusters(p)
    got, bad = tracker.encode_clusters(p)
    assert bad == bad_w > 0
    _same(got, want)


@pytest.mark.parametrize("n", [0, 1, 3, 4, 5, 1023, 4097])
def test_ragged_sizes_device_call(tracker, n):
    import torch
    p = special_values()
    p = {k: v[7:7 + n] for k, v in p.items()}
    want, bad_w = oracle.encode_clusters(p)
    got, bad = tracker.encode_clusters(_to_dev(p, torch))
    assert bad == bad_w
    _same(got, want)


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_unaligned_device_arrays_take_the_scalar_path(tracker, offset):
    import torch
    p = special_values()
    p = {k: v[:50001] for k, v in p.items()}
    want, bad_w = oracle.encode_clusters(p)
    got, bad = tracker.encode_clusters(_to_dev(p, torch, offset))
    assert bad == bad_w
    _same(got, want)


def test_64_event_batch_device_call_in_the_benchmark_configuration(tracker):
    """The benchmark's codec workload (64 uneven events, 16M clusters), device
    resident, launched as the benchmark launches it; every code compared."""
    import torch
    from paper_1910_12214_b300 import synth
    cl = synth.make_batched(seed=1)
    p = synth.cluster_props(cl, seed=1)
    want, bad_w = oracle.encode_clusters(p)
    d = _to_dev(p, torch)
    got, bad = tracker.encode_clusters(d)
    assert bad == bad_w == 0
    _same(got, want)
    # asynchronous form: no count, same codes
    got2, none = tracker.encode_clusters(d, out=None, report_bad=False)
    torch.cuda.synchronize()
    assert none is None
    _same(got2, want)


def test_null_arrays_rejected(tracker):
    from paper_1910_12214_b300 import tpc
    import ctypes as C
    pin = tpc.tpc_cluster_props(None, None, None, None, None, None, None, 5)
    cod = tpc.tpc_cluster_codes(None, None, None, None, None, None, None)
    assert tpc._lib.tpc_encode_clusters(tracker._h, C.byref(pin), C.byref(cod), 0, None) == 1
