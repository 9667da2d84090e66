"""Pins of the cluster-codec oracle (Sec. 4, step 2) against what the paper and
arithmetic fix: hand-worked cases, a brute-force nearest-value definition over
every value of each field, error bounds, and the fixed-point rules."""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dyn_precision.json")


def representable(n, width):
    """Every value of a `width`-bit field with at most n bits after its leading one."""
    vals = {0}
    for k in range(width):
        for m in range(1 << (n + 1)):
            v = m << k
            if v < (1 << width):
                vals.add(v)
    return np.array(sorted(vals), dtype=np.int64)


def nearest_up(S, v):
    """The element of sorted S nearest to v; ties go to the larger one."""
    i = np.searchsorted(S, v)
    hi = S[np.minimum(i, S.size - 1)]
    lo = S[np.maximum(i - 1, 0)]
    return np.where(hi - v <= v - lo, hi, lo)


def test_hand_worked_cases():
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        assert oracle.dyn_round(c["v"], c["n"], c["width"]) == c["expect"], c


@pytest.mark.parametrize("n,width", [(4, 16), (3, 8)])
def test_every_field_value_is_the_nearest_representable(n, width):
    S = representable(n, width)
    v = np.arange(1 << width, dtype=np.int64)
    want = nearest_up(S, v)
    got = np.array([oracle.dyn_round(int(a), n, width) for a in v], dtype=np.int64)
    assert np.array_equal(got, want)
    # idempotent and monotone: a precision reduction, not a reshuffle
    again = np.array([oracle.dyn_round(int(a), n, width) for a in got], dtype=np.int64)
    assert np.array_equal(again, got)
    assert np.all(np.diff(got) >= 0)


@pytest.mark.parametrize("n,width", [(4, 16), (3, 8)])
def test_relative_error_bound(n, width):
    """Below the clamp region the error is at most half a unit of the last kept bit."""
    top = ((1 << (n + 1)) - 1) << (width - n - 1)
    v = np.arange(1, top + 1, dtype=np.int64)
    got = np.array([oracle.dyn_round(int(a), n, width) for a in v], dtype=np.int64)
    assert np.all(np.abs(got - v) <= v * 2.0 ** -(n + 1))


def _props(**kw):
    n = max(len(np.atleast_1d(v)) for v in kw.values())
    base = {"y": np.zeros(n, np.float32), "z": np.zeros(n, np.float32), "row": np.zeros(n, np.int32),
            "q_tot": np.zeros(n, np.float32), "q_max": np.zeros(n, np.float32),
            "sigma_y": np.zeros(n, np.float32), "sigma_z": np.zeros(n, np.float32)}
    for k, v in kw.items():
        base[k] = np.asarray(v, dtype=base[k].dtype)
    return base


def test_positions_fixed_point_round_half_even_and_saturate():
    ys = np.array([0.0, 1.0 / 64, -1.0 / 64, 2.5 / 64, 3.5 / 64, -2.5 / 64, 0.3, 600.0, -600.0], np.float32)
    c, bad = oracle.encode_clusters(_props(y=ys, z=ys * 3))
    assert bad == 0
    assert c["y"].tolist() == [0, 1, -1, 2, 4, -2, 19, 32767, -32768]  # 0.3*64 = 19.2
    zc, _ = oracle.encode_clusters(_props(z=np.array([1e9, -1e9, 1300.0], np.float32)))
    assert zc["z"].tolist() == [2**31 - 1, -2**31, 83200]


def test_charge_and_size_codes():
    c, bad = oracle.encode_clusters(_props(q_tot=[150.4, 1000.0, -3.0, 1e6], q_max=[33.0, 31.0, 0.5, 1.5],
                                           sigma_y=[38.0 / 128, 0.1, 5.0, 0.0], sigma_z=[17.0 / 128, 0.0, 0.0, 1.0]))
    assert bad == 0
    assert c["q_tot"].tolist() == [152, 992, 0, 63488]   # 150, 1000, clamp 0, saturate
    assert c["q_max"].tolist() == [34, 31, 0, 2]         # 0.5 -> 0 and 1.5 -> 2 (ties to even)
    assert c["sigma_y"].tolist() == [40, 13, 240, 0]     # 0.1*128 = 12.8 -> 13
    assert c["sigma_z"].tolist() == [18, 0, 0, 128]


def test_bad_clusters_are_counted_and_coded_deterministically():
    c, bad = oracle.encode_clusters(_props(y=[np.nan, 1.0, 1.0, 1.0], z=[0.0, np.inf, 0.0, 0.0],
                                           row=[3, 3, 152, -1]), n_rows=152)
    assert bad == 4
    assert c["y"].tolist() == [0, 64, 64, 64]
    assert c["z"].tolist() == [0, 2**31 - 1, 0, 0]
    assert c["row"].tolist() == [3, 3, 0, 0]


def test_synthetic_batch_error_bounds():
    from paper_1910_12214_b300 import synth
    cl = synth.make_config1(seed=3)
    p = synth.cluster_props(cl, seed=3)
    c, bad = oracle.encode_clusters(p)
    assert bad == 0
    assert np.all(np.abs(c["y"] / 64.0 - p["y"]) <= 2.0 ** -7)
    assert np.all(np.abs(c["z"] / 64.0 - p["z"]) <= 2.0 ** -7)
    assert np.array_equal(c["row"], p["row"].astype(np.uint8))
    for k, scale, n in (("q_tot", 1.0, 4), ("q_max", 1.0, 4), ("sigma_y", 128.0, 3), ("sigma_z", 128.0, 3)):
        v = p[k].astype(np.float64) * scale
        fits = v < 0.98 * (((1 << (n + 1)) - 1) << ((16 if scale == 1.0 else 8) - n - 1))
        err = np.abs(c[k].astype(np.float64) - v)[fits]
        assert np.all(err <= 0.5 + (v[fits] + 0.5) * 2.0 ** -(n + 1)), k
