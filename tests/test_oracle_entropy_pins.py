"""Pins of the compression oracle (Sec. 4, steps 3 and 4): a hand-worked rANS
chunk, lossless round trips, Shannon's bound on the coded size, and the track
model's prediction against exact circle geometry."""
import math

import numpy as np
import pytest

import oracle
from test_oracle_masks_pins import circle_position, row_x

L = 1 << 16  # initial state of every rANS lane


def stream_fields(blob):
    """(value count, plane count, frequencies, chunk lengths, words) of a one-plane coded stream."""
    b = blob.tobytes()
    n = int.from_bytes(b[0:8], "little")
    planes = int.from_bytes(b[8:12], "little")
    f = np.frombuffer(b[12:12 + 512], np.uint16)
    n_chunks = int.from_bytes(b[524:528], "little")
    lens = np.frombuffer(b[528:528 + 4 * n_chunks], np.uint32)
    words = np.frombuffer(b[528 + 4 * n_chunks:], np.uint16)
    return n, planes, f, lens, words


def test_hand_worked_rans_chunk():
    """Symbols [0, 1] once each: both get frequency 2048 of 4096 (cumulative 0
    and 2048).  Lane 0 encodes symbol 0 from x = 2^16: x < 2048 * 2^20, no
    renormalisation, x' = (2^16 / 2048) * 4096 + 0 + 0 = 2^17.  Lane 1 encodes
    symbol 1: x' = 2^17 + 2048.  Lanes 2..31 keep 2^16.  The chunk is the 32
    final states as (low, high) word pairs and nothing else."""
    n, planes, f, lens, words = stream_fields(oracle.code_stream(np.array([0, 1], np.uint64)))
    assert (n, planes) == (2, 1)
    assert f[0] == 2048 and f[1] == 2048 and f[2:].sum() == 0
    assert lens.tolist() == [64]
    want = [0x0000, 0x0002, 0x0800, 0x0002] + [0x0000, 0x0001] * 30
    assert words.tolist() == want


def test_frequency_scaling_floor_and_excess():
    """The scaling rule worked by hand.  Counts {0: 10000, 1: 1}: f0 =
    floor(10000*4096/10001) = 4095, f1 = max(1, floor(4096/10001) = 0) = 1,
    sum 4096.  Counts {0: 100000, 1..255: 1 each}: f0 = floor(100000*4096/100255)
    = 4085, every other byte is raised to 1 (255 of them), sum 4340: the excess
    of 244 is taken from the largest, f0 = 3841."""
    _, _, f, _, _ = stream_fields(oracle.code_stream(np.array([0] * 10000 + [1], np.uint64)))
    assert f[0] == 4095 and f[1] == 1 and f[2:].sum() == 0
    v = np.concatenate([np.zeros(100000, np.uint64), np.arange(1, 256, dtype=np.uint64)])
    _, _, f, _, _ = stream_fields(oracle.code_stream(v))
    assert f[0] == 3841 and np.all(f[1:] == 1) and int(f.sum()) == 4096
    # two large counts {0: 60000, 1: 40000, 2..255: 1 each}: f0 = floor(60000*4096/100254)
    # = 2451, f1 = floor(40000*4096/100254) = 1634, 254 bytes raised to 1, sum 4339: the
    # excess of 243 is taken one unit at a time from the largest, which stays byte 0
    # (2208 > 1634), so f1 keeps its floor
    v = np.concatenate([np.zeros(60000, np.uint64), np.ones(40000, np.uint64), np.arange(2, 256, dtype=np.uint64)])
    _, _, f, _, _ = stream_fields(oracle.code_stream(v))
    assert f[0] == 2208 and f[1] == 1634 and np.all(f[2:] == 1)


def test_single_symbol_plane_costs_no_words():
    """A plane with one symbol value has frequency 4096: encoding leaves every
    state unchanged, so each chunk is its 32 initial states."""
    n, planes, f, lens, words = stream_fields(oracle.code_stream(np.full(20000, 7, np.uint64)))
    assert f[7] == 4096 and lens.tolist() == [64, 64, 64]
    assert words.tolist() == [0x0000, 0x0001] * 96


@pytest.mark.parametrize("dist", ["geometric", "uniform16", "two", "wide", "empty", "one"])
def test_round_trip_and_shannon_bound(dist):
    rng = np.random.default_rng(11)
    v = {"geometric": lambda: rng.geometric(0.05, 100_001) - 1,
         "uniform16": lambda: rng.integers(0, 1 << 16, 50_000),
         "two": lambda: rng.choice([3, 250], 30_000, p=[0.9, 0.1]),
         "wide": lambda: rng.integers(0, 1 << 40, 9_000) << rng.integers(0, 20, 9_000),
         "empty": lambda: np.zeros(0, np.int64),
         "one": lambda: np.array([123456789])}[dist]().astype(np.uint64)
    blob = oracle.code_stream(v)
    assert np.array_equal(oracle.decode_stream(blob), v)
    if v.size < 1000:
        return
    # size >= the empirical entropy of each byte plane (no code beats it) and
    # within 1% + the fixed costs (tables, 32 states per chunk) of it
    planes = max(1, (int(v.max()).bit_length() + 7) // 8)
    h_bits = 0.0
    for p in range(planes):
        b = ((v >> np.uint64(8 * p)) & np.uint64(255)).astype(np.int64)
        cnt = np.bincount(b, minlength=256)
        pr = cnt[cnt > 0] / v.size
        h_bits += -v.size * float(np.sum(pr * np.log2(pr)))
    chunks = math.ceil(v.size / 8192)
    fixed_bits = 8 * (12 + planes * (512 + 4 + 4 * chunks + 128 * chunks))
    size_bits = 8 * blob.size
    assert size_bits >= h_bits + fixed_bits * 0.0
    assert size_bits <= 1.01 * h_bits + fixed_bits + 64


def test_corrupt_stream_is_rejected():
    rng = np.random.default_rng(3)
    blob = oracle.code_stream(rng.geometric(0.1, 20_000).astype(np.uint64))
    bad = blob.copy()
    bad[-40] ^= 0x5A  # a renormalisation word: the final states no longer return to 2^16
    with pytest.raises(ValueError):
        oracle.decode_stream(bad)
    with pytest.raises(ValueError):
        oracle.decode_stream(blob[:-2])


def test_track_model_prediction_matches_the_exact_helix():
    """The float32 predictor (helix with a truncated arc series) against the
    crossing point from the circle's centre and radius, for tracks of 0.1 to
    10 GeV: within 2^-6 cm plus the series' truncation."""
    rng = np.random.default_rng(4)
    xr = row_x()
    worst = 0.0
    for _ in range(200):
        qpt = rng.choice([-1, 1]) / math.exp(rng.uniform(math.log(0.1), math.log(10.0)))
        st = np.array([xr[0], rng.uniform(-10, 10), rng.uniform(-100, 100), rng.uniform(-0.3, 0.3),
                       rng.uniform(-1, 1), qpt], np.float32)
        for r in range(0, 152, 7):
            P = circle_position(st[1:], float(st[0]), xr[r], 0.5)
            if P is None:
                break
            py, pz = oracle.predict_codes(st, 0.5, xr[r])
            worst = max(worst, abs(py / 64 - P[0]), abs(pz / 64 - P[1]))
    assert worst < 0.02


def test_blob_round_trip_of_a_tracked_event():
    """Every stored cluster comes back: unattached ones in the grid order of
    their pad row, attached ones track by track, with identical codes; the blob
    is smaller than the integer clusters it holds."""
    from paper_1910_12214_b300 import synth
    cl = synth.make_config1(seed=9)
    props = synth.cluster_props(cl, seed=9)
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids", "sorted_id", "rows"])
    tf, ti, ids = oracle.oracle_tracks(ref)
    order, seg = oracle.grid_order(ref)
    blob = oracle.compress(cl, props, order, seg, tf, ti, ids)
    d = oracle.decompress(blob)
    codes, _ = oracle.encode_clusters(props)
    attached = np.zeros(cl.n, bool)
    attached[ids] = True
    un = order[~attached[order]]
    seq = np.concatenate([un, ids.astype(np.int64)])
    assert d["y"].shape[0] == seq.shape[0]
    for k in ("y", "z", "q_tot", "q_max", "sigma_y", "sigma_z"):
        assert np.array_equal(d[k], codes[k][seq].astype(np.int32)), k
    assert np.array_equal(d["row"], cl.row[seq])
    trk_of = np.repeat(np.arange(tf.shape[0]), ti[:, 2])
    assert np.array_equal(d["track"], np.concatenate([np.full(un.shape[0], -1), trk_of]))
    assert blob.size < 13 * seq.shape[0]


def test_removed_clusters_are_not_stored():
    """With a keep mask (Sec. 4, step 5) the blob decodes to exactly the kept
    clusters: unattached ones in grid order, attached ones track by track with
    their row increments across the removed ones; fewer clusters, fewer bytes."""
    from paper_1910_12214_b300 import synth
    cl = synth.make_config1(seed=10)
    props = synth.cluster_props(cl, seed=10)
    ref = oracle.run(cl, what=["trk_f", "trk_i", "trk_ids", "sorted_id", "rows"])
    tf, ti, ids = oracle.oracle_tracks(ref)
    order, seg = oracle.grid_order(ref)
    keep = (np.random.default_rng(3).uniform(size=cl.n) < 0.5).astype(np.uint8)
    full = oracle.compress(cl, props, order, seg, tf, ti, ids)
    part = oracle.compress(cl, props, order, seg, tf, ti, ids, keep=keep)
    d = oracle.decompress(part)
    codes, _ = oracle.encode_clusters(props)
    attached = np.zeros(cl.n, bool)
    attached[ids] = True
    un = order[~attached[order] & (keep[order] == 1)]
    att = ids[keep[ids] == 1].astype(np.int64)
    seq = np.concatenate([un, att])
    for k in ("y", "z", "q_tot", "sigma_z"):
        assert np.array_equal(d[k], codes[k][seq].astype(np.int32)), k
    assert np.array_equal(d["row"], cl.row[seq])
    trk_of = np.repeat(np.arange(tf.shape[0]), ti[:, 2])[keep[ids] == 1]
    assert np.array_equal(d["track"][un.size:], trk_of)
    assert part.size < 0.7 * full.size
