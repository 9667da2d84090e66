"""The allocation-free binning entry point, for callers that cannot allocate GPU
memory while they run.  It must give the same binning, bit for bit, as the
tracker's own binning step, on consecutive calls that share its fixed scratch
array.  This file is collected last (its name) so that a run stopping at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1910_12214_b300 import synth

pytestmark = pytest.mark.gpu


def _noalloc(cl, n_rows=152):
    import torch
    from paper_1910_12214_b300 import tpc
    n = cl.x.shape[0]
    dev = torch.device("cuda", 0)
    y = torch.from_numpy(np.ascontiguousarray(cl.y, np.float32)).to(dev)
    z = torch.from_numpy(np.ascontiguousarray(cl.z, np.float32)).to(dev)
    row = torch.from_numpy(np.ascontiguousarray(cl.row, np.int32)).to(dev)
    # the caller owns every input and output buffer
    sorted_ = torch.full((max(n, 1), 4), -7, dtype=torch.int32, device=dev)
    rows = torch.full((n_rows, 8), -7, dtype=torch.int32, device=dev)
    first = torch.full((2 * n + 3 * n_rows + 1,), -7, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    st = tpc._lib.tpc_bin_sector_noalloc(y.data_ptr(), z.data_ptr(), row.data_ptr(), n, n_rows, sorted_.data_ptr(),
                                         rows.data_ptr(), first.data_ptr(), None)
    return st, sorted_[:n].cpu().numpy(), rows.cpu().numpy(), first.cpu().numpy()


def _reference(cl, n_rows=152):
    from paper_1910_12214_b300 import tpc
    one = type("One", (), {})()
    one.x, one.y, one.z, one.row = cl.x, cl.y, cl.z, cl.row
    one.item_off = np.array([0, cl.x.shape[0]], np.uint64)
    with tpc.Tracker(n_rows=n_rows, row_x_max=85.0 + (n_rows - 1) * 161.0 / 151.0) as t:
        t.load(one).track()
        return t.debug_dump(0).reshape(-1, 3), t.debug_dump(1).reshape(-1, 7), t.debug_dump(2)


def _check(cl, n_rows=152):
    st, s, rows, first = _noalloc(cl, n_rows)
    assert st == 0
    ref0, ref1, ref2 = _reference(cl, n_rows)
    assert np.array_equal(s[:, :3], ref0)
    assert np.array_equal(rows[:, :7], ref1)
    rel = []
    for r in range(rows.shape[0]):
        nb = rows[r, 5] * rows[r, 6] if rows[r, 1] > 0 else 0
        rel.append(first[rows[r, 7]:rows[r, 7] + nb + 1] - rows[r, 0])
    assert np.array_equal(np.concatenate(rel), ref2)
    assert np.array_equal(s[:, 3], cl.row[s[:, 2]])


def _uniform(n, n_rows, seed, same_point=False):
    """n clusters of one sector with rows, y and z uniform (or all at one point)."""
    rng = np.random.default_rng(seed)
    cl = type("Sector", (), {})()
    cl.row = rng.integers(0, n_rows, n).astype(np.int32)
    cl.x = (85.0 + cl.row * (161.0 / 151.0)).astype(np.float32)
    if same_point:
        cl.row[:] = 3
        cl.x[:] = np.float32(85.0 + 3 * 161.0 / 151.0)
        cl.y = np.full(n, 1.25, np.float32)
        cl.z = np.full(n, -40.5, np.float32)
    else:
        cl.y = rng.uniform(-14.0, 14.0, n).astype(np.float32)
        cl.z = rng.uniform(-250.0, 250.0, n).astype(np.float32)
    return cl


def test_noalloc_binning_equals_tracker_binning_on_consecutive_calls():
    for seed in (1, 2):  # two calls in a row share (and reuse) the scratch array
        _check(synth.make_config1(seed=seed))


def test_noalloc_at_the_size_limit_few_rows_and_one_dense_bin():
    from paper_1910_12214_b300 import tpc
    _check(_uniform(tpc.NOALLOC_MAX_CLUSTERS, 152, seed=5))  # the largest accepted input
    _check(_uniform(3000, 8, seed=6), n_rows=8)                # a short sector
    _check(_uniform(5000, 152, seed=7, same_point=True))       # every cluster in one bin of one row


def test_noalloc_empty_input():
    cl = _uniform(0, 152, seed=8)
    st, s, rows, first = _noalloc(cl)
    assert st == 0 and s.shape[0] == 0
    r = np.arange(152)
    # empty rows: no hits, 1 cm bins, no grid, one bin-index entry each
    want = np.stack([0 * r, 0 * r, 0 * r, 0 * r, 10 + 0 * r, 0 * r, 0 * r, r], axis=1)
    assert np.array_equal(rows, want)
    assert np.array_equal(first[:152], np.zeros(152, np.int32))


def test_noalloc_rejects_oversize_and_bad_input():
    from paper_1910_12214_b300 import tpc
    big = tpc.NOALLOC_MAX_CLUSTERS + 1
    # rejected before any GPU work: the pointers are never touched
    assert tpc._lib.tpc_bin_sector_noalloc(1, 1, 1, big, 152, 1, 1, 1, None) == 5
    cl = synth.make_config1(seed=3)
    cl.row = cl.row.copy()
    cl.row[4] = 200
    st, *_ = _noalloc(cl)
    assert st == 7
