"""Host logic of the multi-GPU form (one process per GPU, items sharded, no
data-path collective), checked on CPU: the item partition, the sub-batches,
the concatenation of per-rank tracks and the max-over-ranks timing reduction,
with two gloo ranks running the oracle on their shares."""
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_1910_12214_b300 import shard, synth


def test_lpt_partition_covers_and_balances():
    rng = np.random.default_rng(5)
    for world in (1, 2, 3, 5, 8):
        costs = rng.integers(0, 1000, size=int(rng.integers(0, 40)))
        parts = shard.lpt_partition(costs, world)
        assert len(parts) == world
        allv = np.concatenate(parts) if parts else np.zeros(0, int)
        assert np.array_equal(np.sort(allv), np.arange(costs.size))  # each item exactly once
        for p in parts:
            assert np.all(np.diff(p) > 0)
        loads = np.array([costs[p].sum() for p in parts])
        if costs.size:
            # greedy LPT: no rank exceeds the least loaded by more than the largest item
            assert loads.max() - loads.min() <= costs.max()
        assert all(np.array_equal(a, b) for a, b in zip(parts, shard.lpt_partition(costs, world)))


def test_lpt_partition_known_case():
    # descending cost, ties by index: item 1 (7) -> r0, item 3 (5) -> r1,
    # item 2 (4) -> r1 (load 9), item 0 (3) -> r0 (load 10), item 4 (3) -> r1 (12)
    parts = shard.lpt_partition([3, 7, 4, 5, 3], 2)
    assert parts[0].tolist() == [0, 1] and parts[1].tolist() == [2, 3, 4]


def test_grouped_partition_keeps_events_together():
    """The sectors of one event (which the sector-track merger joins) land on
    one rank; every item exactly once; balanced by events."""
    cl = synth.make_batched(seed=6, n_events=9, mult=(20, 400))
    costs = shard.item_costs(cl)
    for world in (1, 2, 4):
        parts = shard.lpt_partition_grouped(costs, cl.item_event, world)
        allv = np.concatenate(parts)
        assert np.array_equal(np.sort(allv), np.arange(costs.size))
        owner = np.empty(costs.size, int)
        for r, p in enumerate(parts):
            owner[p] = r
        for ev in np.unique(cl.item_event):
            assert np.unique(owner[cl.item_event == ev]).size == 1
        ev_cost = {ev: costs[cl.item_event == ev].sum() for ev in np.unique(cl.item_event)}
        loads = np.array([costs[p].sum() for p in parts])
        assert loads.max() - loads.min() <= max(ev_cost.values())


def test_take_items_slices_the_batch():
    cl = synth.make_batched(seed=4, n_events=3, mult=(5, 30))
    sub, index = shard.take_items(cl, np.arange(cl.n_items))
    assert np.array_equal(sub.y, cl.y) and np.array_equal(sub.item_off, cl.item_off)
    pick = np.array([5, 0, 71, 3])
    sub, index = shard.take_items(cl, pick)
    off = cl.item_off.astype(np.int64)
    for j, i in enumerate(pick):
        a, b = int(sub.item_off[j]), int(sub.item_off[j + 1])
        assert np.array_equal(sub.y[a:b], cl.y[off[i]:off[i + 1]])
        assert np.array_equal(index[a:b], np.arange(off[i], off[i + 1]))
        assert sub.item_sector[j] == cl.item_sector[i] and sub.item_event[j] == cl.item_event[i]


def _track_sets(trk_i, ids, items_map=None):
    out = set()
    for item, first, count, _ in trk_i:
        it = int(item) if items_map is None else int(items_map[int(item)])
        out.add((it, frozenset(int(v) for v in ids[first:first + count])))
    return out


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle
    from paper_1910_12214_b300 import tpc
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cl = synth.make_batched(seed=6, n_events=4, mult=(20, 120))
        parts = shard.lpt_partition(shard.item_costs(cl), world)
        items = parts[rank]
        sub, index = shard.take_items(cl, items)
        ref = oracle.run(sub, what=["trk_i", "trk_ids"])
        trk = np.zeros(ref["trk_i"].shape[0], dtype=tpc.TRACK_DTYPE)
        trk["item"] = ref["trk_i"][:, 0]
        trk["first_cluster"] = ref["trk_i"][:, 1]
        trk["n_clusters"] = ref["trk_i"][:, 2]
        mine = (trk, ref["trk_ids"], index, items)
        got = [None] * world
        dist.all_gather_object(got, mine)
        t_max = shard.max_over_ranks(1.5 + rank, dist)
        assert shard.sum_over_ranks(10 + rank, dist) == 21.0
        if rank == 0:
            trk_all, ids_all = shard.concat_tracks(got)
            full = oracle.run(cl, what=["trk_i", "trk_ids"])
            rows = np.stack([trk_all["item"].astype(np.int64), trk_all["first_cluster"].astype(np.int64),
                             trk_all["n_clusters"].astype(np.int64), np.arange(len(trk_all))], axis=1)
            same = _track_sets(rows, ids_all) == _track_sets(full["trk_i"], full["trk_ids"])
            with open(os.path.join(out_dir, "result.txt"), "w") as f:
                f.write(f"{int(same)} {t_max} {len(trk_all)} {full['trk_i'].shape[0]} {sum(len(p) for p in parts)}\n")
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_sharding_equals_single_process():
    import torch.multiprocessing as mp
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(world, _free_port(), d), nprocs=world, join=True, start_method="spawn")
        same, t_max, n_cat, n_full, n_items = open(os.path.join(d, "result.txt")).read().split()
    assert same == "1", "sharded tracks differ from the single-process result"
    assert float(t_max) == 2.5  # max over ranks of 1.5 + rank
    assert int(n_cat) == int(n_full) > 0
    cl = synth.make_batched(seed=6, n_events=4, mult=(20, 120))
    assert int(n_items) == cl.n_items
