"""Splitting a batch of work items over ranks (one process per GPU).

Items (event, sector[, time slice]) are independent: tracking one item never
reads another, so N GPUs share a batch with no exchange on the data path.  Each
rank takes a static longest-processing-time share of the items (cost = cluster
count), tracks it with its own Tracker, and the tracks are concatenated on the
host.  The only collective is the maximum over ranks of the timed region.
This module is host bookkeeping: it computes nothing of the tracking method.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def lpt_partition(costs, world: int) -> list[np.ndarray]:
    """Items of each rank: descending cost, each to the least-loaded rank (ties:
    lower item index first, lower rank first).  Every item goes to exactly one
    rank; each rank's list is in ascending item order."""
    costs = np.asarray(costs, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.lexsort((np.arange(costs.size), -costs))
    load = np.zeros(world, dtype=np.int64)
    owner = np.empty(costs.size, dtype=np.int64)
    for i in order:
        r = int(np.argmin(load))  # first minimum: lowest rank among equals
        owner[i] = r
        load[r] += costs[i]
    return [np.flatnonzero(owner == r) for r in range(world)]


def lpt_partition_grouped(costs, groups, world: int) -> list[np.ndarray]:
    """As lpt_partition, with the items of one group (e.g. the sectors of one
    event, which the sector-track merger joins) kept on one rank: the groups
    are the units, each costing the sum of its items."""
    costs = np.asarray(costs, dtype=np.int64)
    groups = np.asarray(groups, dtype=np.int64)
    uniq, inv = np.unique(groups, return_inverse=True)
    per_rank = lpt_partition(np.bincount(inv, weights=costs, minlength=uniq.size).astype(np.int64), world)
    return [np.flatnonzero(np.isin(inv, g)) for g in per_rank]


def item_costs(cl) -> np.ndarray:
    """Cluster count of every item of a batch."""
    off = np.asarray(cl.item_off, dtype=np.int64)
    return off[1:] - off[:-1]


def take_items(cl, items):
    """The sub-batch of the given items (in the given order) and, for every
    cluster of it, its index in the full batch."""
    items = np.asarray(items, dtype=np.int64)
    off = np.asarray(cl.item_off, dtype=np.int64)
    lens = off[items + 1] - off[items]
    index = np.concatenate([np.arange(off[i], off[i + 1]) for i in items]) if items.size else np.zeros(0, np.int64)
    sub_off = np.zeros(items.size + 1, dtype=np.uint64)
    sub_off[1:] = np.cumsum(lens)
    pick = lambda a: None if a is None else np.ascontiguousarray(a[index])
    sub = dataclasses.replace(
        cl, x=pick(cl.x), y=pick(cl.y), z=pick(cl.z), row=pick(cl.row), item_off=sub_off,
        item_sector=np.ascontiguousarray(cl.item_sector[items]), item_event=np.ascontiguousarray(cl.item_event[items]),
        item_core=None if cl.item_core is None else np.ascontiguousarray(cl.item_core[items]), mc=pick(cl.mc),
        truth=pick(cl.truth), tracks=None)
    return sub, index


def concat_tracks(parts):
    """Concatenates per-rank results [(tracks, cluster_ids, index, items), ...]
    into one (tracks, cluster_ids) over the full batch: item numbers and cluster
    ids are mapped back through each rank's `items` and `index`, first_cluster
    offsets are shifted."""
    trks, ids = [], []
    base = 0
    for trk, cid, index, items in parts:
        trk = trk.copy()
        trk["item"] = np.asarray(items, dtype=np.int64)[trk["item"].astype(np.int64)].astype(trk["item"].dtype)
        trk["first_cluster"] += base
        trks.append(trk)
        ids.append(np.asarray(index, dtype=np.int64)[np.asarray(cid, dtype=np.int64)].astype(np.uint32))
        base += len(cid)
    if not trks:
        return None, np.zeros(0, np.uint32)
    return np.concatenate(trks), np.concatenate(ids)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank float over the process group (identity without one)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    """Sum of a per-rank number over the process group (identity without one)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
