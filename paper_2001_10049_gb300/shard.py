"""Cost-balanced sharding of one alignment batch across ranks (one GPU each).

Candidate pairs are independent once every rank holds the reads (Sec. 9: after
the reads are exchanged, alignment proceeds independently), but their costs are
not: X-drop stops early on unrelated reads and runs to the end of the shorter
read on related ones, and read lengths vary by two orders of magnitude (Sec. 9
names the resulting imbalance).  So the batch is split by cost, not by count:

* cost key of one seed record = the larger cost bound of its two extensions,
  min(remaining A, remaining B') summed over the left and right extension (the
  same key that orders the GPU's length buckets); a candidate pair's key is
  the sum over its seed records (its records stay together, so the best-seed
  flag of the pair is computed on one rank);
* pairs are dealt longest first to the rank with the smallest total so far
  (greedy LPT: no rank exceeds the mean by more than the largest pair's key);
* every rank aligns its share with its own copy of the read store, and rank 0
  gathers the results back into input order (the one collective, at the end).

Only bytes and keys are handled here; alignment happens in the library.
"""

from __future__ import annotations

import heapq

import numpy as np


def seed_cost_keys(pairs: np.ndarray, read_lengths: np.ndarray, k: int) -> np.ndarray:
    """Per seed record: min(rem A, rem B') of the left plus the right extension
    (0 for a record whose seed lies outside its reads)."""
    la = read_lengths[np.minimum(pairs["read_a"], len(read_lengths) - 1)].astype(np.int64)
    lb = read_lengths[np.minimum(pairs["read_b"], len(read_lengths) - 1)].astype(np.int64)
    pa = pairs["pos_a"].astype(np.int64)
    pb_fwd = pairs["pos_b"].astype(np.int64)
    pb = np.where(pairs["strand"] == 1, lb - pb_fwd - k, pb_fwd)
    valid = ((pairs["read_a"] < len(read_lengths)) & (pairs["read_b"] < len(read_lengths)) &
             (pairs["strand"] <= 1) & (pa + k <= la) & (pb_fwd + k <= lb))
    left = np.minimum(pa, pb)
    right = np.minimum(la - pa - k, lb - pb - k)
    return np.where(valid, np.maximum(left, 0) + np.maximum(right, 0), 0)


def pair_starts(pairs: np.ndarray) -> np.ndarray:
    """Start of every run of records with equal (read_a, read_b), plus len(pairs)."""
    if len(pairs) == 0:
        return np.zeros(1, dtype=np.int64)
    key = pairs["read_a"].astype(np.uint64) << np.uint64(32) | pairs["read_b"].astype(np.uint64)
    starts = np.flatnonzero(np.concatenate([[True], key[1:] != key[:-1]]))
    return np.concatenate([starts, [len(pairs)]]).astype(np.int64)


def partition(pairs: np.ndarray, read_lengths: np.ndarray, k: int, n_ranks: int):
    """Record indices of each rank's share (ascending, whole candidate pairs)
    and each rank's total cost key.  Deterministic: every rank computes the
    same partition from the same inputs."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    g = pair_starts(pairs)
    seed_keys = seed_cost_keys(pairs, read_lengths, k)
    csum = np.concatenate([[0], np.cumsum(seed_keys)])
    pair_keys = csum[g[1:]] - csum[g[:-1]]
    order = np.lexsort((np.arange(len(pair_keys)), -pair_keys))  # longest first, ties by position
    heap = [(0, r) for r in range(n_ranks)]
    owner = np.empty(len(pair_keys), dtype=np.int64)
    totals = np.zeros(n_ranks, dtype=np.int64)
    for p in order:
        tot, r = heapq.heappop(heap)
        owner[p] = r
        totals[r] = tot + pair_keys[p]
        heapq.heappush(heap, (int(totals[r]), r))
    sizes = np.diff(g)
    rec_owner = np.repeat(owner, sizes)
    shares = [np.flatnonzero(rec_owner == r) for r in range(n_ranks)]
    return shares, totals


def gather_results(n: int, shares, results_per_rank, dtype) -> np.ndarray:
    """Results of every rank placed back at their records' input positions."""
    out = np.zeros(n, dtype=dtype)
    for idx, res in zip(shares, results_per_rank):
        if len(idx) != len(res):
            raise ValueError("a rank returned %d results for %d records" % (len(res), len(idx)))
        out[idx] = res
    return out


def align_sharded(pairs: np.ndarray, read_lengths: np.ndarray, k: int, align_fn, group=None):
    """Align one batch across the ranks of ``group`` (torch.distributed): every
    rank computes the same cost-balanced partition, aligns its share with
    ``align_fn(records) -> results`` (on its own GPU and store), and rank 0
    gathers everything into input order.  Returns the gathered results on
    rank 0 and None elsewhere, plus this rank's (share indices, cost total)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    shares, totals = partition(pairs, read_lengths, k, world)
    mine = align_fn(pairs[shares[rank]])
    gathered = [None] * world if rank == 0 else None
    dist.gather_object(mine, gathered, dst=0, group=group)
    if rank != 0:
        return None, (shares[rank], int(totals[rank]))
    return gather_results(len(pairs), shares, gathered, mine.dtype), (shares[rank], int(totals[rank]))
