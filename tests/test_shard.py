"""Cost-balanced sharding of one batch across ranks (host logic, CPU, gloo).

The partition keeps candidate pairs whole, balances the summed cost keys within
the largest pair's key of the mean, and the gathered results equal one batch
aligned in one piece (best-seed flags included).  The per-rank alignment here is
the CPU oracle standing in for each rank's GPU, so the test runs without one;
the GPU path per rank is dibella_xdrop_batch, tested elsewhere."""

import os
import socket
import sys

import numpy as np

import oracle
import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2001_10049_gb300 import shard  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_partition_keeps_pairs_whole_and_balances_cost():
    w = workloads.generate("c2_allseeds_300k")  # up to 75 seeds per candidate pair
    L = w.read_lengths
    for n_ranks in (1, 2, 3, 7):
        shares, totals = shard.partition(w.pairs, L, 17, n_ranks)
        allidx = np.sort(np.concatenate(shares))
        assert np.array_equal(allidx, np.arange(len(w.pairs)))  # every record exactly once
        owner = np.empty(len(w.pairs), dtype=np.int64)
        for r, idx in enumerate(shares):
            owner[idx] = r
            assert np.all(np.diff(idx) > 0)
        g = shard.pair_starts(w.pairs)
        for s, e in zip(g[:-1], g[1:]):
            assert len(set(owner[s:e].tolist())) == 1  # a candidate pair never splits
        keys = shard.seed_cost_keys(w.pairs, L, 17)
        csum = np.concatenate([[0], np.cumsum(keys)])
        pair_keys = csum[g[1:]] - csum[g[:-1]]
        assert totals.sum() == keys.sum()
        assert totals.max() <= totals.mean() + pair_keys.max()
        for r, idx in enumerate(shares):
            assert totals[r] == keys[idx].sum()


def test_cost_key_is_the_extension_bound():
    pairs = np.zeros(3, dtype=workloads.PAIR_DTYPE)
    L = np.array([100, 60], dtype=np.int32)
    pairs["read_a"], pairs["read_b"] = 0, 1
    pairs[0]["pos_a"], pairs[0]["pos_b"] = 10, 20            # L: min(10, 20); R: min(73, 23)
    pairs[1]["pos_a"], pairs[1]["pos_b"], pairs[1]["strand"] = 10, 20, 1  # B': pos 60-20-17 = 23
    pairs[2]["pos_a"], pairs[2]["pos_b"] = 95, 0             # seed beyond read A: invalid
    k = shard.seed_cost_keys(pairs, L, 17)
    assert list(k) == [10 + 23, 10 + 20, 0]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = workloads.generate("c1_tiny")
    res, (mine, tot) = shard.align_sharded(
        w.pairs, w.read_lengths, 17,
        lambda recs: oracle.xdrop_batch(w.reads, w.offsets, recs.view(oracle.PAIR_DTYPE), 17, 1, -1, -1, 25))
    out[rank] = (len(mine), tot)
    if rank == 0:
        exp = oracle.xdrop_batch(w.reads, w.offsets, w.pairs.view(oracle.PAIR_DTYPE), 17, 1, -1, -1, 25)
        out["same"] = res.tobytes() == exp.tobytes()
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_one_batch():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    assert out["same"]
    assert out[0][0] > 0 and out[1][0] > 0
    w = workloads.generate("c1_tiny")
    assert out[0][0] + out[1][0] == len(w.pairs)
