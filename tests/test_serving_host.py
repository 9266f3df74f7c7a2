"""Host logic of the serving loop, on the CPU: the first-fit arena that admits
batches by free device memory, and the merge of waiting requests into a batch
(whole candidate pairs only, requests never sharing a pair run)."""

import random

import numpy as np

from paper_2001_10049_gb300 import PAIR_DTYPE
from paper_2001_10049_gb300.serving import Arena, Request, Server


def test_arena_first_fit_alignment_and_coalescing():
    a = Arena(1 << 16, "cpu")
    x = a.alloc(100)
    y = a.alloc(300)
    z = a.alloc(1000)
    assert x == (0, 256) and y == (256, 512) and z == (768, 1024)
    assert a.free_bytes == (1 << 16) - 1792
    a.release(*y)
    assert a.alloc(200) == (256, 256)  # first fit reuses the hole
    a.release(256, 256)
    a.release(*x)
    a.release(*z)
    assert a.free == [(0, 1 << 16)]  # everything coalesced back
    assert a.alloc((1 << 16) + 1) is None


def test_arena_random_sequence_keeps_blocks_disjoint():
    rng = random.Random(7)
    size = 1 << 20
    a = Arena(size, "cpu")
    live = []
    for _ in range(2000):
        if live and rng.random() < 0.45:
            a.release(*live.pop(rng.randrange(len(live))))
        else:
            got = a.alloc(rng.randint(1, 40000))
            if got is not None:
                live.append(got)
        spans = sorted(live + a.free)
        assert sum(n for _, n in spans) == size
        for (o1, n1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + n1 <= o2
        assert all(o % 256 == 0 for o, _ in live)


def make_request(rid, runs, start_read):
    """A request whose records form `runs` candidate pairs (seed counts given)."""
    recs = []
    for i, n in enumerate(runs):
        for s in range(n):
            recs.append((start_read + i, start_read + i + 1000, 10 * s, 5 * s, 0, s))
    p = np.zeros(len(recs), dtype=PAIR_DTYPE)
    for t, (a, b, pa, pb, st, sid) in enumerate(recs):
        p[t]["read_a"], p[t]["read_b"], p[t]["pos_a"], p[t]["pos_b"], p[t]["strand"], p[t]["seed_id"] = \
            a, b, pa, pb, st, sid
    r = Request(rid, 0.0, 25, p)
    r._next, r._left = 0, len(p)
    return r


def merged(max_batch, q):
    srv = Server.__new__(Server)
    srv.max_batch = max_batch
    return [(r.rid, s, n) for r, s, n in Server._merge(srv, q)]


def test_merge_takes_oldest_whole_pairs_up_to_the_batch_size():
    q = [make_request(0, [2, 1, 3], 0), make_request(1, [1, 1], 100), make_request(2, [4], 200)]
    assert merged(100, q) == [(0, 0, 6), (1, 0, 2), (2, 0, 4)]
    # a batch of 7 seeds: request 0 whole, then request 1 up to its pair boundary
    assert merged(7, q) == [(0, 0, 6), (1, 0, 1)]
    # a batch of 4: request 0 split after its second pair (a pair is never split)
    assert merged(4, q) == [(0, 0, 3)]
    # a batch of 1 cannot hold request 0's first pair (2 seeds): nothing is taken
    assert merged(1, q) == []


def test_merge_never_joins_requests_sharing_a_pair_run():
    a = make_request(0, [2], 0)
    b = make_request(1, [1, 2], 0)  # its first pair is request 0's last pair
    assert merged(100, [a, b]) == [(0, 0, 2)]
