"""GPU traceback (dibella_xdrop_traceback) against the oracle: every result
field and every run of every seed's columns identical; the results also equal
the batch kernels' (dibella_xdrop_batch, best-of-pair flag aside)."""

import random

import numpy as np
import pytest

import oracle
import workloads
from test_oracle_pins import mutate, rand_seq, revcomp

pytestmark = pytest.mark.gpu


def synthetic(seed, n, lo, hi, k):
    """Read pairs from one template each (mutated, some unrelated, both
    strands), a seed per pair (a shared k-mer where one is found, else a random
    position), plus three invalid seeds."""
    rng = random.Random(seed)
    reads, recs = [], []
    for t in range(n):
        base = rand_seq(rng, rng.randint(lo, hi))
        a = mutate(rng, base, rng.choice([0.02, 0.1, 0.2]))
        b = mutate(rng, base, rng.choice([0.02, 0.1, 0.2]))
        if t % 7 == 3:
            b = rand_seq(rng, len(b))
        st = t % 2
        if st:
            b = revcomp(b)
        reads += [a, b]
        if len(a) < k or len(b) < k:
            recs.append((2 * t, 2 * t + 1, 0, 0, st))
            continue
        pa = rng.randint(0, len(a) - k)
        bp = revcomp(b) if st else b
        pbp = rng.randint(0, len(bp) - k)
        if t % 3 == 0:
            f = bp.find(a[pa:pa + k])
            if f >= 0:
                pbp = f
        recs.append((2 * t, 2 * t + 1, pa, len(b) - pbp - k if st else pbp, st))
    recs += [(0, 1, 10 ** 6, 0, 0), (0, 10 ** 6, 0, 0, 0), (0, 1, 0, 0, 2)]
    ascii = np.frombuffer("".join(reads).encode(), dtype=np.uint8)
    offs = np.cumsum([0] + [len(r) for r in reads]).astype(np.int64)
    pairs = np.zeros(len(recs), dtype=oracle.PAIR_DTYPE)
    for t, (ra, rb, pa, pb, st) in enumerate(recs):
        pairs[t]["read_a"], pairs[t]["read_b"], pairs[t]["pos_a"], pairs[t]["pos_b"], pairs[t]["strand"] = \
            ra, rb, pa, pb, st
        pairs[t]["seed_id"] = t
    return ascii, offs, pairs


def gpu_traceback(ascii, offs, pairs, k, scheme, cap, lanes, moves):
    import paper_2001_10049_gb300 as dib
    store = dib.ReadStore.from_ascii(ascii, offs)
    al = dib.Aligner(store, len(pairs), k=k)
    res, ops, n_ops = al.traceback(pairs, scheme, ops_per_seed=cap, n_lanes=lanes, moves_words=moves)
    batch = al.align(pairs, scheme)
    return res, ops, n_ops, batch


def check(ascii, offs, pairs, k, scheme, cap=2048, lanes=64, moves=1 << 20):
    M, S, G, X = scheme
    res, ops, n_ops, batch = gpu_traceback(ascii, offs, pairs, k, scheme, cap, lanes, moves)
    eres, eops, en = oracle.traceback_batch(ascii, offs, pairs, k, M, S, G, X, cap)
    assert res.tobytes() == eres.view(res.dtype).tobytes()
    plain = batch.copy()
    plain["status"] &= ~oracle.STATUS_BEST_OF_PAIR
    assert res.tobytes() == plain.tobytes()
    assert (n_ops == en).all(), np.flatnonzero(n_ops != en)[:5]
    for t in np.flatnonzero(n_ops > 0):
        assert (ops[t, :n_ops[t]] == eops[t, :n_ops[t]]).all(), t
    return res, n_ops


@pytest.mark.parametrize("case", [(1, 60, 30, 300, 5, (1, -1, -1, 7)), (2, 40, 200, 2000, 17, (1, -1, -1, 25)),
                                  (3, 30, 100, 1500, 11, (2, -3, -2, 50)), (4, 30, 50, 800, 9, (1, -4, -1, 1 << 30)),
                                  (5, 60, 20, 200, 3, (5, -4, -3, 0)), (7, 40, 10, 120, 32, (1, 0, -1, 9))],
                         ids=lambda c: "seed%d" % c[0])
def test_matches_oracle(case):
    seed, n, lo, hi, k, scheme = case
    ascii, offs, pairs = synthetic(seed, n, lo, hi, k)
    res, n_ops = check(ascii, offs, pairs, k, scheme, lanes=7)  # fewer lanes than seeds: slots are reused
    valid = (res["status"] & oracle.STATUS_INVALID_SEED) == 0
    assert valid.sum() >= n // 2 and (n_ops[valid] > 0).all()


def test_run_capacity_and_moves_capacity():
    ascii, offs, pairs = synthetic(8, 40, 100, 800, 7)
    _, n_ops = check(ascii, offs, pairs, 7, (1, -1, -1, 25), cap=6)
    assert (n_ops == -1).any() and (n_ops > 0).any()
    # moves that do not fit: -2, the results unchanged
    res, _, n_small, _ = gpu_traceback(ascii, offs, pairs, 7, (1, -1, -1, 25), 2048, 16, 64)
    eres, _, _ = oracle.traceback_batch(ascii, offs, pairs, 7, 1, -1, -1, 25, 2048)
    assert res.tobytes() == eres.view(res.dtype).tobytes()
    assert (n_small == -2).any() and (n_small >= -2).all()


def test_c1_tiny_sample():
    """Every third seed of the c1_tiny batch (reads of 2-6 kb, X = 7)."""
    w = workloads.generate("c1_tiny")
    pairs = np.ascontiguousarray(w.pairs[::3]).view(oracle.PAIR_DTYPE)
    _, n_ops = check(w.reads, w.offsets, pairs, w.params["k"], (1, -1, -1, 7), cap=8192, lanes=256)
    assert (n_ops > 0).sum() >= len(pairs) * 0.9
