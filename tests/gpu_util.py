"""Shared helpers for the GPU tests: build read sets and seed records, run the
CUDA path through the C ABI and the oracle on the same inputs, compare."""

from __future__ import annotations

import numpy as np

import oracle
import paper_2001_10049_gb300 as dib

FIELDS = ("score", "score_left", "score_right", "begin_a", "end_a", "begin_b", "end_b", "status", "cells")
COMP = str.maketrans("ACGT", "TGCA")


def rc(s: str) -> str:
    return s.translate(COMP)[::-1]


def reads_to_arrays(reads):
    ascii = np.frombuffer("".join(reads).encode(), dtype=np.uint8) if reads else np.zeros(0, np.uint8)
    offs = np.cumsum([0] + [len(r) for r in reads]).astype(np.int64)
    return ascii, offs


def make_pairs(recs):
    pairs = np.zeros(len(recs), dtype=dib.PAIR_DTYPE)
    for t, r in enumerate(recs):
        a, b, pa, pb, st = r[:5]
        sid = r[5] if len(r) > 5 else 0
        pairs[t]["read_a"], pairs[t]["read_b"], pairs[t]["pos_a"] = a, b, pa
        pairs[t]["pos_b"], pairs[t]["strand"], pairs[t]["seed_id"] = pb, st, sid
    return pairs


def gpu_align(ascii, offs, pairs, k, scoring, sched=None, per_pair=False, aligner=None):
    if aligner is None:
        store = dib.ReadStore.from_ascii(ascii, offs)
        aligner = dib.Aligner(store, max(1, len(pairs)), k=k)
    return aligner.align(pairs, dib.Scoring(*scoring), sched=sched, per_pair=per_pair)


def oracle_align(ascii, offs, pairs, k, scoring):
    M, S, G, X = scoring
    return oracle.xdrop_batch(ascii, offs, pairs.view(oracle.PAIR_DTYPE), k, M, S, G, X)


def assert_same(got, exp, context=""):
    assert len(got) == len(exp)
    bad = []
    for f in FIELDS:
        diff = np.flatnonzero(got[f].astype(np.int64) != exp[f].astype(np.int64))
        if len(diff):
            bad.append((f, int(diff[0]), int(got[f][diff[0]]), int(exp[f][diff[0]]), len(diff)))
    assert not bad, "%s mismatches (field, first idx, gpu, oracle, count): %s" % (context, bad)


def schedule(**kw):
    s = dib.dibella_get_default_schedule().as_dict()
    s.update(kw)
    return dib.Schedule.from_dict(s)


# Schedules that force each kernel form (results must not depend on them).
NARROW_ALL = dict(narrow_max_xdrop=1 << 30, narrow_max_len=1 << 30)
WIDE_ALL = dict(narrow_max_xdrop=-1)
