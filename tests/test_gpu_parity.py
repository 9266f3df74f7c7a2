"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Bar: bit-exact on every result field (score, both extension scores, all four
coordinates, status bits and the evaluated-cell count): the method is integer
arithmetic with a fixed tie-break, so there is no tolerance to allow.
"""

import random

import numpy as np
import pytest

import workloads
from pair_flags import expected_best_of_pair
from gpu_util import (NARROW_ALL, WIDE_ALL, assert_same, gpu_align, make_pairs, oracle_align, rc,
                      reads_to_arrays, schedule)

pytestmark = pytest.mark.gpu

INF = 1 << 30


@pytest.fixture(scope="module")
def c1():
    return workloads.generate("c1_tiny")


@pytest.mark.parametrize("X", [7, 25])
def test_c1_all_pairs(c1, X):
    sc = (1, -1, -1, X)
    got = gpu_align(c1.reads, c1.offsets, c1.pairs, 17, sc)
    exp = oracle_align(c1.reads, c1.offsets, c1.pairs, 17, sc)
    assert_same(got, exp, "c1 X=%d" % X)
    assert ((got["status"] & 4) != 0).sum() == len(workloads.pair_groups(c1.pairs)) - 1


@pytest.mark.parametrize("form", ["narrow32", "narrow48", "narrow64", "unroll4", "unroll8", "track32", "track48",
                                  "split16", "split64",
                                  "mid128", "mid192", "mid256", "nomid",
                                  "packed8", "packed16", "packed24", "packed32",
                                  "int16", "int32", "grp16x16", "grp16x24", "grp16x32", "grp8x16", "grp8x24"])
@pytest.mark.parametrize("X", [0, 3, 7, 25])
def test_every_kernel_form_matches(c1, form, X):
    """Route every extension to one form; escalations must reproduce the result."""
    if form.startswith("grp"):
        lanes, slots = form[3:].split("x")
        sched = schedule(wide_group_lanes=int(lanes), wide_slots=int(slots), wide_packed=1, **WIDE_ALL)
    elif form.startswith("packed"):
        sched = schedule(wide_slots=int(form[6:]), wide_packed=1, wide_group_lanes=32, **WIDE_ALL)
    elif form.startswith("int"):
        sched = schedule(wide_slots=int(form[3:]), wide_packed=0, **WIDE_ALL)
    elif form.startswith("mid"):
        # every extension through the 32-cell narrow form, its escalations through the mid form
        sched = schedule(narrow_band_cap=32, mid_band_cap=int(form[3:]), narrow_track=0, **NARROW_ALL)
    elif form.startswith("unroll"):
        # the narrow band walked in groups of 4 or 8 cells (32-cell rows: more escalations too)
        sched = schedule(narrow_band_cap=32, narrow_unroll=int(form[6:]), narrow_track=0, **NARROW_ALL)
    elif form.startswith("track"):
        # the live range and maximum kept in registers during the band walk
        sched = schedule(narrow_band_cap=int(form[5:]), narrow_track=1, **NARROW_ALL)
    elif form.startswith("split"):
        # the narrow form in two passes, the first stopping at antidiagonal 16 or 64
        sched = schedule(narrow_split_d=int(form[5:]), narrow_track=0, **NARROW_ALL)
    elif form == "nomid":
        sched = schedule(narrow_band_cap=32, mid_band_cap=0, narrow_track=0, **NARROW_ALL)
    else:
        # the band walked in 16-cell groups, live range and maximum found by scans of the row
        sched = schedule(narrow_band_cap=int(form[6:]), narrow_track=0, **NARROW_ALL)
    pairs = c1.pairs[:300]
    sc = (1, -1, -1, X)
    got = gpu_align(c1.reads, c1.offsets, pairs, 17, sc, sched=sched)
    exp = oracle_align(c1.reads, c1.offsets, pairs, 17, sc)
    assert_same(got, exp, "%s X=%d" % (form, X))


def random_overlap_reads(rng, n_reads, lo, hi, err):
    genome = "".join(rng.choice("ACGT") for _ in range(hi * 3))
    reads = []
    for _ in range(n_reads):
        L = rng.randint(lo, hi)
        s = rng.randint(0, len(genome) - L)
        t = genome[s:s + L]
        if rng.random() < 0.5:
            t = rc(t)
        out = []
        for ch in t:
            r = rng.random()
            if r < err * 0.2:
                out.append(rng.choice([c for c in "ACGT" if c != ch]))
            elif r < err * 0.7:
                out.append(ch)
                out.append(rng.choice("ACGT"))
            elif r >= err:
                out.append(ch)
        reads.append("".join(out))
    return reads


def shared_kmer_pairs(reads, k, max_pairs, rng):
    index = {}
    for r, s in enumerate(reads):
        for p in range(len(s) - k + 1):
            km = s[p:p + k]
            index.setdefault(km, []).append((r, p, 0))
            index.setdefault(rc(km), []).append((r, p, 1))
    recs = []
    for km, occ in index.items():
        for (ra, pa, oa) in occ:
            for (rb, pb, ob) in occ:
                if ra < rb:
                    recs.append((ra, rb, pa, pb, oa ^ ob))
    rng.shuffle(recs)
    recs = recs[:max_pairs]
    recs.sort()
    return recs


@pytest.mark.parametrize("scoring", [(1, -1, -1), (2, -3, -2), (1, -4, -1), (5, -4, -3), (1, 0, -1)])
def test_fuzz_medium(scoring):
    rng = random.Random(hash(scoring) & 0xffff)
    reads = random_overlap_reads(rng, 30, 200, 2500, 0.12)
    k = 11
    recs = shared_kmer_pairs(reads, k, 400, rng)
    ascii, offs = reads_to_arrays(reads)
    pairs = make_pairs(recs)
    for X in (0, 1, 5, 12, 40):
        sc = scoring + (X,)
        exp = oracle_align(ascii, offs, pairs, k, sc)
        for sched in (None, schedule(**NARROW_ALL), schedule(**WIDE_ALL),
                      schedule(narrow_band_cap=32, mid_band_cap=128, narrow_track=0, **NARROW_ALL),
                      schedule(mid_band_cap=0, narrow_track=0, **NARROW_ALL),
                      schedule(narrow_split_d=40, narrow_track=0, **NARROW_ALL),
                      schedule(narrow_unroll=4, narrow_track=0, **NARROW_ALL),
                      schedule(narrow_unroll=8, narrow_split_d=64, narrow_track=0, **NARROW_ALL),
                      schedule(narrow_track=0, **NARROW_ALL), schedule(narrow_track=1, **NARROW_ALL),
                      schedule(wide_packed=0, **WIDE_ALL), schedule(wide_slots=16, wide_group_lanes=32, **WIDE_ALL),
                      schedule(wide_group_lanes=16, **WIDE_ALL), schedule(wide_group_lanes=8, **WIDE_ALL)):
            got = gpu_align(ascii, offs, pairs, k, sc, sched=sched)
            assert_same(got, exp, "scoring %s X=%d" % (sc, X))


@pytest.mark.parametrize("lengths,counter", [((900, 1300), "escalated_wide"),
                                              ((4300, 4800), "cells_smem"),
                                              ((8400, 8800), "escalated_smem")])
def test_infinite_x_escalations(lengths, counter):
    """X = infinity: the band is the whole matrix (and X is above the packed
    form's limit, so the int32 register form runs).  Extensions wider than its
    band go to the CTA form (one block per extension, band in shared memory),
    and wider than 8189 cells to the global-memory form."""
    import paper_2001_10049_gb300 as dib
    rng = random.Random(lengths[0])
    reads = random_overlap_reads(rng, 5, lengths[0], lengths[1], 0.1)
    k = 9
    recs = shared_kmer_pairs(reads, k, 100000, rng)
    recs.sort(key=lambda r: r[2] + r[3])
    recs = sorted(recs[:3] + rng.sample(recs[3:], 3))
    ascii, offs = reads_to_arrays(reads)
    pairs = make_pairs(recs)
    sc = (1, -1, -1, INF)
    store = dib.ReadStore.from_ascii(ascii, offs)
    al = dib.Aligner(store, len(pairs), k=k)
    got = al.align(pairs, dib.Scoring(*sc))
    exp = oracle_align(ascii, offs, pairs, k, sc)
    assert_same(got, exp, "X=inf")
    c = dib.dibella_batch_counters(al.workspace)
    assert c[counter] > 0 and c["band_overflow"] == 0


def test_edge_cases():
    k = 5
    reads = ["ACGTACGTAC", "ACGTACGTAC", "AAAAAAAAAAAAAAAAAAAA", "CCCCCCCCCCCCCCCCCCCC", "ACG",
             "GTACGTACGT", "TTTTTAAAAA" * 30, "ACGTT"]
    recs = [
        (0, 1, 0, 0, 0),      # seed at the start of both reads (empty left extension)
        (0, 1, 5, 5, 0),      # seed ending at the read end (empty right extension)
        (0, 1, 2, 2, 0),
        (2, 3, 0, 0, 0),      # seed bases mismatch everywhere: status bit 0
        (2, 2, 3, 9, 0),      # self pair, homopolymer
        (0, 4, 0, 0, 0),      # read shorter than k: invalid
        (0, 9, 0, 0, 0),      # read id out of range: invalid
        (0, 1, 6, 0, 0),      # pos_a + k beyond the read: invalid
        (0, 1, 0, 0, 2),      # strand out of range: invalid
        (0, 5, 1, 0, 1),      # reverse strand
        (6, 6, 0, 150, 0),    # long self alignment at an offset
        (7, 0, 0, 0, 1),
    ]
    ascii, offs = reads_to_arrays(reads)
    pairs = make_pairs(recs)
    for X in (0, 2, 7, INF):
        for M, S, G in ((1, -1, -1), (3, -2, -5)):
            sc = (M, S, G, X)
            got = gpu_align(ascii, offs, pairs, k, sc)
            exp = oracle_align(ascii, offs, pairs, k, sc)
            assert_same(got, exp, "edge X=%d" % X)
    assert got["status"][5] == 2 and got["status"][6] == 2 and got["status"][7] == 2 and got["status"][8] == 2


def test_empty_batch():
    reads = ["ACGTACGTACGT"]
    ascii, offs = reads_to_arrays(reads)
    got = gpu_align(ascii, offs, make_pairs([]), 5, (1, -1, -1, 7))
    assert len(got) == 0


def test_per_pair_baseline_matches(c1):
    pairs = c1.pairs[:120]
    sc = (1, -1, -1, 25)
    got = gpu_align(c1.reads, c1.offsets, pairs, 17, sc, per_pair=True)
    exp = oracle_align(c1.reads, c1.offsets, pairs, 17, sc)
    assert_same(got, exp, "per-pair")


def test_host_entry_point_and_determinism(c1):
    import torch
    import paper_2001_10049_gb300 as dib
    store = dib.ReadStore.from_ascii(c1.reads, c1.offsets)
    al = dib.Aligner(store, len(c1.pairs), k=17)
    sc = dib.Scoring(1, -1, -1, 7)
    first = al.align(c1.pairs, sc)
    host_pairs = torch.from_numpy(c1.pairs.view(np.uint8).reshape(-1, 24).copy()).pin_memory()
    host_res = torch.empty((len(c1.pairs), 40), dtype=torch.uint8).pin_memory()
    staging = torch.empty(dib.dibella_staging_bytes(len(c1.pairs)), dtype=torch.uint8, device="cuda")
    dib.dibella_xdrop_batch_host(store.words, store.word_offsets, store.lengths, store.n_reads, host_pairs,
                                 len(c1.pairs), 17, sc, host_res, staging, al.workspace, al.workspace_bytes)
    again = host_res.numpy().reshape(-1).view(dib.RESULT_DTYPE)
    assert first.tobytes() == again.tobytes()
    for _ in range(3):
        assert al.align(c1.pairs, sc).tobytes() == first.tobytes()


def test_counters_report_routing(c1):
    import paper_2001_10049_gb300 as dib
    store = dib.ReadStore.from_ascii(c1.reads, c1.offsets)
    al = dib.Aligner(store, len(c1.pairs), k=17)
    al.align(c1.pairs, dib.Scoring(1, -1, -1, 25), sched=schedule(narrow_band_cap=32, mid_band_cap=0, **NARROW_ALL))
    # expand, scan, scatter; narrow; wide twice; ladder 16/24/32; CTA; global; combine, best of pair
    assert dib.dibella_last_launch_count() == 13
    c = dib.dibella_batch_counters(al.workspace)
    assert c["narrow"] == 2 * len(c1.pairs) and c["wide"] == 0
    assert c["escalated_narrow"] > 0 and c["band_overflow"] == 0
    # the narrow escalations are finished by the wide launch on them (or above)
    assert c["cells_wide"] == c["cells_wide_esc"] + c["cells_ladder"] and c["cells_wide_esc"] > 0
    assert c["cells_mid"] == 0 and c["escalated_mid"] == 0
    # with the mid form (one more launch) it takes the narrow escalations first
    al.align(c1.pairs, dib.Scoring(1, -1, -1, 25), sched=schedule(narrow_band_cap=32, mid_band_cap=128,
                                                                  **NARROW_ALL))
    assert dib.dibella_last_launch_count() == 14
    c2 = dib.dibella_batch_counters(al.workspace)
    assert c2["escalated_narrow"] == c["escalated_narrow"] and c2["cells_mid"] > 0
    assert c2["cells_wide_esc"] < c["cells_wide_esc"]
    total = lambda d: sum(d[f] for f in ("cells_narrow", "cells_wide", "cells_smem", "cells_global", "cells_mid"))
    # escalated extensions restart, so the finished cells of both runs agree
    assert total(c2) == total(c)
    # the narrow form in two passes: one launch more, the long extensions run again from the origin
    al.align(c1.pairs, dib.Scoring(1, -1, -1, 25), sched=schedule(narrow_band_cap=32, narrow_split_d=50,
                                                                  **NARROW_ALL))
    assert dib.dibella_last_launch_count() == 14
    c3 = dib.dibella_batch_counters(al.workspace)
    assert c3["narrow_second_pass"] > 0 and c3["cells_restarted"] > c["cells_restarted"]
    assert total(c3) == total(c)


def test_c2_full_size_sampled():
    """The E. coli-sized batch in the bench's launch configuration; a seeded
    sample of outputs is recomputed one by one by the oracle."""
    w = workloads.generate("c2_ecoli")
    rng = np.random.default_rng(11)
    idx = np.sort(rng.choice(len(w.pairs), 3000, replace=False))
    for X in (7, 25):
        sc = (1, -1, -1, X)
        got = gpu_align(w.reads, w.offsets, w.pairs, 17, sc)
        exp = oracle_align(w.reads, w.offsets, w.pairs[idx], 17, sc)
        sub = got[idx].copy()
        sub["status"] &= ~4  # best-of-pair flags depend on the whole run; checked below
        e2 = exp.copy()
        e2["status"] &= ~4
        assert_same(sub, e2, "c2 sample X=%d" % X)
        g = workloads.pair_groups(w.pairs)
        assert ((got["status"] & 4) != 0).sum() == len(g) - 1
        assert ((got["status"] & 8) != 0).sum() == 0


@pytest.mark.parametrize("scoring,X", [((20, -20, -20), 150), ((64, -30, -64), 500), ((64, -64, -64), 8000),
                                       ((64, -64, -64), 8001)])
def test_packed_form_large_scores(c1, scoring, X):
    """Scores far above the int16 range: the packed form rebases its 16-bit
    cells as the best grows (X <= 8000), and X = 8001 takes the int32 form."""
    pairs = c1.pairs[:150]
    sc = scoring + (X,)
    exp = oracle_align(c1.reads, c1.offsets, pairs, 17, sc)
    for slots in (16, 24):
        for lanes in (32, 16, 8):
            got = gpu_align(c1.reads, c1.offsets, pairs, 17, sc,
                            sched=schedule(wide_slots=slots, wide_group_lanes=lanes, **WIDE_ALL))
            assert_same(got, exp, "scoring %s X=%d slots=%d lanes=%d" % (scoring, X, slots, lanes))


@pytest.mark.parametrize("scoring,X", [((20, -20, -20), 150), ((64, -30, -64), 500), ((64, -64, -64), 8000),
                                       ((64, -64, -64), 8001)])
def test_narrow_form_large_scores(c1, scoring, X):
    """The narrow form keeps int16 cells relative to a moving base for X <= 8000
    (rebased as the best grows) and int32 cells above; scores run far beyond the
    int16 range here."""
    pairs = c1.pairs[:150]
    sc = scoring + (X,)
    exp = oracle_align(c1.reads, c1.offsets, pairs, 17, sc)
    for cap in (32, 48, 64):
        got = gpu_align(c1.reads, c1.offsets, pairs, 17, sc, sched=schedule(narrow_band_cap=cap, **NARROW_ALL))
        assert_same(got, exp, "scoring %s X=%d narrow cap %d" % (scoring, X, cap))


@pytest.mark.parametrize("name,X,n_check", [("c3_uneven", 50, 120), ("c4_repeats_small", 15, 400)])
def test_full_batch_sampled(name, X, n_check):
    """The uneven-length (X = 50) and repeat-rich (X = 15) batches launched whole,
    as the benchmark runs them; a seeded sample of records recomputed by the
    oracle one by one."""
    w = workloads.generate(name)
    rng = np.random.default_rng(13)
    idx = np.sort(rng.choice(len(w.pairs), n_check, replace=False))
    sc = (1, -1, -1, X)
    got = gpu_align(w.reads, w.offsets, w.pairs, 17, sc)
    exp = oracle_align(w.reads, w.offsets, w.pairs[idx], 17, sc)
    sub = got[idx].copy()
    sub["status"] &= ~4
    e2 = exp.copy()
    e2["status"] &= ~4
    assert_same(sub, e2, "%s sample X=%d" % (name, X))
    assert ((got["status"] & 8) != 0).sum() == 0


@pytest.mark.parametrize("name,X,n_check", [("c2_allseeds_300k", 25, 300), ("c2_ecoli_1kb", 25, 120)])
def test_seed_options_full_batch(name, X, n_check):
    """The seed options of Sec. 5 (every seed at least k apart; every seed at
    least 1,000 bp apart): the whole batch launched as the benchmark runs it, a
    seeded sample of records recomputed by the oracle, and the per-pair best
    flags equal to the reduction of the scores over each pair's seeds."""
    w = workloads.generate(name)
    rng = np.random.default_rng(17)
    idx = np.sort(rng.choice(len(w.pairs), n_check, replace=False))
    sc = (1, -1, -1, X)
    got = gpu_align(w.reads, w.offsets, w.pairs, 17, sc)
    exp = oracle_align(w.reads, w.offsets, w.pairs[idx], 17, sc)
    sub = got[idx].copy()
    sub["status"] &= ~4
    e2 = exp.copy()
    e2["status"] &= ~4
    assert_same(sub, e2, "%s sample X=%d" % (name, X))
    assert np.array_equal((got["status"] & 4) != 0, expected_best_of_pair(w.pairs, got))
    assert ((got["status"] & 8) != 0).sum() == 0
