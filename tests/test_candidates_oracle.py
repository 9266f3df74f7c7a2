"""Candidate-pair oracle (k-mer counting, multiplicity filter, pairs per
retained k-mer, seed selection) pinned against a brute force written with
Python strings and against the workload generator's independent C++ index;
host-side checks of the GPU entry points' argument validation."""

import random

import numpy as np
import pytest

import workloads
from oracle import candidates as oc

COMP = str.maketrans("ACGT", "TGCA")


def rc(s):
    return s.translate(COMP)[::-1]


def brute(reads, k, lo, hi, max_seeds, gap):
    """Sec. 3 / Sec. 8 from their wording: canonical = the lexicographically
    smaller of the k-mer and its reverse complement (A<C<G<T)."""
    occ = {}
    for r, s in enumerate(reads):
        for p in range(len(s) - k + 1):
            km = s[p:p + k]
            c = min(km, rc(km))
            occ.setdefault(c, []).append((r, p, 0 if km <= rc(km) else 1))
    raw = []
    for c, lst in occ.items():
        if not lo <= len(lst) <= hi:
            continue
        lst = sorted(lst)
        for i in range(len(lst)):
            for j in range(i + 1, len(lst)):
                (ra, pa, oa), (rb, pb, ob) = lst[i], lst[j]
                if ra != rb:
                    raw.append((ra, rb, pa, pb, oa ^ ob))
    raw.sort()
    gap = gap if gap > 0 else k
    out = []
    i = 0
    while i < len(raw):
        j = i
        while j < len(raw) and raw[j][:2] == raw[i][:2]:
            j += 1
        taken, last = 0, None
        for t in range(i, j):
            if taken < max_seeds and (taken == 0 or raw[t][2] >= last + gap):
                out.append(raw[t] + (taken,))
                last = raw[t][2]
                taken += 1
        i = j
    return out, len(raw)


def as_tuples(rec):
    return [(int(r["read_a"]), int(r["read_b"]), int(r["pos_a"]), int(r["pos_b"]), int(r["strand"]),
             int(r["seed_id"])) for r in rec]


def to_arrays(reads):
    ascii = np.frombuffer("".join(reads).encode(), dtype=np.uint8)
    offs = np.cumsum([0] + [len(r) for r in reads]).astype(np.int64)
    return ascii, offs


@pytest.mark.parametrize("k,lo,hi,max_seeds,gap", [(5, 2, 6, 1, 0), (5, 2, 6, 1000, 0), (7, 2, 4, 1000, 9),
                                                   (4, 2, 8, 3, 0), (6, 1, 3, 2, 20)])
def test_oracle_matches_brute_force(k, lo, hi, max_seeds, gap):
    rng = random.Random(k * 100 + hi)
    base = "".join(rng.choice("ACGT") for _ in range(120))
    reads = []
    for _ in range(9):  # overlapping substrings of one template, random strand, a few errors
        a = rng.randint(0, 80)
        s = list(base[a:a + rng.randint(20, 40)])
        for _ in range(2):
            s[rng.randrange(len(s))] = rng.choice("ACGT")
        s = "".join(s)
        reads.append(rc(s) if rng.random() < 0.5 else s)
    reads.append("ACG")  # shorter than k: no occurrences
    ascii, offs = to_arrays(reads)
    rec, stats = oc.candidate_pairs(ascii, offs, k, lo, hi, max_seeds, gap)
    exp, n_raw = brute(reads, k, lo, hi, max_seeds, gap)
    assert as_tuples(rec) == exp
    assert stats["occurrence_pairs"] == n_raw
    assert stats["instances"] == sum(max(0, len(r) - k + 1) for r in reads)


@pytest.mark.parametrize("name", ["c1_tiny", "c2_allseeds_300k"])
def test_oracle_matches_generator_index(name):
    """Two independent implementations of the same steps: this oracle (numpy)
    and the workload generator's partitioned C++ index."""
    w = workloads.generate(name)
    p = w.params
    rec, stats = oc.candidate_pairs(w.reads, w.offsets, p["k"], p["mult_lo"], p["mult_hi"], p["max_seeds"],
                                    p["min_seed_gap"])
    assert rec.tobytes() == w.pairs.view(oc.PAIR_DTYPE).tobytes()
    assert stats["instances"] == w.stats["instances"]
    assert stats["retained_kmers"] == w.stats["retained_kmers"]
    assert stats["candidate_pairs"] == w.stats["candidate_pairs"]


def test_oracle_matches_generator_with_repeats_and_gap():
    w = workloads.generate("c4_repeats_small", genome_len=400_000, repeat_families=4, tandem_bases=20_000,
                           coverage=8.0, max_seeds=50, min_seed_gap=500)
    p = w.params
    rec, _ = oc.candidate_pairs(w.reads, w.offsets, p["k"], p["mult_lo"], p["mult_hi"], p["max_seeds"],
                                p["min_seed_gap"])
    assert rec.tobytes() == w.pairs.view(oc.PAIR_DTYPE).tobytes()


def test_gpu_entry_points_validate_arguments_on_the_host():
    import paper_2001_10049_gb300 as dib
    assert dib.dibella_candidate_workspace_bytes(10, 1000, 17, 8) > 0
    a = dib.dibella_candidate_workspace_bytes(10, 10_000, 17, 8)
    b = dib.dibella_candidate_workspace_bytes(10, 10_000, 17, 12)
    assert b > a
    for bad in ((10, 1000, 0, 8), (10, 1000, 33, 8), (10, 1000, 17, 0), (10, 1000, 17, 33), (-1, 10, 17, 8)):
        with pytest.raises(dib.DibellaError):
            dib.dibella_candidate_workspace_bytes(*bad)
    ws = 1 << 20  # a fake, aligned device address: every call below fails before touching it
    good = dict(k=17, mult_lo=2, mult_hi=8, max_seeds=1, min_seed_gap=0)
    cases = [dict(good, k=0), dict(good, mult_lo=0), dict(good, mult_lo=9), dict(good, max_seeds=0),
             dict(good, min_seed_gap=-1)]
    for c in cases:
        with pytest.raises(dib.DibellaError) as e:
            dib.dibella_candidate_pairs(ws, ws, ws, 10, 1000, 100, c["k"], c["mult_lo"], c["mult_hi"],
                                        c["max_seeds"], c["min_seed_gap"], ws, 100, ws, ws, 1 << 40, stream=0)
        assert e.value.code == dib.DIBELLA_EINVAL
    with pytest.raises(dib.DibellaError) as e:  # too small a workspace
        dib.dibella_candidate_pairs(ws, ws, ws, 10, 1000, 100, 17, 2, 8, 1, 0, ws, 100, ws, ws, 1024, stream=0)
    assert e.value.code == dib.DIBELLA_ENOMEM
    with pytest.raises(dib.DibellaError) as e:  # read and position fields wider than one sort key
        dib.dibella_candidate_pairs(ws, ws, ws, 1 << 20, 1000, 1 << 24, 17, 2, 8, 1, 0, ws, 100, ws, ws, 1 << 40,
                                    stream=0)
    assert e.value.code == dib.DIBELLA_EINVAL
