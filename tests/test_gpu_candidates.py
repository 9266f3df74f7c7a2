"""GPU candidate-pair generation (dibella_candidate_pairs) against the oracle
and the generator's independent index: the seed records must be identical,
byte for byte, and the counts equal."""

import random

import numpy as np
import pytest

import workloads
from oracle import candidates as oc

pytestmark = pytest.mark.gpu


def gpu_candidates(reads_ascii, offsets, k, lo, hi, max_seeds, gap):
    import paper_2001_10049_gb300 as dib
    store = dib.ReadStore.from_ascii(reads_ascii, offsets)
    return store.candidate_pairs(k=k, mult_lo=lo, mult_hi=hi, max_seeds=max_seeds, min_seed_gap=gap)


@pytest.mark.parametrize("name", ["c1_tiny", "c2_allseeds_300k"])
def test_matches_oracle(name):
    w = workloads.generate(name)
    p = w.params
    got, st = gpu_candidates(w.reads, w.offsets, p["k"], p["mult_lo"], p["mult_hi"], p["max_seeds"],
                             p["min_seed_gap"])
    exp, est = oc.candidate_pairs(w.reads, w.offsets, p["k"], p["mult_lo"], p["mult_hi"], p["max_seeds"],
                                  p["min_seed_gap"])
    assert got.tobytes() == exp.view(got.dtype).tobytes()
    assert st["seeds"] == len(exp) and st["status"] == 0
    for key in ("instances", "retained_kmers", "candidate_pairs", "occurrence_pairs"):
        assert st[key] == est[key], key


@pytest.mark.parametrize("k,lo,hi,max_seeds,gap", [(31, 2, 8, 1000, 0), (32, 2, 8, 2, 0), (15, 3, 12, 5, 100),
                                                   (9, 2, 32, 1, 0)])
def test_parameters_match_oracle(k, lo, hi, max_seeds, gap):
    w = workloads.generate("c2_allseeds_300k", genome_len=120_000, coverage=12.0)
    got, st = gpu_candidates(w.reads, w.offsets, k, lo, hi, max_seeds, gap)
    exp, est = oc.candidate_pairs(w.reads, w.offsets, k, lo, hi, max_seeds, gap)
    assert got.tobytes() == exp.view(got.dtype).tobytes()
    assert st["occurrence_pairs"] == est["occurrence_pairs"] and st["status"] == 0


def test_edge_reads():
    rng = random.Random(3)
    base = "".join(rng.choice("ACGT") for _ in range(300))
    reads = ["ACG", base[:50], base[20:90], "A" * 40, "A" * 45, base[100:101], base[80:200], base[80:200]]
    ascii = np.frombuffer("".join(reads).encode(), dtype=np.uint8)
    offs = np.cumsum([0] + [len(r) for r in reads]).astype(np.int64)
    for k in (5, 17):
        got, st = gpu_candidates(ascii, offs, k, 2, 32, 1000, 0)
        exp, est = oc.candidate_pairs(ascii, offs, k, 2, 32, 1000, 0)
        assert got.tobytes() == exp.view(got.dtype).tobytes()
        assert st["instances"] == est["instances"]


def test_full_size_matches_generator():
    """The E. coli-sized read set at its configuration (k = 17, [2, 8], up to 2
    seeds): byte-identical to the generator's own index."""
    w = workloads.generate("c2_ecoli")
    p = w.params
    got, st = gpu_candidates(w.reads, w.offsets, p["k"], p["mult_lo"], p["mult_hi"], p["max_seeds"],
                             p["min_seed_gap"])
    assert got.tobytes() == w.pairs.view(got.dtype).tobytes()
    assert st["instances"] == w.stats["instances"] and st["candidate_pairs"] == w.stats["candidate_pairs"]
    assert st["retained_kmers"] == w.stats["retained_kmers"]


# ---- the partitioned count (dibella_candidate_pairs_parts) -------------------

def gpu_candidates_parts(reads_ascii, offsets, k, lo, hi, max_seeds, gap, n_parts, max_read_len=None):
    import paper_2001_10049_gb300 as dib
    store = dib.ReadStore.from_ascii(reads_ascii, offsets)
    return store.candidate_pairs_parts(k=k, mult_lo=lo, mult_hi=hi, max_seeds=max_seeds, min_seed_gap=gap,
                                       n_parts=n_parts, max_read_len=max_read_len)


@pytest.mark.parametrize("name", ["c1_tiny", "c2_allseeds_300k"])
@pytest.mark.parametrize("n_parts", [1, 3, 8])
@pytest.mark.parametrize("wide_keys", [False, True])
def test_parts_match_oracle(name, n_parts, wide_keys):
    """Hash-partitioned passes give the oracle's records whatever the number of
    parts; a stated read-length bound of 2^24 bases makes the occurrence-pair
    fields exceed 64 bits, so the two-word key sort runs on the same reads."""
    import paper_2001_10049_gb300 as dib
    w = workloads.generate(name)
    p = w.params
    got, st = gpu_candidates_parts(w.reads, w.offsets, p["k"], p["mult_lo"], p["mult_hi"], p["max_seeds"],
                                   p["min_seed_gap"], n_parts,
                                   max_read_len=dib.DIBELLA_MAX_READ_LEN if wide_keys else None)
    exp, est = oc.candidate_pairs(w.reads, w.offsets, p["k"], p["mult_lo"], p["mult_hi"], p["max_seeds"],
                                  p["min_seed_gap"])
    assert got.tobytes() == exp.view(got.dtype).tobytes()
    assert st["seeds"] == len(exp) and st["status"] == 0
    for key in ("instances", "retained_kmers", "candidate_pairs", "occurrence_pairs"):
        assert st[key] == est[key], key
    assert st["instances"] / n_parts <= st["max_pass"] <= st["instances"]


@pytest.mark.parametrize("k,lo,hi,max_seeds,gap,n_parts", [(15, 3, 12, 5, 100, 4), (9, 2, 32, 1, 0, 2),
                                                           (21, 2, 8, 3, 0, 5)])
def test_parts_parameters_match_oracle(k, lo, hi, max_seeds, gap, n_parts):
    w = workloads.generate("c2_allseeds_300k", genome_len=120_000, coverage=12.0)
    got, st = gpu_candidates_parts(w.reads, w.offsets, k, lo, hi, max_seeds, gap, n_parts, max_read_len=1 << 24)
    exp, est = oc.candidate_pairs(w.reads, w.offsets, k, lo, hi, max_seeds, gap)
    assert got.tobytes() == exp.view(got.dtype).tobytes()
    assert st["occurrence_pairs"] == est["occurrence_pairs"] and st["status"] == 0


def test_parts_full_size_matches_generator():
    """The E. coli-sized reads in 6 passes with two-word keys: byte-identical to
    the generator's index."""
    w = workloads.generate("c2_ecoli")
    p = w.params
    got, st = gpu_candidates_parts(w.reads, w.offsets, p["k"], p["mult_lo"], p["mult_hi"], p["max_seeds"],
                                   p["min_seed_gap"], 6, max_read_len=1 << 24)
    assert got.tobytes() == w.pairs.view(got.dtype).tobytes()
    assert st["instances"] == w.stats["instances"] and st["candidate_pairs"] == w.stats["candidate_pairs"]


def test_parts_capacity_overflow_is_reported():
    """Too few parts for the pass capacity: EINVAL when the key cannot hold the
    slot bits; too small an occurrence-pair capacity: status bit 1, never a
    write past the buffers."""
    import torch
    import paper_2001_10049_gb300 as dib
    w = workloads.generate("c1_tiny")
    store = dib.ReadStore.from_ascii(w.reads, w.offsets)
    with pytest.raises(RuntimeError) as e:
        store.candidate_pairs_parts(k=17, n_parts=1, occ_pair_capacity=10)
    assert "status" in str(e.value)
    with pytest.raises(dib.DibellaError) as e2:  # 2k + bits(capacity) > 64 at k = 32
        store.candidate_pairs_parts(k=32, n_parts=1)
    assert e2.value.code == dib.DIBELLA_EINVAL
