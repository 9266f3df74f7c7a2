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
