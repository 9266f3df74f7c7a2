"""The seeded input generator: deterministic, and its pairs and seeds obey the
stated rules (shared retained k-mer at the seed, seed spacing, orientation)."""

import numpy as np

import workloads

COMP = str.maketrans("ACGT", "TGCA")


def rc(s):
    return s.translate(COMP)[::-1]


def test_deterministic_and_thread_independent():
    a = workloads.generate("c1_tiny", cache=False, n_threads=1)
    b = workloads.generate("c1_tiny", cache=False, n_threads=5)
    assert a.reads.tobytes() == b.reads.tobytes()
    assert a.pairs.tobytes() == b.pairs.tobytes()
    assert a.stats == b.stats


def test_c1_shape():
    w = workloads.generate("c1_tiny")
    L = w.read_lengths
    assert 100 <= w.n_reads <= 160
    # 15% error: template lengths in [2000, 6000]; read length within ~12% of template
    assert w.tmpl_len.min() >= 2000 and w.tmpl_len.max() <= 6000
    assert abs(L.sum() / w.tmpl_len.sum() - 1.03) < 0.02  # +0.5*15% ins, -0.3*15% del
    assert set(np.unique(w.reads)) <= set(b"ACGT")
    assert 500 <= len(w.pairs) <= 5000


def test_seeds_are_shared_kmers():
    w = workloads.generate("c2_ecoli", genome_len=300_000, coverage=10.0)
    k = w.params["k"]
    rng = np.random.default_rng(1)
    for t in rng.choice(len(w.pairs), 300, replace=False):
        p = w.pairs[t]
        A, B = w.read(p["read_a"]), w.read(p["read_b"])
        ka = A[p["pos_a"]:p["pos_a"] + k]
        kb = B[p["pos_b"]:p["pos_b"] + k]
        assert p["read_a"] < p["read_b"]
        assert (ka == kb) if p["strand"] == 0 else (ka == rc(kb))


def test_seed_selection_rules():
    w = workloads.generate("c2_ecoli", genome_len=300_000, coverage=10.0)
    g = workloads.pair_groups(w.pairs)
    k = w.params["k"]
    assert np.all(np.diff(g) >= 1) and np.all(np.diff(g) <= w.params["max_seeds"])
    multi = 0
    for s, e in zip(g[:-1], g[1:]):
        run = w.pairs[s:e]
        assert list(run["seed_id"]) == list(range(e - s))
        for u in range(1, len(run)):
            multi += 1
            assert run[u]["pos_a"] >= run[u - 1]["pos_a"] + k
    assert multi > 0


def test_multiplicity_window_and_counts():
    w = workloads.generate("c1_tiny")
    k = 17
    assert w.stats["instances"] == int(sum(max(0, l - k + 1) for l in w.read_lengths))
    assert w.stats["candidate_pairs"] == len(workloads.pair_groups(w.pairs)) - 1


def test_repeat_genome_has_repeats():
    w = workloads.generate("c4_repeats", genome_len=400_000, repeat_families=4, tandem_bases=20_000,
                           coverage=1.0)
    g = w.genome.tobytes().decode()
    # a tandem array repeats its unit: look for a long run with a short period
    found = False
    for p in range(2, 51):
        for start in range(0, len(g) - 600, 97):
            if g[start:start + 500] == g[start + p:start + p + 500]:
                found = True
                break
        if found:
            break
    assert found


def test_serving_requests_shape():
    w = workloads.generate("c1_tiny")
    reqs = workloads.serving_requests(w.pairs, 50, rate_per_s=100.0, seed=5, max_size=64)
    times = [r[0] for r in reqs]
    assert all(b > a for a, b in zip(times, times[1:]))
    for _, x, idx in reqs:
        assert x in (7, 25, 50) and len(idx) >= 1


def test_stratified_sample_keeps_whole_pairs_and_longest():
    w = workloads.generate("c1_tiny")
    s = workloads.stratified_pair_groups(w.pairs, w.read_lengths, 50)
    g = workloads.pair_groups(s)
    assert len(g) - 1 == 50
    L = w.read_lengths
    key_all = np.minimum(L[w.pairs["read_a"]], L[w.pairs["read_b"]])
    key_s = np.minimum(L[s["read_a"]], L[s["read_b"]])
    assert key_s.max() == key_all.max()


def test_seed_options_of_sec5():
    """One seed, all seeds at least k apart, all seeds at least 1,000 bp apart:
    the same first seed per pair, the stated spacing, and more records as the
    spacing shrinks."""
    base = dict(genome_len=300_000, coverage=20.0, len_dist=1, len_a=1000.0, len_b=60000.0, seed=9)
    one = workloads.generate(None, **base, max_seeds=1)
    allk = workloads.generate(None, **base, max_seeds=1 << 30)
    kb = workloads.generate(None, **base, max_seeds=1 << 30, min_seed_gap=1000)
    k = allk.params["k"]
    g1, gk, gb = (workloads.pair_groups(w.pairs) for w in (one, allk, kb))
    assert len(g1) == len(gk) == len(gb)  # the same candidate pairs
    assert np.all(np.diff(g1) == 1)
    assert len(one.pairs) < len(kb.pairs) < len(allk.pairs)
    for w, g, gap in ((allk, gk, k), (kb, gb, 1000)):
        first = w.pairs[g[:-1]]
        assert np.array_equal(first["pos_a"], one.pairs["pos_a"]) and np.array_equal(first["pos_b"], one.pairs["pos_b"])
        pa = w.pairs["pos_a"].astype(np.int64)
        same = np.ones(len(pa), dtype=bool)
        same[g[:-1]] = False  # records after the first of their pair
        assert np.all(pa[1:][same[1:]] - pa[:-1][same[1:]] >= gap)
        assert np.all(w.pairs["seed_id"][same] == w.pairs["seed_id"][np.flatnonzero(same) - 1] + 1)


def _restrict(pairs, ranges):
    m = np.zeros(len(pairs), bool)
    for lo, hi in ranges:
        m |= (pairs["read_a"] >= lo) & (pairs["read_a"] < hi)
    return pairs[m]


def test_read_range_index_equals_the_full_index():
    """pairs_mode PAIRS_RANGES builds only the k-mers of the chosen reads (the
    way the full-size repeat genome's pairs are checked in read blocks) and must
    give exactly the full index's records with read_a in those ranges."""
    for name, over in (("c1_tiny", {}),
                       ("c4_repeats_small", dict(genome_len=400_000, repeat_families=3, tandem_bases=20_000,
                                                 max_seeds=3, min_seed_gap=200))):
        full = workloads.generate(name, **over)
        n = full.n_reads
        ranges = [(0, n // 7), (n // 3, n // 3 + n // 10), (n - 5, n + 3)]
        part = workloads.generate(name, pairs_mode=workloads.PAIRS_RANGES, read_ranges=ranges, cache=False,
                                  **over)
        exp = _restrict(full.pairs, ranges)
        assert len(exp) > 0
        assert part.reads.tobytes() == full.reads.tobytes()
        assert part.pairs.tobytes() == exp.tobytes(), name
        assert part.stats["instances"] == full.stats["instances"]


def test_reads_only_mode():
    full = workloads.generate("c1_tiny")
    none = workloads.generate("c1_tiny", pairs_mode=workloads.PAIRS_NONE, cache=False)
    assert none.reads.tobytes() == full.reads.tobytes() and none.offsets.tobytes() == full.offsets.tobytes()
    assert len(none.pairs) == 0
