"""Pins for the CPU oracle: checks against things other than the oracle itself.

* golden files of hand-worked extensions and seeded alignments;
* X = infinity reduces X-drop to the full dynamic program of diBELLA Sec. 2
  (optimal alignment, quadratic DP); it is computed here by a separate
  row-by-row Needleman-Wunsch-style recurrence over prefixes;
* brute-force enumeration of every alignment (Sec. 2 alignment definition:
  equal-length gapped strings, no all-gap column) on tiny inputs;
* invariants: mirror symmetry, score(X) <= score(inf), cell bounds, the
  empty and all-mismatch degenerate cases, best-of-pair flags.
"""

import os
import random

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = 1 << 30
COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}


def revcomp(s):
    return "".join(COMP[c] for c in reversed(s))


def rand_seq(rng, n):
    return "".join(rng.choice("ACGT") for _ in range(n))


def mutate(rng, s, rate):
    out = []
    for c in s:
        r = rng.random()
        if r < rate * 0.2:
            out.append(rng.choice([x for x in "ACGT" if x != c]))
        elif r < rate * 0.7:
            out.append(c)
            out.append(rng.choice("ACGT"))
        elif r < rate:
            pass
        else:
            out.append(c)
    return "".join(out)


def full_dp_extension(a, b, match, mismatch, gap):
    """Best global score over all prefix pairs a[:i], b[:j] (linear gap), with the
    tie-break "smallest i+j, then smallest i"; the start (0,0) scores 0."""
    m, n = len(a), len(b)
    F = [[0] * (n + 1) for _ in range(m + 1)]
    for i in range(1, m + 1):
        F[i][0] = i * gap
    for j in range(1, n + 1):
        F[0][j] = j * gap
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            s = match if a[i - 1] == b[j - 1] else mismatch
            F[i][j] = max(F[i - 1][j - 1] + s, F[i - 1][j] + gap, F[i][j - 1] + gap)
    best, bi, bj = 0, 0, 0
    for d in range(1, m + n + 1):
        for i in range(max(0, d - n), min(d, m) + 1):
            if F[i][d - i] > best:
                best, bi, bj = F[i][d - i], i, d - i
    return best, bi, bj


def brute_force_extension(a, b, match, mismatch, gap):
    """Enumerate every alignment path from (0,0); keep the best score per end cell."""
    m, n = len(a), len(b)
    best_at = {}

    def walk(i, j, score):
        if best_at.get((i, j), None) is None or score > best_at[(i, j)]:
            best_at[(i, j)] = score
        if i < m and j < n:
            walk(i + 1, j + 1, score + (match if a[i] == b[j] else mismatch))
        if i < m:
            walk(i + 1, j, score + gap)
        if j < n:
            walk(i, j + 1, score + gap)

    walk(0, 0, 0)
    best, bi, bj = 0, 0, 0
    for (i, j), s in sorted(best_at.items(), key=lambda kv: (kv[0][0] + kv[0][1], kv[0][0])):
        if s > best:
            best, bi, bj = s, i, j
    return best, bi, bj


def _parse(path):
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([part.split() for part in line.split("|")])
    return rows


@pytest.mark.parametrize("row", _parse(os.path.join(GOLDEN, "xdrop_extend_examples.txt")),
                         ids=lambda r: r[0][0])
def test_golden_extensions(row):
    (name, a, b, M, S, G, X), expect, bands = row
    a = "" if a == "-" else a
    b = "" if b == "-" else b
    best, i_end, j_end, cells, _ = oracle.extend(a, b, int(M), int(S), int(G), int(X))
    assert (best, i_end, j_end, cells) == tuple(int(v) for v in expect), name
    want_bands = [] if bands[0] == "-" else [int(v) for v in bands[0].split(",")]
    assert oracle.extend_bands(a, b, int(M), int(S), int(G), int(X)) == want_bands, name


@pytest.mark.parametrize("row", _parse(os.path.join(GOLDEN, "xdrop_seed_examples.txt")),
                         ids=lambda r: r[0][0])
def test_golden_seeded(row):
    (name, A, B, pa, pb, strand, k, M, S, G, X), expect = row
    res, _, _ = oracle.align_one(A, B, int(pa), int(pb), int(strand), int(k), int(M), int(S),
                                 int(G), int(X))
    got = (res["score"], res["score_left"], res["score_right"], res["begin_a"], res["end_a"],
           res["begin_b"], res["end_b"], res["status"], res["cells"])
    assert tuple(int(v) for v in got) == tuple(int(v) for v in expect), name


SCHEMES = [(1, -1, -1), (2, -3, -2), (1, -4, -1), (5, -4, -3), (1, 0, -1)]


@pytest.mark.parametrize("scheme", SCHEMES)
def test_infinite_x_equals_full_dp(scheme):
    M, S, G = scheme
    rng = random.Random(1000 + M * 7 + S)
    for trial in range(60):
        m, n = rng.randint(0, 40), rng.randint(0, 40)
        a = rand_seq(rng, m)
        b = mutate(rng, a, 0.3)[:n] if trial % 2 else rand_seq(rng, n)
        best, i_end, j_end, cells, _ = oracle.extend(a, b, M, S, G, INF)
        assert (best, i_end, j_end) == full_dp_extension(a, b, M, S, G), (a, b)
        assert cells == len(a) * len(b) + len(a) + len(b)


def test_infinite_x_equals_full_dp_long():
    rng = random.Random(7)
    for _ in range(4):
        a = rand_seq(rng, 200)
        b = mutate(rng, a, 0.15)[:200]
        best, i_end, j_end, cells, _ = oracle.extend(a, b, 1, -1, -1, INF)
        assert (best, i_end, j_end) == full_dp_extension(a, b, 1, -1, -1)
        assert cells == len(a) * len(b) + len(a) + len(b)


@pytest.mark.parametrize("scheme", SCHEMES[:3])
def test_brute_force_tiny(scheme):
    M, S, G = scheme
    rng = random.Random(55 + M)
    for _ in range(40):
        a = rand_seq(rng, rng.randint(0, 5))
        b = rand_seq(rng, rng.randint(0, 5))
        best, i_end, j_end, _, _ = oracle.extend(a, b, M, S, G, INF)
        assert (best, i_end, j_end) == brute_force_extension(a, b, M, S, G), (a, b)


def test_x_bounds_and_monotone_bound():
    """I2/I4/I5: 0 <= best(X) <= best(inf); cells(X) <= cells(inf); the cell that
    X-drop reports is reachable with at least its score (full DP on the prefixes)."""
    rng = random.Random(3)
    for _ in range(150):
        a = rand_seq(rng, rng.randint(0, 60))
        b = mutate(rng, a, rng.choice([0.05, 0.15, 0.35]))[: rng.randint(0, 60)]
        if rng.random() < 0.3:
            b = rand_seq(rng, len(b))
        full = oracle.extend(a, b, 1, -1, -1, INF)
        for X in (0, 1, 3, 7, 15, 25):
            best, i_end, j_end, cells, _ = oracle.extend(a, b, 1, -1, -1, X)
            assert 0 <= best <= full[0]
            assert cells <= full[3]
            assert full_dp_extension(a[:i_end], b[:j_end], 1, -1, -1)[0] >= best
            if best == 0:
                assert (i_end, j_end) == (0, 0)


def test_mirror_symmetry():
    """I3: swapping a and b mirrors the result; cells and score never change, and
    coordinates swap whenever the winning antidiagonal has a unique maximum."""
    rng = random.Random(11)
    for _ in range(300):
        a = rand_seq(rng, rng.randint(0, 50))
        b = mutate(rng, a, 0.2)[: rng.randint(0, 50)]
        X = rng.choice([0, 2, 5, 7, 12, INF])
        f = oracle.extend(a, b, 1, -1, -1, X)
        r = oracle.extend(b, a, 1, -1, -1, X)
        assert f[0] == r[0] and f[3] == r[3] and f[4] == r[4]
        if not f[4]:
            assert (f[1], f[2]) == (r[2], r[1])


def test_identical_sequences():
    """I1: identical reads seeded at equal positions align end to end with X >= -gap."""
    rng = random.Random(5)
    for _ in range(20):
        L = rng.randint(20, 300)
        A = rand_seq(rng, L)
        k = 17
        p = rng.randint(0, L - k)
        res, _, _ = oracle.align_one(A, A, p, p, 0, k, 1, -1, -1, 1)
        assert int(res["score"]) == L
        assert (int(res["begin_a"]), int(res["end_a"]), int(res["begin_b"]), int(res["end_b"])) == (0, L, 0, L)
        resrc, _, _ = oracle.align_one(A, revcomp(A), p, L - p - k, 1, k, 1, -1, -1, 1)
        assert int(resrc["score"]) == L
        assert (int(resrc["begin_b"]), int(resrc["end_b"])) == (0, L)


def test_all_mismatch_stops_early():
    """I5: with no matching character the best stays 0 and the search dies within
    O(X) antidiagonals (cell (i,j) scores -max(i,j) for match 1, mismatch/gap -1)."""
    for X in (0, 1, 5, 7, 25, 50):
        a, b = "A" * 1000, "C" * 1000
        best, i_end, j_end, cells, _ = oracle.extend(a, b, 1, -1, -1, X)
        assert (best, i_end, j_end) == (0, 0, 0)
        bands = oracle.extend_bands(a, b, 1, -1, -1, X)
        assert len(bands) <= 2 * X + 2
        assert cells == sum(bands) <= (2 * X + 3) ** 2


def test_homopolymer_band_width():
    """Identical homopolymers: cell (i,j) = min(i,j) - |i-j|; live cells satisfy
    3|i-j| <= X + 1 roughly, so the band stays O(X) for any length."""
    for X in (5, 10, 20):
        bands = oracle.extend_bands("A" * 400, "A" * 400, 1, -1, -1, X)
        assert max(bands) <= X + 3
        best, i_end, j_end, _, _ = oracle.extend("A" * 400, "A" * 400, 1, -1, -1, X)
        assert (best, i_end, j_end) == (400, 400, 400)


def test_strand_swap_mirror():
    """I3 at the seeded level: swapping (A,pos_a) with (B,pos_b) keeps the score;
    with strand 1 the left and right extensions exchange."""
    rng = random.Random(21)
    k = 11
    for trial in range(80):
        T = rand_seq(rng, 400)
        A = mutate(rng, T[50:300], 0.1)
        B0 = mutate(rng, T[120:380], 0.1)
        strand = trial % 2
        B = revcomp(B0) if strand else B0
        # plant a shared k-mer so the seed is exact
        kmer = rand_seq(rng, k)
        pa = rng.randint(0, len(A) - k)
        pb0 = rng.randint(0, len(B0) - k)
        A = A[:pa] + kmer + A[pa + k:]
        B0 = B0[:pb0] + kmer + B0[pb0 + k:]
        B = revcomp(B0) if strand else B0
        pb = len(B) - pb0 - k if strand else pb0
        X = rng.choice([3, 7, 25])
        r1, L1, R1 = oracle.align_one(A, B, pa, pb, strand, k, 1, -1, -1, X)
        r2, L2, R2 = oracle.align_one(B, A, pb, pa, strand, k, 1, -1, -1, X)
        assert int(r1["status"]) == 0 and int(r2["status"]) == 0
        assert int(r1["score"]) == int(r2["score"])
        assert int(r1["cells"]) == int(r2["cells"])
        if strand:
            assert (L1[0], R1[0]) == (R2[0], L2[0])
        else:
            assert (L1[0], R1[0]) == (L2[0], R2[0])
        if not (L1[4] or R1[4]):
            assert (int(r1["begin_a"]), int(r1["end_a"])) == (int(r2["begin_b"]), int(r2["end_b"]))
            assert (int(r1["begin_b"]), int(r1["end_b"])) == (int(r2["begin_a"]), int(r2["end_a"]))


def test_seeded_score_bound():
    """I2: score <= seed + full DP of the left part + full DP of the right part."""
    rng = random.Random(8)
    k = 7
    for _ in range(60):
        T = rand_seq(rng, 120)
        A = mutate(rng, T, 0.15)
        B = mutate(rng, T, 0.15)
        pa = rng.randint(0, len(A) - k)
        pb = rng.randint(0, len(B) - k)
        for X in (3, 10):
            r, L, R = oracle.align_one(A, B, pa, pb, 0, k, 1, -1, -1, X)
            seed = sum(1 if A[pa + t] == B[pb + t] else -1 for t in range(k))
            fl = full_dp_extension(A[:pa][::-1], B[:pb][::-1], 1, -1, -1)[0]
            fr = full_dp_extension(A[pa + k:], B[pb + k:], 1, -1, -1)[0]
            assert int(r["score"]) == seed + L[0] + R[0]
            assert int(r["score"]) <= seed + fl + fr
            assert (int(r["status"]) & 1) == (0 if A[pa:pa + k] == B[pb:pb + k] else 1)


def test_batch_threads_and_best_of_pair():
    rng = random.Random(9)
    reads = [rand_seq(rng, rng.randint(30, 200)) for _ in range(12)]
    ascii = np.frombuffer("".join(reads).encode(), dtype=np.uint8)
    offsets = np.cumsum([0] + [len(r) for r in reads]).astype(np.int64)
    recs = []
    for a in range(12):
        for b in range(a + 1, 12, 3):
            for s in range(rng.randint(1, 3)):
                recs.append((a, b, rng.randint(0, len(reads[a]) - 5),
                             rng.randint(0, len(reads[b]) - 5), rng.randint(0, 1), s))
    recs.append((3, 40, 0, 0, 0, 0))      # read id out of range
    recs.append((3, 4, 10 ** 6, 0, 0, 0))  # seed beyond the read
    pairs = np.zeros(len(recs), dtype=oracle.PAIR_DTYPE)
    for t, (a, b, pa, pb, st, sid) in enumerate(recs):
        pairs[t]["read_a"], pairs[t]["read_b"], pairs[t]["pos_a"] = a, b, pa
        pairs[t]["pos_b"], pairs[t]["strand"], pairs[t]["seed_id"] = pb, st, sid
    r1 = oracle.xdrop_batch(ascii, offsets, pairs, 5, 1, -1, -1, 7, n_threads=1)
    r4 = oracle.xdrop_batch(ascii, offsets, pairs, 5, 1, -1, -1, 7, n_threads=4)
    assert r1.tobytes() == r4.tobytes()
    assert r1[-2]["status"] == oracle.STATUS_INVALID_SEED and r1[-1]["status"] == oracle.STATUS_INVALID_SEED
    # each record equals the single-seed entry point, up to the best-of-pair flag
    for t in range(len(recs) - 2):
        a, b, pa, pb, st, _ = recs[t]
        one, _, _ = oracle.align_one(reads[a], reads[b], pa, pb, st, 5, 1, -1, -1, 7)
        got = r1[t].copy()
        got["status"] &= ~oracle.STATUS_BEST_OF_PAIR
        assert got.tobytes() == np.array(one, dtype=oracle.RESULT_DTYPE).tobytes()
    # best-of-pair: exactly one flag per run of equal (read_a, read_b), on the max
    t = 0
    while t < len(recs):
        u = t
        while u < len(recs) and recs[u][:2] == recs[t][:2]:
            u += 1
        run = r1[t:u]
        valid = [v for v in range(u - t) if not run[v]["status"] & oracle.STATUS_INVALID_SEED]
        flags = [v for v in range(u - t) if run[v]["status"] & oracle.STATUS_BEST_OF_PAIR]
        if valid:
            top = max(int(run[v]["score"]) for v in valid)
            assert flags == [min(v for v in valid if int(run[v]["score"]) == top)]
        else:
            assert flags == []
        t = u


def test_best_of_pair_definition_on_multi_seed_pairs():
    """The numpy statement of the best-of-pair flag (used on whole GPU batches)
    agrees with the oracle's flags on pairs with many seeds (the all-seed
    option of Sec. 5)."""
    import workloads
    from pair_flags import expected_best_of_pair
    w = workloads.generate("c2_allseeds_300k")
    g = workloads.pair_groups(w.pairs)
    many = np.flatnonzero(np.diff(g) >= 4)[:40]
    sub = np.concatenate([w.pairs[g[i]:g[i + 1]] for i in many])
    res = oracle.xdrop_batch(w.reads, w.offsets, sub.view(oracle.PAIR_DTYPE), 17, 1, -1, -1, 7)
    flags = (res["status"] & oracle.STATUS_BEST_OF_PAIR) != 0
    assert flags.sum() == len(many)
    assert np.array_equal(flags, expected_best_of_pair(sub, res))
