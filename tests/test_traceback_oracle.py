"""Pins for the oracle's traceback (the edits of the best alignment, diBELLA
Sec. 1-2), each against something other than the oracle:

* hand-worked columns of the golden extensions and seeds;
* X = infinity: every cell is live and the band is the whole matrix, so the
  columns must equal those of a separate full-matrix dynamic program traced
  back here with the same move order (diagonal, step in a, step in b);
* at any X, the columns must consume exactly the aligned ranges and add up,
  rescored here against the sequences, to the reported score.
"""

import os
import random

import numpy as np
import pytest

import oracle
from test_oracle_pins import GOLDEN, INF, SCHEMES, full_dp_extension, mutate, rand_seq, revcomp


def _rows(kind):
    out = []
    with open(os.path.join(GOLDEN, "xdrop_traceback_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if line.startswith(kind + " "):
                left, right = line.split("|")
                out.append((left.split()[1:], right.strip()))
    return out


@pytest.mark.parametrize("row", _rows("ext"), ids=lambda r: r[0][0])
def test_golden_extension_columns(row):
    (name, a, b, M, S, G, X), want = row
    a = "" if a == "-" else a
    b = "" if b == "-" else b
    assert oracle.extend_columns(a, b, int(M), int(S), int(G), int(X)) == ("" if want == "-" else want), name


@pytest.mark.parametrize("row", _rows("seed"), ids=lambda r: r[0][0])
def test_golden_seed_cigars(row):
    (name, A, B, pa, pb, strand, k, M, S, G, X), want = row
    ascii = np.frombuffer((A + B).encode(), dtype=np.uint8)
    offs = np.array([0, len(A), len(A) + len(B)], dtype=np.int64)
    pair = np.zeros(1, dtype=oracle.PAIR_DTYPE)
    pair["read_a"], pair["read_b"], pair["pos_a"], pair["pos_b"], pair["strand"] = 0, 1, int(pa), int(pb), int(strand)
    res, ops, n_ops = oracle.traceback_batch(ascii, offs, pair, int(k), int(M), int(S), int(G), int(X), 16)
    assert oracle.cigar_string(ops[0, :max(n_ops[0], 0)]) == ("" if want == "-" else want), name


def full_dp_columns(a, b, match, mismatch, gap):
    """Full-matrix DP (every cell, no pruning) traced back from the full-DP best
    cell (smallest i+j, then smallest i) with the move order diagonal, step in
    a, step in b."""
    m, n = len(a), len(b)
    NEG = -(1 << 60)
    F = [[NEG] * (n + 1) for _ in range(m + 1)]
    mv = [[None] * (n + 1) for _ in range(m + 1)]
    F[0][0] = 0
    for i in range(m + 1):
        for j in range(n + 1):
            if i == 0 and j == 0:
                continue
            best, how = NEG, None
            if i and j and F[i - 1][j - 1] + (match if a[i - 1] == b[j - 1] else mismatch) > best:
                best, how = F[i - 1][j - 1] + (match if a[i - 1] == b[j - 1] else mismatch), "diag"
            if i and F[i - 1][j] + gap > best:
                best, how = F[i - 1][j] + gap, "a"
            if j and F[i][j - 1] + gap > best:
                best, how = F[i][j - 1] + gap, "b"
            F[i][j], mv[i][j] = best, how
    _, i, j = full_dp_extension(a, b, match, mismatch, gap)
    cols = []
    while i or j:
        how = mv[i][j]
        if how == "diag":
            cols.append("=" if a[i - 1] == b[j - 1] else "X")
            i, j = i - 1, j - 1
        elif how == "a":
            cols.append("D")
            i -= 1
        else:
            cols.append("I")
            j -= 1
    return "".join(reversed(cols))


def rescore(cols, a, b, match, mismatch, gap):
    """Score of the columns walked over a and b from their starts; also the
    characters of each consumed."""
    i = j = s = 0
    for c in cols:
        if c in "=X":
            assert (a[i] == b[j]) == (c == "="), "column letter disagrees with the bases"
            s += match if c == "=" else mismatch
            i, j = i + 1, j + 1
        elif c == "D":
            s, i = s + gap, i + 1
        else:
            assert c == "I"
            s, j = s + gap, j + 1
    return s, i, j


@pytest.mark.parametrize("scheme", SCHEMES)
def test_infinite_x_columns_equal_full_dp_traceback(scheme):
    M, S, G = scheme
    rng = random.Random(500 + 13 * M - S)
    for trial in range(40):
        a = rand_seq(rng, rng.randint(0, 40))
        b = mutate(rng, a, 0.3) if trial % 2 else rand_seq(rng, rng.randint(0, 40))
        assert oracle.extend_columns(a, b, M, S, G, INF) == full_dp_columns(a, b, M, S, G), (a, b)


def test_columns_rescore_to_the_best_at_finite_x():
    rng = random.Random(77)
    for trial in range(300):
        M, S, G = SCHEMES[trial % len(SCHEMES)]
        a = rand_seq(rng, rng.randint(0, 300))
        b = mutate(rng, a, rng.choice([0.05, 0.15, 0.3]))
        X = rng.choice([0, 1, 3, 7, 25, 50])
        best, i_end, j_end, _, _ = oracle.extend(a, b, M, S, G, X)
        cols = oracle.extend_columns(a, b, M, S, G, X)
        assert rescore(cols, a, b, M, S, G) == (best, i_end, j_end), (trial, X)


def test_seed_batch_columns_rescore_and_match_the_batch():
    rng = random.Random(9)
    reads, recs = [], []
    for t in range(40):
        base = rand_seq(rng, rng.randint(60, 400))
        a = mutate(rng, base, 0.12)
        b = mutate(rng, base, 0.12)
        strand = t % 2
        if strand:
            b = revcomp(b)
        reads += [a, b]
        k = 5
        pa = rng.randint(0, len(a) - k)
        bp = revcomp(b) if strand else b
        pbp = rng.randint(0, len(bp) - k)
        pb = len(b) - pbp - k if strand else pbp
        recs.append((2 * t, 2 * t + 1, pa, pb, strand))
    recs.append((0, 1, 10 ** 6, 0, 0))  # an invalid seed
    ascii = np.frombuffer("".join(reads).encode(), dtype=np.uint8)
    offs = np.cumsum([0] + [len(r) for r in reads]).astype(np.int64)
    pairs = np.zeros(len(recs), dtype=oracle.PAIR_DTYPE)
    for t, (ra, rb, pa, pb, st) in enumerate(recs):
        pairs[t]["read_a"], pairs[t]["read_b"], pairs[t]["pos_a"], pairs[t]["pos_b"], pairs[t]["strand"] = \
            ra, rb, pa, pb, st
        pairs[t]["seed_id"] = t
    M, S, G, X, k = 1, -1, -1, 7, 5
    res, ops, n_ops = oracle.traceback_batch(ascii, offs, pairs, k, M, S, G, X, 1024)
    plain = oracle.xdrop_batch(ascii, offs, pairs, k, M, S, G, X, n_threads=1)
    plain["status"] &= ~oracle.STATUS_BEST_OF_PAIR
    assert res.tobytes() == plain.tobytes()
    for t, (ra, rb, pa, pb, st) in enumerate(recs):
        if res[t]["status"] & oracle.STATUS_INVALID_SEED:
            assert n_ops[t] == 0
            continue
        A, B = reads[ra], reads[rb]
        Bp = revcomp(B) if st else B
        r = res[t]
        bb = len(B) - int(r["end_b"]) if st else int(r["begin_b"])  # begin in B'
        cols = "".join(oracle.CIGAR_OPS[int(w) & 15] * (int(w) >> 4) for w in ops[t, :n_ops[t]])
        s, i, j = rescore(cols, A[int(r["begin_a"]):], Bp[bb:], M, S, G)
        assert (s, i, j) == (int(r["score"]), int(r["end_a"]) - int(r["begin_a"]),
                             int(r["end_b"]) - int(r["begin_b"])), t
    # too small a capacity: -1, nothing claimed
    _, _, few = oracle.traceback_batch(ascii, offs, pairs, k, M, S, G, X, 1)
    assert all(v == -1 or v == n for v, n in zip(few, n_ops)) and (few == -1).any()


def test_gpu_traceback_entry_points_validate_arguments_on_the_host():
    import paper_2001_10049_gb300 as dib
    assert dib.dibella_traceback_workspace_bytes(4, 100, 64) == 4 * 1536  # 3 x 102 x 4 + 64 x 4, to 256 B
    for bad in ((0, 100, 64), (4, -1, 64), (4, 100, 1), (4, (1 << 24) + 1, 64), ((1 << 24) + 1, 100, 64)):
        with pytest.raises(dib.DibellaError):
            dib.dibella_traceback_workspace_bytes(*bad)
    ws = 1 << 20  # a fake, aligned device address: every call below fails before touching it
    sc = dib.Scoring(1, -1, -1, 7)
    good = dict(n_reads=2, max_len=100, n_pairs=3, k=17, sc=sc, ops_per_seed=8, lanes=4, moves=64, ws_bytes=1 << 30)
    cases = [dict(good, k=0), dict(good, k=33), dict(good, sc=dib.Scoring(0, -1, -1, 7)),
             dict(good, sc=dib.Scoring(1, 1, -1, 7)), dict(good, sc=dib.Scoring(1, -1, 0, 7)),
             dict(good, sc=dib.Scoring(1, -1, -1, -1)), dict(good, ops_per_seed=0), dict(good, lanes=0),
             dict(good, moves=1), dict(good, n_pairs=-1), dict(good, max_len=-1)]
    for c in cases:
        with pytest.raises(dib.DibellaError) as e:
            dib.dibella_xdrop_traceback(ws, ws, ws, c["n_reads"], c["max_len"], ws, c["n_pairs"], c["k"], c["sc"], ws,
                                        ws, c["ops_per_seed"], ws, c["lanes"], c["moves"], ws, c["ws_bytes"], stream=0)
        assert e.value.code == dib.DIBELLA_EINVAL
    with pytest.raises(dib.DibellaError) as e:  # a misaligned workspace
        dib.dibella_xdrop_traceback(ws, ws, ws, 2, 100, ws, 3, 17, sc, ws, ws, 8, ws, 4, 64, ws + 16, 1 << 30, stream=0)
    assert e.value.code == dib.DIBELLA_EINVAL
    with pytest.raises(dib.DibellaError) as e:  # too small a workspace
        dib.dibella_xdrop_traceback(ws, ws, ws, 2, 100, ws, 3, 17, sc, ws, ws, 8, ws, 4, 64, ws, 6143, stream=0)
    assert e.value.code == dib.DIBELLA_ENOMEM
