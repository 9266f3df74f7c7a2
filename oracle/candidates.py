"""Oracle for candidate-pair generation: plain numpy, test infrastructure.

Only the test suite and ``bench.py``'s CPU-baseline leg may import this module;
it shares no code with the CUDA path.  It computes, step by step, what diBELLA
does before alignment:

* Sec. 3 (k-mer analysis): every k-mer occurrence of every read, taken in its
  canonical orientation (the smaller 2-bit code of the k-mer and its reverse
  complement, A<C<G<T), counted over all occurrences;
* Sec. 3-4 (reliable k-mers): a k-mer is retained when its multiplicity lies in
  [mult_lo, mult_hi];
* Sec. 8 (overlap detection, Algorithm 1): every pair of distinct reads that
  share a retained k-mer, once per pair of occurrences, with the occurrence
  positions and the strand (1 when the two occurrences have opposite
  orientations);
* Sec. 8 (seed constraints) and Sec. 5 (seed options): per read pair, the
  occurrence pairs sorted by (pos_a, pos_b, strand); the first is seed 0 and
  each next seed is the first whose pos_a is at least min_seed_gap (0 = k) past
  the previous seed's, up to max_seeds.

The readings this takes where the paper is silent (A<C<G<T, odd k so that no
k-mer is its own reverse complement, read_a < read_b, orientation of a k-mer
whose code equals its reverse complement's taken as forward) are the ones the
workload generator states.  Records come out sorted by (read_a, read_b, seed_id)
in the ABI's 24-byte pair layout.
"""

from __future__ import annotations

import numpy as np

from . import PAIR_DTYPE

_CODE = np.full(256, 255, dtype=np.uint8)
for _i, _c in enumerate(b"ACGT"):
    _CODE[_c] = _i
    _CODE[ord(chr(_c).lower())] = _i


def kmer_instances(ascii: np.ndarray, offsets: np.ndarray, k: int):
    """Every k-mer occurrence: (canonical code, read id, position, orientation)."""
    if not 1 <= k <= 32:
        raise ValueError("k in 1..32")
    canon, rid, pos, orient = [], [], [], []
    mask = np.uint64((1 << (2 * k)) - 1) if k < 32 else np.uint64(0xFFFFFFFFFFFFFFFF)
    for r in range(len(offsets) - 1):
        b = _CODE[np.asarray(ascii[offsets[r]:offsets[r + 1]], dtype=np.uint8)].astype(np.uint64)
        n = len(b) - k + 1
        if n <= 0:
            continue
        fw = np.zeros(n, dtype=np.uint64)
        rc = np.zeros(n, dtype=np.uint64)
        for t in range(k):  # base t of the k-mer: most significant in fw, least in rc
            fw = (fw << np.uint64(2)) | b[t:t + n]
            rc = rc | ((np.uint64(3) - b[t:t + n]) << np.uint64(2 * t))
        fw &= mask
        canon.append(np.minimum(fw, rc))
        orient.append((fw > rc).astype(np.uint8))
        rid.append(np.full(n, r, dtype=np.uint32))
        pos.append(np.arange(n, dtype=np.uint32))
    if not canon:
        z = np.zeros(0, dtype=np.uint64)
        return z, z.astype(np.uint32), z.astype(np.uint32), z.astype(np.uint8)
    return np.concatenate(canon), np.concatenate(rid), np.concatenate(pos), np.concatenate(orient)


def candidate_pairs(ascii: np.ndarray, offsets: np.ndarray, k: int, mult_lo: int, mult_hi: int,
                    max_seeds: int, min_seed_gap: int = 0):
    """Seed records of every candidate pair, and (instances, retained k-mers,
    candidate pairs, occurrence pairs)."""
    canon, rid, pos, orient = kmer_instances(ascii, offsets, k)
    order = np.lexsort((orient, pos, rid, canon))  # by k-mer, then read, position
    canon, rid, pos, orient = canon[order], rid[order], pos[order], orient[order]
    starts = np.flatnonzero(np.concatenate([[True], canon[1:] != canon[:-1]])) if len(canon) else np.zeros(0, int)
    ends = np.concatenate([starts[1:], [len(canon)]]).astype(np.int64)
    mult = ends - starts
    keep = (mult >= mult_lo) & (mult <= mult_hi)
    ra, rb, pa, pb, st = [], [], [], [], []
    for s, e in zip(starts[keep], ends[keep]):
        for x in range(s, e):
            for y in range(x + 1, e):
                if rid[x] == rid[y]:
                    continue
                ra.append(rid[x]); rb.append(rid[y]); pa.append(pos[x]); pb.append(pos[y])
                st.append(orient[x] ^ orient[y])
    ra, rb, pa, pb, st = (np.array(v, dtype=np.int64) for v in (ra, rb, pa, pb, st))
    o = np.lexsort((st, pb, pa, rb, ra))
    ra, rb, pa, pb, st = ra[o], rb[o], pa[o], pb[o], st[o]
    gap = min_seed_gap if min_seed_gap > 0 else k
    out = []
    n_cand = 0
    u = 0
    while u < len(ra):
        v = u + 1
        while v < len(ra) and ra[v] == ra[u] and rb[v] == rb[u]:
            v += 1
        n_cand += 1
        taken, last = 0, None
        for t in range(u, v):
            if taken >= max_seeds:
                break
            if taken > 0 and pa[t] < last + gap:
                continue
            out.append((ra[t], rb[t], pa[t], pb[t], st[t], taken))
            last = pa[t]
            taken += 1
        u = v
    rec = np.zeros(len(out), dtype=PAIR_DTYPE)
    if out:
        a = np.array(out, dtype=np.int64)
        rec["read_a"], rec["read_b"], rec["pos_a"] = a[:, 0], a[:, 1], a[:, 2]
        rec["pos_b"], rec["strand"], rec["seed_id"] = a[:, 3], a[:, 4], a[:, 5]
    stats = {"instances": int(len(canon)), "retained_kmers": int(keep.sum()), "candidate_pairs": n_cand,
             "occurrence_pairs": int(len(ra))}
    return rec, stats
