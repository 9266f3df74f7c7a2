"""Whole-genome alignment in bounded pieces: candidate pairs generated on the
GPU, kept on the host, and streamed back through the X-drop kernels in chunks.

This is the shape of diBELLA's pipeline for inputs larger than one phase can
hold (Sec. 4: memory-limited streaming phases; Sec. 6-7: k-mer counting in
passes; Sec. 8-9: candidate pairs, then alignment of every pair), on one GPU:

1. dibella_candidate_pairs_parts counts the k-mers of the resident read store
   in hash-partitioned passes and writes every seed record (device memory);
2. the records are copied to host memory (the device buffers are released);
3. windows of whole candidate pairs are copied into pinned host buffers and
   aligned by dibella_xdrop_stream, which moves chunks of ``chunk_pairs``
   records through two device slots (copies of one chunk overlap the kernels
   of the other) with the store resident in HBM;
4. per window only summaries are kept, plus the records and results of the
   read ranges the caller asks for.

No alignment or counting arithmetic happens here; this module moves bytes and
keeps time.
"""

from __future__ import annotations

import time

import numpy as np


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the dibella X-drop path needs a CUDA GPU; none is visible")
    return torch


def pair_boundary(read_a: np.ndarray, read_b: np.ndarray, end: int, start: int) -> int:
    """The largest e <= end, e > start, at which no candidate pair is split."""
    n = len(read_a)
    if end >= n:
        return n
    e = end
    while e > start and read_a[e] == read_a[e - 1] and read_b[e] == read_b[e - 1]:
        e -= 1
    if e == start:
        raise ValueError("one candidate pair has more seed records than a window holds")
    return e


def align_all_candidates(store, scoring, k: int = 17, mult_lo: int = 2, mult_hi: int = 12, max_seeds: int = 1,
                         min_seed_gap: int = 0, n_parts: int = 8, occ_pair_capacity: int | None = None,
                         pairs_capacity: int | None = None, max_read_len: int | None = None,
                         chunk_pairs: int = 4_000_000, window_pairs: int = 32_000_000, keep_ranges=(),
                         sched=None, log=None) -> dict:
    """Candidate pairs of every read of ``store`` and the X-drop alignment of
    each of their seed records.

    Returns a dict with the candidate counts, timings (seconds) of the
    candidate call, the copy to host and the streamed alignment, the number of
    records, chunks and evaluated cells, status and score summaries, and under
    "kept" one (records, results) pair of numpy arrays per requested read range
    (half-open read_a ranges)."""
    from . import (PAIR_DTYPE, RESULT_DTYPE, Scoring, dibella_staging_bytes, dibella_xdrop_stream,
                   dibella_xdrop_workspace_bytes)
    torch = _torch()
    dev = store.words.device
    sc = scoring if isinstance(scoring, Scoring) else Scoring(*scoring)
    say = log or (lambda *a: None)

    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    recs_dev, cstats = store.candidate_pairs_parts(k=k, mult_lo=mult_lo, mult_hi=mult_hi, max_seeds=max_seeds,
                                                   min_seed_gap=min_seed_gap, n_parts=n_parts,
                                                   occ_pair_capacity=occ_pair_capacity,
                                                   pairs_capacity=pairs_capacity, max_read_len=max_read_len,
                                                   to_host=False)
    t_cand = time.perf_counter() - t0
    say("candidates: %s in %.1f s" % (cstats, t_cand))
    t0 = time.perf_counter()
    pairs = recs_dev.cpu().numpy().reshape(-1).view(PAIR_DTYPE)
    del recs_dev
    torch.cuda.empty_cache()
    t_host = time.perf_counter() - t0
    n = len(pairs)
    say("%d seed records on the host in %.1f s" % (n, t_host))

    ra, rb = pairs["read_a"], pairs["read_b"]
    spans = [(int(np.searchsorted(ra, lo, "left")), int(np.searchsorted(ra, hi, "left"))) for lo, hi in keep_ranges]
    kept = [(pairs[a:b].copy(), np.zeros(b - a, dtype=RESULT_DTYPE)) for a, b in spans]

    chunk = max(1, min(chunk_pairs, n))
    window = max(chunk, min(window_pairs, n))
    wsb = dibella_xdrop_workspace_bytes(chunk, max(store.max_len, 1))
    staging = [torch.empty(dibella_staging_bytes(chunk), dtype=torch.uint8, device=dev) for _ in range(2)]
    ws = [torch.empty(wsb, dtype=torch.uint8, device=dev) for _ in range(2)]
    streams = [torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)]
    hp = torch.empty((window, 24), dtype=torch.uint8).pin_memory()
    hr = torch.empty((window, 40), dtype=torch.uint8).pin_memory()
    hp_np = hp.numpy().reshape(-1).view(PAIR_DTYPE)
    hr_np = hr.numpy().reshape(-1).view(RESULT_DTYPE)

    cells = 0
    n_chunks = 0
    status = {}
    score_sum = 0
    best_of_pair = 0
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    s = 0
    while s < n:
        e = pair_boundary(ra, rb, s + window, s)
        m = e - s
        hp_np[:m] = pairs[s:e]
        n_chunks += dibella_xdrop_stream(store.words, store.word_offsets, store.lengths, store.n_reads, hp, m, chunk,
                                         k, sc, hr, staging, ws, wsb, streams, sched)
        res = hr_np[:m]
        cells += int(res["cells"].sum())
        score_sum += int(res["score"].sum())
        best_of_pair += int(((res["status"] & 4) != 0).sum())
        for v, c in zip(*np.unique(res["status"], return_counts=True)):
            status[int(v)] = status.get(int(v), 0) + int(c)
        for (a, b), (_, kr) in zip(spans, kept):
            lo, hi = max(a, s), min(b, e)
            if lo < hi:
                kr[lo - a:hi - a] = res[lo - s:hi - s]
        s = e
        say("aligned %d / %d records, %.1f s" % (s, n, time.perf_counter() - t0))
    t_stream = time.perf_counter() - t0
    return {"candidates": cstats, "records": n, "t_candidates": t_cand, "t_to_host": t_host, "t_stream": t_stream,
            "chunks": n_chunks, "chunk_pairs": chunk, "window_pairs": window, "cells": cells, "status": status,
            "score_sum": score_sum, "best_of_pair": best_of_pair, "kept": kept}
