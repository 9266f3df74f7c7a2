"""The best-of-pair flag written from its definition (numpy only): used to pin
the oracle's flags and to check the CUDA path's on whole batches."""

import numpy as np

import workloads


def expected_best_of_pair(pairs, res):
    """Best-of-pair flags implied by the scores: in each run of records with the
    same (read_a, read_b), the valid record with the highest score, earliest on
    ties."""
    g = workloads.pair_groups(pairs)
    valid = (res["status"] & 2) == 0
    score = np.where(valid, res["score"].astype(np.int64), np.iinfo(np.int64).min)
    top = np.repeat(np.maximum.reduceat(score, g[:-1]), np.diff(g))
    cand = valid & (score == top)
    run = np.repeat(np.arange(len(g) - 1), np.diff(g))
    idx = np.flatnonzero(cand)
    first = idx[np.concatenate([[True], run[idx][1:] != run[idx][:-1]])] if len(idx) else idx
    flags = np.zeros(len(pairs), dtype=bool)
    flags[first] = True
    return flags

