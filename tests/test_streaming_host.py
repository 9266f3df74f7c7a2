"""Host logic of the whole-genome streaming helper: window ends never split the
seed records of one candidate pair."""

import numpy as np
import pytest

from paper_2001_10049_gb300.streaming import pair_boundary


def test_window_ends_fall_between_candidate_pairs():
    ra = np.array([0, 0, 0, 1, 1, 2, 3, 3, 3, 3], dtype=np.uint32)
    rb = np.array([5, 5, 6, 2, 2, 9, 4, 4, 4, 7], dtype=np.uint32)
    with pytest.raises(ValueError):
        pair_boundary(ra, rb, 1, 0)                  # a window shorter than the first pair
    assert pair_boundary(ra, rb, 2, 0) == 2          # (0,5) ends at 2
    assert pair_boundary(ra, rb, 4, 2) == 3          # (1,2) spans 3..4: back to 3
    assert pair_boundary(ra, rb, 8, 5) == 6          # (3,4) spans 6..8: back to 6
    assert pair_boundary(ra, rb, 100, 3) == 10       # past the end: everything
    with pytest.raises(ValueError):
        pair_boundary(ra, rb, 7, 6)                  # one pair longer than the window


def test_windows_cover_every_record_once():
    rng = np.random.default_rng(3)
    sizes = rng.integers(1, 6, size=500)
    ra = np.repeat(np.arange(500, dtype=np.uint32) // 3, sizes)
    rb = np.repeat(np.arange(500, dtype=np.uint32), sizes)
    n, s, seen = len(ra), 0, 0
    while s < n:
        e = pair_boundary(ra, rb, s + 37, s)
        assert e > s and (e == n or (ra[e], rb[e]) != (ra[e - 1], rb[e - 1]))
        seen += e - s
        s = e
    assert seen == n
