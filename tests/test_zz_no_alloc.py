"""The no-allocation entry point, dibella_xdrop_batch_noalloc.

It is meant for callers that may not allocate device memory themselves (a
runtime whose pool owns the GPU's memory, a latency-critical loop, plug-in
code).  It must give exactly what dibella_xdrop_batch gives on the same
inputs, call after call, although every call reuses the library's one fixed
scratch array.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes on its own.
"""

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_noalloc_matches_batch_on_two_calls_in_a_row():
    import torch
    import paper_2001_10049_gb300 as dib

    w = workloads.generate("c1_tiny")
    store = dib.ReadStore.from_ascii(w.reads, w.offsets)
    pairs = w.pairs[:1000]
    n = len(pairs)
    ref_al = dib.Aligner(store, n, k=17)
    dev_pairs = torch.from_numpy(pairs.view(np.uint8).reshape(n, 24).copy()).cuda()
    for X in (7, 25):  # two calls in a row, different work in the shared scratch
        sc = dib.Scoring(1, -1, -1, X)
        expected = ref_al.align(pairs, sc)
        out = torch.full((n, 40), 0xAB, dtype=torch.uint8, device="cuda")
        dib.dibella_xdrop_batch_noalloc(store.words, store.word_offsets, store.lengths, store.n_reads,
                                        dev_pairs, n, 17, sc, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(-1).view(dib.RESULT_DTYPE)
        # integer results: the tolerance is zero
        assert got.tobytes() == expected.tobytes(), "X=%d" % X


def test_noalloc_rejects_oversize_batches():
    import paper_2001_10049_gb300 as dib

    with pytest.raises(dib.DibellaError) as e:
        dib.dibella_xdrop_batch_noalloc(0, 0, 0, 0, 0, dib.NOALLOC_MAX_PAIRS + 1, 17,
                                        dib.Scoring(1, -1, -1, 7), 0, stream=0)
    assert e.value.code == dib.DIBELLA_ENOMEM
    assert "maximum" in str(e.value)


def test_noalloc_band_beyond_its_scratch_is_reported():
    """The fixed scratch holds bands of at most NOALLOC_MAX_BAND cells.  Two
    identical 10 kb reads seeded at their first base at X = infinity keep the
    whole antidiagonal live (about 10,000 cells), so the no-allocation call
    must flag that seed's band overflow and leave its fields zero, while the
    entry point with a workspace sized for the read length aligns it in full
    (length x match)."""
    import random

    import torch
    import paper_2001_10049_gb300 as dib

    rng = random.Random(5)
    read = "".join(rng.choice("ACGT") for _ in range(10000))
    ascii = np.frombuffer((read * 3).encode(), dtype=np.uint8)
    offs = np.arange(4, dtype=np.int64) * len(read)
    pairs = np.zeros(2, dtype=dib.PAIR_DTYPE)  # two candidate pairs, (0, 1) and (0, 2)
    pairs["read_a"] = 0
    pairs["read_b"] = [1, 2]
    pairs[1]["pos_a"] = pairs[1]["pos_b"] = 4990  # both extensions 5 kb: within the limit
    store = dib.ReadStore.from_ascii(ascii, offs)
    sc = dib.Scoring(1, -1, -1, dib.XDROP_INF)
    sized = dib.Aligner(store, 2, k=17).align(pairs, sc)
    assert list(sized["score"]) == [len(read), len(read)] and not (sized["status"] & dib.RES_BAND_OVERFLOW).any()
    dev_pairs = torch.from_numpy(pairs.view(np.uint8).reshape(2, 24).copy()).cuda()
    for _ in range(2):
        out = torch.full((2, 40), 0xAB, dtype=torch.uint8, device="cuda")
        dib.dibella_xdrop_batch_noalloc(store.words, store.word_offsets, store.lengths, store.n_reads,
                                        dev_pairs, 2, 17, sc, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(-1).view(dib.RESULT_DTYPE)
        assert got[0]["status"] & dib.RES_BAND_OVERFLOW
        assert got[0]["score"] == 0 and got[0]["cells"] == 0
        assert got[1].tobytes() == sized[1].tobytes()
