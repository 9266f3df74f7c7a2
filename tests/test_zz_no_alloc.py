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
