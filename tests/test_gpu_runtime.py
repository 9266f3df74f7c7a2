"""The batching runtime around the kernels: autotuner, chunked streaming and the
continuous-batching serving loop.  None of them may change a result."""

import numpy as np
import pytest

import workloads
from gpu_util import assert_same, oracle_align

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1():
    return workloads.generate("c1_tiny")


@pytest.fixture(scope="module")
def store(c1):
    import paper_2001_10049_gb300 as dib
    return dib.ReadStore.from_ascii(c1.reads, c1.offsets)


def test_autotune_returns_valid_schedule_and_exact_results(c1, store):
    import paper_2001_10049_gb300 as dib
    al = dib.Aligner(store, len(c1.pairs), k=17)
    al.upload_pairs(c1.pairs)
    sc = dib.Scoring(1, -1, -1, 25)
    best, ms, tried = dib.dibella_autotune(store.words, store.word_offsets, store.lengths, store.n_reads, al.pairs,
                                           len(c1.pairs), 17, sc, al.results, al.workspace, al.workspace_bytes,
                                           repeats=1)
    assert tried >= 10 and ms > 0
    d = best.as_dict()
    assert d["narrow_band_cap"] in (32, 48, 64) and d["wide_slots"] in (0, 8, 16, 24, 32)
    exp = oracle_align(c1.reads, c1.offsets, c1.pairs, 17, (1, -1, -1, 25))
    assert_same(al.results_host(len(c1.pairs)), exp, "after autotune")
    assert_same(al.align(c1.pairs, sc, sched=best), exp, "tuned schedule")


@pytest.mark.parametrize("chunk", [1, 7, 100, 5000])
def test_stream_equals_one_batch(c1, store, chunk):
    import torch
    import paper_2001_10049_gb300 as dib
    pairs = c1.pairs
    n = len(pairs)
    sc = dib.Scoring(1, -1, -1, 7)
    ref = dib.Aligner(store, n, k=17).align(pairs, sc)
    chunk_eff = chunk  # C1 pairs have one seed each, so any chunk size holds a whole pair
    host_pairs = torch.from_numpy(pairs.view(np.uint8).reshape(n, 24).copy()).pin_memory()
    host_res = torch.zeros((n, 40), dtype=torch.uint8).pin_memory()
    wsb = dib.dibella_xdrop_workspace_bytes(chunk_eff, store.max_len)
    staging = [torch.empty(dib.dibella_staging_bytes(chunk_eff), dtype=torch.uint8, device="cuda") for _ in range(2)]
    ws = [torch.empty(wsb, dtype=torch.uint8, device="cuda") for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    n_chunks = dib.dibella_xdrop_stream(store.words, store.word_offsets, store.lengths, store.n_reads, host_pairs, n,
                                        chunk_eff, 17, sc, host_res, staging, ws, wsb, streams)
    got = host_res.numpy().reshape(-1).view(dib.RESULT_DTYPE)
    assert got.tobytes() == ref.tobytes()
    assert n_chunks >= (n + chunk_eff - 1) // chunk_eff


def test_stream_keeps_candidate_pairs_whole():
    """Two-seed pairs: a chunk end never separates the seeds of one pair, so the
    best-seed flags equal those of one batch."""
    import torch
    import paper_2001_10049_gb300 as dib
    w = workloads.generate("c2_ecoli", genome_len=200_000, coverage=10.0)
    pairs = w.pairs[:3000]
    n = len(pairs)
    st = dib.ReadStore.from_ascii(w.reads, w.offsets)
    sc = dib.Scoring(1, -1, -1, 7)
    ref = dib.Aligner(st, n, k=17).align(pairs, sc)
    host_pairs = torch.from_numpy(pairs.view(np.uint8).reshape(n, 24).copy()).pin_memory()
    host_res = torch.zeros((n, 40), dtype=torch.uint8).pin_memory()
    chunk = 97
    wsb = dib.dibella_xdrop_workspace_bytes(chunk, st.max_len)
    staging = [torch.empty(dib.dibella_staging_bytes(chunk), dtype=torch.uint8, device="cuda") for _ in range(2)]
    ws = [torch.empty(wsb, dtype=torch.uint8, device="cuda") for _ in range(2)]
    dib.dibella_xdrop_stream(st.words, st.word_offsets, st.lengths, st.n_reads, host_pairs, n, chunk, 17, sc,
                             host_res, staging, ws, wsb, [torch.cuda.Stream(), torch.cuda.Stream()])
    assert host_res.numpy().reshape(-1).view(dib.RESULT_DTYPE).tobytes() == ref.tobytes()


@pytest.mark.parametrize("rate", [0.0, 400.0])
def test_serving_result_alone_equals_in_mix(c1, store, rate):
    """Requests served concurrently (merged into batches, overlapping on several
    streams) get exactly the result each gets alone."""
    import paper_2001_10049_gb300 as dib
    from paper_2001_10049_gb300.serving import Request, Server
    specs = workloads.serving_requests(c1.pairs, 40, rate_per_s=max(rate, 1.0), seed=3, max_size=200)
    reqs = [Request(i, 0.0 if rate == 0 else t, x, c1.pairs[idx]) for i, (t, x, idx) in enumerate(specs)]
    srv = Server(store, k=17, arena_bytes=1 << 28, max_batch=256, n_streams=4)
    stats = srv.run(reqs, timeout_s=120)
    assert stats["requests"] == len(reqs) and all(r.done is not None for r in reqs)
    if rate == 0:
        assert stats["batches"] < len(reqs)  # requests were merged
    alone = dib.Aligner(store, 512, k=17)
    for r in reqs:
        exp = alone.align(r.pairs, dib.Scoring(1, -1, -1, r.xdrop))
        assert r.result.tobytes() == exp.tobytes(), "request %d differs in the mix" % r.rid


def test_serving_admission_by_memory(c1, store):
    """An arena that holds only one batch at a time still serves everything,
    one batch in flight at a time."""
    from paper_2001_10049_gb300.serving import Request, Server
    probe = Server(store, k=17, arena_bytes=1 << 28, max_batch=64, n_streams=4)
    one = probe.batch_bytes(64)
    srv = Server(store, k=17, arena_bytes=one + 4096, max_batch=64, n_streams=4)
    specs = workloads.serving_requests(c1.pairs, 12, rate_per_s=1.0, seed=4, max_size=100)
    reqs = [Request(i, 0.0, x, c1.pairs[idx]) for i, (t, x, idx) in enumerate(specs)]
    stats = srv.run(reqs, timeout_s=120)
    assert stats["max_inflight"] == 1
    assert all(r.done is not None for r in reqs)


def test_serving_c5_shaped_requests_match_whole_batches():
    """C5's request mix on the E. coli-sized store: Poisson arrivals of requests
    of 1..4096 candidate pairs (log-uniform) with X drawn from {7, 25, 50},
    admitted by device memory and overlapping on several streams.  Each served
    result equals the same records of the whole batch aligned at that X in one
    call (whole candidate pairs, so even the best-seed flags agree); the whole
    batches are checked record by record against the oracle in
    test_gpu_full_parity.py."""
    import paper_2001_10049_gb300 as dib
    from paper_2001_10049_gb300.serving import Request, Server
    w = workloads.generate("c2_ecoli")
    st = dib.ReadStore.from_ascii(w.reads, w.offsets)
    specs = workloads.serving_requests(w.pairs, 48, rate_per_s=300.0, seed=45)
    reqs = [Request(i, t, x, w.pairs[idx]) for i, (t, x, idx) in enumerate(specs)]
    srv = Server(st, k=17, arena_bytes=2 << 30, max_batch=65536, n_streams=8)
    stats = srv.run(reqs, timeout_s=600)
    assert stats["requests"] == len(reqs) and all(r.done is not None for r in reqs)
    assert stats["max_inflight"] > 1  # batches overlapped on the device
    al = dib.Aligner(st, len(w.pairs), k=17)
    for X in sorted({x for _, x, _ in specs}):
        whole = al.align(w.pairs, dib.Scoring(1, -1, -1, X))
        for r, (_, x, idx) in zip(reqs, specs):
            if x == X:
                assert r.result.tobytes() == whole[idx].tobytes(), "request %d (X=%d) differs" % (r.rid, X)


def test_warp_clock_of_a_launch(c1, store):
    """The per-warp clock of one launch: every warp of the clocked launch
    reports a start and an end, in order; other launches are not clocked."""
    import paper_2001_10049_gb300 as dib
    al = dib.Aligner(store, len(c1.pairs), k=17)
    dib.dibella_enable_warp_clock(1)  # the narrow form
    try:
        ref = al.align(c1.pairs, dib.Scoring(1, -1, -1, 7))
        wc = dib.dibella_warp_clock()
    finally:
        dib.dibella_enable_warp_clock(0)
    assert len(wc) > 0 and np.all(wc[:, 1] >= wc[:, 0]) and np.all(wc[:, 0] > 0)
    assert al.align(c1.pairs, dib.Scoring(1, -1, -1, 7)).tobytes() == ref.tobytes()  # clocking changes nothing
