"""The repeat-rich workload (C4) end to end on the GPU: reads only from the
generator, candidate pairs from dibella_candidate_pairs_parts (hash-partitioned
k-mer passes, two-word occurrence-pair keys), every seed record streamed from
host memory through dibella_xdrop_stream in chunks, the read store resident.

The oracle's inputs never come from the GPU: the generator's own index (whole,
or restricted to read_a ranges) gives the seed records, which must equal the
GPU's byte for byte; the oracle aligns them and every compared result must be
identical.

* test_c4_rules_scaled: every rule of the configuration on a 0.8 Mb genome,
  every record checked.
* test_c4_full_size (runs only with DIBELLA_SLOW=1; about an hour on a
  GB300): the configured 100 Mb genome.  Read blocks play the part of chunks:
  all records of two blocks of at least 4M records each, and a seeded sample
  of records from a seeded 5% of the 2,000-read blocks (their seed records in
  full).  The oracle runs on the host cores while the GPU streams.
"""

import json
import os
import threading
import time

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import assert_same

pytestmark = pytest.mark.gpu

X = 15
K = 17


def _c4(genome_len, **over):
    scale = genome_len / 100_000_000
    return dict(genome_len=genome_len, repeat_families=max(1, int(round(200 * scale))),
                tandem_bases=int(1_000_000 * scale), **over)


def _stream(w, ranges, n_parts, chunk, window, max_read_len=None):
    import paper_2001_10049_gb300 as dib
    from paper_2001_10049_gb300.streaming import align_all_candidates
    store = dib.ReadStore.from_ascii(w.reads, w.offsets)
    p = w.params
    occ_cap = None
    return align_all_candidates(store, dib.Scoring(1, -1, -1, X), k=K, mult_lo=p["mult_lo"], mult_hi=p["mult_hi"],
                                max_seeds=p["max_seeds"], n_parts=n_parts, occ_pair_capacity=occ_cap,
                                max_read_len=max_read_len, chunk_pairs=chunk, window_pairs=window,
                                keep_ranges=ranges)


def test_c4_rules_scaled():
    import paper_2001_10049_gb300 as dib
    over = _c4(800_000)
    w = workloads.generate("c4_repeats", **over)
    out = _stream(w, [(0, w.n_reads)], n_parts=5, chunk=9_000, window=40_000, max_read_len=dib.DIBELLA_MAX_READ_LEN)
    recs, res = out["kept"][0]
    assert out["candidates"]["status"] == 0
    assert recs.tobytes() == w.pairs.view(recs.dtype).tobytes()  # the generator's index, byte for byte
    assert out["chunks"] >= len(w.pairs) // 9_000
    exp = oracle.xdrop_batch(w.reads, w.offsets, w.pairs.view(oracle.PAIR_DTYPE), K, 1, -1, -1, X)
    assert_same(res, exp, "c4 rules, 0.8 Mb")
    assert out["cells"] == int(exp["cells"].sum())


@pytest.mark.skipif(os.environ.get("DIBELLA_SLOW") != "1", reason="about an hour on a GB300; DIBELLA_SLOW=1")
def test_c4_full_size():
    report = {}
    t_all = time.time()
    w = workloads.generate("c4_repeats", pairs_mode=workloads.PAIRS_NONE, cache=False)
    n = w.n_reads
    report.update(reads=int(n), bases=int(len(w.reads)), t_generate=round(time.time() - t_all, 1))
    # Parity blocks: two full blocks (sized for >= 4M records each at this
    # workload's pair density) and a seeded 5% of the 2,000-read blocks.
    full = [(0, 1300), (n // 2, n // 2 + 2600)]
    B = 2000
    rng = np.random.default_rng(20240)
    cand = [b for b in range(n // B) if not any(lo < (b + 1) * B and b * B < hi for lo, hi in full)]
    picked = sorted(rng.choice(cand, size=max(1, int(round(0.05 * (n // B)))), replace=False).tolist())
    blocks = sorted(full + [(b * B, (b + 1) * B) for b in picked])
    report["blocks"] = blocks

    expected = {}

    def cpu_side():
        t0 = time.time()
        g = workloads.generate("c4_repeats", pairs_mode=workloads.PAIRS_RANGES, read_ranges=blocks, cache=False)
        expected["pairs"] = g.pairs
        expected["t_index"] = time.time() - t0
        ra = g.pairs["read_a"]
        res = {}
        t0 = time.time()
        for lo, hi in blocks:
            a, b = np.searchsorted(ra, lo), np.searchsorted(ra, hi)
            recs = g.pairs[a:b]
            if (lo, hi) in full:
                idx = np.arange(len(recs))
            else:  # a seeded sample of 1000 records of this block
                idx = np.sort(np.random.default_rng(lo).choice(len(recs), min(1000, len(recs)), replace=False))
            res[(lo, hi)] = (idx, oracle.xdrop_batch(g.reads, g.offsets, recs[idx].view(oracle.PAIR_DTYPE), K,
                                                     1, -1, -1, X, n_threads=max(1, (os.cpu_count() or 2) - 1)))
        expected["results"] = res
        expected["t_oracle"] = time.time() - t0

    th = threading.Thread(target=cpu_side)
    th.start()
    out = _stream(w, blocks, n_parts=8, chunk=4_000_000, window=32_000_000)
    th.join()
    report.update({k: v for k, v in out.items() if k != "kept"})
    report.update(t_index=expected["t_index"], t_oracle=expected["t_oracle"])
    exp_pairs = expected["pairs"]
    ra = exp_pairs["read_a"]
    checked = 0
    for (lo, hi), (recs, res) in zip(blocks, out["kept"]):
        a, b = np.searchsorted(ra, lo), np.searchsorted(ra, hi)
        assert recs.tobytes() == exp_pairs[a:b].view(recs.dtype).tobytes(), "block %s: seed records differ" % ((lo, hi),)
        idx, exp = expected["results"][(lo, hi)]
        assert_same(res[idx], exp, "block %s" % ((lo, hi),))
        checked += len(idx)
    report["records_checked"] = checked
    report["full_block_records"] = [int(len(r)) for (lo, hi), (r, _) in zip(blocks, out["kept"]) if (lo, hi) in full]
    report["t_total"] = round(time.time() - t_all, 1)
    print("C4 full-size parity:", json.dumps(report, default=str))
    d = os.environ.get("DIBELLA_REPORT_DIR")
    if d:
        with open(os.path.join(d, "c4_full_parity.json"), "w") as f:
            json.dump(report, f, default=str)
    assert all(x >= 4_000_000 for x in report["full_block_records"]), report["full_block_records"]
