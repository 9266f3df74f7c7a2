"""Whole benchmark batches on the GPU against the oracle, every record.

The expected results are stored as BLAKE2b digests of consecutive blocks of
4096 result records (40 bytes each, every field including cells and the
best-of-pair flag), written by ``tests/golden/make_full_parity.py``, which runs
only the input generator and the CPU oracle.  Equal digests mean equal bytes
for every record of the block; for a block whose digest differs, the oracle is
run again on that block here and the differing fields are reported.  The batch
runs as ``bench.py`` runs it: the whole seed set in one dibella_xdrop_batch call
with the default schedule."""

import glob
import json
import os

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import assert_same

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
FILES = sorted(glob.glob(os.path.join(HERE, "golden", "full_parity_*.json")))


def _load_make():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_full_parity", os.path.join(HERE, "golden",
                                                                                  "make_full_parity.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(f)[len("full_parity_"):-5] for f in FILES])
def test_whole_batch_matches_oracle(path):
    import paper_2001_10049_gb300 as dib
    mk = _load_make()
    doc = json.load(open(path))
    w = workloads.generate(doc["workload"])
    assert mk.input_digest(w) == doc["input_digest"], "generated inputs differ from the ones the digests cover"
    assert len(w.pairs) == doc["n_records"]
    store = dib.ReadStore.from_ascii(w.reads, w.offsets)
    al = dib.Aligner(store, len(w.pairs), k=doc["k"])
    M, S, G = doc["scoring"]
    got = al.align(w.pairs, dib.Scoring(M, S, G, doc["xdrop"]))
    digests = mk.block_digests(got)
    bad = [b for b, (x, y) in enumerate(zip(digests, doc["digests"])) if x != y]
    if bad:
        B = doc["block"]
        for b in bad[:3]:
            sl = slice(b * B, (b + 1) * B)
            exp = oracle.xdrop_batch(w.reads, w.offsets, w.pairs[sl].view(oracle.PAIR_DTYPE), doc["k"], M, S, G,
                                     doc["xdrop"])
            g2, e2 = got[sl].copy(), exp.copy()
            g2["status"] &= ~4  # best-of-pair flags of a block edge depend on the next block
            e2["status"] &= ~4
            assert_same(g2, e2, "%s X=%d block %d" % (doc["workload"], doc["xdrop"], b))
    assert not bad, "%d of %d blocks differ (first %s)" % (len(bad), len(digests), bad[:5])
    assert int(got["cells"].sum()) == doc["cells"]
