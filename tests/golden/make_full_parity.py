#!/usr/bin/env python3
"""Write the expected results of whole benchmark batches, as block digests.

For each (workload, X) named on the command line, every seed record of the
workload is aligned by the CPU oracle (``oracle.xdrop_batch``, all host
threads) and the 40-byte result records are hashed in blocks of BLOCK records
(BLAKE2b, 8-byte digests).  The JSON file written next to this script holds the
digests together with a digest of the inputs (reads, offsets, seed records), so
a test on another machine first checks that it generated the same inputs.

This script calls only the input generator (``workloads``) and the oracle; no
value in its output comes from the CUDA path.

  python tests/golden/make_full_parity.py c2_ecoli:7 c2_ecoli:25 c3_uneven:50
"""

from __future__ import annotations

import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

BLOCK = 4096


def input_digest(w) -> str:
    h = hashlib.blake2b(digest_size=16)
    for a in (w.reads, w.offsets, w.pairs):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def block_digests(results: np.ndarray) -> list[str]:
    raw = np.ascontiguousarray(results).view(np.uint8).reshape(-1, 40)
    return [hashlib.blake2b(raw[s:s + BLOCK].tobytes(), digest_size=8).hexdigest()
            for s in range(0, len(raw), BLOCK)]


def path_for(workload: str, xdrop: int) -> str:
    return os.path.join(HERE, "full_parity_%s_x%d.json" % (workload, xdrop))


def main(argv):
    import oracle
    import workloads
    out_dir = HERE
    if argv and argv[0].startswith("--out="):
        out_dir = argv[0][len("--out="):]
        argv = argv[1:]
    for spec in argv:
        name, x = spec.split(":")
        x = int(x)
        w = workloads.generate(name)
        t0 = time.time()
        sc = workloads.SCORING
        res = oracle.xdrop_batch(w.reads, w.offsets, w.pairs, w.params["k"], sc["match"], sc["mismatch"],
                                 sc["gap"], x)
        dt = time.time() - t0
        doc = {"workload": name, "xdrop": x, "k": w.params["k"], "scoring": [sc["match"], sc["mismatch"], sc["gap"]],
               "n_records": int(len(w.pairs)), "block": BLOCK, "input_digest": input_digest(w),
               "digests": block_digests(res), "oracle_seconds": round(dt, 1), "host_threads": os.cpu_count(),
               "cells": int(res["cells"].sum())}
        p = os.path.join(out_dir, os.path.basename(path_for(name, x)))
        with open(p, "w") as f:
            json.dump(doc, f)
        print("%s X=%d: %d records, %.1f s -> %s" % (name, x, len(w.pairs), dt, p), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
