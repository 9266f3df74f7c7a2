"""The bounds-checked debug build on the GPU: the same results as the oracle,
with every kernel's store reads, shared-memory slots, queue pushes, item
indices and band slots checked and the fault record left clean.  Runs in a
child process so that the debug library is the one loaded."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import numpy as np
import paper_2001_10049_gb300 as dib, workloads
from gpu_util import oracle_align, schedule, NARROW_ALL, WIDE_ALL
assert dib.debug_build() and "libdibella_debug" in dib.library_path()
w = workloads.generate("c1_tiny")
store = dib.ReadStore.from_ascii(w.reads, w.offsets)
al = dib.Aligner(store, len(w.pairs), k=17)
dib.dibella_bounds_check(reset=True)
out = {"cases": 0, "mismatch": []}
for X in (0, 7, 25, 1 << 30):
    exp = oracle_align(w.reads, w.offsets, w.pairs, 17, (1, -1, -1, X))
    for name, sch in (("default", None), ("narrow32", schedule(narrow_band_cap=32, narrow_track=0, **NARROW_ALL)),
                      ("track32", schedule(narrow_band_cap=32, narrow_track=1, **NARROW_ALL)),
                      ("mid128", schedule(narrow_band_cap=32, mid_band_cap=128, narrow_track=0, **NARROW_ALL)),
                      ("wide", schedule(**WIDE_ALL)), ("int32", schedule(wide_packed=0, **WIDE_ALL))):
        got = al.align(w.pairs, dib.Scoring(1, -1, -1, X), sched=sch)
        out["cases"] += 1
        if got.tobytes() != exp.tobytes():
            out["mismatch"].append((name, X))
got = al.align(w.pairs[:200], dib.Scoring(1, -1, -1, 25), per_pair=True)
exp = oracle_align(w.reads, w.offsets, w.pairs[:200], 17, (1, -1, -1, 25))
if got.tobytes() != exp.tobytes():
    out["mismatch"].append(("per_pair", 25))
is_debug, rec = dib.dibella_bounds_check()
out["is_debug"] = is_debug
out["record"] = rec
print(json.dumps(out))
"""


def test_debug_build_is_clean_and_exact():
    env = dict(os.environ, DIBELLA_LIB_VARIANT="debug")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["is_debug"] and out["cases"] == 24  # 4 X values x 6 schedules
    assert out["mismatch"] == []
    assert out["record"] == {"code": 0, "index": 0, "limit": 0, "count": 0}, out["record"]
