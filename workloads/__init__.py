"""Seeded synthetic long-read workloads (inputs only; no alignment arithmetic).

Both the CUDA path and the CPU oracle read what this module produces.  The
generator itself is ``gen.cpp`` (see its header for the generation rules); this
module compiles it, exposes the named configurations and caches results.

Named configurations (stand-ins for the paper's PacBio E. coli inputs, diBELLA
Sec. 5, which are not available here):

* ``c1_tiny``   50 kb uniform genome, 10x, lengths U[2000, 6000], 15% error,
                k=17, multiplicity [2, 8], one seed per pair;
* ``c2_ecoli``  4.6 Mb genome, 30x, lognormal lengths (mean 9 kb, sd 7 kb)
                clipped to [1 kb, 60 kb], 15% error, k=17, [2, 8], up to 2 seeds;
* ``c3_uneven`` 2 Mb genome, 20x, log-uniform lengths [500, 100k], per-read
                error U[5%, 35%], k=17, [2, 8], one seed;
* ``c4_repeats`` 100 Mb genome with 200 families x 2 copies of 5 kb repeats (3%
                divergence) and 1 Mb of tandem arrays (period 2-50), 40x, C2
                lengths, 15% error, k=17, [2, 12], one seed.  ``c4_repeats_small``
                keeps every rule at 1/20 of the genome.

Error split everywhere: 20% substitution, 50% insertion, 30% deletion.
"""

from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import tempfile
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.cpp")
_LIB = os.path.join(_HERE, "libworkloads.so")
_lock = threading.Lock()
_lib = None

PAIR_DTYPE = np.dtype(
    [("read_a", "<u4"), ("read_b", "<u4"), ("pos_a", "<u4"), ("pos_b", "<u4"),
     ("strand", "u1"), ("pad", "u1", (3,)), ("seed_id", "<u4")])


class _Config(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64), ("genome_len", ctypes.c_int64),
        ("repeat_families", ctypes.c_int32), ("repeat_unit_len", ctypes.c_int32),
        ("repeat_copies", ctypes.c_int32), ("tandem_period_lo", ctypes.c_int32),
        ("tandem_period_hi", ctypes.c_int32), ("tandem_array_lo", ctypes.c_int32),
        ("tandem_array_hi", ctypes.c_int32), ("len_dist", ctypes.c_int32),
        ("tandem_bases", ctypes.c_int64), ("repeat_divergence", ctypes.c_double),
        ("coverage", ctypes.c_double), ("len_a", ctypes.c_double), ("len_b", ctypes.c_double),
        ("len_mean", ctypes.c_double), ("len_sd", ctypes.c_double),
        ("err_lo", ctypes.c_double), ("err_hi", ctypes.c_double),
        ("p_sub", ctypes.c_double), ("p_ins", ctypes.c_double), ("p_del", ctypes.c_double),
        ("k", ctypes.c_int32), ("mult_lo", ctypes.c_int32), ("mult_hi", ctypes.c_int32),
        ("max_seeds", ctypes.c_int32), ("n_threads", ctypes.c_int32), ("min_seed_gap", ctypes.c_int32),
        ("pairs_mode", ctypes.c_int32), ("n_ranges", ctypes.c_int64), ("ranges", ctypes.c_void_p),
    ]

# pairs_mode of the generator: every candidate pair, none (reads only), or the
# candidate pairs whose read_a lies in given read-id ranges (same records as the
# full index restricted to those read_a, from an index of the ranges' k-mers only).
PAIRS_ALL, PAIRS_NONE, PAIRS_RANGES = 0, 1, 2


_BASE = dict(seed=1, genome_len=50_000, repeat_families=0, repeat_unit_len=5000, repeat_copies=2,
             tandem_period_lo=2, tandem_period_hi=50, tandem_array_lo=500, tandem_array_hi=5000,
             len_dist=0, tandem_bases=0, repeat_divergence=0.03, coverage=10.0, len_a=2000.0,
             len_b=6000.0, len_mean=9000.0, len_sd=7000.0, err_lo=0.15, err_hi=0.15, p_sub=0.2,
             p_ins=0.5, p_del=0.3, k=17, mult_lo=2, mult_hi=8, max_seeds=1, min_seed_gap=0)

CONFIGS = {
    "c1_tiny": dict(_BASE),
    "c2_ecoli": dict(_BASE, seed=2, genome_len=4_600_000, coverage=30.0, len_dist=1,
                     len_a=1000.0, len_b=60000.0, max_seeds=2),
    "c3_uneven": dict(_BASE, seed=3, genome_len=2_000_000, coverage=20.0, len_dist=2,
                      len_a=500.0, len_b=100000.0, err_lo=0.05, err_hi=0.35),
    "c4_repeats": dict(_BASE, seed=4, genome_len=100_000_000, repeat_families=200,
                       tandem_bases=1_000_000, coverage=40.0, len_dist=1, len_a=1000.0,
                       len_b=60000.0, mult_hi=12),
    "c4_repeats_small": dict(_BASE, seed=4, genome_len=5_000_000, repeat_families=10,
                             tandem_bases=50_000, coverage=40.0, len_dist=1, len_a=1000.0,
                             len_b=60000.0, mult_hi=12),
    # The seed options of Sec. 5 on the E. coli-sized reads: every seed at least
    # 1,000 bp apart, and (on a smaller genome) every seed at least k apart.
    "c2_ecoli_1kb": dict(_BASE, seed=2, genome_len=4_600_000, coverage=30.0, len_dist=1,
                         len_a=1000.0, len_b=60000.0, max_seeds=1 << 30, min_seed_gap=1000),
    "c2_allseeds_300k": dict(_BASE, seed=5, genome_len=300_000, coverage=30.0, len_dist=1,
                             len_a=1000.0, len_b=60000.0, max_seeds=1 << 30),
}

# Scoring of every configuration: match +1, mismatch -1, gap -1 (int32).
SCORING = dict(match=1, mismatch=-1, gap=-1)
XDROP = {"c1_tiny": (7,), "c2_ecoli": (7, 25), "c3_uneven": (50,), "c4_repeats": (15,),
         "c4_repeats_small": (15,), "c2_ecoli_1kb": (7, 25), "c2_allseeds_300k": (7, 25)}


def build(force: bool = False) -> str:
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + ".tmp%d" % os.getpid()
            subprocess.check_call(
                ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.wl_generate.argtypes = [ctypes.POINTER(_Config)]
        lib.wl_generate.restype = vp
        for name in ("wl_genome_len", "wl_n_reads", "wl_n_bases", "wl_n_pairs"):
            getattr(lib, name).argtypes = [vp]
            getattr(lib, name).restype = i64
        for name in ("wl_genome", "wl_reads", "wl_offsets", "wl_tmpl_start", "wl_tmpl_len",
                     "wl_tmpl_strand", "wl_pairs"):
            getattr(lib, name).argtypes = [vp]
            getattr(lib, name).restype = vp
        lib.wl_stat.argtypes = [vp, ctypes.c_int]
        lib.wl_stat.restype = i64
        lib.wl_free.argtypes = [vp]
        lib.wl_free.restype = None
        _lib = lib
    return _lib


@dataclass
class Workload:
    name: str
    params: dict
    genome: np.ndarray          # uint8 ASCII
    reads: np.ndarray           # uint8 ASCII, concatenated
    offsets: np.ndarray         # int64, n_reads + 1
    tmpl_start: np.ndarray      # int64 template start of each read
    tmpl_len: np.ndarray        # int32 template length
    tmpl_strand: np.ndarray     # uint8
    pairs: np.ndarray           # PAIR_DTYPE seed records, grouped by (read_a, read_b)
    stats: dict = field(default_factory=dict)

    @property
    def n_reads(self) -> int:
        return len(self.offsets) - 1

    @property
    def read_lengths(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int32)

    def read(self, r: int) -> str:
        return self.reads[self.offsets[r]:self.offsets[r + 1]].tobytes().decode()


def _copy(ptr, dtype, n):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    buf = (ctypes.c_char * (n * np.dtype(dtype).itemsize)).from_address(ptr)
    return np.frombuffer(buf, dtype=dtype).copy()


def _cache_dir() -> str:
    d = os.environ.get("DIBELLA_WORKLOAD_CACHE", os.path.join(tempfile.gettempdir(), "dibella_workloads"))
    os.makedirs(d, exist_ok=True)
    return d


def generate(name: str | None = None, *, cache: bool = True, n_threads: int = 0, pairs_mode: int = PAIRS_ALL,
             read_ranges=None, **overrides) -> Workload:
    """Generate (or load from the cache) a named configuration, optionally overridden.

    pairs_mode PAIRS_NONE skips the candidate pairs (reads only); PAIRS_RANGES
    keeps the candidate pairs whose read_a lies in one of ``read_ranges``
    (half-open (lo, hi) read-id ranges, ascending and disjoint)."""
    params = dict(CONFIGS[name] if name else _BASE)
    params.update(overrides)
    ranges = np.ascontiguousarray(np.asarray(read_ranges if read_ranges is not None else [], dtype=np.int64)
                                  .reshape(-1, 2))
    if pairs_mode == PAIRS_RANGES and len(ranges) and (np.any(ranges[:, 1] < ranges[:, 0]) or
                                                       np.any(ranges[1:, 0] < ranges[:-1, 1])):
        raise ValueError("read ranges must be ascending and disjoint")
    key_src = repr(sorted(params.items())) + repr((pairs_mode, ranges.tolist()))
    key = hashlib.sha256(key_src.encode() + open(_SRC, "rb").read()).hexdigest()[:16]
    path = os.path.join(_cache_dir(), "%s_%s.npz" % (name or "custom", key))
    if cache and os.path.exists(path):
        z = np.load(path)
        return Workload(name or "custom", params, z["genome"], z["reads"], z["offsets"], z["tmpl_start"],
                        z["tmpl_len"], z["tmpl_strand"], z["pairs"].view(PAIR_DTYPE).reshape(-1),
                        dict(zip(["instances", "retained_kmers", "candidate_pairs"], z["stats"].tolist())))
    lib = _load()
    cfg = _Config(**{k: v for k, v in params.items()}, n_threads=n_threads, pairs_mode=pairs_mode,
                  n_ranges=len(ranges), ranges=ranges.ctypes.data if len(ranges) else None)
    h = lib.wl_generate(ctypes.byref(cfg))
    if not h:
        raise ValueError("the generator rejected its configuration")
    try:
        gl, nr, nb, npairs = lib.wl_genome_len(h), lib.wl_n_reads(h), lib.wl_n_bases(h), lib.wl_n_pairs(h)
        w = Workload(
            name or "custom", params,
            _copy(lib.wl_genome(h), np.uint8, gl), _copy(lib.wl_reads(h), np.uint8, nb),
            _copy(lib.wl_offsets(h), np.int64, nr + 1), _copy(lib.wl_tmpl_start(h), np.int64, nr),
            _copy(lib.wl_tmpl_len(h), np.int32, nr), _copy(lib.wl_tmpl_strand(h), np.uint8, nr),
            _copy(lib.wl_pairs(h), PAIR_DTYPE, npairs),
            {"instances": lib.wl_stat(h, 0), "retained_kmers": lib.wl_stat(h, 1),
             "candidate_pairs": lib.wl_stat(h, 2)})
    finally:
        lib.wl_free(h)
    if cache:
        tmp = path + ".tmp%d.npz" % os.getpid()
        np.savez(tmp, genome=w.genome, reads=w.reads, offsets=w.offsets, tmpl_start=w.tmpl_start,
                 tmpl_len=w.tmpl_len, tmpl_strand=w.tmpl_strand, pairs=w.pairs.view(np.uint8),
                 stats=np.array([w.stats["instances"], w.stats["retained_kmers"],
                                 w.stats["candidate_pairs"]], dtype=np.int64))
        os.replace(tmp, path)
    return w


def pair_groups(pairs: np.ndarray) -> np.ndarray:
    """Start index of every run of consecutive records sharing (read_a, read_b),
    plus a final entry len(pairs)."""
    if len(pairs) == 0:
        return np.zeros(1, dtype=np.int64)
    key = pairs["read_a"].astype(np.uint64) << np.uint64(32) | pairs["read_b"].astype(np.uint64)
    starts = np.flatnonzero(np.concatenate([[True], key[1:] != key[:-1]]))
    return np.concatenate([starts, [len(pairs)]]).astype(np.int64)


def sample_pair_groups(pairs: np.ndarray, n_groups: int, seed: int) -> np.ndarray:
    """A seeded random subset of whole candidate pairs (all their seed records)."""
    g = pair_groups(pairs)
    n = len(g) - 1
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(n, size=min(n_groups, n), replace=False))
    idx = np.concatenate([np.arange(g[i], g[i + 1]) for i in pick]) if len(pick) else np.zeros(0, np.int64)
    return pairs[idx]


def stratified_pair_groups(pairs: np.ndarray, read_lengths: np.ndarray, n_groups: int) -> np.ndarray:
    """Every k-th whole candidate pair in order of decreasing min(len_a, len_b):
    a sample whose length mix (including the longest pairs) follows the batch."""
    g = pair_groups(pairs)
    n = len(g) - 1
    if n == 0 or n_groups <= 0:
        return pairs[:0]
    starts = g[:-1]
    key = np.minimum(read_lengths[pairs["read_a"][starts]], read_lengths[pairs["read_b"][starts]])
    order = np.argsort(-key, kind="stable")
    step = max(1, n // min(n_groups, n))
    pick = np.sort(order[::step][:n_groups])
    idx = np.concatenate([np.arange(g[i], g[i + 1]) for i in pick])
    return pairs[idx]


def serving_requests(pairs: np.ndarray, n_requests: int, rate_per_s: float, seed: int,
                     max_size: int = 4096, xdrops=(7, 25, 50)):
    """Poisson arrivals of requests, each a log-uniform number (1..max_size) of whole
    candidate pairs drawn from ``pairs`` with X drawn uniformly from ``xdrops``.

    Returns a list of (arrival_s, xdrop, record index array)."""
    rng = np.random.default_rng(seed)
    g = pair_groups(pairs)
    n_groups = len(g) - 1
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        size = int(np.floor(np.exp(rng.uniform(0.0, np.log(max_size + 1)))))
        size = max(1, min(max_size, size))
        start = int(rng.integers(0, max(1, n_groups - size)))
        idx = np.arange(g[start], g[min(n_groups, start + size)])
        out.append((t, int(rng.choice(xdrops)), idx))
    return out
