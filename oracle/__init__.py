"""Oracle for the X-drop seed-and-extend path: plain CPU code, test infrastructure.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA path (no headers,
helpers or tables) and the product never falls back to it.

The arithmetic lives in ``xdrop_oracle.cpp`` (plain C++, int64); this module only
compiles it and marshals numpy arrays through ctypes.  What it computes is the
X-drop extension of diBELLA Sec. 2 (alignment definition and X-drop paragraph)
applied per seed as in Sec. 8-9, under the readings R1-R5 stated in the C++
file's header.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xdrop_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Byte layouts (independent declarations; same bytes as the library's ABI).
PAIR_DTYPE = np.dtype(
    [("read_a", "<u4"), ("read_b", "<u4"), ("pos_a", "<u4"), ("pos_b", "<u4"),
     ("strand", "u1"), ("pad", "u1", (3,)), ("seed_id", "<u4")])
RESULT_DTYPE = np.dtype(
    [("score", "<i4"), ("score_left", "<i4"), ("score_right", "<i4"),
     ("begin_a", "<u4"), ("end_a", "<u4"), ("begin_b", "<u4"), ("end_b", "<u4"),
     ("status", "<i4"), ("cells", "<i8")])
assert PAIR_DTYPE.itemsize == 24 and RESULT_DTYPE.itemsize == 40

STATUS_SEED_MISMATCH = 1
STATUS_INVALID_SEED = 2
STATUS_BEST_OF_PAIR = 4


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (portable C++, no intrinsics)."""
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
        i64, i32, vp, cp = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_char_p
        lib.oracle_extend.argtypes = [cp, i64, cp, i64, i32, i32, i32, i32, vp]
        lib.oracle_extend.restype = i32
        lib.oracle_extend_bands.argtypes = [cp, i64, cp, i64, i32, i32, i32, i32, vp, i64]
        lib.oracle_extend_bands.restype = i64
        lib.oracle_align_one.argtypes = [cp, i64, cp, i64, vp, i32, i32, i32, i32, i32, vp, vp]
        lib.oracle_align_one.restype = i32
        lib.oracle_xdrop_batch.argtypes = [vp, vp, i64, vp, i64, i32, i32, i32, i32, i32, vp, i32]
        lib.oracle_xdrop_batch.restype = i32
        lib.oracle_extend_columns.argtypes = [cp, i64, cp, i64, i32, i32, i32, i32, vp, i64]
        lib.oracle_extend_columns.restype = i64
        lib.oracle_traceback_batch.argtypes = [vp, vp, i64, vp, i64, i32, i32, i32, i32, i32, vp, vp, i64,
                                               vp]
        lib.oracle_traceback_batch.restype = i32
        _lib = lib
    return _lib


def extend(a: str | bytes, b: str | bytes, match: int, mismatch: int, gap: int, xdrop: int):
    """One-direction X-drop extension of a against b from cell (0,0).

    Returns (best, i_end, j_end, cells, tie)."""
    a = a.encode() if isinstance(a, str) else a
    b = b.encode() if isinstance(b, str) else b
    out = np.zeros(5, dtype=np.int64)
    _load().oracle_extend(a, len(a), b, len(b), match, mismatch, gap, xdrop,
                          out.ctypes.data_as(ctypes.c_void_p))
    return tuple(int(v) for v in out)


def extend_bands(a: str | bytes, b: str | bytes, match: int, mismatch: int, gap: int,
                 xdrop: int) -> list[int]:
    """Band size (evaluated cells) of every antidiagonal d >= 1 of one extension."""
    a = a.encode() if isinstance(a, str) else a
    b = b.encode() if isinstance(b, str) else b
    cap = len(a) + len(b) + 1
    out = np.zeros(cap, dtype=np.int64)
    n = _load().oracle_extend_bands(a, len(a), b, len(b), match, mismatch, gap, xdrop,
                                    out.ctypes.data_as(ctypes.c_void_p), cap)
    return [int(v) for v in out[:n]]


def align_one(a: str | bytes, b: str | bytes, pos_a: int, pos_b: int, strand: int, k: int,
              match: int, mismatch: int, gap: int, xdrop: int):
    """One seeded alignment; returns (result record, left ext tuple, right ext tuple)."""
    a = a.encode() if isinstance(a, str) else a
    b = b.encode() if isinstance(b, str) else b
    pair = np.zeros(1, dtype=PAIR_DTYPE)
    pair["read_a"], pair["read_b"], pair["pos_a"], pair["pos_b"], pair["strand"] = 0, 1, pos_a, pos_b, strand
    res = np.zeros(1, dtype=RESULT_DTYPE)
    ext = np.zeros(10, dtype=np.int64)
    _load().oracle_align_one(a, len(a), b, len(b), pair.ctypes.data_as(ctypes.c_void_p), k,
                             match, mismatch, gap, xdrop, res.ctypes.data_as(ctypes.c_void_p),
                             ext.ctypes.data_as(ctypes.c_void_p))
    e = [int(v) for v in ext]
    return res[0], tuple(e[:5]), tuple(e[5:])


def xdrop_batch(ascii: np.ndarray, offsets: np.ndarray, pairs: np.ndarray, k: int, match: int,
                mismatch: int, gap: int, xdrop: int, n_threads: int = 0) -> np.ndarray:
    """Align every seed record of ``pairs`` (PAIR_DTYPE) against the reads given as
    concatenated uint8 ASCII plus int64 offsets (n_reads + 1 entries)."""
    ascii = np.ascontiguousarray(ascii, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    pairs = np.ascontiguousarray(pairs, dtype=PAIR_DTYPE)
    out = np.zeros(len(pairs), dtype=RESULT_DTYPE)
    rc = _load().oracle_xdrop_batch(
        ascii.ctypes.data_as(ctypes.c_void_p), offsets.ctypes.data_as(ctypes.c_void_p),
        len(offsets) - 1, pairs.ctypes.data_as(ctypes.c_void_p), len(pairs), k, match,
        mismatch, gap, xdrop, out.ctypes.data_as(ctypes.c_void_p), n_threads)
    if rc != 0:
        raise ValueError("oracle_xdrop_batch rejected its arguments (rc=%d)" % rc)
    return out


# SAM/BAM op numbers of the run-length encoded traceback words (run << 4 | op).
CIGAR_OPS = {7: "=", 8: "X", 1: "I", 2: "D"}


def extend_columns(a: str | bytes, b: str | bytes, match: int, mismatch: int, gap: int,
                   xdrop: int) -> str:
    """Columns of one extension's best alignment from the origin on: '=' equal
    pair, 'X' unequal pair, 'D' a character of a only, 'I' a character of b only."""
    a = a.encode() if isinstance(a, str) else a
    b = b.encode() if isinstance(b, str) else b
    cap = len(a) + len(b) + 1
    buf = ctypes.create_string_buffer(cap)
    n = _load().oracle_extend_columns(a, len(a), b, len(b), match, mismatch, gap, xdrop, buf, cap)
    if n < 0:
        raise RuntimeError("oracle traceback failed")
    return buf.raw[:n].decode()


def cigar_string(words) -> str:
    """Text form of run-length encoded traceback words, e.g. '12=1X3=1D'."""
    return "".join("%d%s" % (int(w) >> 4, CIGAR_OPS[int(w) & 15]) for w in words)


def traceback_batch(ascii: np.ndarray, offsets: np.ndarray, pairs: np.ndarray, k: int, match: int,
                    mismatch: int, gap: int, xdrop: int, cap_per_seed: int):
    """Every seed's result (no best-of-pair flag) and its run-length encoded
    columns: (results, ops[n, cap_per_seed] uint32, n_ops[n] int32 with -1 when
    more than cap_per_seed runs were needed)."""
    ascii = np.ascontiguousarray(ascii, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    pairs = np.ascontiguousarray(pairs, dtype=PAIR_DTYPE)
    res = np.zeros(len(pairs), dtype=RESULT_DTYPE)
    ops = np.zeros((len(pairs), max(cap_per_seed, 1)), dtype=np.uint32)
    n_ops = np.zeros(len(pairs), dtype=np.int32)
    rc = _load().oracle_traceback_batch(
        ascii.ctypes.data_as(ctypes.c_void_p), offsets.ctypes.data_as(ctypes.c_void_p),
        len(offsets) - 1, pairs.ctypes.data_as(ctypes.c_void_p), len(pairs), k, match, mismatch, gap,
        xdrop, res.ctypes.data_as(ctypes.c_void_p), ops.ctypes.data_as(ctypes.c_void_p), ops.shape[1],
        n_ops.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError("oracle_traceback_batch failed (rc=%d)" % rc)
    return res, ops, n_ops
