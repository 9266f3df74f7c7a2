"""GB300 seed-and-extend X-drop alignment (diBELLA's per-pair alignment stage).

Thin ctypes binding over the C ABI of ``libdibella.so`` (declared in
``include/dibella.h``).  Every function named ``dibella_*`` here marshals its
arguments to the C entry point of the same name; all computation runs in the
library's CUDA kernels.  PyTorch is used only for device memory and streams.
There is no CPU fallback: if the library cannot be loaded, importing the
binding's functions raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

PAIR_DTYPE = np.dtype(
    [("read_a", "<u4"), ("read_b", "<u4"), ("pos_a", "<u4"), ("pos_b", "<u4"),
     ("strand", "u1"), ("pad", "u1", (3,)), ("seed_id", "<u4")])
RESULT_DTYPE = np.dtype(
    [("score", "<i4"), ("score_left", "<i4"), ("score_right", "<i4"),
     ("begin_a", "<u4"), ("end_a", "<u4"), ("begin_b", "<u4"), ("end_b", "<u4"),
     ("status", "<i4"), ("cells", "<i8")])

DIBELLA_OK, DIBELLA_EINVAL, DIBELLA_EBASE, DIBELLA_ENOMEM, DIBELLA_ECUDA, DIBELLA_ETIMEOUT = 0, -1, -2, -3, -4, -5
RES_SEED_MISMATCH, RES_INVALID_SEED, RES_BEST_OF_PAIR, RES_BAND_OVERFLOW = 1, 2, 4, 8
XDROP_INF = 1 << 30
DIBELLA_MAX_READ_LEN = 1 << 24
MAX_BUCKETS = 8

_ERRORS = {DIBELLA_EINVAL: "invalid argument", DIBELLA_EBASE: "non-ACGT base",
           DIBELLA_ENOMEM: "workspace too small", DIBELLA_ECUDA: "CUDA error",
           DIBELLA_ETIMEOUT: "device wait timed out"}


class DibellaError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = "%s failed: %s (%d)" % (where, _ERRORS.get(code, "error"), code)
        if code in (DIBELLA_ECUDA, DIBELLA_ENOMEM):
            detail = _lib().dibella_last_error().decode()
            if detail:
                msg += ": " + detail
        super().__init__(msg)
        self.code = code


class Scoring(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32),
                ("gap", ctypes.c_int32), ("xdrop", ctypes.c_int32)]


class Schedule(ctypes.Structure):
    _fields_ = [("narrow_max_xdrop", ctypes.c_int32), ("narrow_max_len", ctypes.c_int32),
                ("narrow_band_cap", ctypes.c_int32), ("wide_slots", ctypes.c_int32),
                ("wide_packed", ctypes.c_int32), ("wide_group_lanes", ctypes.c_int32),
                ("wide_blocks_per_sm", ctypes.c_int32),
                ("narrow_blocks_per_sm", ctypes.c_int32), ("n_buckets", ctypes.c_int32),
                ("bucket_bounds", ctypes.c_int32 * MAX_BUCKETS), ("mid_band_cap", ctypes.c_int32),
                ("narrow_split_d", ctypes.c_int32), ("narrow_unroll", ctypes.c_int32),
                ("narrow_track", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"narrow_max_xdrop": self.narrow_max_xdrop, "narrow_max_len": self.narrow_max_len,
                "narrow_band_cap": self.narrow_band_cap, "wide_slots": self.wide_slots,
                "wide_packed": self.wide_packed, "wide_group_lanes": self.wide_group_lanes,
                "wide_blocks_per_sm": self.wide_blocks_per_sm,
                "narrow_blocks_per_sm": self.narrow_blocks_per_sm, "n_buckets": self.n_buckets,
                "bucket_bounds": list(self.bucket_bounds)[: max(0, self.n_buckets - 1)],
                "mid_band_cap": self.mid_band_cap, "narrow_split_d": self.narrow_split_d,
                "narrow_unroll": self.narrow_unroll, "narrow_track": self.narrow_track}

    @classmethod
    def from_dict(cls, d: dict) -> "Schedule":
        s = cls()
        for key in ("narrow_max_xdrop", "narrow_max_len", "narrow_band_cap", "wide_slots", "wide_packed",
                    "wide_group_lanes", "wide_blocks_per_sm",
                    "narrow_blocks_per_sm", "n_buckets"):
            setattr(s, key, int(d[key]))
        s.mid_band_cap = int(d.get("mid_band_cap", 0))
        s.narrow_split_d = int(d.get("narrow_split_d", 0))
        s.narrow_unroll = int(d.get("narrow_unroll", 0))
        s.narrow_track = int(d.get("narrow_track", 0))
        bounds = list(d.get("bucket_bounds", []))
        for b in range(MAX_BUCKETS):
            s.bucket_bounds[b] = int(bounds[b]) if b < len(bounds) else 0
        return s


_LIB = None


def debug_build() -> bool:
    """True when DIBELLA_LIB_VARIANT=debug selects the bounds-checked library."""
    return os.environ.get("DIBELLA_LIB_VARIANT", "") == "debug"


def _lib():
    """Load libdibella.so, or libdibella_debug.so when DIBELLA_LIB_VARIANT=debug
    (compiling it first if its sources are newer)."""
    global _LIB
    if _LIB is None:
        path = _build.lib_path(debug_build())
        if not os.path.exists(path) or _build._stale(path, _build.SOURCES + _build.HEADERS):
            _build.build(debug=debug_build())
        lib = ctypes.CDLL(path)
        vp, i64, i32, p64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)
        sig = {
            "dibella_packed_words": ([vp, i64, p64], i32),
            "dibella_pack_reads": ([vp, vp, i64, vp, vp, vp, p64, i32], i32),
            "dibella_get_default_schedule": ([ctypes.POINTER(Schedule)], i32),
            "dibella_set_default_schedule": ([ctypes.POINTER(Schedule)], i32),
            "dibella_xdrop_workspace_bytes": ([i64, i32, p64], i32),
            "dibella_staging_bytes": ([i64, p64], i32),
            "dibella_xdrop_batch": ([vp, vp, vp, i64, vp, i64, i32, Scoring, vp, vp, i64, vp,
                                     ctypes.POINTER(Schedule)], i32),
            "dibella_xdrop_batch_noalloc": ([vp, vp, vp, i64, vp, i64, i32, Scoring, vp, vp], i32),
            "dibella_xdrop_batch_host": ([vp, vp, vp, i64, vp, i64, i32, Scoring, vp, vp, vp, i64, vp,
                                          ctypes.POINTER(Schedule)], i32),
            "dibella_xdrop_stream": ([vp, vp, vp, i64, vp, i64, i64, i32, Scoring, vp, ctypes.POINTER(vp),
                                      ctypes.POINTER(vp), i64, ctypes.POINTER(vp), ctypes.POINTER(Schedule),
                                      p64], i32),
            "dibella_xdrop_per_pair": ([vp, vp, vp, i64, vp, i64, i32, Scoring, vp, vp, i64, vp], i32),
            "dibella_autotune": ([vp, vp, vp, i64, vp, i64, i32, Scoring, vp, vp, i64, vp, i32,
                                  ctypes.POINTER(Schedule), ctypes.POINTER(ctypes.c_float),
                                  ctypes.POINTER(ctypes.c_int32)], i32),
            "dibella_enable_phase_timing": ([ctypes.c_int], i32),
            "dibella_phase_times": ([ctypes.POINTER(ctypes.c_float), ctypes.c_int], i32),
            "dibella_batch_counters": ([vp, vp, p64, ctypes.c_int], i32),
            "dibella_last_launch_count": ([], i32),
            "dibella_enable_warp_clock": ([ctypes.c_int], i32),
            "dibella_warp_clock": ([vp, ctypes.c_int], i32),
            "dibella_int_peak": ([i32, i64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp],
                                 i32),
            "dibella_candidate_workspace_bytes": ([i64, i64, i32, i32, p64], i32),
            "dibella_candidate_pairs": ([vp, vp, vp, i64, i64, i32, i32, i32, i32, i32, i32, vp, i64, vp, vp, i64,
                                         vp], i32),
            "dibella_candidate_workspace_bytes_parts": ([i64, i64, i32, i32, i32, i64, p64], i32),
            "dibella_candidate_pairs_parts": ([vp, vp, vp, i64, i64, i32, i32, i32, i32, i32, i32, i32, i64, vp, i64,
                                               vp, vp, i64, vp], i32),
            "dibella_traceback_workspace_bytes": ([i64, i32, i64, p64], i32),
            "dibella_xdrop_traceback": ([vp, vp, vp, i64, i32, vp, i64, i32, Scoring, vp, vp, i32, vp, i64, i64,
                                         vp, i64, vp], i32),
            "dibella_bounds_check": ([p64, ctypes.c_int], i32),
            "dibella_last_error": ([], ctypes.c_char_p),
            "dibella_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = lib
    return _LIB


def library_path() -> str:
    return _build.lib_path(debug_build())


def dibella_bounds_check(reset: bool = False):
    """(is_debug_build, {code, index, limit, count}) of the kernels' bounds record."""
    buf = (ctypes.c_int64 * 4)()
    rc = _lib().dibella_bounds_check(buf, 1 if reset else 0)
    if rc < 0:
        _check(rc, "dibella_bounds_check")
    return rc == 1, dict(zip(("code", "index", "limit", "count"), (int(v) for v in buf)))


def exported_symbols() -> list[str]:
    """Names the binding resolves in the loaded library."""
    lib = _lib()
    return [n for n in dir(lib) if n.startswith("dibella_")]


def _check(rc: int, where: str) -> None:
    if rc != DIBELLA_OK:
        raise DibellaError(rc, where)


def _ptr(x) -> int:
    """Address of a numpy array or a torch tensor (host or device)."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- C ABI, one Python function per entry point -----------------------------

def dibella_packed_words(ascii_offsets: np.ndarray) -> int:
    offs = np.ascontiguousarray(ascii_offsets, dtype=np.int64)
    out = ctypes.c_int64(0)
    _check(_lib().dibella_packed_words(offs.ctypes.data, len(offs) - 1, ctypes.byref(out)),
           "dibella_packed_words")
    return out.value


def dibella_pack_reads(ascii: np.ndarray, ascii_offsets: np.ndarray, n_threads: int = 0):
    """Pack ASCII reads; returns (packed_words uint32, read_word_offsets int64, read_lengths int32)."""
    ascii = np.ascontiguousarray(ascii, dtype=np.uint8)
    offs = np.ascontiguousarray(ascii_offsets, dtype=np.int64)
    n = len(offs) - 1
    words = np.empty(dibella_packed_words(offs), dtype=np.uint32)
    woffs = np.empty(n, dtype=np.int64)
    lens = np.empty(n, dtype=np.int32)
    bad = ctypes.c_int64(-1)
    rc = _lib().dibella_pack_reads(ascii.ctypes.data, offs.ctypes.data, n, words.ctypes.data,
                                   woffs.ctypes.data, lens.ctypes.data, ctypes.byref(bad), n_threads)
    if rc == DIBELLA_EBASE:
        raise DibellaError(rc, "dibella_pack_reads (byte %d)" % bad.value)
    _check(rc, "dibella_pack_reads")
    return words, woffs, lens


def dibella_get_default_schedule() -> Schedule:
    s = Schedule()
    _check(_lib().dibella_get_default_schedule(ctypes.byref(s)), "dibella_get_default_schedule")
    return s


def dibella_set_default_schedule(s: Schedule) -> None:
    _check(_lib().dibella_set_default_schedule(ctypes.byref(s)), "dibella_set_default_schedule")


def dibella_xdrop_workspace_bytes(n_pairs: int, max_read_len: int) -> int:
    out = ctypes.c_int64(0)
    _check(_lib().dibella_xdrop_workspace_bytes(n_pairs, max_read_len, ctypes.byref(out)),
           "dibella_xdrop_workspace_bytes")
    return out.value


def dibella_candidate_workspace_bytes(n_reads: int, n_bases: int, k: int, mult_hi: int) -> int:
    out = ctypes.c_int64(0)
    _check(_lib().dibella_candidate_workspace_bytes(n_reads, n_bases, k, mult_hi, ctypes.byref(out)),
           "dibella_candidate_workspace_bytes")
    return out.value


def dibella_candidate_pairs(words, word_offsets, lengths, n_reads: int, n_bases: int, max_read_len: int, k: int,
                            mult_lo: int, mult_hi: int, max_seeds: int, min_seed_gap: int, pairs_out,
                            pairs_capacity: int, counts_out, workspace, workspace_bytes: int, stream=None) -> None:
    _check(_lib().dibella_candidate_pairs(_ptr(words), _ptr(word_offsets), _ptr(lengths), n_reads, n_bases,
                                          max_read_len, k, mult_lo, mult_hi, max_seeds, min_seed_gap,
                                          _ptr(pairs_out), pairs_capacity, _ptr(counts_out), _ptr(workspace),
                                          workspace_bytes, _stream_handle(stream)), "dibella_candidate_pairs")


def dibella_candidate_workspace_bytes_parts(n_reads: int, n_bases: int, max_read_len: int, k: int, n_parts: int,
                                            occ_pair_capacity: int) -> int:
    out = ctypes.c_int64(0)
    _check(_lib().dibella_candidate_workspace_bytes_parts(n_reads, n_bases, max_read_len, k, n_parts,
                                                          occ_pair_capacity, ctypes.byref(out)),
           "dibella_candidate_workspace_bytes_parts")
    return out.value


def dibella_candidate_pairs_parts(words, word_offsets, lengths, n_reads: int, n_bases: int, max_read_len: int,
                                  k: int, mult_lo: int, mult_hi: int, max_seeds: int, min_seed_gap: int, n_parts: int,
                                  occ_pair_capacity: int, pairs_out, pairs_capacity: int, counts_out, workspace,
                                  workspace_bytes: int, stream=None) -> None:
    _check(_lib().dibella_candidate_pairs_parts(_ptr(words), _ptr(word_offsets), _ptr(lengths), n_reads, n_bases,
                                                max_read_len, k, mult_lo, mult_hi, max_seeds, min_seed_gap, n_parts,
                                                occ_pair_capacity, _ptr(pairs_out), pairs_capacity, _ptr(counts_out),
                                                _ptr(workspace), workspace_bytes, _stream_handle(stream)),
           "dibella_candidate_pairs_parts")


def dibella_traceback_workspace_bytes(n_lanes: int, max_read_len: int, moves_words: int) -> int:
    out = ctypes.c_int64(0)
    _check(_lib().dibella_traceback_workspace_bytes(n_lanes, max_read_len, moves_words, ctypes.byref(out)),
           "dibella_traceback_workspace_bytes")
    return out.value


def dibella_xdrop_traceback(packed_words, read_word_offsets, read_lengths, n_reads: int, max_read_len: int, pairs,
                            n_pairs: int, k: int, scoring: Scoring, results, ops, ops_per_seed: int, n_ops,
                            n_lanes: int, moves_words: int, workspace, workspace_bytes: int, stream=None) -> None:
    _check(_lib().dibella_xdrop_traceback(_ptr(packed_words), _ptr(read_word_offsets), _ptr(read_lengths), n_reads,
                                          max_read_len, _ptr(pairs), n_pairs, k, scoring, _ptr(results),
                                          _ptr(ops), ops_per_seed, _ptr(n_ops), n_lanes, moves_words,
                                          _ptr(workspace), workspace_bytes, _stream_handle(stream)),
           "dibella_xdrop_traceback")


# Op letters of the run-length encoded traceback words (run << 4 | op).
CIGAR_LETTERS = {1: "I", 2: "D", 7: "=", 8: "X"}


def cigar_string(words) -> str:
    """Text form of one seed's run words, e.g. '120=1X40=1I8='."""
    return "".join("%d%s" % (int(w) >> 4, CIGAR_LETTERS[int(w) & 15]) for w in words)


def dibella_staging_bytes(n_pairs: int) -> int:
    out = ctypes.c_int64(0)
    _check(_lib().dibella_staging_bytes(n_pairs, ctypes.byref(out)), "dibella_staging_bytes")
    return out.value


def dibella_xdrop_batch(packed_words, read_word_offsets, read_lengths, n_reads: int, pairs, n_pairs: int,
                        k: int, scoring: Scoring, results, workspace, workspace_bytes: int,
                        stream=None, sched: Schedule | None = None) -> None:
    rc = _lib().dibella_xdrop_batch(_ptr(packed_words), _ptr(read_word_offsets), _ptr(read_lengths),
                                    n_reads, _ptr(pairs), n_pairs, k, scoring, _ptr(results),
                                    _ptr(workspace), workspace_bytes, _stream_handle(stream),
                                    ctypes.byref(sched) if sched is not None else None)
    _check(rc, "dibella_xdrop_batch")


NOALLOC_MAX_PAIRS = 16384
NOALLOC_MAX_BAND = 8189


def dibella_xdrop_batch_noalloc(packed_words, read_word_offsets, read_lengths, n_reads: int, pairs,
                                n_pairs: int, k: int, scoring: Scoring, results, stream=None) -> None:
    """dibella_xdrop_batch without a caller workspace and without allocating
    (the library's fixed scratch; at most NOALLOC_MAX_PAIRS seeds per call)."""
    rc = _lib().dibella_xdrop_batch_noalloc(_ptr(packed_words), _ptr(read_word_offsets), _ptr(read_lengths),
                                            n_reads, _ptr(pairs), n_pairs, k, scoring, _ptr(results),
                                            _stream_handle(stream))
    _check(rc, "dibella_xdrop_batch_noalloc")


def dibella_xdrop_batch_host(packed_words, read_word_offsets, read_lengths, n_reads: int, host_pairs,
                             n_pairs: int, k: int, scoring: Scoring, host_results, staging, workspace,
                             workspace_bytes: int, stream=None, sched: Schedule | None = None) -> None:
    rc = _lib().dibella_xdrop_batch_host(_ptr(packed_words), _ptr(read_word_offsets), _ptr(read_lengths),
                                         n_reads, _ptr(host_pairs), n_pairs, k, scoring,
                                         _ptr(host_results), _ptr(staging), _ptr(workspace),
                                         workspace_bytes, _stream_handle(stream),
                                         ctypes.byref(sched) if sched is not None else None)
    _check(rc, "dibella_xdrop_batch_host")


def dibella_xdrop_stream(packed_words, read_word_offsets, read_lengths, n_reads: int, host_pairs, n_pairs: int,
                         chunk_pairs: int, k: int, scoring: Scoring, host_results, staging, workspace,
                         workspace_bytes: int, streams, sched: Schedule | None = None) -> int:
    """staging / workspace / streams are pairs (two slots); returns the number of chunks."""
    st = (ctypes.c_void_p * 2)(*[_ptr(x) for x in staging])
    ws = (ctypes.c_void_p * 2)(*[_ptr(x) for x in workspace])
    ss = (ctypes.c_void_p * 2)(*[_stream_handle(x) for x in streams])
    n_chunks = ctypes.c_int64(0)
    rc = _lib().dibella_xdrop_stream(_ptr(packed_words), _ptr(read_word_offsets), _ptr(read_lengths), n_reads,
                                     _ptr(host_pairs), n_pairs, chunk_pairs, k, scoring, _ptr(host_results), st, ws,
                                     workspace_bytes, ss, ctypes.byref(sched) if sched is not None else None,
                                     ctypes.byref(n_chunks))
    _check(rc, "dibella_xdrop_stream")
    return int(n_chunks.value)


def dibella_xdrop_per_pair(packed_words, read_word_offsets, read_lengths, n_reads: int, pairs, n_pairs: int,
                           k: int, scoring: Scoring, results, workspace, workspace_bytes: int,
                           stream=None) -> None:
    rc = _lib().dibella_xdrop_per_pair(_ptr(packed_words), _ptr(read_word_offsets), _ptr(read_lengths),
                                       n_reads, _ptr(pairs), n_pairs, k, scoring, _ptr(results),
                                       _ptr(workspace), workspace_bytes, _stream_handle(stream))
    _check(rc, "dibella_xdrop_per_pair")


def dibella_autotune(packed_words, read_word_offsets, read_lengths, n_reads: int, pairs, n_pairs: int, k: int,
                     scoring: Scoring, results, workspace, workspace_bytes: int, stream=None, repeats: int = 2):
    """Returns (best Schedule, its median ms, number of schedules timed)."""
    best = Schedule()
    ms = ctypes.c_float(0)
    tried = ctypes.c_int32(0)
    rc = _lib().dibella_autotune(_ptr(packed_words), _ptr(read_word_offsets), _ptr(read_lengths), n_reads,
                                 _ptr(pairs), n_pairs, k, scoring, _ptr(results), _ptr(workspace),
                                 workspace_bytes, _stream_handle(stream), repeats, ctypes.byref(best),
                                 ctypes.byref(ms), ctypes.byref(tried))
    _check(rc, "dibella_autotune")
    return best, float(ms.value), int(tried.value)


def dibella_enable_phase_timing(enable: bool) -> None:
    _check(_lib().dibella_enable_phase_timing(1 if enable else 0), "dibella_enable_phase_timing")


def dibella_phase_times(n_max: int = 8) -> list[float]:
    buf = (ctypes.c_float * n_max)()
    n = _lib().dibella_phase_times(buf, n_max)
    if n < 0:
        _check(n, "dibella_phase_times")
    return [float(buf[i]) for i in range(n)]


def dibella_batch_counters(workspace, stream=None) -> dict:
    buf = (ctypes.c_int64 * 16)()
    n = _lib().dibella_batch_counters(_ptr(workspace), _stream_handle(stream), buf, 16)
    if n < 0:
        _check(n, "dibella_batch_counters")
    keys = ["narrow", "wide", "escalated_narrow", "escalated_wide", "escalated_smem", "band_overflow",
            "cells_narrow", "cells_wide", "cells_smem", "cells_global", "cells_wide_esc", "cells_ladder",
            "cells_mid", "escalated_mid", "cells_restarted", "narrow_second_pass"]
    return {keys[i]: int(buf[i]) for i in range(n)}


WARP_CLOCK_LAUNCHES = {"narrow form": 1, "narrow form, second pass": 5, "wide form, first launch": 2,
                       "mid form on the narrow escalations": 3, "wide form on the escalations": 4}


def dibella_enable_warp_clock(launch: int) -> None:
    _check(_lib().dibella_enable_warp_clock(launch), "dibella_enable_warp_clock")


def dibella_warp_clock(max_warps: int = 1 << 16) -> np.ndarray:
    """(start, end) global-timer ns of every warp of the last clocked launch."""
    buf = np.zeros((max_warps, 2), dtype=np.uint64)
    n = _lib().dibella_warp_clock(buf.ctypes.data, max_warps)
    if n < 0:
        _check(n, "dibella_warp_clock")
    return buf[:n]


INT_PEAK_CLASSES = {0: "IADD", 1: "IMNMX", 2: "VIADDMNMX int16x2", 3: "VIMNMX3 int16x2",
                    4: "int32 DP cell (8 ops)"}


def dibella_int_peak(op_class: int, iters: int, stream=None) -> tuple[float, float]:
    """Measured lane-ops/s of one integer instruction class and the timed launch's ms."""
    ops = ctypes.c_double(0)
    ms = ctypes.c_double(0)
    _check(_lib().dibella_int_peak(op_class, iters, ctypes.byref(ops), ctypes.byref(ms), _stream_handle(stream)),
           "dibella_int_peak")
    return float(ops.value), float(ms.value)


def dibella_last_launch_count() -> int:
    return int(_lib().dibella_last_launch_count())


def dibella_last_error() -> str:
    return _lib().dibella_last_error().decode()


def dibella_version() -> str:
    return _lib().dibella_version().decode()


from .store import ReadStore, Aligner  # noqa: E402  (device-memory plumbing)

__all__ = [n for n in dir() if n.startswith("dibella_")] + [
    "PAIR_DTYPE", "RESULT_DTYPE", "Scoring", "Schedule", "DibellaError", "ReadStore", "Aligner"]
