"""Continuous-batching X-drop service over a device-resident read store.

Requests (a set of seed records plus an X-drop value) arrive over time.  The
loop keeps the GPU busy without a fixed batch size:

* arrived requests wait in one queue per X (a batch has one scoring);
* whenever device memory and a stream are free, the oldest waiting requests
  of one X are merged (up to ``max_batch`` seeds) into one batch, which is
  admitted only if its staging + workspace bytes fit in what is left of the
  device arena (admission by free device memory);
* the batch runs dibella_xdrop_batch on its own stream, so batches admitted
  while others are running overlap on the device; its results come back by an
  asynchronous copy into pinned memory and an event marks completion;
* a request completes when its batch's event has fired; its latency is
  completion minus its scheduled arrival.

Every result is computed by the library's kernels; this module only moves
bytes and keeps time.  Merging never changes a result: records are
independent, and two requests are not placed back to back when the last seed of
one and the first seed of the next belong to the same read pair (which would
join their runs for the best-seed flag).
"""

from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import (RESULT_DTYPE, Scoring, dibella_staging_bytes, dibella_xdrop_batch,
               dibella_xdrop_workspace_bytes)


@dataclass
class Request:
    rid: int
    arrival: float                  # seconds after the start of the run
    xdrop: int
    pairs: np.ndarray               # PAIR_DTYPE seed records
    done: float | None = None
    result: np.ndarray | None = None


@dataclass
class _Batch:
    xdrop: int
    members: list                   # (request, start, count)
    n: int
    offset: int                     # arena offset
    nbytes: int
    stream: int                     # slot index (stream, pinned buffers)
    event: object
    host_res: object
    launched: float = 0.0


class Arena:
    """First-fit allocator over one device buffer (bytes, 256-byte aligned)."""

    def __init__(self, nbytes: int, device):
        import torch
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.size = nbytes
        self.free = [(0, nbytes)]

    def alloc(self, n: int):
        n = (n + 255) & ~255
        for i, (off, sz) in enumerate(self.free):
            if sz >= n:
                if sz == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, sz - n)
                return off, n
        return None

    def release(self, off: int, n: int):
        self.free.append((off, n))
        self.free.sort()
        merged = []
        for o, s in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + s)
            else:
                merged.append((o, s))
        self.free = merged

    @property
    def free_bytes(self) -> int:
        return sum(s for _, s in self.free)


class Server:
    def __init__(self, store, k: int = 17, scoring=(1, -1, -1), arena_bytes: int = 2 << 30,
                 max_batch: int = 65536, n_streams: int = 8, device="cuda"):
        import torch
        self.store, self.k, self.scoring, self.device = store, k, scoring, device
        self.max_batch = max_batch
        self.arena = Arena(arena_bytes, device)
        self.streams = [torch.cuda.Stream(device=device) for _ in range(n_streams)]
        self.free_slots = collections.deque(range(n_streams))
        self.host_pairs = torch.empty((n_streams, max_batch, 24), dtype=torch.uint8).pin_memory()
        self.host_res = torch.empty((n_streams, max_batch, 40), dtype=torch.uint8).pin_memory()
        self.max_len = max(1, store.max_len)
        need = self.batch_bytes(max_batch)
        if need > arena_bytes:
            raise ValueError("arena of %d bytes cannot hold one batch of %d seeds (%d bytes)"
                             % (arena_bytes, max_batch, need))

    def batch_bytes(self, n: int) -> int:
        return dibella_staging_bytes(n) + dibella_xdrop_workspace_bytes(n, self.max_len) + 256

    # -- launching --------------------------------------------------------------
    def _launch(self, members, xdrop: int, now: float):
        import torch
        n = sum(c for _, _, c in members)
        got = self.arena.alloc(self.batch_bytes(n))
        if got is None:
            return None
        off, nbytes = got
        slot = self.free_slots.popleft()
        stream = self.streams[slot]
        host = self.host_pairs[slot, :n]
        pos = 0
        for req, start, cnt in members:
            host[pos:pos + cnt].copy_(torch.from_numpy(req.pairs[start:start + cnt].view(np.uint8).reshape(cnt, 24)))
            pos += cnt
        base = self.arena.buf[off:off + nbytes]
        res_off = (n * 24 + 255) // 256 * 256
        ws_off = (dibella_staging_bytes(n) + 255) // 256 * 256
        pairs_dev, res_dev, ws = base[:n * 24], base[res_off:res_off + n * 40], base[ws_off:]
        event = torch.cuda.Event()
        with torch.cuda.stream(stream):
            pairs_dev.copy_(host.reshape(-1), non_blocking=True)
            M, S, G = self.scoring
            dibella_xdrop_batch(self.store.words, self.store.word_offsets, self.store.lengths, self.store.n_reads,
                                pairs_dev, n, self.k, Scoring(M, S, G, xdrop), res_dev, ws, nbytes - ws_off,
                                stream=stream)
            self.host_res[slot, :n].reshape(-1).copy_(res_dev, non_blocking=True)
            event.record(stream)
        return _Batch(xdrop, members, n, off, nbytes, slot, event, None, now)

    def _finish(self, b: _Batch, now: float):
        res = self.host_res[b.stream, :b.n].numpy().reshape(-1).view(RESULT_DTYPE)
        pos = 0
        for req, start, cnt in b.members:
            req.result[start:start + cnt] = res[pos:pos + cnt]
            pos += cnt
            req._left -= cnt
            if req._left == 0:
                req.done = now
        self.arena.release(b.offset, b.nbytes)
        self.free_slots.append(b.stream)

    def _merge(self, q):
        """The oldest waiting work of one X, up to max_batch seeds, split only at
        candidate-pair boundaries; runs of different requests never touch."""
        members, n, last_key = [], 0, None
        for r in q:
            remaining = len(r.pairs) - r._next
            take = min(remaining, self.max_batch - n)
            if take < remaining:
                p, e = r.pairs, r._next + take
                while e > r._next and p[e]["read_a"] == p[e - 1]["read_a"] and p[e]["read_b"] == p[e - 1]["read_b"]:
                    e -= 1
                take = e - r._next
                if take == 0:
                    break
            first = r.pairs[r._next]
            if last_key is not None and (int(first["read_a"]), int(first["read_b"])) == last_key:
                break
            members.append((r, r._next, take))
            n += take
            last = r.pairs[r._next + take - 1]
            last_key = (int(last["read_a"]), int(last["read_b"]))
            if take < remaining or n >= self.max_batch:
                break
        return members

    # -- the loop ---------------------------------------------------------------
    def run(self, requests: list[Request], timeout_s: float = 600.0) -> dict:
        """Serve `requests` in real time (arrivals relative to the start).  Returns
        latency statistics; each request's `result` and `done` are filled in."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            r._left, r._next, r.done = len(r.pairs), 0, None
            r.result = np.zeros(len(r.pairs), dtype=RESULT_DTYPE)
        pending = collections.deque(reqs)
        waiting = collections.defaultdict(collections.deque)
        inflight: list[_Batch] = []
        t0 = time.perf_counter()
        n_batches = max_inflight = 0
        while True:
            now = time.perf_counter() - t0
            if now > timeout_s:
                raise TimeoutError("serving loop exceeded %.0f s" % timeout_s)
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                if r._left == 0:
                    r.done = max(now, r.arrival)
                else:
                    waiting[r.xdrop].append(r)
            still = []
            for b in inflight:
                if b.event.query():
                    self._finish(b, time.perf_counter() - t0)
                else:
                    still.append(b)
            inflight = still
            launched = False
            while self.free_slots:
                heads = [(q[0].arrival, x) for x, q in waiting.items() if q]
                if not heads:
                    break
                x = min(heads)[1]
                q = waiting[x]
                members = self._merge(q)
                if not members:
                    break
                b = self._launch(members, x, now)
                if b is None:  # admission refused: not enough free device memory yet
                    break
                for r, start, cnt in members:
                    r._next = start + cnt
                while q and q[0]._next == len(q[0].pairs):
                    q.popleft()
                inflight.append(b)
                n_batches += 1
                launched = True
            max_inflight = max(max_inflight, len(inflight))
            if not pending and not inflight and not any(waiting.values()):
                break
            if not launched:
                time.sleep(0.0001)
        lat = np.array([r.done - r.arrival for r in reqs])
        span = max(r.done for r in reqs) - min(r.arrival for r in reqs) if reqs else 0.0
        total_pairs = sum(len(workloads_groups(r.pairs)) for r in reqs)
        return {"requests": len(reqs), "batches": n_batches, "max_inflight": max_inflight,
                "p50_ms": float(np.percentile(lat, 50, method="nearest") * 1e3) if len(lat) else 0.0,
                "p99_ms": float(np.percentile(lat, 99, method="nearest") * 1e3) if len(lat) else 0.0,
                "mean_ms": float(lat.mean() * 1e3) if len(lat) else 0.0,
                "span_s": span, "pairs": total_pairs,
                "pairs_per_s": total_pairs / span if span > 0 else 0.0}


def workloads_groups(pairs: np.ndarray) -> list[int]:
    """Start index of each run of seed records sharing (read_a, read_b)."""
    if len(pairs) == 0:
        return []
    key = pairs["read_a"].astype(np.uint64) << np.uint64(32) | pairs["read_b"].astype(np.uint64)
    return list(np.flatnonzero(np.concatenate([[True], key[1:] != key[:-1]])))
