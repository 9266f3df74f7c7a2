"""Device-memory plumbing around the C ABI: a resident packed read store and an
aligner that owns its workspace.  No alignment arithmetic happens here."""

from __future__ import annotations

import numpy as np


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the dibella X-drop path needs a CUDA GPU; none is visible")
    return torch


class ReadStore:
    """Reads packed by dibella_pack_reads and resident in HBM (diBELLA Sec. 3's
    2-bit encoding, both orientations; layout in include/dibella.h)."""

    def __init__(self, words: np.ndarray, word_offsets: np.ndarray, lengths: np.ndarray, device="cuda"):
        torch = _torch()
        self.n_reads = int(len(lengths))
        self.max_len = int(lengths.max()) if len(lengths) else 0
        self.n_bases = int(lengths.sum()) if len(lengths) else 0
        self.words = torch.from_numpy(words.view(np.int32)).to(device)
        self.word_offsets = torch.from_numpy(np.ascontiguousarray(word_offsets)).to(device)
        self.lengths = torch.from_numpy(np.ascontiguousarray(lengths)).to(device)
        self.lengths_host = np.ascontiguousarray(lengths)

    @classmethod
    def from_ascii(cls, ascii: np.ndarray, offsets: np.ndarray, device="cuda", n_threads: int = 0):
        from . import dibella_pack_reads
        words, woffs, lens = dibella_pack_reads(ascii, offsets, n_threads)
        return cls(words, woffs, lens, device)

    @property
    def nbytes(self) -> int:
        return self.words.numel() * 4 + self.word_offsets.numel() * 8 + self.lengths.numel() * 4

    def candidate_pairs(self, k: int = 17, mult_lo: int = 2, mult_hi: int = 8, max_seeds: int = 1,
                        min_seed_gap: int = 0, stream=None, workspace=None):
        """Seed records of every candidate pair of the store's reads, computed on
        the GPU by dibella_candidate_pairs (k-mer counting, multiplicity filter,
        pairs per retained k-mer, seed selection), and its counts.  Synchronous:
        returns (records as a numpy PAIR_DTYPE array, dict of counts)."""
        from . import PAIR_DTYPE, dibella_candidate_pairs, dibella_candidate_workspace_bytes
        torch = _torch()
        dev = self.words.device
        ws_bytes = dibella_candidate_workspace_bytes(self.n_reads, self.n_bases, k, mult_hi)
        if workspace is None or workspace.numel() < ws_bytes:
            workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        counts = torch.zeros(6, dtype=torch.int64, device=dev)
        cap = max(1024, self.n_bases // 16)
        for _ in range(2):
            out = torch.empty((cap, 24), dtype=torch.uint8, device=dev)
            dibella_candidate_pairs(self.words, self.word_offsets, self.lengths, self.n_reads, self.n_bases,
                                    self.max_len, k, mult_lo, mult_hi, max_seeds, min_seed_gap, out, cap, counts,
                                    workspace, ws_bytes, stream)
            torch.cuda.synchronize(dev)
            c = counts.cpu().numpy()
            if not (int(c[5]) & 4):
                break
            cap = int(c[0])  # the seed records did not fit: once more, exactly sized
        stats = dict(zip(["seeds", "candidate_pairs", "instances", "retained_kmers", "occurrence_pairs", "status"],
                         (int(v) for v in c)))
        if stats["status"]:
            raise RuntimeError("dibella_candidate_pairs incomplete, status %d" % stats["status"])
        recs = out[:stats["seeds"]].cpu().numpy().reshape(-1).view(PAIR_DTYPE)
        return recs, stats


    def candidate_pairs_parts(self, k: int = 17, mult_lo: int = 2, mult_hi: int = 8, max_seeds: int = 1,
                              min_seed_gap: int = 0, n_parts: int = 1, occ_pair_capacity: int | None = None,
                              pairs_capacity: int | None = None, max_read_len: int | None = None, stream=None,
                              to_host: bool = True):
        """dibella_candidate_pairs_parts: the same seed records, counted in
        n_parts hash passes (for read sets beyond one sort key).  Synchronous:
        returns (records, dict of counts); records are a numpy PAIR_DTYPE array,
        or with to_host=False a device uint8 tensor of shape (seeds, 24)."""
        from . import PAIR_DTYPE, dibella_candidate_pairs_parts, dibella_candidate_workspace_bytes_parts
        torch = _torch()
        dev = self.words.device
        mrl = self.max_len if max_read_len is None else max_read_len
        occ_cap = occ_pair_capacity
        if occ_cap is None:
            # The most occurrence pairs the multiplicity window allows, or as many
            # as 85% of the free device memory holds (workspace plus one 24-byte
            # output record per occurrence pair), whichever is smaller.
            worst = max(1024, self.n_bases * (mult_hi - 1) // 2 + 1)
            base = dibella_candidate_workspace_bytes_parts(self.n_reads, self.n_bases, mrl, k, n_parts, 0)
            per = dibella_candidate_workspace_bytes_parts(self.n_reads, self.n_bases, mrl, k, n_parts, 1 << 20) - base
            free = torch.cuda.mem_get_info(dev)[0]
            fit = int((0.85 * free - base) / (per / float(1 << 20) + 24))
            occ_cap = max(1024, min(worst, fit))
        cap = pairs_capacity if pairs_capacity is not None else max(1024, occ_cap)
        ws_bytes = dibella_candidate_workspace_bytes_parts(self.n_reads, self.n_bases, mrl, k, n_parts, occ_cap)
        workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        counts = torch.zeros(7, dtype=torch.int64, device=dev)
        out = torch.empty((cap, 24), dtype=torch.uint8, device=dev)
        dibella_candidate_pairs_parts(self.words, self.word_offsets, self.lengths, self.n_reads, self.n_bases, mrl, k,
                                      mult_lo, mult_hi, max_seeds, min_seed_gap, n_parts, occ_cap, out, cap, counts,
                                      workspace, ws_bytes, stream)
        torch.cuda.synchronize(dev)
        del workspace
        c = counts.cpu().numpy()
        stats = dict(zip(["seeds", "candidate_pairs", "instances", "retained_kmers", "occurrence_pairs", "status",
                          "max_pass"], (int(v) for v in c)))
        if stats["status"]:
            raise RuntimeError("dibella_candidate_pairs_parts incomplete, status %d" % stats["status"])
        recs = out[:stats["seeds"]]
        if to_host:
            recs = recs.cpu().numpy().reshape(-1).view(PAIR_DTYPE)
        return recs, stats


class Aligner:
    """Runs dibella_xdrop_batch on a ReadStore with a reusable workspace."""

    def __init__(self, store: ReadStore, max_pairs: int, k: int = 17, device="cuda"):
        from . import dibella_xdrop_workspace_bytes
        torch = _torch()
        self.store, self.k, self.device = store, k, device
        self.max_pairs = max(1, int(max_pairs))
        self.workspace_bytes = dibella_xdrop_workspace_bytes(self.max_pairs, max(store.max_len, 1))
        self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=device)
        self.pairs = torch.empty((self.max_pairs, 24), dtype=torch.uint8, device=device)
        self.results = torch.empty((self.max_pairs, 40), dtype=torch.uint8, device=device)

    def upload_pairs(self, pairs: np.ndarray, non_blocking: bool = False):
        torch = _torch()
        n = len(pairs)
        if n > self.max_pairs:
            raise ValueError("batch of %d seeds exceeds this aligner's capacity %d" % (n, self.max_pairs))
        if n:
            src = torch.from_numpy(np.ascontiguousarray(pairs).view(np.uint8).reshape(n, 24))
            self.pairs[:n].copy_(src, non_blocking=non_blocking)
        return n

    def run(self, n_pairs: int, scoring, stream=None, sched=None, per_pair: bool = False):
        """Align the first n_pairs uploaded seeds into self.results (device, async)."""
        from . import Scoring, dibella_xdrop_batch, dibella_xdrop_per_pair
        s = scoring if isinstance(scoring, Scoring) else Scoring(*scoring)
        st = self.store
        if per_pair:
            dibella_xdrop_per_pair(st.words, st.word_offsets, st.lengths, st.n_reads, self.pairs, n_pairs,
                                   self.k, s, self.results, self.workspace, self.workspace_bytes, stream)
        else:
            dibella_xdrop_batch(st.words, st.word_offsets, st.lengths, st.n_reads, self.pairs, n_pairs,
                                self.k, s, self.results, self.workspace, self.workspace_bytes, stream, sched)

    def results_host(self, n_pairs: int) -> np.ndarray:
        from . import RESULT_DTYPE
        return self.results[:n_pairs].cpu().numpy().reshape(-1).view(RESULT_DTYPE)

    def traceback(self, pairs: np.ndarray, scoring, ops_per_seed: int = 4096, n_lanes: int | None = None,
                  moves_words: int = 1 << 18):
        """The seeds' results and the run-length encoded columns of their best
        alignments (dibella_xdrop_traceback; synchronous): (results,
        ops[n, ops_per_seed] uint32, n_ops[n] int32).  Scratch: n_lanes warp
        slots (default 24 per SM, where one warp per seed is no longer latency
        bound) of 3 x (longest read + 2) int32 plus moves_words words."""
        from . import RESULT_DTYPE, Scoring, dibella_traceback_workspace_bytes, dibella_xdrop_traceback
        torch = _torch()
        s = scoring if isinstance(scoring, Scoring) else Scoring(*scoring)
        n = self.upload_pairs(pairs)
        ops = torch.zeros((max(n, 1), ops_per_seed), dtype=torch.int32, device=self.device)
        n_ops = torch.zeros(max(n, 1), dtype=torch.int32, device=self.device)
        if n_lanes is None:
            n_lanes = 24 * torch.cuda.get_device_properties(self.device).multi_processor_count
        lanes = max(1, min(n_lanes, n))
        st = self.store
        ws_bytes = dibella_traceback_workspace_bytes(lanes, max(st.max_len, 1), moves_words)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=self.device)
        dibella_xdrop_traceback(st.words, st.word_offsets, st.lengths, st.n_reads, max(st.max_len, 1), self.pairs,
                                n, self.k, s, self.results, ops, ops_per_seed, n_ops, lanes, moves_words, ws,
                                ws_bytes)
        torch.cuda.synchronize()
        res = self.results[:n].cpu().numpy().reshape(-1).view(RESULT_DTYPE)
        return res, ops[:n].cpu().numpy().view(np.uint32), n_ops[:n].cpu().numpy()

    def align(self, pairs: np.ndarray, scoring, sched=None, per_pair: bool = False) -> np.ndarray:
        """Upload, align and download one batch (synchronous convenience)."""
        torch = _torch()
        n = self.upload_pairs(pairs)
        self.run(n, scoring, sched=sched, per_pair=per_pair)
        torch.cuda.synchronize()
        return self.results_host(n)
