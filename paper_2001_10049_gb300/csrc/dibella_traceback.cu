// Traceback of seeded X-drop alignments: the edits of each seed's best
// alignment as run-length encoded columns (diBELLA Sec. 1: an alignment is
// the list of edits that makes two overlapping regions identical; Sec. 2: an
// alignment's columns pair two characters, or a character with a gap).
//
// The extension is the one dibella_xdrop_batch computes (band of antidiagonal
// d from the live cells of d-1 widened by one, live iff H >= best(<d) - X,
// strict improvement with the smallest i on ties, both extensions from the
// seed); each evaluated cell also keeps the move that gave its value, taking
// the diagonal first, then the step in A, then the step in B' on equal
// values.  The walk from the best cell back to the seed follows those moves.
//
// A warp per seed re-runs both extensions with the band's cells across its
// lanes.  Its scratch (a slot of the caller's workspace per warp) holds three
// rows of H indexed by the position in A, read and written coalesced, and a
// stream of 32-bit words with, per evaluated antidiagonal, two header words
// (the band's first i and its width), the band's moves at 2 bits per cell
// (packed by warp reductions), and a trailer word (the width again), so that
// lane 0 can walk back one antidiagonal at a time from the best cell.

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/dibella.h"

namespace {

constexpr int kTbThreads = 128;
constexpr int32_t kDead = INT32_MIN / 2;  // dead, or outside its antidiagonal's band
constexpr uint32_t kMoveNone = 0, kMoveDiag = 1, kMoveA = 2, kMoveB = 3;
constexpr uint32_t kOpEq = DIBELLA_OP_EQ, kOpX = DIBELLA_OP_DIFF, kOpIns = DIBELLA_OP_INS, kOpDel = DIBELLA_OP_DEL;

struct TbArgs {
  const uint32_t* words;
  const int64_t* word_offsets;
  const int32_t* lengths;
  long long n_reads;
  const dibella_pair_t* pairs;
  long long n_pairs;
  int k, M, S, G, X;
  int max_len;
  dibella_result_t* results;
  uint32_t* ops;
  int ops_per_seed;
  int32_t* n_ops;
  long long n_lanes;
  long long moves_words;
  char* workspace;
  long long lane_bytes;
};

__host__ __device__ inline long long tb_copy_words(long long len) { return ((len + 15) / 16 + 3) / 4 * 4; }

// Base q of the copy whose first base is base index `start` of the store.
__host__ __device__ inline uint32_t tb_base(const uint32_t* words, long long start, long long q) {
  const long long g = start + q;
  return (words[g >> 4] >> (2 * (g & 15))) & 3u;
}

// One extension's sequences: a(i) = base a0 + sa * i of the store (sa = +1 or
// -1), likewise b(j); m and n characters.
struct TbSeq {
  long long a0, b0;
  int sa, sb;
  int m, n;
};

struct TbExt {
  int best, i_end, j_end;
  long long cells;
  long long best_rec;  // stream index of the best antidiagonal's header (-1: the origin)
  bool recorded;       // every antidiagonal up to the best one fit the stream
};

// The X-drop extension from the origin, run by the 32 lanes of a warp (every
// lane calls it; lane l computes cell i = i0 + l of each 32-cell chunk of the
// band), recording moves into mv (capacity cap words) while they fit.  The
// rows r0..r2 (antidiagonals d, d-1, d-2, indexed by i) live in the warp's
// workspace slot, read and written coalesced.  Each chunk's 2-bit moves are
// packed 16 cells to a word by two warp OR-reductions; lane 0 writes the
// stream, so its format is the one tb_walk reads.  All lanes return the same
// result.
__device__ TbExt tb_extend_warp(const TbArgs& p, const TbSeq& s, int32_t* r0, int32_t* r1, int32_t* r2,
                                uint32_t* mv, long long cap) {
  constexpr unsigned kAll = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  TbExt e{0, 0, 0, 0, -1, true};
  int lo2 = 1, hi2 = 0, lo1 = 0, hi1 = 0;
  if (lane == 0) r1[0] = 0;
  __syncwarp();
  int live_lo = 0, live_hi = 0;
  int best = 0;
  long long w = 0;
  bool streaming = true;
  const int last_d = s.m + s.n;
  for (int d = 1; d <= last_d; ++d) {
    int lo = live_lo > d - s.n ? live_lo : d - s.n;
    if (lo < 0) lo = 0;
    int hi = live_hi + 1 < d ? live_hi + 1 : d;
    if (hi > s.m) hi = s.m;
    if (lo > hi) break;
    const int width = hi - lo + 1;
    const long long rec = w;
    const bool keep = streaming && w + 3 + (width + 15) / 16 <= cap;
    streaming = keep;
    if (keep && lane == 0) {
      mv[w] = (uint32_t)lo;
      mv[w + 1] = (uint32_t)width;
    }
    if (keep) w += 2;
    const int threshold = best - p.X;
    int row_best = kDead, row_best_i = -1, new_lo = -1, new_hi = -1;
    for (int i0 = lo; i0 <= hi; i0 += 32) {
      const int i = i0 + lane;
      const int j = d - i;
      int h = kDead;
      uint32_t from = kMoveNone;
      bool live = false;
      if (i <= hi) {
        if (i >= 1 && j >= 1 && i - 1 >= lo2 && i - 1 <= hi2 && r2[i - 1] != kDead) {
          const uint32_t x = tb_base(p.words, s.a0, (long long)s.sa * (i - 1));
          const uint32_t y = tb_base(p.words, s.b0, (long long)s.sb * (j - 1));
          const int v = r2[i - 1] + (x == y ? p.M : p.S);
          if (v > h) {
            h = v;
            from = kMoveDiag;
          }
        }
        if (i >= 1 && i - 1 >= lo1 && i - 1 <= hi1 && r1[i - 1] != kDead && r1[i - 1] + p.G > h) {
          h = r1[i - 1] + p.G;
          from = kMoveA;
        }
        if (j >= 1 && i >= lo1 && i <= hi1 && r1[i] != kDead && r1[i] + p.G > h) {
          h = r1[i] + p.G;
          from = kMoveB;
        }
        live = h != kDead && h >= threshold;
        r0[i] = live ? h : kDead;
      }
      const uint32_t bits = live ? from : kMoveNone;
      const uint32_t wlo = __reduce_or_sync(kAll, lane < 16 ? bits << (2 * lane) : 0u);
      const uint32_t whi = __reduce_or_sync(kAll, lane >= 16 ? bits << (2 * (lane - 16)) : 0u);
      const int c0 = i0 - lo;  // cell offset of the chunk; a multiple of 32
      if (keep && lane == 0) {
        mv[w + c0 / 16] = wlo;
        if (c0 + 16 < width) mv[w + c0 / 16 + 1] = whi;
      }
      const unsigned bl = __ballot_sync(kAll, live);
      if (bl) {
        if (new_lo < 0) new_lo = i0 + __ffs(bl) - 1;
        new_hi = i0 + 31 - __clz(bl);
        const int cmax = __reduce_max_sync(kAll, live ? h : kDead);
        if (cmax > row_best) {  // strictly larger: an earlier chunk (smaller i) keeps a tie
          row_best = cmax;
          row_best_i = i0 + __ffs(__ballot_sync(kAll, live && h == cmax)) - 1;
        }
      }
    }
    e.cells += width;
    if (keep) {
      w += (width + 15) / 16;
      if (lane == 0) mv[w] = (uint32_t)width;
      w += 1;
    }
    __syncwarp();  // the row of d is complete before any lane reads it as d-1
    if (new_lo < 0) break;
    if (row_best > best) {
      best = row_best;
      e.best = best;
      e.i_end = row_best_i;
      e.j_end = d - row_best_i;
      e.best_rec = rec;
      e.recorded = keep;
    }
    live_lo = new_lo;
    live_hi = new_hi;
    int32_t* t = r2;  // rotate: d-1 -> d-2, d -> d-1
    r2 = r1;
    r1 = r0;
    r0 = t;
    lo2 = lo1;
    hi2 = hi1;
    lo1 = lo;
    hi1 = hi;
  }
  return e;
}

// Run-length writer over one seed's op words.
struct TbRuns {
  uint32_t* out;
  int cap;
  int n;       // runs written
  bool full;   // more runs than cap were needed
  uint32_t op;  // pending run
  uint32_t len;
  __host__ __device__ void push(uint32_t o) { push_run(o, 1); }
  __host__ __device__ void push_run(uint32_t o, uint32_t l) {
    if (len && o == op) {
      len += l;
      return;
    }
    flush();
    op = o;
    len = l;
  }
  __host__ __device__ void flush() {
    if (!len) return;
    if (n < cap)
      out[n] = (len << 4) | op;
    else
      full = true;
    ++n;
    len = 0;
  }
};

// Walks back from the extension's best cell to the origin, pushing each
// column's op.  Returns false if a visited cell lies outside its recorded
// band or has no move.
__host__ __device__ bool tb_walk(const TbArgs& p, const TbSeq& s, const TbExt& e, const uint32_t* mv, TbRuns* runs) {
  int i = e.i_end, j = e.j_end;
  long long rec = e.best_rec;
  while (i > 0 || j > 0) {
    if (rec < 0) return false;
    const int lo = (int)mv[rec], width = (int)mv[rec + 1];
    const int c = i - lo;
    if (c < 0 || c >= width) return false;
    const uint32_t move = (mv[rec + 2 + c / 16] >> (2 * (c & 15))) & 3u;
    int steps;  // antidiagonals stepped back
    if (move == kMoveDiag) {
      const uint32_t x = tb_base(p.words, s.a0, (long long)s.sa * (i - 1));
      const uint32_t y = tb_base(p.words, s.b0, (long long)s.sb * (j - 1));
      runs->push(x == y ? kOpEq : kOpX);
      --i;
      --j;
      steps = 2;
    } else if (move == kMoveA) {
      runs->push(kOpDel);
      --i;
      steps = 1;
    } else if (move == kMoveB) {
      runs->push(kOpIns);
      --j;
      steps = 1;
    } else {
      return false;
    }
    if (i == 0 && j == 0) break;
    for (int t = 0; t < steps; ++t) {  // the record before starts after its trailer
      if (rec < 1) return false;
      const long long prev_width = mv[rec - 1];
      rec -= 3 + (prev_width + 15) / 16;
    }
  }
  return true;
}

// Everything for seed t with one warp and its workspace slot: the result
// record (as dibella_xdrop_batch writes it, without the best-of-pair flag) and
// the run-length encoded columns from (begin_a, begin_b') to (end_a, end_b').
// Every lane runs both extensions; lane 0 walks back and writes.
__device__ void tb_seed(const TbArgs& p, long long t, char* scratch) {
  const int lane = threadIdx.x & 31;
  const dibella_pair_t pr = p.pairs[t];
  dibella_result_t r;
  r.score = r.score_left = r.score_right = 0;
  r.begin_a = r.end_a = r.begin_b = r.end_b = 0;
  r.status = 0;
  r.cells = 0;
  const int k = p.k;
  bool valid = (long long)pr.read_a < p.n_reads && (long long)pr.read_b < p.n_reads && pr.strand <= 1;
  long long lenA = 0, lenB = 0;
  if (valid) {
    lenA = p.lengths[pr.read_a];
    lenB = p.lengths[pr.read_b];
    valid = (long long)pr.pos_a + k <= lenA && (long long)pr.pos_b + k <= lenB;
  }
  if (!valid) {
    r.status = DIBELLA_RES_INVALID_SEED;
    if (lane == 0) {
      p.results[t] = r;
      p.n_ops[t] = 0;
    }
    return;
  }
  if (lenA > p.max_len || lenB > p.max_len) {  // the H rows would not hold the band
    r.status = DIBELLA_RES_BAND_OVERFLOW;
    if (lane == 0) {
      p.results[t] = r;
      p.n_ops[t] = -3;
    }
    return;
  }
  const long long fA = p.word_offsets[pr.read_a] * 16;
  const long long fB = p.word_offsets[pr.read_b] * 16;
  const long long bp0 = pr.strand ? fB + tb_copy_words(lenB) * 16 : fB;  // B': forward or reverse-complement copy
  const long long pa = pr.pos_a;
  const long long pb = pr.strand ? lenB - pr.pos_b - k : (long long)pr.pos_b;
  int seed = 0;
  bool exact = true;
  for (int q = 0; q < k; ++q) {
    const bool eq = tb_base(p.words, fA, pa + q) == tb_base(p.words, bp0, pb + q);
    seed += eq ? p.M : p.S;
    exact = exact && eq;
  }
  const long long hw = (long long)p.max_len + 2;
  int32_t* rows = (int32_t*)scratch;
  uint32_t* mv = (uint32_t*)(scratch + 3 * hw * 4);
  // Left: a(i) = A[pa-1-i], b(j) = B'[pb-1-j]; right: a(i) = A[pa+k+i], b(j) = B'[pb+k+j].
  const TbSeq L{fA + pa - 1, bp0 + pb - 1, -1, -1, (int)pa, (int)pb};
  const TbSeq R{fA + pa + k, bp0 + pb + k, 1, 1, (int)(lenA - pa - k), (int)(lenB - pb - k)};
  TbRuns runs{p.ops + t * (long long)p.ops_per_seed, p.ops_per_seed, 0, false, 0, 0};
  bool ok = true;
  // The left walk runs from its best cell (the alignment's start) toward the
  // seed: its columns come out in alignment order.
  const TbExt el = tb_extend_warp(p, L, rows, rows + hw, rows + 2 * hw, mv, p.moves_words);
  if (lane == 0) {
    ok = el.recorded && tb_walk(p, L, el, mv, &runs);
    for (int q = 0; q < k && ok; ++q)
      runs.push(tb_base(p.words, fA, pa + q) == tb_base(p.words, bp0, pb + q) ? kOpEq : kOpX);
  }
  __syncwarp();  // the left walk has read the stream before the right extension rewrites it
  // The right walk yields its columns last to first: its runs go to the H
  // rows (free once the extension is done; at most m + n runs fit there),
  // then into the seed's runs in reverse order.
  const TbExt er = tb_extend_warp(p, R, rows, rows + hw, rows + 2 * hw, mv, p.moves_words);
  if (lane == 0) {
    if (ok) {
      TbRuns back{(uint32_t*)rows, (int)(3 * hw < 0x7FFFFFFF ? 3 * hw : 0x7FFFFFFF), 0, false, 0, 0};
      ok = er.recorded && tb_walk(p, R, er, mv, &back);
      back.flush();
      ok = ok && !back.full;
      for (int x = back.n - 1; x >= 0 && ok; --x) runs.push_run(back.out[x] & 15u, back.out[x] >> 4);
    }
    runs.flush();
  }
  r.score = seed + el.best + er.best;
  r.score_left = el.best;
  r.score_right = er.best;
  r.begin_a = (uint32_t)(pa - el.i_end);
  r.end_a = (uint32_t)(pa + k + er.i_end);
  const long long bb = pb - el.j_end, eb = pb + k + er.j_end;
  r.begin_b = (uint32_t)(pr.strand ? lenB - eb : bb);
  r.end_b = (uint32_t)(pr.strand ? lenB - bb : eb);
  r.status = exact ? 0 : DIBELLA_RES_SEED_MISMATCH;
  r.cells = el.cells + er.cells;
  if (lane == 0) {
    p.results[t] = r;
    p.n_ops[t] = !ok ? -2 : (runs.full ? -1 : runs.n);
  }
  __syncwarp();  // lane 0's use of the rows ends before the next seed
}

// A warp per seed: warp w (of n_lanes warps, one workspace slot each) takes
// seeds w, w + n_lanes, ...
__global__ void __launch_bounds__(kTbThreads) traceback_kernel(TbArgs p) {
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (warp >= p.n_lanes) return;
  char* scratch = p.workspace + warp * p.lane_bytes;
  for (long long t = warp; t < p.n_pairs; t += p.n_lanes) tb_seed(p, t, scratch);
}

long long tb_lane_bytes(long long max_len, long long moves_words) {
  const long long b = 3 * (max_len + 2) * 4 + moves_words * 4;
  return (b + 255) / 256 * 256;
}

}  // namespace

extern "C" {

int dibella_traceback_workspace_bytes(int64_t n_lanes, int32_t max_read_len, int64_t moves_words,
                                      int64_t* bytes_out) {
  if (!bytes_out || n_lanes < 1 || n_lanes > (1ll << 24) || max_read_len < 0 ||
      max_read_len > DIBELLA_MAX_READ_LEN || moves_words < 2 || moves_words > (1ll << 34))
    return DIBELLA_EINVAL;
  *bytes_out = (int64_t)(n_lanes * tb_lane_bytes(max_read_len, moves_words));
  return DIBELLA_OK;
}

int dibella_xdrop_traceback(const uint32_t* packed_words, const int64_t* read_word_offsets,
                            const int32_t* read_lengths, int64_t n_reads, int32_t max_read_len,
                            const dibella_pair_t* pairs, int64_t n_pairs, int32_t k, dibella_scoring_t scoring,
                            dibella_result_t* results, uint32_t* ops, int32_t ops_per_seed, int32_t* n_ops,
                            int64_t n_lanes, int64_t moves_words, void* workspace, int64_t workspace_bytes,
                            void* stream) {
  if (n_reads < 0 || n_pairs < 0 || n_pairs > (1ll << 29) || k < 1 || k > DIBELLA_MAX_K) return DIBELLA_EINVAL;
  if (scoring.match <= 0 || scoring.match > DIBELLA_MAX_SCORE || scoring.mismatch > 0 ||
      scoring.mismatch < -DIBELLA_MAX_SCORE || scoring.gap >= 0 || scoring.gap < -DIBELLA_MAX_SCORE ||
      scoring.xdrop < 0 || scoring.xdrop > DIBELLA_XDROP_INF)
    return DIBELLA_EINVAL;
  if (ops_per_seed < 1 || max_read_len < 0 || max_read_len > DIBELLA_MAX_READ_LEN) return DIBELLA_EINVAL;
  int64_t need = 0;
  if (dibella_traceback_workspace_bytes(n_lanes, max_read_len, moves_words, &need) != DIBELLA_OK)
    return DIBELLA_EINVAL;
  if (n_pairs > 0 && (!packed_words || !read_word_offsets || !read_lengths || !pairs || !results || !ops ||
                      !n_ops))
    return DIBELLA_EINVAL;
  if (!workspace || ((uintptr_t)workspace & 255)) return DIBELLA_EINVAL;
  if (workspace_bytes < need) return DIBELLA_ENOMEM;
  if (n_pairs == 0) return DIBELLA_OK;
  TbArgs a;
  a.words = packed_words;
  a.word_offsets = read_word_offsets;
  a.lengths = read_lengths;
  a.n_reads = n_reads;
  a.pairs = pairs;
  a.n_pairs = n_pairs;
  a.k = k;
  a.M = scoring.match;
  a.S = scoring.mismatch;
  a.G = scoring.gap;
  a.X = scoring.xdrop;
  a.max_len = max_read_len;
  a.results = results;
  a.ops = ops;
  a.ops_per_seed = ops_per_seed;
  a.n_ops = n_ops;
  a.n_lanes = n_lanes < n_pairs ? n_lanes : n_pairs;
  a.moves_words = moves_words;
  a.workspace = (char*)workspace;
  a.lane_bytes = tb_lane_bytes(max_read_len, moves_words);
  const long long blocks = (a.n_lanes * 32 + kTbThreads - 1) / kTbThreads;
  traceback_kernel<<<(unsigned)blocks, kTbThreads, 0, (cudaStream_t)stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? DIBELLA_OK : DIBELLA_ECUDA;
}

}  // extern "C"
