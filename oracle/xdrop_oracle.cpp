// Oracle: plain, slow, CPU reference of seed-and-extend X-drop alignment.
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
// bench's CPU-baseline leg load this library.  It shares no code, header,
// table or helper with the CUDA path and must never be used as a fallback
// for it.
//
// What it computes (diBELLA, Sec. 2 "Read-to-Read Alignment"):
//   * a pairwise alignment of s and t is a pair of equal-length gapped strings
//     with no column holding two gaps; its score rewards matches and penalises
//     mismatches, insertions and deletions (Sec. 2, alignment definition);
//   * instead of full O(|s||t|) dynamic programming, each candidate pair is
//     extended from a shared k-mer seed with an X-drop search that abandons a
//     path once its score falls X below the best seen so far (Sec. 2, X-drop
//     paragraph, after Zhang et al. 2000), once per seed (Sec. 8, seed
//     selection; Sec. 9, per-pair alignment).
// The paper gives no recurrence, band rule or tie-break, so this file commits
// to one reading, written out step by step in the order of the antidiagonal
// algorithm:
//   R1  the cells evaluated on antidiagonal d are the i in
//       [lo(d-1), hi(d-1)+1] clipped to the matrix, where lo/hi are the
//       smallest/largest i of LIVE cells on d-1;
//   R2  a cell is live iff H >= best(<d) - X (threshold fixed for the whole
//       antidiagonal); dead cells act as -infinity;
//   R3  best improves only on a strictly larger value; within the improving
//       antidiagonal the live cell of smallest i wins;
//   R4  `cells` counts every evaluated cell on antidiagonals d >= 1;
//   R5  seeded score = seed score + left best + right best, half-open
//       coordinates, read B reported in forward coordinates;
//   R12 the traceback (the edits of the alignment, Sec. 1) follows, from the
//       best cell back to the origin, the move that gave each cell its value,
//       taking the diagonal first, then the step in a, then the step in b
//       when values are equal; the seeded alignment's columns are the left
//       extension's reversed, the seed's, then the right extension's, in A
//       and B' (B reverse complemented for strand 1).
// Arithmetic is int64 (the paper fixes no precision; scores are integers).
//
// Parity pinned by the tests: hand-worked examples (golden files), an
// independent full dynamic program for X = infinity, brute-force enumeration
// of all alignments on tiny inputs, and invariants (mirror symmetry, X
// monotonicity bound, cell bounds); the traceback by hand-worked columns, by
// an independent full-matrix traceback at X = infinity, and by rescoring the
// columns against the sequences (they must consume exactly the aligned
// ranges and add up to the reported score).

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

namespace {

const int64_t kNegInf = INT64_MIN / 4;   // "dead" / outside the band

struct ExtOut {
  int64_t best;    // best score of the extension (>= 0: the empty extension)
  int64_t i_end;   // characters of a consumed by the best extension
  int64_t j_end;   // characters of b consumed by the best extension
  int64_t cells;   // evaluated cells, antidiagonals d >= 1 (R4)
  int64_t tie;     // 1 if the winning antidiagonal held >1 cell of the best value
};

// Score of aligning character x against character y (Sec. 2 scoring scheme).
inline int64_t substitution(char x, char y, int64_t match, int64_t mismatch) {
  return x == y ? match : mismatch;
}

// One antidiagonal of the DP: H values indexed by i, valid on [lo, hi].
struct Antidiagonal {
  std::vector<int64_t> h;
  int64_t lo = 1, hi = 0;   // evaluated band; empty when lo > hi
  int64_t at(int64_t i) const {
    if (i < lo || i > hi) return kNegInf;
    return h[(size_t)i];
  }
};

// One-direction X-drop extension of a[0..m) against b[0..n), starting from
// the cell (0,0) that holds score 0.  i indexes a, j indexes b, d = i + j.
// Predecessor of an evaluated cell, for the traceback: the move that gave its
// value, taking on equal values the diagonal first, then the step in a, then
// the step in b (kFromNone: no live predecessor, the cell is dead).
enum : uint8_t { kFromNone = 0, kFromDiag = 1, kFromUp = 2, kFromLeft = 3 };

// Predecessors of every evaluated cell: moves[d] holds antidiagonal d's band
// [move_lo[d], move_lo[d] + moves[d].size()).
struct Moves {
  std::vector<std::vector<uint8_t>> moves;
  std::vector<int64_t> move_lo;
};

ExtOut extend(const char* a, int64_t m, const char* b, int64_t n, int64_t match,
              int64_t mismatch, int64_t gap, int64_t xdrop,
              std::vector<int64_t>* band_sizes = nullptr, Moves* record = nullptr) {
  ExtOut out{0, 0, 0, 0, 0};
  Antidiagonal d2, d1, d0;  // antidiagonals d-2, d-1, d
  d2.h.assign((size_t)m + 1, kNegInf);
  d1.h.assign((size_t)m + 1, kNegInf);
  d0.h.assign((size_t)m + 1, kNegInf);

  // Antidiagonal 0: the single cell (0,0) with score 0, live.
  d1.lo = 0;
  d1.hi = 0;
  d1.h[0] = 0;
  int64_t live_lo = 0, live_hi = 0;  // live cells of antidiagonal d-1
  int64_t best = 0;
  if (record) {  // antidiagonal 0: the origin, reached by no move
    record->moves.assign(1, std::vector<uint8_t>(1, kFromNone));
    record->move_lo.assign(1, 0);
  }

  for (int64_t d = 1; d <= m + n; ++d) {
    // R1: band of d from the live cells of d-1, clipped to 0<=i<=m, 0<=j<=n.
    int64_t lo = std::max<int64_t>(std::max<int64_t>(live_lo, d - n), 0);
    int64_t hi = std::min<int64_t>(std::min<int64_t>(live_hi + 1, d), m);
    if (lo > hi) break;
    d0.lo = lo;
    d0.hi = hi;
    const int64_t threshold = best - xdrop;  // R2: fixed for this antidiagonal
    if (record) {
      record->moves.emplace_back((size_t)(hi - lo + 1), kFromNone);
      record->move_lo.push_back(lo);
    }

    int64_t row_best = kNegInf, row_best_i = -1, row_best_count = 0;
    int64_t new_live_lo = -1, new_live_hi = -1;
    for (int64_t i = lo; i <= hi; ++i) {
      const int64_t j = d - i;
      int64_t h = kNegInf;
      uint8_t from = kFromNone;
      // H(i-1, j-1) + s(a[i-1], b[j-1]): antidiagonal d-2, index i-1.
      if (i >= 1 && j >= 1) {
        const int64_t diag = d2.at(i - 1);
        if (diag != kNegInf) {
          const int64_t v = diag + substitution(a[i - 1], b[j - 1], match, mismatch);
          if (v > h) {
            h = v;
            from = kFromDiag;
          }
        }
      }
      // H(i-1, j) + gap: antidiagonal d-1, index i-1.
      if (i >= 1) {
        const int64_t up = d1.at(i - 1);
        if (up != kNegInf && up + gap > h) {
          h = up + gap;
          from = kFromUp;
        }
      }
      // H(i, j-1) + gap: antidiagonal d-1, index i.
      if (j >= 1) {
        const int64_t left = d1.at(i);
        if (left != kNegInf && left + gap > h) {
          h = left + gap;
          from = kFromLeft;
        }
      }
      out.cells += 1;  // R4: every cell of the band is evaluated
      const bool live = (h != kNegInf) && (h >= threshold);  // R2
      d0.h[(size_t)i] = live ? h : kNegInf;
      if (!live) continue;
      if (record) record->moves.back()[(size_t)(i - lo)] = from;
      if (new_live_lo < 0) new_live_lo = i;
      new_live_hi = i;
      if (h > row_best) {  // ascending i: first maximum = smallest i
        row_best = h;
        row_best_i = i;
        row_best_count = 1;
      } else if (h == row_best) {
        row_best_count += 1;
      }
    }

    if (band_sizes) band_sizes->push_back(hi - lo + 1);
    if (new_live_lo < 0) break;  // no live cell on d: the extension stops
    if (row_best > best) {       // R3: strict improvement only
      best = row_best;
      out.best = best;
      out.i_end = row_best_i;
      out.j_end = d - row_best_i;
      out.tie = row_best_count > 1 ? 1 : 0;
    }
    live_lo = new_live_lo;
    live_hi = new_live_hi;
    // Rotate: d-1 becomes d-2, d becomes d-1.
    std::swap(d2, d1);
    std::swap(d1, d0);
  }
  return out;
}

// The edits of the best extension (Sec. 1: an alignment is the list of edits
// that makes the two overlapping regions identical; Sec. 2: its columns pair
// two characters or a character with a gap).  Walks the recorded moves back
// from the best cell to the origin and returns the columns from the origin
// on: '=' equal pair, 'X' unequal pair, 'D' a character of a against a gap,
// 'I' a character of b against a gap.  Returns false if a cell on the way has
// no move (cannot happen for a cell the extension reported).
bool trace_columns(const char* a, const char* b, int64_t i, int64_t j, const Moves& mv,
                   std::string* cols) {
  std::string rev;
  while (i > 0 || j > 0) {
    const int64_t d = i + j;
    if (d >= (int64_t)mv.moves.size()) return false;
    const int64_t at = i - mv.move_lo[(size_t)d];
    if (at < 0 || at >= (int64_t)mv.moves[(size_t)d].size()) return false;
    switch (mv.moves[(size_t)d][(size_t)at]) {
      case kFromDiag:
        rev.push_back(a[i - 1] == b[j - 1] ? '=' : 'X');
        --i;
        --j;
        break;
      case kFromUp:
        rev.push_back('D');
        --i;
        break;
      case kFromLeft:
        rev.push_back('I');
        --j;
        break;
      default:
        return false;
    }
  }
  cols->assign(rev.rbegin(), rev.rend());
  return true;
}

char complement(char c) {
  switch (c) {
    case 'A': return 'T';
    case 'C': return 'G';
    case 'G': return 'C';
    case 'T': return 'A';
    default: return 'N';
  }
}

std::string reverse_complement(const std::string& s) {
  std::string r(s.rbegin(), s.rend());
  for (char& c : r) c = complement(c);
  return r;
}

std::string reversed(const std::string& s) { return std::string(s.rbegin(), s.rend()); }

// Byte layout of one candidate seed (24 bytes, little endian):
//   u32 read_a, u32 read_b, u32 pos_a, u32 pos_b, u8 strand, u8 pad[3], u32 seed_id
struct OraclePair {
  uint32_t read_a, read_b, pos_a, pos_b;
  uint8_t strand;
  uint8_t pad[3];
  uint32_t seed_id;
};
static_assert(sizeof(OraclePair) == 24, "pair record is 24 bytes");

// Byte layout of one result (40 bytes):
//   i32 score, i32 score_left, i32 score_right,
//   u32 begin_a, u32 end_a, u32 begin_b, u32 end_b, i32 status, i64 cells
struct OracleResult {
  int32_t score, score_left, score_right;
  uint32_t begin_a, end_a, begin_b, end_b;
  int32_t status;
  int64_t cells;
};
static_assert(sizeof(OracleResult) == 40, "result record is 40 bytes");

const int32_t kStatusSeedMismatch = 1;  // seed bases are not identical
const int32_t kStatusInvalidSeed = 2;   // read id or seed position out of range
const int32_t kStatusBestOfPair = 4;    // best seed of its candidate pair

// Seeded alignment of one candidate (R5).  The seed is the shared k-mer at
// pos_a in A and pos_b in forward B; strand 1 means B is read reverse
// complemented (B' = revcomp(B), seed at len_B - pos_b - k in B').
OracleResult align_seed(const std::string& A, const std::string& B, const OraclePair& p,
                        int64_t k, int64_t match, int64_t mismatch, int64_t gap,
                        int64_t xdrop, ExtOut* left_out, ExtOut* right_out) {
  OracleResult r;
  std::memset(&r, 0, sizeof(r));
  const int64_t len_a = (int64_t)A.size(), len_b = (int64_t)B.size();
  if (p.strand > 1 || (int64_t)p.pos_a + k > len_a || (int64_t)p.pos_b + k > len_b) {
    r.status = kStatusInvalidSeed;
    return r;
  }
  const std::string Bp = p.strand ? reverse_complement(B) : B;
  const int64_t pa = p.pos_a;
  const int64_t pb = p.strand ? len_b - (int64_t)p.pos_b - k : (int64_t)p.pos_b;

  int64_t seed_score = 0;
  bool seed_exact = true;
  for (int64_t t = 0; t < k; ++t) {
    seed_score += substitution(A[(size_t)(pa + t)], Bp[(size_t)(pb + t)], match, mismatch);
    if (A[(size_t)(pa + t)] != Bp[(size_t)(pb + t)]) seed_exact = false;
  }

  // Left extension: reversed prefixes before the seed.
  const std::string la = reversed(A.substr(0, (size_t)pa));
  const std::string lb = reversed(Bp.substr(0, (size_t)pb));
  // Right extension: suffixes after the seed.
  const std::string ra = A.substr((size_t)(pa + k));
  const std::string rb = Bp.substr((size_t)(pb + k));
  const ExtOut L = extend(la.data(), (int64_t)la.size(), lb.data(), (int64_t)lb.size(),
                          match, mismatch, gap, xdrop);
  const ExtOut R = extend(ra.data(), (int64_t)ra.size(), rb.data(), (int64_t)rb.size(),
                          match, mismatch, gap, xdrop);
  if (left_out) *left_out = L;
  if (right_out) *right_out = R;

  r.score = (int32_t)(seed_score + L.best + R.best);
  r.score_left = (int32_t)L.best;
  r.score_right = (int32_t)R.best;
  r.begin_a = (uint32_t)(pa - L.i_end);
  r.end_a = (uint32_t)(pa + k + R.i_end);
  const int64_t begin_bp = pb - L.j_end, end_bp = pb + k + R.j_end;
  if (p.strand) {
    r.begin_b = (uint32_t)(len_b - end_bp);
    r.end_b = (uint32_t)(len_b - begin_bp);
  } else {
    r.begin_b = (uint32_t)begin_bp;
    r.end_b = (uint32_t)end_bp;
  }
  r.status = seed_exact ? 0 : kStatusSeedMismatch;
  r.cells = L.cells + R.cells;
  return r;
}

// Columns of the whole seeded alignment, from (begin_a, begin_b') to
// (end_a, end_b') in A and B' (B reverse complemented when strand = 1): the
// left extension's columns in reverse order (it ran on reversed prefixes), the
// k seed columns, then the right extension's columns.  Empty for an invalid
// seed; false if a traceback failed.
bool seed_columns(const std::string& A, const std::string& B, const OraclePair& p, int64_t k,
                  int64_t match, int64_t mismatch, int64_t gap, int64_t xdrop,
                  OracleResult* res, std::string* cols) {
  cols->clear();
  *res = align_seed(A, B, p, k, match, mismatch, gap, xdrop, nullptr, nullptr);
  if (res->status & kStatusInvalidSeed) return true;
  const int64_t len_b = (int64_t)B.size();
  const std::string Bp = p.strand ? reverse_complement(B) : B;
  const int64_t pa = p.pos_a;
  const int64_t pb = p.strand ? len_b - (int64_t)p.pos_b - k : (int64_t)p.pos_b;
  const std::string la = reversed(A.substr(0, (size_t)pa));
  const std::string lb = reversed(Bp.substr(0, (size_t)pb));
  const std::string ra = A.substr((size_t)(pa + k));
  const std::string rb = Bp.substr((size_t)(pb + k));
  Moves lm, rm;
  const ExtOut L = extend(la.data(), (int64_t)la.size(), lb.data(), (int64_t)lb.size(), match,
                          mismatch, gap, xdrop, nullptr, &lm);
  const ExtOut R = extend(ra.data(), (int64_t)ra.size(), rb.data(), (int64_t)rb.size(), match,
                          mismatch, gap, xdrop, nullptr, &rm);
  std::string lc, rc;
  if (!trace_columns(la.data(), lb.data(), L.i_end, L.j_end, lm, &lc)) return false;
  if (!trace_columns(ra.data(), rb.data(), R.i_end, R.j_end, rm, &rc)) return false;
  cols->assign(lc.rbegin(), lc.rend());
  for (int64_t t = 0; t < k; ++t) cols->push_back(A[(size_t)(pa + t)] == Bp[(size_t)(pb + t)] ? '=' : 'X');
  cols->append(rc);
  return true;
}

// Run-length encoding of columns as 32-bit words (run length << 4 | op), with
// the SAM/BAM op numbers: 7 '=', 8 'X', 1 'I', 2 'D'.
std::vector<uint32_t> run_length(const std::string& cols) {
  std::vector<uint32_t> out;
  size_t t = 0;
  while (t < cols.size()) {
    size_t u = t;
    while (u < cols.size() && cols[u] == cols[t]) ++u;
    const uint32_t op = cols[t] == '=' ? 7u : cols[t] == 'X' ? 8u : cols[t] == 'I' ? 1u : 2u;
    out.push_back(((uint32_t)(u - t) << 4) | op);
    t = u;
  }
  return out;
}

// Per candidate pair (a run of consecutive records with equal read ids), flag
// the valid seed with the highest score; ties go to the earlier record.
void flag_best_of_pair(const OraclePair* pairs, OracleResult* res, int64_t n) {
  int64_t start = 0;
  while (start < n) {
    int64_t end = start + 1;
    while (end < n && pairs[end].read_a == pairs[start].read_a &&
           pairs[end].read_b == pairs[start].read_b)
      ++end;
    int64_t best_idx = -1;
    for (int64_t t = start; t < end; ++t) {
      if (res[t].status & kStatusInvalidSeed) continue;
      if (best_idx < 0 || res[t].score > res[best_idx].score) best_idx = t;
    }
    if (best_idx >= 0) res[best_idx].status |= kStatusBestOfPair;
    start = end;
  }
}

}  // namespace

extern "C" {

// One extension; out5 = {best, i_end, j_end, cells, tie}.  Returns 0.
int oracle_extend(const char* a, int64_t m, const char* b, int64_t n, int32_t match,
                  int32_t mismatch, int32_t gap, int32_t xdrop, int64_t* out5) {
  const ExtOut e = extend(a, m, b, n, match, mismatch, gap, xdrop);
  out5[0] = e.best;
  out5[1] = e.i_end;
  out5[2] = e.j_end;
  out5[3] = e.cells;
  out5[4] = e.tie;
  return 0;
}

// Band size of every evaluated antidiagonal d >= 1 of one extension; returns
// how many there were (at most `cap` are written).
int64_t oracle_extend_bands(const char* a, int64_t m, const char* b, int64_t n,
                            int32_t match, int32_t mismatch, int32_t gap, int32_t xdrop,
                            int64_t* bands, int64_t cap) {
  std::vector<int64_t> sizes;
  extend(a, m, b, n, match, mismatch, gap, xdrop, &sizes);
  for (int64_t t = 0; t < (int64_t)sizes.size() && t < cap; ++t) bands[t] = sizes[(size_t)t];
  return (int64_t)sizes.size();
}

// One seed with the details of both extensions:
//   ext10 = {L.best, L.i_end, L.j_end, L.cells, L.tie, R.best, R.i_end, R.j_end, R.cells, R.tie}
int oracle_align_one(const char* a, int64_t len_a, const char* b, int64_t len_b,
                     const void* pair, int32_t k, int32_t match, int32_t mismatch,
                     int32_t gap, int32_t xdrop, void* result, int64_t* ext10) {
  const std::string A(a, (size_t)len_a), B(b, (size_t)len_b);
  ExtOut L{0, 0, 0, 0, 0}, R{0, 0, 0, 0, 0};
  const OracleResult r = align_seed(A, B, *static_cast<const OraclePair*>(pair), k, match,
                                    mismatch, gap, xdrop, &L, &R);
  std::memcpy(result, &r, sizeof(r));
  if (ext10) {
    const int64_t v[10] = {L.best, L.i_end, L.j_end, L.cells, L.tie,
                           R.best, R.i_end, R.j_end, R.cells, R.tie};
    std::memcpy(ext10, v, sizeof(v));
  }
  return 0;
}

// A batch of seeds over a read set given as concatenated ASCII with n_reads+1
// offsets.  Results are 40-byte records in input order, with the best-of-pair
// flag set per run of consecutive records sharing (read_a, read_b).
// n_threads <= 0 means one thread per hardware thread.  Returns 0, or -1 on a
// bad argument.
int oracle_xdrop_batch(const char* ascii, const int64_t* offsets, int64_t n_reads,
                       const void* pairs_v, int64_t n_pairs, int32_t k, int32_t match,
                       int32_t mismatch, int32_t gap, int32_t xdrop, void* results_v,
                       int32_t n_threads) {
  if (n_pairs < 0 || n_reads < 0 || k < 1) return -1;
  const OraclePair* pairs = static_cast<const OraclePair*>(pairs_v);
  OracleResult* results = static_cast<OracleResult*>(results_v);
  if (n_threads <= 0) n_threads = (int32_t)std::max(1u, std::thread::hardware_concurrency());

  std::atomic<int64_t> next(0);
  const int64_t chunk = 16;
  auto worker = [&]() {
    for (;;) {
      const int64_t start = next.fetch_add(chunk);
      if (start >= n_pairs) return;
      const int64_t end = std::min(n_pairs, start + chunk);
      for (int64_t t = start; t < end; ++t) {
        const OraclePair& p = pairs[t];
        if ((int64_t)p.read_a >= n_reads || (int64_t)p.read_b >= n_reads) {
          std::memset(&results[t], 0, sizeof(OracleResult));
          results[t].status = kStatusInvalidSeed;
          continue;
        }
        const std::string A(ascii + offsets[p.read_a],
                            (size_t)(offsets[p.read_a + 1] - offsets[p.read_a]));
        const std::string B(ascii + offsets[p.read_b],
                            (size_t)(offsets[p.read_b + 1] - offsets[p.read_b]));
        results[t] = align_seed(A, B, p, k, match, mismatch, gap, xdrop, nullptr, nullptr);
      }
    }
  };
  if (n_threads == 1) {
    worker();
  } else {
    std::vector<std::thread> pool;
    for (int32_t t = 0; t < n_threads; ++t) pool.emplace_back(worker);
    for (auto& th : pool) th.join();
  }
  flag_best_of_pair(pairs, results, n_pairs);
  return 0;
}

// Columns of one extension's best alignment as characters ('=', 'X', 'D',
// 'I'; see trace_columns).  Returns their number (at most `cap` are written),
// or -1 if the traceback failed.
int64_t oracle_extend_columns(const char* a, int64_t m, const char* b, int64_t n, int32_t match,
                              int32_t mismatch, int32_t gap, int32_t xdrop, char* cols,
                              int64_t cap) {
  Moves mv;
  const ExtOut e = extend(a, m, b, n, match, mismatch, gap, xdrop, nullptr, &mv);
  std::string c;
  if (!trace_columns(a, b, e.i_end, e.j_end, mv, &c)) return -1;
  for (int64_t t = 0; t < (int64_t)c.size() && t < cap; ++t) cols[t] = c[(size_t)t];
  return (int64_t)c.size();
}

// A batch of seeds with the traceback of each: results as oracle_xdrop_batch
// (without the best-of-pair flag) and, per seed t, its run-length encoded
// columns in ops[t * cap_per_seed ...] with n_ops[t] runs; n_ops[t] = -1 when
// more than cap_per_seed runs were needed (nothing written), 0 for an invalid
// seed.  Single-threaded.  Returns 0, -1 on a bad argument, -2 if a traceback
// failed.
int oracle_traceback_batch(const char* ascii, const int64_t* offsets, int64_t n_reads,
                           const void* pairs_v, int64_t n_pairs, int32_t k, int32_t match,
                           int32_t mismatch, int32_t gap, int32_t xdrop, void* results_v,
                           uint32_t* ops, int64_t cap_per_seed, int32_t* n_ops) {
  if (n_pairs < 0 || n_reads < 0 || k < 1 || cap_per_seed < 0) return -1;
  const OraclePair* pairs = static_cast<const OraclePair*>(pairs_v);
  OracleResult* results = static_cast<OracleResult*>(results_v);
  for (int64_t t = 0; t < n_pairs; ++t) {
    const OraclePair& p = pairs[t];
    n_ops[t] = 0;
    if ((int64_t)p.read_a >= n_reads || (int64_t)p.read_b >= n_reads) {
      std::memset(&results[t], 0, sizeof(OracleResult));
      results[t].status = kStatusInvalidSeed;
      continue;
    }
    const std::string A(ascii + offsets[p.read_a], (size_t)(offsets[p.read_a + 1] - offsets[p.read_a]));
    const std::string B(ascii + offsets[p.read_b], (size_t)(offsets[p.read_b + 1] - offsets[p.read_b]));
    std::string cols;
    if (!seed_columns(A, B, p, k, match, mismatch, gap, xdrop, &results[t], &cols)) return -2;
    const std::vector<uint32_t> runs = run_length(cols);
    if ((int64_t)runs.size() > cap_per_seed) {
      n_ops[t] = -1;
      continue;
    }
    for (size_t r = 0; r < runs.size(); ++r) ops[t * cap_per_seed + (int64_t)r] = runs[r];
    n_ops[t] = (int32_t)runs.size();
  }
  return 0;
}

}  // extern "C"
