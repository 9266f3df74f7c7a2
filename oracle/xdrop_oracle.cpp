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
//       coordinates, read B reported in forward coordinates.
// Arithmetic is int64 (the paper fixes no precision; scores are integers).
//
// Parity pinned by the tests: hand-worked examples (golden files), an
// independent full dynamic program for X = infinity, brute-force enumeration
// of all alignments on tiny inputs, and invariants (mirror symmetry, X
// monotonicity bound, cell bounds).

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
ExtOut extend(const char* a, int64_t m, const char* b, int64_t n, int64_t match,
              int64_t mismatch, int64_t gap, int64_t xdrop,
              std::vector<int64_t>* band_sizes = nullptr) {
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

  for (int64_t d = 1; d <= m + n; ++d) {
    // R1: band of d from the live cells of d-1, clipped to 0<=i<=m, 0<=j<=n.
    int64_t lo = std::max<int64_t>(std::max<int64_t>(live_lo, d - n), 0);
    int64_t hi = std::min<int64_t>(std::min<int64_t>(live_hi + 1, d), m);
    if (lo > hi) break;
    d0.lo = lo;
    d0.hi = hi;
    const int64_t threshold = best - xdrop;  // R2: fixed for this antidiagonal

    int64_t row_best = kNegInf, row_best_i = -1, row_best_count = 0;
    int64_t new_live_lo = -1, new_live_hi = -1;
    for (int64_t i = lo; i <= hi; ++i) {
      const int64_t j = d - i;
      int64_t h = kNegInf;
      // H(i-1, j-1) + s(a[i-1], b[j-1]): antidiagonal d-2, index i-1.
      if (i >= 1 && j >= 1) {
        const int64_t diag = d2.at(i - 1);
        if (diag != kNegInf)
          h = std::max(h, diag + substitution(a[i - 1], b[j - 1], match, mismatch));
      }
      // H(i-1, j) + gap: antidiagonal d-1, index i-1.
      if (i >= 1) {
        const int64_t up = d1.at(i - 1);
        if (up != kNegInf) h = std::max(h, up + gap);
      }
      // H(i, j-1) + gap: antidiagonal d-1, index i.
      if (j >= 1) {
        const int64_t left = d1.at(i);
        if (left != kNegInf) h = std::max(h, left + gap);
      }
      out.cells += 1;  // R4: every cell of the band is evaluated
      const bool live = (h != kNegInf) && (h >= threshold);  // R2
      d0.h[(size_t)i] = live ? h : kNegInf;
      if (!live) continue;
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

}  // extern "C"
