// X-drop seed-and-extend on GB300 (sm_103a): kernels and the C ABI.
//
// Computes, per candidate seed, the alignment of diBELLA Sec. 2 (pairwise
// alignment, linear-gap scoring, X-drop search after Zhang et al. 2000) from
// a shared k-mer seed (Sec. 2 Fig. 1, Sec. 8 seed selection), which is the
// per-pair work of the alignment stage (Sec. 9).  The exact reading of the
// X-drop rule (band from the live cells of the previous antidiagonal, live
// iff H >= best - X, strict improvement, smallest i on ties, evaluated-cell
// count) is documented on dibella_xdrop_batch in include/dibella.h.
//
// Pipeline of one batch (all on the caller's stream, no host sync):
//   expand   one thread per seed: validate, seed score, two extension items
//            (left, right) with the copy/offset of both sequences; count
//            items per (kernel class, length bucket)
//   scan     bucket offsets, longest bucket first (work queues are ordered
//            so long extensions start early: Sec. 9 load imbalance from
//            read length and X-drop early exit)
//   scatter  item ids into the narrow and wide queues
//   extend   persistent kernel; every warp first takes wide items (one warp
//            per extension, band in shared memory in chunks of 32 cells),
//            then narrow items (one lane per extension, band in per-lane
//            shared memory); a band that outgrows its storage is re-queued
//            for the next wider form
//   extend   again for narrow->wide escalations
//   global   one warp per extension with the band in workspace memory
//   combine  seed + left + right, coordinates, cells; best seed per pair
//
// Arithmetic is int32 (limits on scores and read lengths in dibella.h keep
// every value inside (-2^31, 2^31)); no tensor cores: this is not a dense
// contraction.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/dibella.h"

namespace {

constexpr int kNeg = -(1 << 30) - (1 << 29);  // dead / outside band; below any threshold
constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerBlock = 4;
constexpr int kBlockThreads = kWarpsPerBlock * 32;
constexpr int kGlobalWarps = 64;  // warps of the global-band kernel (and its band slots)

// One extension of one seed: a[x] = base (a0 + x) of the packed store
// (ascending), b[y] = base (b0 - y) (descending); a is always read in the
// opposite complement sense of b (see expand), so a match is a 2-bit XOR of 3.
struct Item {
  long long a0, b0;
  int m, n;
  int tag;  // class << 8 | bucket, or -1 for no item
  int pad;
};
static_assert(sizeof(Item) == 32, "item is 32 bytes");

struct ExtOut {
  int best, i_end, j_end, status;
  long long cells;
};
static_assert(sizeof(ExtOut) == 24, "ext out is 24 bytes");

// Queues: routed narrow / wide; narrow escalations (to the wide form); one
// queue per step of the wide-form slot ladder (8 -> 16 -> 24 -> 32 slots);
// the shared-memory form's input; the global-band form's input.
// The mid form's escalations (extensions whose band outgrew it) go to kQEsc2;
// with a split narrow launch, the extensions still running after the first
// pass's antidiagonal limit go to kQLong for the second pass.
enum { kQNarrow = 0, kQWide = 1, kQEsc1 = 2, kQLadder = 3, kQSmem = 7, kQGlobal = 8, kQEsc2 = 9, kQLong = 10,
       kNumQ = 11 };

struct Counters {
  unsigned int tail[kNumQ];   // queue sizes (see the kQ* names)
  unsigned int head[kNumQ];   // pop cursors
  unsigned int pad_[2];
  unsigned int bucket_count[2][DIBELLA_MAX_BUCKETS];
  unsigned int bucket_cursor[2][DIBELLA_MAX_BUCKETS];
  unsigned int stat[8];   // routed narrow, routed wide, escalated from narrow / wide /
                          // shared-memory form, band overflows, escalated from the mid form,
                          // moved to the second narrow pass
  // cells of finished extensions: 0 narrow, 1 wide (first launch), 2 CTA,
  // 3 global, 4 wide launch on the narrow escalations, 5 slot-ladder rungs,
  // 6 mid form (the narrow escalations, one lane per extension, wide band),
  // 7 cells the one-lane forms evaluated for extensions they then handed to a
  // wider form (which restarts them: work done twice)
  unsigned long long cells[8];
};



struct Scoring {
  int M, S, G, X;
};

struct ExtendParams {
  const uint32_t* __restrict__ words;
  const Item* __restrict__ items;
  ExtOut* ext;
  Counters* cnt;
  const int* wide_q;  // queue popped one item per warp (wide forms)
  int wide_q_id;      // its head/tail index in Counters
  const int* narrow_q;  // queue popped one item per lane (narrow form)
  int narrow_q_id;
  int* esc_q;         // where extensions that outgrow the form go
  int esc_q_id;
  // A slot-ladder rung whose queue holds at most this many extensions passes
  // them all on to esc_q unextended: so few are latency bound, and the CTA
  // form above the ladder walks a wide band faster than one warp (0 = never).
  unsigned forward_max;
  int cells_idx;  // Counters::cells entry the wide forms add to
  int narrow_cells_idx;  // Counters::cells entry of the one-lane forms (0 narrow, 6 mid)
  int narrow_esc_stat;   // Counters::stat entry counting their escalations (2 narrow, 6 mid)
  // Per-warp clock of one launch (null unless requested): warp w writes the
  // global timer (ns) when it starts, at [2w], and when it leaves, at [2w+1].
  unsigned long long* wclock;
  long long q_cap;  // entries of every queue and of items / ext (2 x seed records)
  // Split narrow launch: an extension still running after antidiagonal
  // narrow_max_d (0 = no limit) stops and goes to long_q, to be run again
  // from the origin by the second pass.
  int narrow_max_d;
  int* long_q;
  Scoring sc;
  int* gband;
  int gcap;
};

// ---- bounds checks of the debug build ---------------------------------------
// Built with -DDIBELLA_BOUNDS_CHECK (libdibella_debug.so), every store word
// read, per-lane shared-memory slot, queue push, item index and global band
// slot is checked; a failed check records (code, index, limit) of the first
// fault and a count in g_bounds_fault and the access is skipped (store reads
// give 0, slots fall back to slot 0, pushes and items are dropped), so the
// kernel finishes and the host reads the record (dibella_bounds_check).  No
// trap.  Codes: 1 narrow slot, 2 queue push, 3 item index, 4 store word,
// 5 global band slot.  In the release build the checks compile to nothing.
#ifdef DIBELLA_BOUNDS_CHECK
__device__ unsigned long long g_bounds_fault[4];
__device__ long long g_store_words;  // words of the batch's store, set by store_extent_kernel
__device__ __noinline__ bool bounds_fault(int code, long long v, long long lim) {
  if (atomicCAS(&g_bounds_fault[0], 0ull, (unsigned long long)code) == 0ull) {
    g_bounds_fault[1] = (unsigned long long)v;
    g_bounds_fault[2] = (unsigned long long)lim;
  }
  atomicAdd(&g_bounds_fault[3], 1ull);
  return false;
}
#define DIBELLA_IN_BOUNDS(v, lim, code) \
  ((unsigned long long)(long long)(v) < (unsigned long long)(long long)(lim) ? true \
                                                                            : bounds_fault((code), (long long)(v), (long long)(lim)))
#define DIBELLA_STORE_WORDS g_store_words
#else
#define DIBELLA_IN_BOUNDS(v, lim, code) true
#define DIBELLA_STORE_WORDS 0
#endif

// One word of the packed store (checked in the debug build).
__device__ __forceinline__ uint32_t ldg_word(const uint32_t* __restrict__ words, long long w) {
  return DIBELLA_IN_BOUNDS(w, DIBELLA_STORE_WORDS, 4) ? __ldg(words + w) : 0u;
}

__device__ __forceinline__ uint32_t base_window(const uint32_t* __restrict__ words, long long idx) {
  // 16 bases starting at base index idx (>= 0), base t at bits 2t.
  const long long w = idx >> 4;
  const uint32_t lo = ldg_word(words, w), hi = ldg_word(words, w + 1);
  return __funnelshift_r(lo, hi, (unsigned)(idx & 15) * 2u);
}

__device__ __forceinline__ int base_at(const uint32_t* __restrict__ words, long long idx) {
  return (int)((ldg_word(words, idx >> 4) >> ((unsigned)(idx & 15) * 2u)) & 3u);
}

constexpr int kMaxClockedWarps = 1 << 16;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Start (at = 0) or end (at = 1) of this warp's work in a clocked launch,
// written at once by lane 0 so that no timer value stays live in registers
// across the persistent loop.
__device__ __forceinline__ void warp_clock(unsigned long long* wclock, int at) {
  if (wclock == nullptr || (threadIdx.x & 31) != 0) return;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w < kMaxClockedWarps) wclock[2 * w + at] = global_ns();
}

__device__ __forceinline__ unsigned pop_warp(Counters* cnt, int q) {
  unsigned idx = 0;
  if ((threadIdx.x & 31) == 0) idx = atomicAdd(&cnt->head[q], 1u);
  return __shfl_sync(kFull, idx, 0);
}

// ---------------------------------------------------------------------------
// Wide form: one warp per extension.  Three antidiagonals in a circular array
// of `cap` (power of two) cells; lane l computes cell i = i0 + l of each chunk
// of 32 cells.  Returns false if the band outgrew cap - 3 cells.
template <bool kGlobalBand>
__device__ bool extend_warp(const uint32_t* __restrict__ words, const Item& it, const Scoring sc,
                            int* arr, int cap, ExtOut* out) {
  const int lane = threadIdx.x & 31;
  const int mask = cap - 1;
  int* H2 = arr;            // antidiagonal d-2
  int* H1 = arr + cap;      // d-1
  int* H0 = arr + 2 * cap;  // d
  const int m = it.m, n = it.n;
  // d = 0: cell (0,0) = 0 with guards; d = -1: no cell (guards read as dead).
  if (lane == 0) {
    H1[0] = 0;
    H1[mask] = kNeg;      // i = -1
    H1[1 & mask] = kNeg;  // i = 1
    H2[mask] = kNeg;
    H2[0] = kNeg;
  }
  __syncwarp();
  int live_lo = 0, live_hi = 0, best = 0, bi = 0, bj = 0;
  long long cells = 0;
  for (int d = 1; d <= m + n; ++d) {
    const int lo = max(live_lo, d - n);
    const int hi = min(min(live_hi + 1, d), m);
    if (hi - lo + 3 > cap) return false;
    const int thr = best - sc.X;
    const long long abase = it.a0 - 1, bbase = it.b0 + 1 - d;
    int vmax = kNeg, first = INT32_MAX, last = -1;
    for (int i0 = lo; i0 <= hi; i0 += 32) {
      const int i = i0 + lane;
      int h = kNeg;
      if (i <= hi) {
        const int lf = H1[i & mask];
        const int u = H1[(i - 1) & mask];
        const int dg = H2[(i - 1) & mask];
        const int ca = base_at(words, abase + i), cb = base_at(words, bbase + i);
        const int sub = (ca ^ cb) == 3 ? sc.M : sc.S;
        h = max(max(u, lf) + sc.G, dg + sub);
        h = h >= thr ? h : kNeg;
        H0[i & mask] = h;
      }
      vmax = max(vmax, h);
      const unsigned bl = __ballot_sync(kFull, h != kNeg);
      if (bl) {
        if (first == INT32_MAX) first = i0 + __ffs(bl) - 1;
        last = i0 + 31 - __clz(bl);
      }
    }
    cells += hi - lo + 1;
    if (lane == 0) H0[(lo - 1) & mask] = kNeg;
    if (lane == 1) H0[(hi + 1) & mask] = kNeg;
    vmax = __reduce_max_sync(kFull, vmax);
    __syncwarp();
    if (vmax == kNeg) break;
    if (vmax > best) {
      for (int i0 = first;; i0 += 32) {
        const int i = i0 + lane;
        const unsigned bl = __ballot_sync(kFull, i <= last && H0[i & mask] == vmax);
        if (bl) {
          bi = i0 + __ffs(bl) - 1;
          break;
        }
      }
      best = vmax;
      bj = d - bi;
    }
    live_lo = first;
    live_hi = last;
    int* t = H2;
    H2 = H1;
    H1 = H0;
    H0 = t;
  }
  if (lane == 0) {
    out->best = best;
    out->i_end = bi;
    out->j_end = bj;
    out->status = 0;
    out->cells = cells;
  }
  __syncwarp();
  return true;
}

// ---------------------------------------------------------------------------
// Register form: one warp per extension, the band held in registers.
// Cells are grouped in chunks of 32 consecutive i (lane l of chunk c holds
// cell i = 32c + l).  NC register slots hold chunks cbase .. cbase+NC-1;
// slot 0 is a guard below the band (chunk lo/32 - 1) and the band plus the
// chunk holding hi+1 must fit in slots 1..NC-1, else the extension is handed
// to a wider form.  Per lane and slot: H (antidiagonal d-1), Up (the up
// neighbour read on d-1, i.e. H(d-2, i-1), the diagonal predecessor on d) and
// Bb (b base of the cell on d-1); the a base of every slot is packed 2 bits
// per slot in one register.  Moving from d-1 to d, every cell takes its up
// neighbour and its b base from the cell below (lane - 1, or lane 31 of the
// slot below for lane 0), so a chunk costs two shuffles and no memory access;
// slots are processed top down so the slot below still holds d-1.  The lowest
// chunk's lane 0 reads its new b base from memory.
__device__ __forceinline__ int base_of(const uint32_t* __restrict__ words, long long idx) {
  return (int)((ldg_word(words, idx >> 4) >> ((unsigned)(idx & 15) * 2u)) & 3u);
}

template <int NC>
__device__ bool extend_reg(const uint32_t* __restrict__ words, const Item& it, const Scoring sc,
                           ExtOut* out) {
  const int lane = threadIdx.x & 31;
  const int src_lane = (lane + 31) & 31;
  const bool top_lane = lane == 31;
  const int m = it.m, n = it.n;
  const long long a_lo = it.a0 - 1;   // store index of a[i-1] is a_lo + i
  const long long b_lo = it.b0 + 1;   // store index of b[d-i-1] is b_lo - d + i
  int H[NC], Up[NC], Bb[NC];
  // a base of every slot, 2 bits per slot (64-bit once there are more than 16 slots)
  using AWord = typename std::conditional<(NC > 16), unsigned long long, unsigned>::type;
  AWord Aall = 0;
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    H[s] = kNeg;
    Up[s] = kNeg;
    Bb[s] = 0;
  }
  // Antidiagonal 0: cell (0,0) = 0 in chunk 0 (slot 1); slot 0 guards chunk -1.
  int cbase = -1, ctop = 0;
  if (lane == 0) H[1] = 0;
  Aall = (AWord)base_of(words, a_lo + lane) << 2;
  Bb[1] = base_of(words, b_lo + lane);  // b base of cell i on "d = 0": b_lo - 0 + i
  int live_lo = 0, live_hi = 0, best = 0, bi = 0, bj = 0;
  long long cells = 0;
  for (int d = 1; d <= m + n; ++d) {
    const int lo = max(live_lo, d - n);
    const int hi = min(min(live_hi + 1, d), m);
    const int c0 = lo >> 5;
    while (cbase < c0 - 1) {  // keep slot 0 = chunk c0 - 1
#pragma unroll
      for (int s = 0; s + 1 < NC; ++s) {
        H[s] = H[s + 1];
        Up[s] = Up[s + 1];
        Bb[s] = Bb[s + 1];
      }
      H[NC - 1] = kNeg;
      Up[NC - 1] = kNeg;
      Aall >>= 2;
      ++cbase;
    }
    const int cneed = (hi + 1) >> 5;
    if (cneed - cbase > NC - 1) return false;
    if (cneed > ctop) {  // at most one new chunk per antidiagonal
      const int snew = cneed - cbase;
      const int ab = base_of(words, a_lo + 32 * cneed + lane);
      const int bb = base_of(words, b_lo + 1 - d + 32 * cneed + lane);
#pragma unroll
      for (int s = 1; s < NC; ++s) {
        if (s == snew) {
          H[s] = kNeg;
          Up[s] = kNeg;
          Bb[s] = bb;
        }
      }
      Aall = (Aall & ~((AWord)3 << (2 * snew))) | ((AWord)ab << (2 * snew));
    }
    ctop = cneed;
    const int thr = best - sc.X;
    const int bfresh = base_of(words, b_lo - d + 32 * c0);  // lane 0 of chunk c0
    const unsigned span = (unsigned)(hi - lo);
    int vmax = kNeg, first = 0, last = -1;
#pragma unroll
    for (int s = NC - 1; s >= 1; --s) {
      const int c = cbase + s;
      if (c <= ctop) {
        const int u = __shfl_sync(kFull, top_lane ? H[s - 1] : H[s], src_lane);
        int bn = __shfl_sync(kFull, top_lane ? Bb[s - 1] : Bb[s], src_lane);
        if (s == 1 && lane == 0) bn = bfresh;
        const int i = 32 * c + lane;
        const int a = (int)((Aall >> (2 * s)) & 3u);  // s is a compile-time constant
        const int sub = (a ^ bn) == 3 ? sc.M : sc.S;
        int h = max(max(u, H[s]) + sc.G, Up[s] + sub);
        const bool live = ((unsigned)(i - lo) <= span) && h >= thr;
        h = live ? h : kNeg;
        Up[s] = u;
        H[s] = h;
        Bb[s] = bn;
        vmax = max(vmax, h);
        const unsigned bl = __ballot_sync(kFull, live);
        if (bl) {
          first = 32 * c + __ffs(bl) - 1;
          if (last < 0) last = 32 * c + 31 - __clz(bl);
        }
      }
    }
    H[0] = kNeg;
    cells += hi - lo + 1;
    vmax = __reduce_max_sync(kFull, vmax);
    if (vmax == kNeg) break;
    if (vmax > best) {
      int cand = INT32_MAX;
#pragma unroll
      for (int s = 1; s < NC; ++s) {
        if (cbase + s <= ctop) {
          const unsigned bl = __ballot_sync(kFull, H[s] == vmax);
          if (bl) cand = min(cand, 32 * (cbase + s) + __ffs(bl) - 1);
        }
      }
      best = vmax;
      bi = cand;
      bj = d - cand;
    }
    live_lo = first;
    live_hi = last;
  }
  if (lane == 0) {
    out->best = best;
    out->i_end = bi;
    out->j_end = bj;
    out->status = 0;
    out->cells = cells;
  }
  __syncwarp();
  return true;
}

// ---------------------------------------------------------------------------
// Packed form: one warp per extension, two cells per 32-bit register.
// Scores are held as int16 pairs relative to a per-extension base `rb`
// (rebased when the best score gets 4096 above it), which is exact while
// X <= kPackedMaxX: every live value then lies within [-X, 4096 + 2*match] of
// rb and dead cells hold kNeg16 = -16384, far from both int16 limits, so no
// packed add can wrap.  Chunk c covers cells 64c .. 64c+63; lane l holds cells
// 64c + 2l (low half) and 64c + 2l + 1 (high half).  Slots, guard and
// escalation follow the register form.  The a and b bases of every cell are
// 2-bit fields in NC/8 words per lane (slot s of word w = s/8: low cell at bits
// 2(s%8), high cell at bits 2(s%8)+16), so one word XOR gives the match bits
// of 16 cells and one shuffle per word moves every b base to the next cell.
constexpr int kPackedMaxX = 8000;
constexpr unsigned kNeg2 = 0xC000C000u;  // kNeg16 in both halves
constexpr int kRebase = 4096;

__device__ __forceinline__ unsigned pk_pair(int lo, int hi) {
  return ((unsigned)lo & 0xFFFFu) | ((unsigned)hi << 16);
}
// x in both 16-bit halves (x within int16)
__device__ __forceinline__ unsigned pk_dup(int x) { return __byte_perm((unsigned)x, 0u, 0x1010u); }
__device__ __forceinline__ int pk_lo(unsigned v) { return (int)(short)(v & 0xFFFFu); }
// 0xFFFF in each 16-bit half of x whose top bit (bit 15 / bit 31) is set, else
// 0: PTX prmt with sign-replicating selectors (byte 1's sign into bytes 0-1,
// byte 3's sign into bytes 2-3).
__device__ __forceinline__ unsigned half_sign_mask(unsigned x) {
  unsigned r;
  asm("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(r) : "r"(x));
  return r;
}
__device__ __forceinline__ int pk_hi(unsigned v) { return (int)(short)(v >> 16); }

template <int NC>
__device__ bool extend_pk(const uint32_t* __restrict__ words, const Item& it, const Scoring sc, ExtOut* out) {
  static_assert(NC % 8 == 0 && NC >= 8 && NC <= 32, "slots come in words of 8");
  constexpr int NW = NC / 8;
  const int lane = threadIdx.x & 31;
  const int src_lane = (lane + 31) & 31;
  const bool top_lane = lane == 31;
  const int m = it.m, n = it.n;
  const long long a_lo = it.a0 - 1;
  const long long b_lo = it.b0 + 1;
  // The lowest chunk's fresh b base is read every antidiagonal: address it with
  // 32-bit offsets from a word pointer below every index it can take.
  const long long b_floor = (b_lo - n - 128) & ~15ll;
  const uint32_t* __restrict__ bwords = words + (b_floor >> 4);
  const int b_rel = (int)(b_lo - b_floor);
  unsigned H[NC], Up[NC], Aw[NW], Bw[NW];
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    H[s] = kNeg2;
    Up[s] = kNeg2;
  }
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    Aw[w] = 0;
    Bw[w] = 0;
  }
  const unsigned M2 = pk_pair(sc.M, sc.M), S2 = pk_pair(sc.S, sc.S), G2 = pk_pair(sc.G, sc.G);
  int cbase = -1, ctop = 0, rb = 0;
  // d = 0: cell (0,0) = 0 at chunk 0 (slot 1), lane 0, low half.
  if (lane == 0) H[1] = pk_pair(0, -16384);
  {  // bases of chunk 0 (cells 2l, 2l+1): a[i-1] and b on "d = 0"
    const int i0 = 2 * lane;
    const unsigned a0b = base_of(words, a_lo + i0), a1b = base_of(words, a_lo + i0 + 1);
    const unsigned b0b = base_of(words, b_lo + i0), b1b = base_of(words, b_lo + i0 + 1);
    Aw[0] = (a0b << 2) | (a1b << 18);
    Bw[0] = (b0b << 2) | (b1b << 18);
  }
  int live_lo = 0, live_hi = 0, best = 0, bi = 0, bj = 0;
  int bq_idx = INT32_MIN;  // store word of the fresh b base, cached
  unsigned bq = 0;
  long long cells = 0;
  for (int d = 1; d <= m + n; ++d) {
    const int lo = max(live_lo, d - n);
    const int hi = min(min(live_hi + 1, d), m);
    const int c0 = lo >> 6;
    const int cneed = (hi + 1) >> 6;
    // Window moves, chunk (de)activation and rebasing are rare: one test for all.
    if ((c0 - 1 != cbase) | (cneed != ctop) | (best - rb >= kRebase)) {
      while (cbase < c0 - 1) {  // keep slot 0 = chunk c0 - 1
#pragma unroll
        for (int s = 0; s + 1 < NC; ++s) {
          H[s] = H[s + 1];
          Up[s] = Up[s + 1];
        }
        H[NC - 1] = kNeg2;
        Up[NC - 1] = kNeg2;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const int wn = w + 1 < NW ? w + 1 : w;
          const unsigned na = w + 1 < NW ? Aw[wn] : 0u, nb = w + 1 < NW ? Bw[wn] : 0u;
          Aw[w] = ((Aw[w] >> 2) & 0x3FFF3FFFu) | ((na & 0x00030003u) << 14);
          Bw[w] = ((Bw[w] >> 2) & 0x3FFF3FFFu) | ((nb & 0x00030003u) << 14);
        }
        ++cbase;
      }
      if (cneed - cbase > NC - 1) return false;
      if (cneed > ctop) {  // activate the chunk holding hi + 1 (at most one per antidiagonal)
        const int snew = cneed - cbase;
        const int i0 = 64 * cneed + 2 * lane;
        const unsigned a0b = base_of(words, a_lo + i0), a1b = base_of(words, a_lo + i0 + 1);
        const unsigned b0b = base_of(words, b_lo + 1 - d + i0), b1b = base_of(words, b_lo + 2 - d + i0);
        const int sh = 2 * (snew & 7);
        const unsigned clear = ~((3u << sh) | (3u << (sh + 16)));
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          if (w == (snew >> 3)) {
            Aw[w] = (Aw[w] & clear) | (a0b << sh) | (a1b << (sh + 16));
            Bw[w] = (Bw[w] & clear) | (b0b << sh) | (b1b << (sh + 16));
          }
        }
#pragma unroll
        for (int s = 1; s < NC; ++s) {
          if (s == snew) {
            H[s] = kNeg2;
            Up[s] = kNeg2;
          }
        }
      }
      ctop = cneed;
      // Rebase the packed scores when the best has run 4096 above the base.
      if (best - rb >= kRebase) {
        const int delta = best - rb;
        const unsigned dn = pk_pair(-delta, -delta);
#pragma unroll
        for (int s = 0; s < NC; ++s) {
          H[s] = __vmaxs2(__vadd2(H[s], dn), kNeg2);
          Up[s] = __vmaxs2(__vadd2(Up[s], dn), kNeg2);
        }
        rb = best;
      }
    }
    // Move every b base to the next cell (cell i takes the base of cell i-1),
    // for the words that hold active slots, and form their mismatch bits.
    const int ntop = ctop - cbase;
    const int wtop = ntop >> 3;
    unsigned MM[NW];
    {
      const int r = b_rel - d + 64 * c0;  // lane 0, low cell of slot 1: store index b_lo - d + 64*c0
      if ((r >> 4) != bq_idx) {  // r falls by one per antidiagonal: one load per 16
        bq_idx = r >> 4;
#ifdef DIBELLA_BOUNDS_CHECK
        bq = ldg_word(words, (long long)(bwords - words) + bq_idx);
#else
        bq = __ldg(bwords + bq_idx);
#endif
      }
      const int bfresh = (int)((bq >> ((unsigned)(r & 15) * 2u)) & 3u);
      unsigned prev_top = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        MM[w] = 0;
        if (w <= wtop) {
          const unsigned t = __shfl_sync(kFull, Bw[w], src_lane);
          unsigned lo_new = t >> 16;                                  // lane-1's high cells
          const unsigned lo_lane0 = ((t >> 14) & 0xFFFCu) | prev_top;  // lane 31's high cells, one slot up
          prev_top = (t >> 30) & 3u;
          if (lane == 0) lo_new = (w == 0) ? ((lo_lane0 & ~0xCu) | ((unsigned)bfresh << 2)) : lo_lane0;
          Bw[w] = (Bw[w] << 16) | lo_new;
          const unsigned x = ~(Aw[w] ^ Bw[w]);
          MM[w] = (x | (x >> 1)) & 0x55555555u;  // bit 2k set: mismatch
        }
      }
    }
    const int thr_rel = best - rb - sc.X;
    const unsigned nthr2 = pk_pair(-thr_rel, -thr_rel);
    // Band test as int16 pairs: a = i - lo >= 0 and b = hi - i >= 0.
    const unsigned lane2 = pk_pair(2 * lane, 2 * lane + 1);  // the lane's two cell offsets
    const unsigned A2 = __vsub2(lane2, pk_dup(lo - 64 * cbase));
    const unsigned B2 = __vsub2(pk_dup(hi - 64 * cbase), lane2);
    // Live bits of this lane: word s/16, bit s%16 = low cell of slot s live,
    // bit 16 + s%16 = high cell live (one LOP3 per slot, no vote).
    constexpr int NL = (NC + 15) / 16;
    unsigned vmax2 = kNeg2, lm[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) lm[q] = 0;
#define DIBELLA_PK_I(S) ((S) < NC ? (S) : NC - 1)
#define DIBELLA_PK_SLOT(S)                                                                         \
  if (S < NC) {                                                                                    \
    constexpr int s_ = DIBELLA_PK_I(S), p_ = s_ > 0 ? s_ - 1 : 0;                                  \
    const unsigned prevH = __shfl_sync(kFull, top_lane ? H[p_] : H[s_], src_lane);                 \
    const unsigned u2 = __byte_perm(H[s_], prevH, 0x1076u);                                        \
    /* mismatch flags of the two cells moved to bits 15 and 31, then spread */                     \
    const unsigned mis = half_sign_mask(MM[s_ >> 3] << (15 - 2 * (s_ & 7)));                       \
    const unsigned sub2 = (mis & S2) | (~mis & M2);                                                \
    const unsigned ds = __viaddmax_s16x2(Up[s_], sub2, kNeg2);                                     \
    unsigned h2 = __viaddmax_s16x2(__vmaxs2(u2, H[s_]), G2, ds);                                   \
    const unsigned f = __vimin3_s16x2(__vadd2(h2, nthr2), __vadd2(A2, 0x00400040u * s_),          \
                                      __vsub2(B2, 0x00400040u * s_));                              \
    const unsigned dead = half_sign_mask(f); /* 0xFFFF in every half with f < 0 */                 \
    h2 = (h2 & ~dead) | (kNeg2 & dead);                                                            \
    Up[s_] = u2;                                                                                   \
    H[s_] = h2;                                                                                    \
    vmax2 = __vmaxs2(vmax2, h2);                                                                   \
    lm[s_ >> 4] |= ~dead & (0x00010001u << (s_ & 15));                                             \
  }
    switch (ntop) {
      case 31: DIBELLA_PK_SLOT(31) [[fallthrough]];
      case 30: DIBELLA_PK_SLOT(30) [[fallthrough]];
      case 29: DIBELLA_PK_SLOT(29) [[fallthrough]];
      case 28: DIBELLA_PK_SLOT(28) [[fallthrough]];
      case 27: DIBELLA_PK_SLOT(27) [[fallthrough]];
      case 26: DIBELLA_PK_SLOT(26) [[fallthrough]];
      case 25: DIBELLA_PK_SLOT(25) [[fallthrough]];
      case 24: DIBELLA_PK_SLOT(24) [[fallthrough]];
      case 23: DIBELLA_PK_SLOT(23) [[fallthrough]];
      case 22: DIBELLA_PK_SLOT(22) [[fallthrough]];
      case 21: DIBELLA_PK_SLOT(21) [[fallthrough]];
      case 20: DIBELLA_PK_SLOT(20) [[fallthrough]];
      case 19: DIBELLA_PK_SLOT(19) [[fallthrough]];
      case 18: DIBELLA_PK_SLOT(18) [[fallthrough]];
      case 17: DIBELLA_PK_SLOT(17) [[fallthrough]];
      case 16: DIBELLA_PK_SLOT(16) [[fallthrough]];
      case 15: DIBELLA_PK_SLOT(15) [[fallthrough]];
      case 14: DIBELLA_PK_SLOT(14) [[fallthrough]];
      case 13: DIBELLA_PK_SLOT(13) [[fallthrough]];
      case 12: DIBELLA_PK_SLOT(12) [[fallthrough]];
      case 11: DIBELLA_PK_SLOT(11) [[fallthrough]];
      case 10: DIBELLA_PK_SLOT(10) [[fallthrough]];
      case 9: DIBELLA_PK_SLOT(9) [[fallthrough]];
      case 8: DIBELLA_PK_SLOT(8) [[fallthrough]];
      case 7: DIBELLA_PK_SLOT(7) [[fallthrough]];
      case 6: DIBELLA_PK_SLOT(6) [[fallthrough]];
      case 5: DIBELLA_PK_SLOT(5) [[fallthrough]];
      case 4: DIBELLA_PK_SLOT(4) [[fallthrough]];
      case 3: DIBELLA_PK_SLOT(3) [[fallthrough]];
      case 2: DIBELLA_PK_SLOT(2) [[fallthrough]];
      case 1: DIBELLA_PK_SLOT(1) [[fallthrough]];
      default: break;
    }
#undef DIBELLA_PK_SLOT
#undef DIBELLA_PK_I
    H[0] = kNeg2;
    cells += hi - lo + 1;
    // Lowest and highest live cell of the lane (relative to chunk cbase), then of
    // the warp: two reductions per antidiagonal.
    int my_first = INT32_MAX, my_last = -1;
#pragma unroll
    for (int q = NL - 1; q >= 0; --q) {
      const unsigned comb = (lm[q] | (lm[q] >> 16)) & 0xFFFFu;
      if (comb) {
        const int s_lo = __ffs(comb) - 1;
        my_first = 64 * (16 * q + s_lo) + 2 * lane + (int)(((lm[q] >> s_lo) & 1u) ^ 1u);
      }
    }
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const unsigned comb = (lm[q] | (lm[q] >> 16)) & 0xFFFFu;
      if (comb) {
        const int s_hi = 31 - __clz(comb);
        my_last = 64 * (16 * q + s_hi) + 2 * lane + (int)((lm[q] >> (16 + s_hi)) & 1u);
      }
    }
    // The three reductions are independent: issue them together so that their
    // latencies overlap on the antidiagonal's dependency chain.
    const int last_rel = __reduce_max_sync(kFull, my_last);
    const int first_rel = __reduce_min_sync(kFull, my_first);
    const int vrel = __reduce_max_sync(kFull, max(pk_lo(vmax2), pk_hi(vmax2)));
    if (last_rel < 0) break;
    const int first = 64 * cbase + first_rel, last = 64 * cbase + last_rel;
    if (vrel + rb > best) {
      // Smallest i holding the new best: each lane's smallest matching cell
      // over slots 1..sh, then one warp minimum.  Slots below the live range's
      // are dead on this antidiagonal (every cell holds kNeg16), so they never
      // match; slots above sh are not scanned (they may hold older values).
      const int sh = last_rel >> 6;
      const unsigned v2 = pk_pair(vrel, vrel);
      int my_c = INT32_MAX;
#pragma unroll
      for (int s = 1; s < NC; ++s) {
        if (s > sh) break;
        const unsigned e = H[s] ^ v2;
        const int c = 64 * s + 2 * lane;
        my_c = min(my_c, (e & 0xFFFFu) == 0 ? c : ((e >> 16) == 0 ? c + 1 : INT32_MAX));
      }
      const int cand = 64 * cbase + __reduce_min_sync(kFull, my_c);
      best = vrel + rb;
      bi = cand;
      bj = d - cand;
    }
    live_lo = first;
    live_hi = last;
  }
  if (lane == 0) {
    out->best = best;
    out->i_end = bi;
    out->j_end = bj;
    out->status = 0;
    out->cells = cells;
  }
  __syncwarp();
  return true;
}

// ---------------------------------------------------------------------------
// Narrow form: one lane per extension.  Two antidiagonal arrays of WT cells
// per lane, lane-interleaved in shared memory (cell slot s of array A of a
// lane at element ((A*WT + s) * 32 + lane), so the 32 lanes never conflict).
// Slot s holds cell i = f + s; the frame f moves up when the band reaches the
// top.  The band is walked cell by cell; the array of d-2 is overwritten in
// place with d (its value is read one cell ahead).
// Cells are stored as T: int32 scores, or (for X <= kNarrow16MaxX) int16
// scores relative to a per-lane base rb, rebased when the best has run 4096
// above it.  As in the packed wide form this is exact: live values then lie in
// [-X, 4096 + 64] of rb and dead cells hold -16384, so the halved rows (and the
// doubled residency they allow) change no result.
template <typename T>
struct NarrowCell;
template <>
struct NarrowCell<int> {
  static constexpr int kDead = kNeg;
  static constexpr bool kRelative = false;
};
template <>
struct NarrowCell<short> {
  static constexpr int kDead = -16384;
  static constexpr bool kRelative = true;
};
constexpr int kNarrow16MaxX = 8000;
constexpr int kNarrowRebase = 4096;

template <int WT>
struct NarrowLane {
  long long a0, b0;
  int m, n, item;
  int d, live_lo, live_hi, best, bi, bj, f, h1, rb;
  long long cells;
};

template <int WT, typename T>
__device__ __forceinline__ T& nslot(T* wbase, int A, int s, int lane) {
  if (!DIBELLA_IN_BOUNDS(s, WT, 1)) s = 0;
  return wbase[((A * WT + s) << 5) + lane];
}

template <int WT, typename T>
__device__ void narrow_init(NarrowLane<WT>& L, const Item& it, int item, T* wbase, int lane) {
  constexpr int kD = NarrowCell<T>::kDead;
  L.a0 = it.a0;
  L.b0 = it.b0;
  L.m = it.m;
  L.n = it.n;
  L.item = item;
  L.d = 1;
  L.live_lo = 0;
  L.live_hi = 0;
  L.best = 0;
  L.bi = 0;
  L.bj = 0;
  L.f = -1;
  L.h1 = 0;
  L.rb = 0;
  L.cells = 0;
  nslot<WT>(wbase, 0, 0, lane) = (T)kD;  // d = 0: i = -1
  nslot<WT>(wbase, 0, 1, lane) = (T)0;   //        i = 0
  nslot<WT>(wbase, 0, 2, lane) = (T)kD;  //        i = 1
  nslot<WT>(wbase, 1, 0, lane) = (T)kD;  // d = -1: i = -1
  nslot<WT>(wbase, 1, 1, lane) = (T)kD;  //         i = 0
}

// One antidiagonal for one lane.  Returns 1 when the extension finished,
// 2 when its band outgrew the lane's storage, 0 otherwise.  The band is walked
// in groups of U cells (unrolled, each cell guarded by the band's end): a lane
// issues the instructions of every cell of its last group, so U = 16 wastes up
// to 15 cell slots on a narrow band and U = 4 at most 3, for one loop step
// per group.  With TRACK the first and last live cell and the first cell of
// the maximum are kept in registers while the band is walked (selects on every
// lane), instead of being found afterwards by scans of the new row whose
// lengths differ from lane to lane.
template <int WT, typename T, int U, bool TRACK>
__device__ int narrow_step(NarrowLane<WT>& L, const uint32_t* __restrict__ words, const Scoring sc,
                           T* wbase, int lane) {
  static_assert(U == 4 || U == 8 || U == 16, "groups of 4, 8 or 16 cells");
  constexpr int kD = NarrowCell<T>::kDead;
  const int d = L.d;
  const int lo = max(L.live_lo, d - L.n);
  const int hi = min(min(L.live_hi + 1, d), L.m);
  const int h1 = L.h1, h2 = 1 - h1;
  if (hi + 1 - L.f >= WT) {
    if (hi - lo + 3 > WT) return 2;
    const int nf = lo - 1;
    for (int i = lo - 1; i <= hi; ++i) nslot<WT>(wbase, h1, i - nf, lane) = nslot<WT>(wbase, h1, i - L.f, lane);
    for (int i = lo - 1; i <= hi - 1; ++i) nslot<WT>(wbase, h2, i - nf, lane) = nslot<WT>(wbase, h2, i - L.f, lane);
    L.f = nf;
  }
  if (NarrowCell<T>::kRelative && L.best - L.rb >= kNarrowRebase) {
    // Both rows, every slot: live values stay above -X, dead ones stay dead.
    const int delta = L.best - L.rb;
    for (int A = 0; A < 2; ++A)
      for (int t = 0; t < WT; ++t) {
        T& c = nslot<WT>(wbase, A, t, lane);
        c = (T)max((int)c - delta, kD);
      }
    L.rb = L.best;
  }
  const int f = L.f;
  const int thr = L.best - L.rb - sc.X;
  int u = nslot<WT>(wbase, h1, lo - 1 - f, lane);
  int dg = nslot<WT>(wbase, h2, lo - 1 - f, lane);
  int vmax = kD;
  int tr_first = INT32_MAX, tr_last = -1, tr_best = -1;  // TRACK: first / last live cell, first maximum
  const long long abase = L.a0 - 1, bbase = L.b0 + 1 - d;
  for (int i = lo; i <= hi; i += 16) {
    const uint32_t wa = base_window(words, abase + i);
    const uint32_t wb = base_window(words, bbase + i);
    const uint32_t x = ~(wa ^ wb);
    const uint32_t mm = (x | (x >> 1)) & 0x55555555u;
    const int cnt = min(16, hi - i + 1);
    for (int g = 0; g < cnt; g += U) {
      T* p1 = &nslot<WT>(wbase, h1, i + g - f, lane);
      T* p2 = &nslot<WT>(wbase, h2, i + g - f, lane);
      const uint32_t mg = mm >> (2 * g);
      // Four cells at a time: their d-1 and d-2 values are loaded before any of
      // them is stored.  The compiler cannot tell that the two rows never
      // overlap, so a load of row d-1 issued after a store to row d-2 would wait
      // for it, and each cell would wait out a shared-memory latency.
      int lfv[U], dnv[U];
#pragma unroll
      for (int t = 0; t < U; ++t) {
        if ((t & 3) == 0) {
#pragma unroll
          for (int k = t; k < t + 4; ++k) {
            if (g + k < cnt) {
              lfv[k] = p1[k * 32];
              dnv[k] = p2[k * 32];
            }
          }
        }
        if (g + t < cnt) {
          const int lf = lfv[t];
          const int dn = dnv[t];
          const int sub = ((mg >> (2 * t)) & 1u) ? sc.S : sc.M;
          int h = __viaddmax_s32(max(u, lf), sc.G, dg + sub);  // max(max(u, lf) + G, dg + sub)
          h = h >= thr ? h : kD;
          p2[t * 32] = (T)h;
          if (TRACK) {
            const int ii = i + g + t;
            const bool lv = h != kD;
            tr_first = min(tr_first, lv ? ii : INT32_MAX);
            tr_last = lv ? ii : tr_last;
            tr_best = h > vmax ? ii : tr_best;  // strictly larger: the smallest i keeps a tie
          }
          vmax = max(vmax, h);
          u = lf;
          dg = dn;
        }
      }
    }
  }
  nslot<WT>(wbase, h2, lo - 1 - f, lane) = (T)kD;
  nslot<WT>(wbase, h2, hi + 1 - f, lane) = (T)kD;
  L.cells += hi - lo + 1;
  L.h1 = h2;
  if (vmax == kD) return 1;
  int llo = tr_first, lhi = tr_last;
  if (!TRACK) {
    llo = lo;
    while ((int)nslot<WT>(wbase, h2, llo - f, lane) == kD) ++llo;
    lhi = hi;
    while ((int)nslot<WT>(wbase, h2, lhi - f, lane) == kD) --lhi;
  }
  if (vmax + L.rb > L.best) {
    int b = tr_best;
    if (!TRACK) {
      b = llo;
      while ((int)nslot<WT>(wbase, h2, b - f, lane) != vmax) ++b;
    }
    L.best = vmax + L.rb;
    L.bi = b;
    L.bj = d - b;
  }
  L.live_lo = llo;
  L.live_hi = lhi;
  if (d == L.m + L.n) return 1;
  L.d = d + 1;
  return 0;
}

// ---------------------------------------------------------------------------
// Persistent kernels.  Each pops items from one queue until it is empty;
// an extension whose band outgrows the form is appended to p.esc_q.

// Register form, one warp per extension.
template <int NC>
__global__ void __launch_bounds__(kBlockThreads) wide_reg_kernel(ExtendParams p) {
  const int lane = threadIdx.x & 31;
  warp_clock(p.wclock, 0);
  const unsigned tail = *((volatile unsigned*)&p.cnt->tail[p.wide_q_id]);
  const bool fwd = tail <= p.forward_max;
  for (;;) {
    const unsigned q = pop_warp(p.cnt, p.wide_q_id);
    if (q >= tail) break;
    const int item = p.wide_q[q];
    if (!DIBELLA_IN_BOUNDS(item, p.q_cap, 3)) continue;
    if (fwd) {
      if (lane == 0) {
        const unsigned s = atomicAdd(&p.cnt->tail[p.esc_q_id], 1u);
        if (DIBELLA_IN_BOUNDS(s, p.q_cap, 2)) p.esc_q[s] = item;
      }
      __syncwarp();
      continue;
    }
    const Item it = p.items[item];
    if (!extend_reg<NC>(p.words, it, p.sc, p.ext + item)) {
      if (lane == 0) {
        const unsigned s = atomicAdd(&p.cnt->tail[p.esc_q_id], 1u);
        if (DIBELLA_IN_BOUNDS(s, p.q_cap, 2)) p.esc_q[s] = item;
        atomicAdd(&p.cnt->stat[3], 1u);
      }
    } else if (lane == 0) {
      atomicAdd(&p.cnt->cells[p.cells_idx], (unsigned long long)p.ext[item].cells);
    }
    __syncwarp();
  }
  warp_clock(p.wclock, 1);
}

// Packed form, one warp per extension (routed here only when X <= kPackedMaxX).
// Resident CTAs per SM asked of the compiler, by measurement: 9 for 8 slots (a
// little faster than the unconstrained 8, and than 10 or 12, where the slot
// code recomputes values it can no longer keep in registers), 6 for 16 slots,
// 4 for 24 slots (c3: 14% faster than the unconstrained 3, without spills).
// The per-warp clock is a separate instantiation (CLOCK), launched only for a
// clocked batch: even two untaken clock branches at entry and exit changed this
// kernel's code enough to cost 5% on the E. coli-sized escalations.
template <int NC, bool CLOCK = false>
__global__ void __launch_bounds__(kBlockThreads, NC == 8 ? 9 : (NC == 16 ? 6 : (NC == 24 ? 4 : 1)))
    wide_pk_kernel(ExtendParams p) {
  const int lane = threadIdx.x & 31;
  if (CLOCK) warp_clock(p.wclock, 0);
  const unsigned tail = *((volatile unsigned*)&p.cnt->tail[p.wide_q_id]);
  const bool fwd = NC > 8 && tail <= p.forward_max;  // 8 slots is never a ladder rung
  for (;;) {
    const unsigned q = pop_warp(p.cnt, p.wide_q_id);
    if (q >= tail) break;
    const int item = p.wide_q[q];
    if (!DIBELLA_IN_BOUNDS(item, p.q_cap, 3)) continue;
    if (fwd) {
      if (lane == 0) {
        const unsigned s = atomicAdd(&p.cnt->tail[p.esc_q_id], 1u);
        if (DIBELLA_IN_BOUNDS(s, p.q_cap, 2)) p.esc_q[s] = item;
      }
      __syncwarp();
      continue;
    }
    const Item it = p.items[item];
    if (!extend_pk<NC>(p.words, it, p.sc, p.ext + item)) {
      if (lane == 0) {
        const unsigned s = atomicAdd(&p.cnt->tail[p.esc_q_id], 1u);
        if (DIBELLA_IN_BOUNDS(s, p.q_cap, 2)) p.esc_q[s] = item;
        atomicAdd(&p.cnt->stat[3], 1u);
      }
    } else if (lane == 0) {
      atomicAdd(&p.cnt->cells[p.cells_idx], (unsigned long long)p.ext[item].cells);
    }
    __syncwarp();
  }
  if (CLOCK) warp_clock(p.wclock, 1);
}

// Grouped packed form: a warp runs NG = 32/GL extensions at once, GL lanes
// each, chunks of 2*GL cells (same cell encoding, slots, guard and base words
// as the packed form).  Every per-extension scalar lives in the lanes of its
// group, so one pass of the per-antidiagonal control serves all groups.  The
// jump table enters at the highest slot any group needs; a group whose band is
// lower processes the extra slots too, and its band test kills them (their
// cells lie above its hi; a slot it activates later is reset first).  Live
// range, maximum and argmax come from per-lane masks and one full-warp
// reduction per group.  The rare steps (window move, activation, rebase) run
// under a warp vote with per-group predicates.  Each group pops its next
// extension as soon as its current one ends.
template <int NG>
__device__ __forceinline__ int grp_reduce_max(int v, int g) {
  int r = 0;
#pragma unroll
  for (int k = 0; k < NG; ++k) {
    const int t = __reduce_max_sync(kFull, g == k ? v : INT32_MIN);
    r = g == k ? t : r;
  }
  return r;
}
template <int NG>
__device__ __forceinline__ int grp_reduce_min(int v, int g) {
  int r = 0;
#pragma unroll
  for (int k = 0; k < NG; ++k) {
    const int t = __reduce_min_sync(kFull, g == k ? v : INT32_MAX);
    r = g == k ? t : r;
  }
  return r;
}

template <int GL, int NC>
__global__ void __launch_bounds__(kBlockThreads) wide_grp_kernel(ExtendParams p) {
  static_assert(GL == 8 || GL == 16, "group of 8 or 16 lanes");
  warp_clock(p.wclock, 0);
  static_assert(NC % 8 == 0 && NC >= 8 && NC <= 32, "slots come in words of 8");
  constexpr int NW = NC / 8;
  constexpr int NG = 32 / GL;
  constexpr int CH = 2 * GL;                 // cells per chunk
  constexpr int LOG_CH = GL == 8 ? 4 : 5;
  constexpr int NL = (NC + 15) / 16;
  const int lane = threadIdx.x & 31;
  const int g = lane / GL, gl = lane % GL;
  const int src = (gl + GL - 1) & (GL - 1);
  const bool top = gl == GL - 1;
  const Scoring sc = p.sc;
  const unsigned M2 = pk_pair(sc.M, sc.M), S2 = pk_pair(sc.S, sc.S), G2 = pk_pair(sc.G, sc.G);
  const unsigned lane2 = pk_pair(2 * gl, 2 * gl + 1);
  const unsigned tail = *((volatile unsigned*)&p.cnt->tail[p.wide_q_id]);
  const uint32_t* __restrict__ words = p.words;

  bool active = false, exhausted = false;
  int item = 0, m = 0, n = 0, d = 0, live_lo = 0, live_hi = 0, best = 0, bi = 0, bj = 0;
  int cbase = 0, ctop = 0, rb = 0, bq_idx = INT32_MIN;
  unsigned bq = 0;
  long long a_lo = 0, b_lo = 0, cells = 0;
  unsigned H[NC], Up[NC], Aw[NW], Bw[NW];
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    H[s] = kNeg2;
    Up[s] = kNeg2;
  }
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    Aw[w] = 0;
    Bw[w] = 0;
  }

  for (;;) {
    // Refill: every group without work pops one extension.
    const bool want = !active && !exhausted;
    if (__any_sync(kFull, want)) {
      unsigned q = 0;
      if (want && gl == 0) q = atomicAdd(&p.cnt->head[p.wide_q_id], 1u);
      q = __shfl_sync(kFull, q, lane & ~(GL - 1));
      if (want) {
        if (q < tail) {
          item = p.wide_q[q];
          if (!DIBELLA_IN_BOUNDS(item, p.q_cap, 3)) item = 0;
          const Item it = p.items[item];
          m = it.m;
          n = it.n;
          a_lo = it.a0 - 1;
          b_lo = it.b0 + 1;
#pragma unroll
          for (int s = 0; s < NC; ++s) {
            H[s] = kNeg2;
            Up[s] = kNeg2;
          }
          if (gl == 0) H[1] = pk_pair(0, -16384);
          const int i0 = 2 * gl;
          Aw[0] = ((unsigned)base_of(words, a_lo + i0) << 2) | ((unsigned)base_of(words, a_lo + i0 + 1) << 18);
          Bw[0] = ((unsigned)base_of(words, b_lo + i0) << 2) | ((unsigned)base_of(words, b_lo + i0 + 1) << 18);
#pragma unroll
          for (int w = 1; w < NW; ++w) {
            Aw[w] = 0;
            Bw[w] = 0;
          }
          cbase = -1;
          ctop = 0;
          rb = 0;
          bq_idx = INT32_MIN;
          d = 1;
          live_lo = live_hi = 0;
          best = bi = bj = 0;
          cells = 0;
          active = true;
          if (m + n == 0) {
            if (gl == 0) {
              ExtOut o;
              o.best = 0; o.i_end = 0; o.j_end = 0; o.status = 0; o.cells = 0;
              p.ext[item] = o;
            }
            active = false;
          }
        } else {
          exhausted = true;
        }
      }
    }
    if (!__any_sync(kFull, active)) {
      if (__all_sync(kFull, exhausted)) {
        warp_clock(p.wclock, 1);
        break;
      }
      continue;
    }

    // One antidiagonal for every active group.
    int lo = max(live_lo, d - n);
    int hi = min(min(live_hi + 1, d), m);
    int c0 = lo >> LOG_CH;
    int cneed = (hi + 1) >> LOG_CH;
    const bool rare = active && ((c0 - 1 != cbase) | (cneed != ctop) | (best - rb >= kRebase));
    if (__any_sync(kFull, rare)) {
      for (;;) {  // keep slot 0 = chunk c0 - 1
        const bool need = rare && cbase < c0 - 1;
        if (!__any_sync(kFull, need)) break;
        if (need) {
#pragma unroll
          for (int s = 0; s + 1 < NC; ++s) {
            H[s] = H[s + 1];
            Up[s] = Up[s + 1];
          }
          H[NC - 1] = kNeg2;
          Up[NC - 1] = kNeg2;
#pragma unroll
          for (int w = 0; w < NW; ++w) {
            const int wn = w + 1 < NW ? w + 1 : w;
            const unsigned na = w + 1 < NW ? Aw[wn] : 0u, nb = w + 1 < NW ? Bw[wn] : 0u;
            Aw[w] = ((Aw[w] >> 2) & 0x3FFF3FFFu) | ((na & 0x00030003u) << 14);
            Bw[w] = ((Bw[w] >> 2) & 0x3FFF3FFFu) | ((nb & 0x00030003u) << 14);
          }
          ++cbase;
        }
      }
      if (rare && cneed - cbase > NC - 1) {  // band outgrew the slots: hand over
        if (gl == 0) {
          const unsigned s2 = atomicAdd(&p.cnt->tail[p.esc_q_id], 1u);
          if (DIBELLA_IN_BOUNDS(s2, p.q_cap, 2)) p.esc_q[s2] = item;
          atomicAdd(&p.cnt->stat[3], 1u);
        }
        active = false;
      }
      const bool act_new = rare && active && cneed > ctop;
      if (__any_sync(kFull, act_new)) {
        if (act_new) {
          const int snew = cneed - cbase;
          const int i0 = CH * cneed + 2 * gl;
          const unsigned a0b = base_of(words, a_lo + i0), a1b = base_of(words, a_lo + i0 + 1);
          const unsigned b0b = base_of(words, b_lo + 1 - d + i0), b1b = base_of(words, b_lo + 2 - d + i0);
          const int sh = 2 * (snew & 7);
          const unsigned clear = ~((3u << sh) | (3u << (sh + 16)));
#pragma unroll
          for (int w = 0; w < NW; ++w) {
            if (w == (snew >> 3)) {
              Aw[w] = (Aw[w] & clear) | (a0b << sh) | (a1b << (sh + 16));
              Bw[w] = (Bw[w] & clear) | (b0b << sh) | (b1b << (sh + 16));
            }
          }
#pragma unroll
          for (int s = 1; s < NC; ++s) {
            if (s == snew) {
              H[s] = kNeg2;
              Up[s] = kNeg2;
            }
          }
        }
      }
      if (rare && active) ctop = cneed;
      const bool reb = rare && active && best - rb >= kRebase;
      if (__any_sync(kFull, reb)) {
        if (reb) {
          const int delta = best - rb;
          const unsigned dn = pk_pair(-delta, -delta);
#pragma unroll
          for (int s = 0; s < NC; ++s) {
            H[s] = __vmaxs2(__vadd2(H[s], dn), kNeg2);
            Up[s] = __vmaxs2(__vadd2(Up[s], dn), kNeg2);
          }
          rb = best;
        }
      }
    }
    if (!active) {  // an idle group computes an empty band
      lo = 1;
      hi = 0;
      c0 = cbase + 1;
    }
    const int ntop = active ? ctop - cbase : 0;
    const int ntop_w = __reduce_max_sync(kFull, ntop);
    const int wtop_w = ntop_w >> 3;
    // Move every b base to the next cell and form the mismatch bits.
    unsigned MM[NW];
    {
      const long long r = b_lo - d + CH * c0;  // lane 0 of the group, low cell of slot 1
      if ((r >> 4) != (long long)bq_idx) {
        bq_idx = (int)(r >> 4);
        bq = active ? ldg_word(words, r >> 4) : 0u;
      }
      const unsigned bfresh = (bq >> ((unsigned)(r & 15) * 2u)) & 3u;
      unsigned prev_top = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        MM[w] = 0;
        if (NW == 1 || w <= wtop_w) {
          const unsigned t = __shfl_sync(kFull, Bw[w], src, GL);
          unsigned lo_new = t >> 16;
          const unsigned lo_lane0 = ((t >> 14) & 0xFFFCu) | prev_top;
          prev_top = (t >> 30) & 3u;
          if (gl == 0) lo_new = (w == 0) ? ((lo_lane0 & ~0xCu) | (bfresh << 2)) : lo_lane0;
          Bw[w] = (Bw[w] << 16) | lo_new;
          const unsigned x = ~(Aw[w] ^ Bw[w]);
          MM[w] = (x | (x >> 1)) & 0x55555555u;
        }
      }
    }
    const int thr_rel = best - rb - sc.X;
    const unsigned nthr2 = pk_pair(-thr_rel, -thr_rel);
    const unsigned A2 = __vsub2(lane2, pk_dup(lo - CH * cbase));
    const unsigned B2 = __vsub2(pk_dup(hi - CH * cbase), lane2);
    unsigned vmax2 = kNeg2, lm[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) lm[q] = 0;
#define DIBELLA_GRP_I(S) ((S) < NC ? (S) : NC - 1)
#define DIBELLA_GRP_SLOT(S)                                                                        \
  if (S < NC) {                                                                                    \
    constexpr int s_ = DIBELLA_GRP_I(S), p_ = s_ > 0 ? s_ - 1 : 0;                                 \
    const unsigned prevH = __shfl_sync(kFull, top ? H[p_] : H[s_], src, GL);                       \
    const unsigned u2 = __byte_perm(H[s_], prevH, 0x1076u);                                        \
    const unsigned mis = half_sign_mask(MM[s_ >> 3] << (15 - 2 * (s_ & 7)));                       \
    const unsigned sub2 = (mis & S2) | (~mis & M2);                                                \
    const unsigned ds = __viaddmax_s16x2(Up[s_], sub2, kNeg2);                                     \
    unsigned h2 = __viaddmax_s16x2(__vmaxs2(u2, H[s_]), G2, ds);                                   \
    const unsigned f = __vimin3_s16x2(__vadd2(h2, nthr2), __vadd2(A2, (unsigned)(CH * 0x00010001u) * s_), \
                                      __vsub2(B2, (unsigned)(CH * 0x00010001u) * s_));             \
    const unsigned dead = half_sign_mask(f);                                                       \
    h2 = (h2 & ~dead) | (kNeg2 & dead);                                                            \
    Up[s_] = u2;                                                                                   \
    H[s_] = h2;                                                                                    \
    vmax2 = __vmaxs2(vmax2, h2);                                                                   \
    lm[s_ >> 4] |= ~dead & (0x00010001u << (s_ & 15));                                             \
  }
    switch (ntop_w) {
      case 31: DIBELLA_GRP_SLOT(31) [[fallthrough]];
      case 30: DIBELLA_GRP_SLOT(30) [[fallthrough]];
      case 29: DIBELLA_GRP_SLOT(29) [[fallthrough]];
      case 28: DIBELLA_GRP_SLOT(28) [[fallthrough]];
      case 27: DIBELLA_GRP_SLOT(27) [[fallthrough]];
      case 26: DIBELLA_GRP_SLOT(26) [[fallthrough]];
      case 25: DIBELLA_GRP_SLOT(25) [[fallthrough]];
      case 24: DIBELLA_GRP_SLOT(24) [[fallthrough]];
      case 23: DIBELLA_GRP_SLOT(23) [[fallthrough]];
      case 22: DIBELLA_GRP_SLOT(22) [[fallthrough]];
      case 21: DIBELLA_GRP_SLOT(21) [[fallthrough]];
      case 20: DIBELLA_GRP_SLOT(20) [[fallthrough]];
      case 19: DIBELLA_GRP_SLOT(19) [[fallthrough]];
      case 18: DIBELLA_GRP_SLOT(18) [[fallthrough]];
      case 17: DIBELLA_GRP_SLOT(17) [[fallthrough]];
      case 16: DIBELLA_GRP_SLOT(16) [[fallthrough]];
      case 15: DIBELLA_GRP_SLOT(15) [[fallthrough]];
      case 14: DIBELLA_GRP_SLOT(14) [[fallthrough]];
      case 13: DIBELLA_GRP_SLOT(13) [[fallthrough]];
      case 12: DIBELLA_GRP_SLOT(12) [[fallthrough]];
      case 11: DIBELLA_GRP_SLOT(11) [[fallthrough]];
      case 10: DIBELLA_GRP_SLOT(10) [[fallthrough]];
      case 9: DIBELLA_GRP_SLOT(9) [[fallthrough]];
      case 8: DIBELLA_GRP_SLOT(8) [[fallthrough]];
      case 7: DIBELLA_GRP_SLOT(7) [[fallthrough]];
      case 6: DIBELLA_GRP_SLOT(6) [[fallthrough]];
      case 5: DIBELLA_GRP_SLOT(5) [[fallthrough]];
      case 4: DIBELLA_GRP_SLOT(4) [[fallthrough]];
      case 3: DIBELLA_GRP_SLOT(3) [[fallthrough]];
      case 2: DIBELLA_GRP_SLOT(2) [[fallthrough]];
      case 1: DIBELLA_GRP_SLOT(1) [[fallthrough]];
      default: break;
    }
#undef DIBELLA_GRP_SLOT
#undef DIBELLA_GRP_I
    H[0] = kNeg2;
    if (active) cells += hi - lo + 1;
    // Lowest and highest live cell of the lane (relative to chunk cbase), then
    // of the group.
    int my_first = INT32_MAX, my_last = -1;
#pragma unroll
    for (int q = NL - 1; q >= 0; --q) {
      const unsigned comb = (lm[q] | (lm[q] >> 16)) & 0xFFFFu;
      if (comb) {
        const int s_lo = __ffs(comb) - 1;
        my_first = CH * (16 * q + s_lo) + 2 * gl + (int)(((lm[q] >> s_lo) & 1u) ^ 1u);
      }
    }
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const unsigned comb = (lm[q] | (lm[q] >> 16)) & 0xFFFFu;
      if (comb) {
        const int s_hi = 31 - __clz(comb);
        my_last = CH * (16 * q + s_hi) + 2 * gl + (int)((lm[q] >> (16 + s_hi)) & 1u);
      }
    }
    const int last_rel = grp_reduce_max<NG>(my_last, g);
    const int first_rel = grp_reduce_min<NG>(my_first, g);
    const int vrel = grp_reduce_max<NG>(max(pk_lo(vmax2), pk_hi(vmax2)), g);
    const bool improved = active && last_rel >= 0 && vrel + rb > best;
    if (__any_sync(kFull, improved)) {
      // Smallest i holding the new best: each lane's first match over the
      // group's live slots, then the group minimum.
      const int sl = improved ? first_rel >> LOG_CH : NC, sh = improved ? last_rel >> LOG_CH : 0;
      const int sh_w = __reduce_max_sync(kFull, sh);
      const unsigned v2 = pk_pair(vrel, vrel);
      int my_c = INT32_MAX;
#pragma unroll
      for (int s = 1; s < NC; ++s) {
        if (s > sh_w) break;
        if (s >= sl && s <= sh && my_c == INT32_MAX) {
          const unsigned e = H[s] ^ v2;
          if ((e & 0xFFFFu) == 0) my_c = CH * s + 2 * gl;
          else if ((e >> 16) == 0) my_c = CH * s + 2 * gl + 1;
        }
      }
      const int cand = grp_reduce_min<NG>(my_c, g);
      if (improved) {
        best = vrel + rb;
        bi = CH * cbase + cand;
        bj = d - bi;
      }
    }
    if (active) {
      if (last_rel < 0 || d == m + n) {
        if (gl == 0) {
          ExtOut o;
          o.best = best; o.i_end = bi; o.j_end = bj; o.status = 0; o.cells = cells;
          p.ext[item] = o;
          atomicAdd(&p.cnt->cells[p.cells_idx], (unsigned long long)cells);
        }
        active = false;
      } else {
        live_lo = CH * cbase + first_rel;
        live_hi = CH * cbase + last_rel;
        ++d;
      }
    }
  }
}

// CTA form: one CTA of kCtaWarps warps per extension, for the widest bands.
// Three antidiagonals of kCtaCap int32 cells in a circular shared-memory array
// (cell i at i mod kCtaCap, as in the warp form); the band's 32-cell chunks
// are dealt round-robin to the warps.  Per antidiagonal each warp reduces its
// own maximum and live range, and one barrier publishes them (double-buffered
// by antidiagonal parity, so the next antidiagonal's writes cannot overtake a
// slow reader); every thread then combines the kCtaWarps entries itself, so
// all threads hold the same band, best and threshold.  The argmax, needed
// only when the best improves, takes one more barrier.
constexpr int kCtaWarps = 8;
constexpr int kCtaThreads = kCtaWarps * 32;
constexpr int kCtaCap = 8192;
struct CtaShared {
  int red[2][kCtaWarps][3];  // per warp: max, first live, last live
  int arg[kCtaWarps];        // per warp: smallest i holding the new best
  int item;
};
constexpr size_t kCtaSmemBytes = sizeof(CtaShared) + (size_t)3 * kCtaCap * sizeof(int);

// Returns false (uniformly across the CTA) when the band outgrew kCtaCap - 3.
__device__ bool extend_cta(const uint32_t* __restrict__ words, const Item& it, const Scoring sc,
                           CtaShared& sh, int* arr, ExtOut* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int mask = kCtaCap - 1;
  int* H2 = arr;
  int* H1 = arr + kCtaCap;
  int* H0 = arr + 2 * kCtaCap;
  const int m = it.m, n = it.n;
  if (threadIdx.x == 0) {
    H1[0] = 0;
    H1[mask] = kNeg;
    H1[1] = kNeg;
    H2[mask] = kNeg;
    H2[0] = kNeg;
  }
  __syncthreads();
  int live_lo = 0, live_hi = 0, best = 0, bi = 0, bj = 0;
  long long cells = 0;
  bool ok = true;
  for (int d = 1; d <= m + n; ++d) {
    const int lo = max(live_lo, d - n);
    const int hi = min(min(live_hi + 1, d), m);
    if (hi - lo + 3 > kCtaCap) {
      ok = false;
      break;
    }
    const int thr = best - sc.X;
    const long long abase = it.a0 - 1, bbase = it.b0 + 1 - d;
    int vmax = kNeg, first = INT32_MAX, last = -1;
    for (int i0 = lo + 32 * warp; i0 <= hi; i0 += 32 * kCtaWarps) {
      const int i = i0 + lane;
      int h = kNeg;
      if (i <= hi) {
        const int lf = H1[i & mask];
        const int u = H1[(i - 1) & mask];
        const int dg = H2[(i - 1) & mask];
        const int ca = base_at(words, abase + i), cb = base_at(words, bbase + i);
        const int sub = (ca ^ cb) == 3 ? sc.M : sc.S;
        h = max(max(u, lf) + sc.G, dg + sub);
        h = h >= thr ? h : kNeg;
        H0[i & mask] = h;
      }
      vmax = max(vmax, h);
      const unsigned bl = __ballot_sync(kFull, h != kNeg);
      if (bl) {
        if (first == INT32_MAX) first = i0 + __ffs(bl) - 1;
        last = i0 + 31 - __clz(bl);
      }
    }
    vmax = __reduce_max_sync(kFull, vmax);
    const int par = d & 1;
    if (lane == 0) {
      sh.red[par][warp][0] = vmax;
      sh.red[par][warp][1] = first;
      sh.red[par][warp][2] = last;
    }
    if (threadIdx.x == 0) H0[(lo - 1) & mask] = kNeg;
    if (threadIdx.x == 1) H0[(hi + 1) & mask] = kNeg;
    __syncthreads();
    int cmax = kNeg, cfirst = INT32_MAX, clast = -1;
#pragma unroll
    for (int w = 0; w < kCtaWarps; ++w) {
      cmax = max(cmax, sh.red[par][w][0]);
      cfirst = min(cfirst, sh.red[par][w][1]);
      clast = max(clast, sh.red[par][w][2]);
    }
    cells += hi - lo + 1;
    if (cmax == kNeg) break;
    if (cmax > best) {
      int cand = INT32_MAX;
      for (int i0 = lo + 32 * warp; i0 <= clast; i0 += 32 * kCtaWarps) {
        if (i0 + 31 < cfirst) continue;
        const int i = i0 + lane;
        const unsigned bl = __ballot_sync(kFull, i >= cfirst && i <= clast && H0[i & mask] == cmax);
        if (bl) {
          cand = i0 + __ffs(bl) - 1;
          break;
        }
      }
      if (lane == 0) sh.arg[warp] = cand;
      __syncthreads();
      int c = INT32_MAX;
#pragma unroll
      for (int w = 0; w < kCtaWarps; ++w) c = min(c, sh.arg[w]);
      best = cmax;
      bi = c;
      bj = d - c;
      __syncthreads();  // sh.arg is read before any warp can write it again
    }
    live_lo = cfirst;
    live_hi = clast;
    int* t = H2;
    H2 = H1;
    H1 = H0;
    H0 = t;
  }
  if (ok && threadIdx.x == 0) {
    out->best = best;
    out->i_end = bi;
    out->j_end = bj;
    out->status = 0;
    out->cells = cells;
  }
  __syncthreads();
  return ok;
}

__global__ void __launch_bounds__(kCtaThreads) wide_cta_kernel(ExtendParams p) {
  extern __shared__ int smem_cta[];
  CtaShared& sh = *reinterpret_cast<CtaShared*>(smem_cta);
  int* arr = smem_cta + sizeof(CtaShared) / sizeof(int);
  const unsigned tail = *((volatile unsigned*)&p.cnt->tail[p.wide_q_id]);
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned q = atomicAdd(&p.cnt->head[p.wide_q_id], 1u);
      sh.item = q < tail ? p.wide_q[q] : -1;
      if (sh.item >= 0 && !DIBELLA_IN_BOUNDS(sh.item, p.q_cap, 3)) sh.item = -1;
    }
    __syncthreads();
    const int item = sh.item;
    __syncthreads();  // every thread has read sh.item before thread 0 may rewrite it
    if (item < 0) break;
    const Item it = p.items[item];
    if (!extend_cta(p.words, it, p.sc, sh, arr, p.ext + item)) {
      if (threadIdx.x == 0) {
        const unsigned s = atomicAdd(&p.cnt->tail[p.esc_q_id], 1u);
        if (DIBELLA_IN_BOUNDS(s, p.q_cap, 2)) p.esc_q[s] = item;
        atomicAdd(&p.cnt->stat[4], 1u);
      }
    } else if (threadIdx.x == 0) {
      atomicAdd(&p.cnt->cells[2], (unsigned long long)p.ext[item].cells);
    }
  }
}

// Narrow form: one lane per extension; lanes refill independently.  Each warp
// owns 2*WT*32 cells of type T in shared memory (see NarrowLane).  The same
// kernel with a wide row (WT = 128..256, one warp per block so that the rows
// of more warps fit an SM) is the mid form: it takes the narrow form's
// escalations, whose bands (about 100-200 cells for reads that share their
// seed by chance) a lane walks for ~12 warp instructions per 32 cells, against
// a fixed per-antidiagonal control cost for a whole warp per extension.
template <int WT, typename T, int NW, int U, bool TRACK = false>
__global__ void __launch_bounds__(NW * 32) narrow_kernel(ExtendParams p) {
  extern __shared__ int smem_words[];
  const int lane = threadIdx.x & 31;
  T* wbase = reinterpret_cast<T*>(smem_words) + (threadIdx.x >> 5) * (2 * WT * 32);
  warp_clock(p.wclock, 0);
  const unsigned ntail = *((volatile unsigned*)&p.cnt->tail[p.narrow_q_id]);
  NarrowLane<WT> L;
  bool active = false, exhausted = false;
  for (;;) {
    const unsigned want = __ballot_sync(kFull, !active && !exhausted);
    if (want) {
      const int leader = __ffs(want) - 1;
      unsigned base = 0;
      if (lane == leader) base = atomicAdd(&p.cnt->head[p.narrow_q_id], (unsigned)__popc(want));
      base = __shfl_sync(kFull, base, leader);
      if (want & (1u << lane)) {
        const unsigned q = base + __popc(want & ((1u << lane) - 1u));
        const int item = q < ntail ? p.narrow_q[q] : -1;
        // (a bad item index, debug build: dropped; the lane stays idle and refills)
        if (q < ntail && DIBELLA_IN_BOUNDS(item, p.q_cap, 3)) {
          const Item it = p.items[item];
          narrow_init<WT, T>(L, it, item, wbase, lane);
          active = true;
          if (it.m + it.n == 0) {
            ExtOut o;
            o.best = 0; o.i_end = 0; o.j_end = 0; o.status = 0; o.cells = 0;
            p.ext[item] = o;
            active = false;
          }
        } else if (q >= ntail) {
          exhausted = true;
        }
      }
    }
    if (!__any_sync(kFull, active)) {
      if (__all_sync(kFull, exhausted)) {
        warp_clock(p.wclock, 1);
        break;
      }
      continue;
    }
    if (active) {
      const int r = narrow_step<WT, T, U, TRACK>(L, p.words, p.sc, wbase, lane);
      if (r == 1) {
        ExtOut o;
        o.best = L.best; o.i_end = L.bi; o.j_end = L.bj; o.status = 0; o.cells = L.cells;
        p.ext[L.item] = o;
        atomicAdd(&p.cnt->cells[p.narrow_cells_idx], (unsigned long long)L.cells);
        active = false;
      } else if (r == 2) {
        const unsigned s = atomicAdd(&p.cnt->tail[p.esc_q_id], 1u);
        if (DIBELLA_IN_BOUNDS(s, p.q_cap, 2)) p.esc_q[s] = L.item;
        atomicAdd(&p.cnt->stat[p.narrow_esc_stat], 1u);
        atomicAdd(&p.cnt->cells[7], (unsigned long long)L.cells);
        active = false;
      } else if (p.narrow_max_d > 0 && L.d > p.narrow_max_d) {
        const unsigned s = atomicAdd(&p.cnt->tail[kQLong], 1u);
        if (DIBELLA_IN_BOUNDS(s, p.q_cap, 2)) p.long_q[s] = L.item;
        atomicAdd(&p.cnt->stat[7], 1u);
        atomicAdd(&p.cnt->cells[7], (unsigned long long)L.cells);
        active = false;
      }
    }
  }
}

// Global-band form: one warp per extension, band in workspace memory.
__global__ void __launch_bounds__(kBlockThreads) global_kernel(ExtendParams p) {
  const int gwarp = (blockIdx.x * kBlockThreads + threadIdx.x) >> 5;
  if (!DIBELLA_IN_BOUNDS(gwarp, kGlobalWarps, 5)) return;
  int* arr = p.gband + (size_t)gwarp * 3 * p.gcap;
  const unsigned tail = *((volatile unsigned*)&p.cnt->tail[p.wide_q_id]);
  for (;;) {
    const unsigned q = pop_warp(p.cnt, p.wide_q_id);
    if (q >= tail) break;
    const int item = p.wide_q[q];
    if (!DIBELLA_IN_BOUNDS(item, p.q_cap, 3)) continue;
    const Item it = p.items[item];
    if (!extend_warp<true>(p.words, it, p.sc, arr, p.gcap, p.ext + item)) {
      if ((threadIdx.x & 31) == 0) {
        ExtOut o;
        o.best = 0; o.i_end = 0; o.j_end = 0; o.status = DIBELLA_RES_BAND_OVERFLOW; o.cells = 0;
        p.ext[item] = o;
        atomicAdd(&p.cnt->stat[5], 1u);
      }
    } else if ((threadIdx.x & 31) == 0) {
      atomicAdd(&p.cnt->cells[3], (unsigned long long)p.ext[item].cells);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
struct ExpandParams {
  const uint32_t* __restrict__ words;
  const long long* __restrict__ read_word_offsets;
  const int* __restrict__ read_lengths;
  long long n_reads;
  const dibella_pair_t* __restrict__ pairs;
  long long n_pairs;
  int k;
  Scoring sc;
  dibella_result_t* results;
  Item* items;
  Counters* cnt;
  int narrow_max_x, narrow_max_len, n_buckets;
  int bounds[DIBELLA_MAX_BUCKETS];
};

__device__ __forceinline__ unsigned long long bases64(const uint32_t* __restrict__ words, long long idx) {
  const long long w = idx >> 4;
  const unsigned sh = (unsigned)(idx & 15) * 2u;
  const uint32_t w0 = ldg_word(words, w), w1 = ldg_word(words, w + 1), w2 = ldg_word(words, w + 2);
  return (unsigned long long)__funnelshift_r(w0, w1, sh) |
         ((unsigned long long)__funnelshift_r(w1, w2, sh) << 32);
}

__device__ __forceinline__ long long copy_words(long long len) { return ((len + 15) / 16 + 3) / 4 * 4; }

__global__ void expand_kernel(ExpandParams p) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < p.n_pairs;
       t += (long long)gridDim.x * blockDim.x) {
    const dibella_pair_t pr = p.pairs[t];
    dibella_result_t r;
    memset(&r, 0, sizeof(r));
    Item L, R;
    L.a0 = L.b0 = R.a0 = R.b0 = 0;
    L.m = L.n = R.m = R.n = 0;
    L.tag = R.tag = -1;
    L.pad = R.pad = 0;
    const int k = p.k;
    bool valid = (long long)pr.read_a < p.n_reads && (long long)pr.read_b < p.n_reads && pr.strand <= 1;
    long long lenA = 0, lenB = 0;
    if (valid) {
      lenA = p.read_lengths[pr.read_a];
      lenB = p.read_lengths[pr.read_b];
      valid = (long long)pr.pos_a + k <= lenA && (long long)pr.pos_b + k <= lenB;
    }
    if (!valid) {
      r.status = DIBELLA_RES_INVALID_SEED;
    } else {
      const long long offA = p.read_word_offsets[pr.read_a], offB = p.read_word_offsets[pr.read_b];
      const long long fA = offA * 16, rA = (offA + copy_words(lenA)) * 16;
      const long long fB = offB * 16, rB = (offB + copy_words(lenB)) * 16;
      const long long pa = pr.pos_a;
      const long long pb = pr.strand ? lenB - pr.pos_b - k : (long long)pr.pos_b;  // in B'
      // Seed score: A[pa, pa+k) against B'[pb, pb+k), B' = F_B or R_B.
      const unsigned long long sa = bases64(p.words, fA + pa);
      const unsigned long long sb = bases64(p.words, (pr.strand ? rB : fB) + pb);
      const unsigned long long x = sa ^ sb;
      const unsigned long long kmask = k == 32 ? ~0ull : ((1ull << (2 * k)) - 1ull);
      const int mism = __popcll((x | (x >> 1)) & 0x5555555555555555ull & kmask);
      r.score = k * p.sc.M + mism * (p.sc.S - p.sc.M);
      r.status = mism ? DIBELLA_RES_SEED_MISMATCH : 0;
      // Left: a[x] = A[pa-1-x] = comp(R_A[lenA-pa+x]); b[y] = B'[pb-1-y].
      L.a0 = rA + (lenA - pa);
      L.m = (int)pa;
      L.b0 = (pr.strand ? rB : fB) + (pb - 1);
      L.n = (int)pb;
      // Right: a[x] = A[pa+k+x]; b[y] = B'[pb+k+y] = comp(copy'[lenB-1-pb-k-y]).
      R.a0 = fA + pa + k;
      R.m = (int)(lenA - pa - k);
      R.b0 = (pr.strand ? fB : rB) + (lenB - 1 - pb - k);
      R.n = (int)(lenB - pb - k);
      Item* both[2] = {&L, &R};
      for (int s = 0; s < 2; ++s) {
        Item* it = both[s];
        const int key = min(it->m, it->n);
        const int cls = (p.sc.X <= p.narrow_max_x && key <= p.narrow_max_len) ? 0 : 1;
        int b = 0;
        while (b < p.n_buckets - 1 && key >= p.bounds[b]) ++b;
        it->tag = (cls << 8) | b;
        atomicAdd(&p.cnt->bucket_count[cls][b], 1u);
      }
    }
    p.results[t] = r;
    p.items[2 * t] = L;
    p.items[2 * t + 1] = R;
  }
}

__global__ void scan_kernel(Counters* cnt, int n_buckets) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int c = 0; c < 2; ++c) {
    unsigned pos = 0;
    for (int b = n_buckets - 1; b >= 0; --b) {
      cnt->bucket_cursor[c][b] = pos;
      pos += cnt->bucket_count[c][b];
    }
    cnt->tail[c == 0 ? kQNarrow : kQWide] = pos;
    cnt->stat[c] = pos;
  }
}

__global__ void scatter_kernel(const Item* __restrict__ items, long long n_items, Counters* cnt,
                               int* narrow_q, int* wide_q) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n_items;
       t += (long long)gridDim.x * blockDim.x) {
    const int tag = items[t].tag;
    if (tag < 0) continue;
    const int cls = tag >> 8, b = tag & 255;
    const unsigned s = atomicAdd(&cnt->bucket_cursor[cls][b], 1u);
    (cls == 0 ? narrow_q : wide_q)[s] = (int)t;
  }
}

#ifdef DIBELLA_BOUNDS_CHECK
// Debug build: the words of the batch's store (the last read's two copies end
// it, followed by the 8 closing zero words), for the store-read checks.
__global__ void store_extent_kernel(const long long* offs, const int* lens, long long n_reads) {
  g_store_words = n_reads > 0 ? offs[n_reads - 1] + 2 * copy_words(lens[n_reads - 1]) + 8 : 8;
}
#endif

// Debug build: set the store extent on `st` (no launch in the release build).
void set_store_extent(const int64_t* offs, const int32_t* lens, int64_t n_reads, cudaStream_t st) {
#ifdef DIBELLA_BOUNDS_CHECK
  store_extent_kernel<<<1, 1, 0, st>>>((const long long*)offs, lens, (long long)n_reads);
#else
  (void)offs;
  (void)lens;
  (void)n_reads;
  (void)st;
#endif
}

struct CombineParams {
  const int* __restrict__ read_lengths;
  const dibella_pair_t* __restrict__ pairs;
  long long n_pairs;
  int k;
  const ExtOut* __restrict__ ext;
  dibella_result_t* results;
};

__global__ void combine_kernel(CombineParams p) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < p.n_pairs;
       t += (long long)gridDim.x * blockDim.x) {
    dibella_result_t r = p.results[t];
    if (r.status & DIBELLA_RES_INVALID_SEED) continue;
    const ExtOut L = p.ext[2 * t], R = p.ext[2 * t + 1];
    if ((L.status | R.status) & DIBELLA_RES_BAND_OVERFLOW) {
      const int st = r.status;
      memset(&r, 0, sizeof(r));
      r.status = st | DIBELLA_RES_BAND_OVERFLOW;
      p.results[t] = r;
      continue;
    }
    const dibella_pair_t pr = p.pairs[t];
    const long long lenB = p.read_lengths[pr.read_b];
    const long long pa = pr.pos_a;
    const long long pb = pr.strand ? lenB - pr.pos_b - p.k : (long long)pr.pos_b;
    r.score += L.best + R.best;
    r.score_left = L.best;
    r.score_right = R.best;
    r.begin_a = (uint32_t)(pa - L.i_end);
    r.end_a = (uint32_t)(pa + p.k + R.i_end);
    const long long bb = pb - L.j_end, be = pb + p.k + R.j_end;
    if (pr.strand) {
      r.begin_b = (uint32_t)(lenB - be);
      r.end_b = (uint32_t)(lenB - bb);
    } else {
      r.begin_b = (uint32_t)bb;
      r.end_b = (uint32_t)be;
    }
    r.cells = L.cells + R.cells;
    p.results[t] = r;
  }
}

__global__ void best_of_pair_kernel(const dibella_pair_t* __restrict__ pairs, long long n,
                                    dibella_result_t* results) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const dibella_pair_t pr = pairs[t];
    if (t > 0 && pairs[t - 1].read_a == pr.read_a && pairs[t - 1].read_b == pr.read_b) continue;
    long long best = -1;
    int best_score = 0;
    for (long long u = t; u < n && pairs[u].read_a == pr.read_a && pairs[u].read_b == pr.read_b; ++u) {
      const dibella_result_t& r = results[u];
      if (r.status & (DIBELLA_RES_INVALID_SEED | DIBELLA_RES_BAND_OVERFLOW)) continue;
      if (best < 0 || r.score > best_score) {
        best = u;
        best_score = r.score;
      }
    }
    if (best >= 0) results[best].status |= DIBELLA_RES_BEST_OF_PAIR;
  }
}

// One launch per candidate pair (the baseline form): one warp aligns, seed by
// seed, the left then the right extension of every seed record in [t0, t1)
// with the same per-extension code as the batched path: the packed register
// form with 8 slots (int32 register form above X = kPackedMaxX), then 32 slots
// when its band outgrows that, then the band in workspace slot 0.  No queues,
// no persistence, no graph: what batching adds is measured against this.
__global__ void __launch_bounds__(32) per_pair_kernel(const uint32_t* __restrict__ words,
                                                      const Item* __restrict__ items, ExtOut* ext, long long t0,
                                                      long long t1, Scoring sc, int* gband, int gcap) {
  for (long long t = t0; t < t1; ++t)
    for (int s = 0; s < 2; ++s) {
      const Item it = items[2 * t + s];
      if (it.tag < 0) continue;
      ExtOut* o = ext + 2 * t + s;
      bool ok;
      if (sc.X <= kPackedMaxX)
        ok = extend_pk<8>(words, it, sc, o) || extend_pk<32>(words, it, sc, o);
      else
        ok = extend_reg<32>(words, it, sc, o);
      if (!ok && !extend_warp<true>(words, it, sc, gband, gcap, o)) {
        if (threadIdx.x == 0) {
          ExtOut b;
          b.best = 0; b.i_end = 0; b.j_end = 0; b.status = DIBELLA_RES_BAND_OVERFLOW; b.cells = 0;
          *o = b;
        }
      }
      __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Host side.

thread_local std::string g_last_error;

std::mutex g_mu;
dibella_schedule_t g_default_schedule = {
    /*narrow_max_xdrop=*/30, /*narrow_max_len=*/1 << 30, /*narrow_band_cap=*/48,
    /*wide_slots=*/0, /*wide_packed=*/1, /*wide_group_lanes=*/0, /*wide_blocks_per_sm=*/0,
    /*narrow_blocks_per_sm=*/0,
    /*n_buckets=*/6, {500, 2000, 5000, 10000, 20000, 0, 0, 0}, /*mid_band_cap=*/0, /*narrow_split_d=*/0,
    /*narrow_unroll=*/0, /*narrow_track=*/1};

struct DeviceInfo {
  bool ready = false;
  int sms = 0;
  int narrow_blocks[2][3][4] = {};  // narrow_kernel<32/48/64, int | short, ., 4/8/16 groups | tracked> per SM
  int mid_blocks[3] = {};        // narrow_kernel<128/192/256, short, 1> (the mid form) blocks per SM
  int reg_blocks[2] = {0, 0};        // wide_reg_kernel<16/32> blocks per SM
  int pk_blocks[4] = {0, 0, 0, 0};   // wide_pk_kernel<16/24/32/8> blocks per SM
  int grp16_blocks[3] = {0, 0, 0};   // wide_grp_kernel<16, 16/24/32> blocks per SM
  int grp8_blocks[2] = {0, 0};       // wide_grp_kernel<8, 16/24> blocks per SM
  int cta_blocks = 0;                // wide_cta_kernel blocks per SM
};
std::mutex g_dev_mu;
DeviceInfo g_dev[64];

bool g_timing = false;
cudaEvent_t g_ev[10] = {};
// Per-warp clock of one launch per batch (dibella_enable_warp_clock): which
// launch (0 none, 1 narrow, 2 first wide, 3 mid, 4 wide on the escalations)
// and how many warps the last clocked launch ran.
__device__ unsigned long long g_warp_clock[2 * kMaxClockedWarps];
int g_clock_launch = 0;
int g_clocked_warps = 0;

// The clock array for launch `which` of this batch, cleared on `st`; null when
// that launch is not clocked.
unsigned long long* clock_for(int which, int warps, cudaStream_t st) {
  if (g_clock_launch != which) return nullptr;
  unsigned long long* p = nullptr;
  if (cudaGetSymbolAddress((void**)&p, g_warp_clock) != cudaSuccess) return nullptr;
  const int n = std::min(warps, kMaxClockedWarps);
  if (cudaMemsetAsync(p, 0, sizeof(unsigned long long) * 2 * (size_t)n, st) != cudaSuccess) return nullptr;
  g_clocked_warps = n;
  return p;
}
thread_local int g_launches = 0;  // kernel launches of this thread's last batch
int g_ev_count = 0;

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return DIBELLA_ECUDA;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int gband_cap_for(int32_t max_read_len) {
  int cap = 64;
  while (cap < max_read_len + 4 && cap < (1 << 25)) cap <<= 1;
  return cap;
}

struct Layout {
  size_t counters, items, ext, queue[kNumQ], gband, total;
};

Layout layout_for(long long n_pairs, int gcap) {
  Layout L;
  size_t off = 0;
  L.counters = off;
  off = align256(off + sizeof(Counters));
  L.items = off;
  off = align256(off + sizeof(Item) * 2 * (size_t)n_pairs);
  L.ext = off;
  off = align256(off + sizeof(ExtOut) * 2 * (size_t)n_pairs);
  for (int q = 0; q < kNumQ; ++q) {
    L.queue[q] = off;
    off = align256(off + sizeof(int) * 2 * (size_t)n_pairs);
  }
  L.gband = off;
  off = align256(off + sizeof(int) * 3 * (size_t)gcap * kGlobalWarps);
  L.total = off;
  return L;
}

// Largest band capacity whose global band region fits in `bytes`.
int gcap_from_workspace(long long n_pairs, long long bytes) {
  int best = 0;
  for (int cap = 64; cap <= (1 << 25); cap <<= 1)
    if ((long long)layout_for(n_pairs, cap).total <= bytes) best = cap;
  return best;
}

template <int WT, typename T, int NW>
size_t narrow_smem() {
  return (size_t)NW * 2 * WT * 32 * sizeof(T);
}

int occupancy(int* out, const void* fn, int threads, size_t smem) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  }
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fn, threads, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (*out < 1) *out = 1;
  return DIBELLA_OK;
}

int device_info(DeviceInfo** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return DIBELLA_EINVAL;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DeviceInfo& D = g_dev[dev];
  if (!D.ready) {
    e = cudaDeviceGetAttribute(&D.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    int rc = DIBELLA_OK;
    if ((rc = occupancy(&D.narrow_blocks[0][0][2], (const void*)narrow_kernel<32, int, kWarpsPerBlock, 16>,
                        kBlockThreads, narrow_smem<32, int, kWarpsPerBlock>())) ||
        (rc = occupancy(&D.narrow_blocks[0][1][2], (const void*)narrow_kernel<48, int, kWarpsPerBlock, 16>,
                        kBlockThreads, narrow_smem<48, int, kWarpsPerBlock>())) ||
        (rc = occupancy(&D.narrow_blocks[0][2][2], (const void*)narrow_kernel<64, int, kWarpsPerBlock, 16>,
                        kBlockThreads, narrow_smem<64, int, kWarpsPerBlock>())) ||
        (rc = occupancy(&D.narrow_blocks[1][0][0], (const void*)narrow_kernel<32, short, kWarpsPerBlock, 4>,
                        kBlockThreads, narrow_smem<32, short, kWarpsPerBlock>())) ||
        (rc = occupancy(&D.narrow_blocks[1][1][0], (const void*)narrow_kernel<48, short, kWarpsPerBlock, 4>,
                        kBlockThreads, narrow_smem<48, short, kWarpsPerBlock>())) ||
        (rc = occupancy(&D.narrow_blocks[1][2][0], (const void*)narrow_kernel<64, short, kWarpsPerBlock, 4>,
                        kBlockThreads, narrow_smem<64, short, kWarpsPerBlock>())) ||
        (rc = occupancy(&D.narrow_blocks[1][0][1], (const void*)narrow_kernel<32, short, kWarpsPerBlock, 8>,
                        kBlockThreads, narrow_smem<32, short, kWarpsPerBlock>())) ||
        (rc = occupancy(&D.narrow_blocks[1][1][1], (const void*)narrow_kernel<48, short, kWarpsPerBlock, 8>,
                        kBlockThreads, narrow_smem<48, short, kWarpsPerBlock>())) ||
        (rc = occupancy(&D.narrow_blocks[1][2][1], (const void*)narrow_kernel<64, short, kWarpsPerBlock, 8>,
                        kBlockThreads, narrow_smem<64, short, kWarpsPerBlock>())) ||
        (rc = occupancy(&D.narrow_blocks[1][0][2], (const void*)narrow_kernel<32, short, kWarpsPerBlock, 16>,
                        kBlockThreads, narrow_smem<32, short, kWarpsPerBlock>())) ||
        (rc = occupancy(&D.narrow_blocks[1][1][2], (const void*)narrow_kernel<48, short, kWarpsPerBlock, 16>,
                        kBlockThreads, narrow_smem<48, short, kWarpsPerBlock>())) ||
        (rc = occupancy(&D.narrow_blocks[1][2][2], (const void*)narrow_kernel<64, short, kWarpsPerBlock, 16>,
                        kBlockThreads, narrow_smem<64, short, kWarpsPerBlock>())) ||
        (rc = occupancy(&D.narrow_blocks[1][0][3], (const void*)narrow_kernel<32, short, kWarpsPerBlock, 16, true>,
                        kBlockThreads, narrow_smem<32, short, kWarpsPerBlock>())) ||
        (rc = occupancy(&D.narrow_blocks[1][1][3], (const void*)narrow_kernel<48, short, kWarpsPerBlock, 16, true>,
                        kBlockThreads, narrow_smem<48, short, kWarpsPerBlock>())) ||
        (rc = occupancy(&D.narrow_blocks[1][2][3], (const void*)narrow_kernel<64, short, kWarpsPerBlock, 16, true>,
                        kBlockThreads, narrow_smem<64, short, kWarpsPerBlock>())) ||
        (rc = occupancy(&D.mid_blocks[0], (const void*)narrow_kernel<128, short, 1, 16>, 32,
                        narrow_smem<128, short, 1>())) ||
        (rc = occupancy(&D.mid_blocks[1], (const void*)narrow_kernel<192, short, 1, 16>, 32,
                        narrow_smem<192, short, 1>())) ||
        (rc = occupancy(&D.mid_blocks[2], (const void*)narrow_kernel<256, short, 1, 16>, 32,
                        narrow_smem<256, short, 1>())) ||
        (rc = occupancy(&D.reg_blocks[0], (const void*)wide_reg_kernel<16>, kBlockThreads, 0)) ||
        (rc = occupancy(&D.reg_blocks[1], (const void*)wide_reg_kernel<32>, kBlockThreads, 0)) ||
        (rc = occupancy(&D.pk_blocks[0], (const void*)wide_pk_kernel<16>, kBlockThreads, 0)) ||
        (rc = occupancy(&D.pk_blocks[1], (const void*)wide_pk_kernel<24>, kBlockThreads, 0)) ||
        (rc = occupancy(&D.pk_blocks[2], (const void*)wide_pk_kernel<32>, kBlockThreads, 0)) ||
        (rc = occupancy(&D.pk_blocks[3], (const void*)wide_pk_kernel<8>, kBlockThreads, 0)) ||
        (rc = occupancy(&D.grp16_blocks[0], (const void*)wide_grp_kernel<16, 16>, kBlockThreads, 0)) ||
        (rc = occupancy(&D.grp16_blocks[1], (const void*)wide_grp_kernel<16, 24>, kBlockThreads, 0)) ||
        (rc = occupancy(&D.grp16_blocks[2], (const void*)wide_grp_kernel<16, 32>, kBlockThreads, 0)) ||
        (rc = occupancy(&D.grp8_blocks[0], (const void*)wide_grp_kernel<8, 16>, kBlockThreads, 0)) ||
        (rc = occupancy(&D.grp8_blocks[1], (const void*)wide_grp_kernel<8, 24>, kBlockThreads, 0)) ||
        (rc = occupancy(&D.cta_blocks, (const void*)wide_cta_kernel, kCtaThreads, kCtaSmemBytes)))
      return rc;
    for (int w = 0; w < 3; ++w)  // the int32 rows come in 16-cell groups only
      D.narrow_blocks[0][w][0] = D.narrow_blocks[0][w][1] = D.narrow_blocks[0][w][3] = D.narrow_blocks[0][w][2];
    D.ready = true;
  }
  *out = &D;
  return DIBELLA_OK;
}

int validate_schedule(const dibella_schedule_t& s) {
  if (s.narrow_band_cap != 32 && s.narrow_band_cap != 48 && s.narrow_band_cap != 64) return DIBELLA_EINVAL;
  if (s.mid_band_cap != 0 && s.mid_band_cap != 128 && s.mid_band_cap != 192 && s.mid_band_cap != 256)
    return DIBELLA_EINVAL;
  if (s.narrow_split_d < 0) return DIBELLA_EINVAL;
  if (s.narrow_unroll != 0 && s.narrow_unroll != 4 && s.narrow_unroll != 8 && s.narrow_unroll != 16)
    return DIBELLA_EINVAL;
  if (s.narrow_track != 0 && s.narrow_track != 1) return DIBELLA_EINVAL;
  if (s.wide_slots != 0 && s.wide_slots != 8 && s.wide_slots != 16 && s.wide_slots != 24 && s.wide_slots != 32)
    return DIBELLA_EINVAL;
  if (s.wide_slots == 8 && s.wide_group_lanes != 0 && s.wide_group_lanes != 32) return DIBELLA_EINVAL;
  if (s.wide_packed != 0 && s.wide_packed != 1) return DIBELLA_EINVAL;
  if (s.wide_group_lanes != 0 && s.wide_group_lanes != 8 && s.wide_group_lanes != 16 && s.wide_group_lanes != 32)
    return DIBELLA_EINVAL;
  if (s.wide_group_lanes == 8 && s.wide_slots == 32) return DIBELLA_EINVAL;
  if (s.n_buckets < 1 || s.n_buckets > DIBELLA_MAX_BUCKETS) return DIBELLA_EINVAL;
  if (s.wide_blocks_per_sm < 0 || s.narrow_blocks_per_sm < 0) return DIBELLA_EINVAL;
  for (int b = 1; b < s.n_buckets - 1; ++b)
    if (s.bucket_bounds[b] < s.bucket_bounds[b - 1]) return DIBELLA_EINVAL;
  return DIBELLA_OK;
}

int validate_common(long long n_reads, long long n_pairs, int k, const dibella_scoring_t& sc) {
  if (n_reads < 0 || n_pairs < 0 || n_pairs > (1ll << 29)) return DIBELLA_EINVAL;
  if (k < 1 || k > DIBELLA_MAX_K) return DIBELLA_EINVAL;
  if (sc.match <= 0 || sc.match > DIBELLA_MAX_SCORE) return DIBELLA_EINVAL;
  if (sc.mismatch > 0 || sc.mismatch < -DIBELLA_MAX_SCORE) return DIBELLA_EINVAL;
  if (sc.gap >= 0 || sc.gap < -DIBELLA_MAX_SCORE) return DIBELLA_EINVAL;
  if (sc.xdrop < 0 || sc.xdrop > DIBELLA_XDROP_INF) return DIBELLA_EINVAL;
  return DIBELLA_OK;
}

int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 65535) g = 65535;
  return (int)g;
}

// Phase events: plain records on a live stream; under stream capture they
// become external event-record nodes, so a replayed graph still times phases.
void record(cudaStream_t st, int idx) {
  if (!g_timing || g_ev[idx] == nullptr) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return;
  if (cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(g_ev[idx], st, cudaEventRecordExternal);
  else
    cudaEventRecord(g_ev[idx], st);
  g_ev_count = idx + 1;
}

// int16 narrow cells (relative scores) when X allows, else int32.
inline int narrow_kind(int xdrop) { return xdrop <= kNarrow16MaxX ? 1 : 0; }

// Index of a schedule's narrow-form variant: cell groups of 4, 8 or 16
// (narrow_unroll 0 means 16), or 16 with the live range tracked (narrow_track;
// int16 rows only).
inline int narrow_variant(int unroll, int track, int xdrop) {
  if (track && xdrop <= 8000) return 3;
  return unroll == 4 ? 0 : (unroll == 8 ? 1 : 2);
}

template <int WT, int U>
void launch_narrow16(int grid, cudaStream_t st, const ExtendParams& ep) {
  narrow_kernel<WT, short, kWarpsPerBlock, U><<<grid, kBlockThreads, narrow_smem<WT, short, kWarpsPerBlock>(), st>>>(ep);
}

template <int WT>
void launch_narrow16_u(int unroll, bool track, int grid, cudaStream_t st, const ExtendParams& ep) {
  if (track)  // 16-cell groups with the live range and maximum tracked in registers
    narrow_kernel<WT, short, kWarpsPerBlock, 16, true>
        <<<grid, kBlockThreads, narrow_smem<WT, short, kWarpsPerBlock>(), st>>>(ep);
  else if (unroll == 4)
    launch_narrow16<WT, 4>(grid, st, ep);
  else if (unroll == 8)
    launch_narrow16<WT, 8>(grid, st, ep);
  else
    launch_narrow16<WT, 16>(grid, st, ep);
}

cudaError_t launch_narrow(int wt, int unroll, bool track, int xdrop, int grid, cudaStream_t st,
                          const ExtendParams& ep) {
  if (narrow_kind(xdrop)) {
    if (wt == 32)
      launch_narrow16_u<32>(unroll, track, grid, st, ep);
    else if (wt == 48)
      launch_narrow16_u<48>(unroll, track, grid, st, ep);
    else
      launch_narrow16_u<64>(unroll, track, grid, st, ep);
  } else {
    if (wt == 32)
      narrow_kernel<32, int, kWarpsPerBlock, 16><<<grid, kBlockThreads, narrow_smem<32, int, kWarpsPerBlock>(), st>>>(ep);
    else if (wt == 48)
      narrow_kernel<48, int, kWarpsPerBlock, 16><<<grid, kBlockThreads, narrow_smem<48, int, kWarpsPerBlock>(), st>>>(ep);
    else
      narrow_kernel<64, int, kWarpsPerBlock, 16><<<grid, kBlockThreads, narrow_smem<64, int, kWarpsPerBlock>(), st>>>(ep);
  }
  ++g_launches;
  return cudaGetLastError();
}

// The mid form (int16 cells only): one lane per extension, WT = 128/192/256.
cudaError_t launch_mid(const DeviceInfo& D, int wt, cudaStream_t st, const ExtendParams& ep) {
  const int vi = wt == 128 ? 0 : (wt == 192 ? 1 : 2);
  const int grid = D.sms * D.mid_blocks[vi];
  if (wt == 128)
    narrow_kernel<128, short, 1, 16><<<grid, 32, narrow_smem<128, short, 1>(), st>>>(ep);
  else if (wt == 192)
    narrow_kernel<192, short, 1, 16><<<grid, 32, narrow_smem<192, short, 1>(), st>>>(ep);
  else
    narrow_kernel<256, short, 1, 16><<<grid, 32, narrow_smem<256, short, 1>(), st>>>(ep);
  ++g_launches;
  return cudaGetLastError();
}

// The wide form of a schedule: packed int16 pairs when allowed, else int32.
cudaError_t launch_wide(const DeviceInfo& D, const dibella_schedule_t& sch_in, int xdrop, cudaStream_t st,
                        const ExtendParams& ep) {
  dibella_schedule_t sch = sch_in;
  const bool packed = sch.wide_packed && xdrop <= kPackedMaxX;
  int lanes = sch.wide_group_lanes;
  if (lanes == 0) lanes = 32;  // auto: one warp per extension (measured fastest at X = 7..50)
  if (!packed) lanes = 32;                                      // the int32 form is one warp per extension
  if (sch.wide_slots == 0) sch.wide_slots = (lanes == 32 && packed) ? (xdrop <= 30 ? 8 : 24) : (xdrop <= 30 ? 16 : 24);
  if (lanes == 8 && sch.wide_slots == 32) sch.wide_slots = 24;
  if (sch.wide_slots == 8 && (lanes != 32 || !packed)) sch.wide_slots = 16;
  const int vi = sch.wide_slots == 8 ? 3 : (sch.wide_slots == 16 ? 0 : (sch.wide_slots == 24 ? 1 : 2));
  int b;
  if (!packed)
    b = D.reg_blocks[sch.wide_slots == 16 ? 0 : 1];
  else if (lanes == 32)
    b = D.pk_blocks[vi];
  else if (lanes == 16)
    b = D.grp16_blocks[vi];
  else
    b = D.grp8_blocks[vi];
  if (sch.wide_blocks_per_sm > 0) b = std::min(b, sch.wide_blocks_per_sm);
  const int grid = D.sms * b;
  if (!packed) {
    if (sch.wide_slots == 16)
      wide_reg_kernel<16><<<grid, kBlockThreads, 0, st>>>(ep);
    else
      wide_reg_kernel<32><<<grid, kBlockThreads, 0, st>>>(ep);
  } else if (lanes == 32) {
    const bool clk = ep.wclock != nullptr;
    if (vi == 3)
      clk ? wide_pk_kernel<8, true><<<grid, kBlockThreads, 0, st>>>(ep)
          : wide_pk_kernel<8><<<grid, kBlockThreads, 0, st>>>(ep);
    else if (vi == 0)
      clk ? wide_pk_kernel<16, true><<<grid, kBlockThreads, 0, st>>>(ep)
          : wide_pk_kernel<16><<<grid, kBlockThreads, 0, st>>>(ep);
    else if (vi == 1)
      clk ? wide_pk_kernel<24, true><<<grid, kBlockThreads, 0, st>>>(ep)
          : wide_pk_kernel<24><<<grid, kBlockThreads, 0, st>>>(ep);
    else
      clk ? wide_pk_kernel<32, true><<<grid, kBlockThreads, 0, st>>>(ep)
          : wide_pk_kernel<32><<<grid, kBlockThreads, 0, st>>>(ep);
  } else if (lanes == 16) {
    if (vi == 0)
      wide_grp_kernel<16, 16><<<grid, kBlockThreads, 0, st>>>(ep);
    else if (vi == 1)
      wide_grp_kernel<16, 24><<<grid, kBlockThreads, 0, st>>>(ep);
    else
      wide_grp_kernel<16, 32><<<grid, kBlockThreads, 0, st>>>(ep);
  } else {
    if (vi == 0)
      wide_grp_kernel<8, 16><<<grid, kBlockThreads, 0, st>>>(ep);
    else
      wide_grp_kernel<8, 24><<<grid, kBlockThreads, 0, st>>>(ep);
  }
  ++g_launches;
  return cudaGetLastError();
}

// All extension launches of one batch, in stream order:
//   narrow form        on Narrow        (outgrown -> Esc1)
//   wide form (S slots) on Wide         (outgrown -> ladder queue of S)
//   mid form           on Esc1          (outgrown -> Esc2; int16 cells only,
//                                        skipped when the schedule has none)
//   wide form (S slots) on Esc2 (or Esc1 without a mid form)
//   wide form, next rung of the slot ladder 8 -> 16 -> 24 -> 32, on the queue
//                      of the rung below (outgrown -> its own queue; the top
//                      rung hands a short queue on unextended)
//   CTA form           on Smem          (outgrown -> Global)
//   global form        on Global
// With narrow_split_d > 0 the narrow form runs twice: the first pass stops
// every extension at antidiagonal narrow_split_d and queues the unfinished
// ones on Long, which the second pass runs from the origin (so that lanes with
// long extensions are not interleaved with the refills of short ones).
// Every launch whose queue is empty returns at once.  Phase events: 2 after
// the (first) narrow launch, 3 after the second narrow pass (at once when
// there is none), 4 after the first wide launch, 5 after the mid form (at
// once when there is none), 6 after the wide launch on the escalations, 7
// after the ladder, CTA and global launches.
int launch_extensions(const DeviceInfo& D, const dibella_schedule_t& sch_in, int xdrop, ExtendParams ep,
                      int* const q[kNumQ], cudaStream_t st) {
  dibella_schedule_t sch = sch_in;
  const bool packed = sch.wide_packed && xdrop <= kPackedMaxX;
  if (sch.wide_group_lanes == 0 || !packed) sch.wide_group_lanes = 32;
  if (sch.wide_slots == 0) sch.wide_slots = (sch.wide_group_lanes == 32 && packed) ? (xdrop <= 30 ? 8 : 24)
                                                                                 : (xdrop <= 30 ? 16 : 24);
  if (sch.wide_slots == 8 && (sch.wide_group_lanes != 32 || !packed)) sch.wide_slots = 16;
  if (sch.wide_group_lanes == 8 && sch.wide_slots == 32) sch.wide_slots = 24;
  // ladder rungs above the configured slot count (the int32 form has 16 and 32 only)
  int rungs[4], n_rungs = 0;
  const int ladder[4] = {8, 16, 24, 32};
  for (int r = 0; r < 4; ++r)
    if (ladder[r] > sch.wide_slots && (packed || ladder[r] == 32)) rungs[n_rungs++] = ladder[r];
  auto rung_queue = [&](int slots) { return kQLadder + (slots / 8 - 1); };  // 8..32 -> 3..6
  const int wt = sch.narrow_band_cap;
  const int vi = wt == 32 ? 0 : (wt == 48 ? 1 : 2);
  const int unroll = sch.narrow_unroll == 0 ? 16 : sch.narrow_unroll;
  const bool track = sch.narrow_track != 0;
  int nb = D.narrow_blocks[narrow_kind(xdrop)][vi][narrow_variant(unroll, sch.narrow_track, xdrop)];
  if (sch.narrow_blocks_per_sm > 0) nb = std::min(nb, sch.narrow_blocks_per_sm);
  cudaError_t e;

  ep.wide_q = nullptr;
  ep.narrow_q = q[kQNarrow];
  ep.narrow_q_id = kQNarrow;
  ep.esc_q = q[kQEsc1];
  ep.esc_q_id = kQEsc1;
  ep.narrow_cells_idx = 0;
  ep.narrow_esc_stat = 2;
  ep.wclock = clock_for(1, D.sms * nb * kWarpsPerBlock, st);
  ep.narrow_max_d = sch.narrow_split_d;
  ep.long_q = q[kQLong];
  if ((e = launch_narrow(wt, unroll, track, xdrop, D.sms * nb, st, ep)) != cudaSuccess)
    return cuda_fail(e, "narrow launch");
  ep.wclock = nullptr;
  ep.narrow_max_d = 0;
  record(st, 2);
  if (sch.narrow_split_d > 0) {  // second pass: the long extensions, from the origin
    ep.narrow_q = q[kQLong];
    ep.narrow_q_id = kQLong;
    ep.wclock = clock_for(5, D.sms * nb * kWarpsPerBlock, st);
    if ((e = launch_narrow(wt, unroll, track, xdrop, D.sms * nb, st, ep)) != cudaSuccess)
      return cuda_fail(e, "narrow launch 2");
    ep.wclock = nullptr;
  }
  record(st, 3);

  // The configured wide form; its escalations climb the ladder.
  ep.narrow_q = nullptr;
  int cur_q = n_rungs ? rung_queue(sch.wide_slots) : kQSmem;
  ep.esc_q = q[cur_q];
  ep.esc_q_id = cur_q;
  ep.wide_q = q[kQWide];
  ep.wide_q_id = kQWide;
  ep.cells_idx = 1;
  ep.wclock = clock_for(2, D.sms * 64, st);  // every warp an SM can hold; rows of absent warps stay 0
  if ((e = launch_wide(D, sch, xdrop, st, ep)) != cudaSuccess) return cuda_fail(e, "wide launch");
  ep.wclock = nullptr;
  record(st, 4);
  int esc_in = kQEsc1;
  if (sch.mid_band_cap > 0 && narrow_kind(xdrop) == 1) {
    const int wide_esc_q = ep.esc_q_id;
    ep.narrow_q = q[kQEsc1];
    ep.narrow_q_id = kQEsc1;
    ep.esc_q = q[kQEsc2];
    ep.esc_q_id = kQEsc2;
    ep.narrow_cells_idx = 6;
    ep.narrow_esc_stat = 6;
    const int mvi = sch.mid_band_cap == 128 ? 0 : (sch.mid_band_cap == 192 ? 1 : 2);
    ep.wclock = clock_for(3, D.sms * D.mid_blocks[mvi], st);
    if ((e = launch_mid(D, sch.mid_band_cap, st, ep)) != cudaSuccess) return cuda_fail(e, "mid launch");
    ep.wclock = nullptr;
    ep.narrow_q = nullptr;
    ep.esc_q = q[wide_esc_q];
    ep.esc_q_id = wide_esc_q;
    esc_in = kQEsc2;
  }
  record(st, 5);
  ep.wide_q = q[esc_in];
  ep.wide_q_id = esc_in;
  ep.cells_idx = 4;
  ep.wclock = clock_for(4, D.sms * 64, st);
  if ((e = launch_wide(D, sch, xdrop, st, ep)) != cudaSuccess) return cuda_fail(e, "wide launch (escalations)");
  ep.wclock = nullptr;
  record(st, 6);
  ep.cells_idx = 5;
  for (int r = 0; r < n_rungs; ++r) {
    dibella_schedule_t up = sch;
    up.wide_slots = rungs[r];
    up.wide_group_lanes = 32;
    const int next_q = r + 1 < n_rungs ? rung_queue(rungs[r]) : kQSmem;
    // Only the top rung hands a short queue straight to the CTA form (the
    // lower rungs' extensions mostly fit the next rung; measured).
    ep.forward_max = r + 1 == n_rungs ? (unsigned)(4 * D.sms * D.cta_blocks) : 0u;
    ep.wide_q = q[cur_q];
    ep.wide_q_id = cur_q;
    ep.esc_q = q[next_q];
    ep.esc_q_id = next_q;
    if ((e = launch_wide(D, up, xdrop, st, ep)) != cudaSuccess) return cuda_fail(e, "wide launch (ladder)");
    cur_q = next_q;
  }
  ep.forward_max = 0;

  ep.wide_q = q[kQSmem];
  ep.wide_q_id = kQSmem;
  ep.esc_q = q[kQGlobal];
  ep.esc_q_id = kQGlobal;
  wide_cta_kernel<<<D.sms * D.cta_blocks, kCtaThreads, kCtaSmemBytes, st>>>(ep);
  ++g_launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "wide_cta launch");

  ep.wide_q = q[kQGlobal];
  ep.wide_q_id = kQGlobal;
  global_kernel<<<kGlobalWarps / kWarpsPerBlock, kBlockThreads, 0, st>>>(ep);
  ++g_launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "global launch");
  record(st, 7);
  return DIBELLA_OK;
}

int expand_and_queue(const uint32_t* words, const int64_t* offs, const int32_t* lens, int64_t n_reads,
                     const dibella_pair_t* pairs, int64_t n_pairs, int32_t k, const dibella_scoring_t& s,
                     dibella_result_t* results, char* ws, const Layout& L, const dibella_schedule_t& sch,
                     cudaStream_t st) {
  Counters* cnt = (Counters*)(ws + L.counters);
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(Counters), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  if (n_pairs == 0) return DIBELLA_OK;
  ExpandParams xp;
  xp.words = words;
  xp.read_word_offsets = (const long long*)offs;
  xp.read_lengths = lens;
  xp.n_reads = n_reads;
  xp.pairs = pairs;
  xp.n_pairs = n_pairs;
  xp.k = k;
  xp.sc = {s.match, s.mismatch, s.gap, s.xdrop};
  xp.results = results;
  xp.items = (Item*)(ws + L.items);
  xp.cnt = cnt;
  xp.narrow_max_x = sch.narrow_max_xdrop;
  xp.narrow_max_len = sch.narrow_max_len;
  xp.n_buckets = sch.n_buckets;
  for (int b = 0; b < DIBELLA_MAX_BUCKETS; ++b) xp.bounds[b] = sch.bucket_bounds[b];
  expand_kernel<<<grid_for(n_pairs, 256), 256, 0, st>>>(xp);
  ++g_launches;
  scan_kernel<<<1, 32, 0, st>>>(cnt, sch.n_buckets);
  ++g_launches;
  scatter_kernel<<<grid_for(2 * n_pairs, 256), 256, 0, st>>>(
      xp.items, 2 * n_pairs, cnt, (int*)(ws + L.queue[kQNarrow]), (int*)(ws + L.queue[kQWide]));
  ++g_launches;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "expand launch");
  return DIBELLA_OK;
}

int finish(const int32_t* lens, const dibella_pair_t* pairs, int64_t n_pairs, int32_t k,
           dibella_result_t* results, const ExtOut* ext, cudaStream_t st) {
  if (n_pairs == 0) return DIBELLA_OK;
  CombineParams cp;
  cp.read_lengths = lens;
  cp.pairs = pairs;
  cp.n_pairs = n_pairs;
  cp.k = k;
  cp.ext = ext;
  cp.results = results;
  combine_kernel<<<grid_for(n_pairs, 256), 256, 0, st>>>(cp);
  ++g_launches;
  best_of_pair_kernel<<<grid_for(n_pairs, 256), 256, 0, st>>>(pairs, n_pairs, results);
  ++g_launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "combine launch");
  return DIBELLA_OK;
}

// ---------------------------------------------------------------------------
// Fixed scratch for dibella_xdrop_batch_noalloc.  Every GPU that loads this
// library holds kNoAllocBytes of it until the process exits.  Host code must
// not use the symbol's name as an address: it resolves the device address with
// cudaGetSymbolAddress, with the caller's device current, on every call (the
// lookup is cheap once the module is loaded, and it stays right if the
// context is destroyed and re-created and the module reloads elsewhere).
constexpr long long kNoAllocMaxPairs = DIBELLA_NOALLOC_MAX_PAIRS;
constexpr int kNoAllocBandCap = 8192;  // global-band cells per warp slot at the maximum batch
static_assert(kNoAllocBandCap - 3 == DIBELLA_NOALLOC_MAX_BAND, "the band limit stated in include/dibella.h");
constexpr size_t up256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kNoAllocBytes =
    up256(sizeof(Counters)) + up256(sizeof(Item) * 2 * kNoAllocMaxPairs) +
    up256(sizeof(ExtOut) * 2 * kNoAllocMaxPairs) + kNumQ * up256(sizeof(int) * 2 * kNoAllocMaxPairs) +
    up256(sizeof(int) * 3 * (size_t)kNoAllocBandCap * kGlobalWarps);
static_assert(kNoAllocBytes == 9568768, "the size stated in include/dibella.h must follow the layout");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array on the current device.
int noalloc_scratch(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
  *out = p;
  return DIBELLA_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

int dibella_get_default_schedule(dibella_schedule_t* out) {
  if (!out) return DIBELLA_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  *out = g_default_schedule;
  return DIBELLA_OK;
}

int dibella_set_default_schedule(const dibella_schedule_t* sched) {
  if (!sched || validate_schedule(*sched) != DIBELLA_OK) return DIBELLA_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  g_default_schedule = *sched;
  return DIBELLA_OK;
}

int dibella_xdrop_workspace_bytes(int64_t n_pairs, int32_t max_read_len, int64_t* bytes_out) {
  if (!bytes_out || n_pairs < 0 || n_pairs > (1ll << 29) || max_read_len < 0 ||
      max_read_len > DIBELLA_MAX_READ_LEN)
    return DIBELLA_EINVAL;
  *bytes_out = (int64_t)layout_for(n_pairs, gband_cap_for(max_read_len)).total;
  return DIBELLA_OK;
}

int dibella_xdrop_batch(const uint32_t* packed_words, const int64_t* read_word_offsets,
                        const int32_t* read_lengths, int64_t n_reads, const dibella_pair_t* pairs,
                        int64_t n_pairs, int32_t k, dibella_scoring_t scoring,
                        dibella_result_t* results, void* workspace, int64_t workspace_bytes,
                        void* stream, const dibella_schedule_t* sched) {
  int rc = validate_common(n_reads, n_pairs, k, scoring);
  if (rc != DIBELLA_OK) return rc;
  if (n_pairs > 0 && (!packed_words || !read_word_offsets || !read_lengths || !pairs || !results))
    return DIBELLA_EINVAL;
  if (!workspace || ((uintptr_t)workspace & 255)) return DIBELLA_EINVAL;
  dibella_schedule_t sch;
  if (sched) {
    if (validate_schedule(*sched) != DIBELLA_OK) return DIBELLA_EINVAL;
    sch = *sched;
  } else {
    dibella_get_default_schedule(&sch);
  }
  const int gcap = gcap_from_workspace(n_pairs, workspace_bytes);
  if (gcap < 64) return DIBELLA_ENOMEM;
  DeviceInfo* D = nullptr;
  rc = device_info(&D);
  if (rc != DIBELLA_OK) return rc;
  const Layout L = layout_for(n_pairs, gcap);
  char* ws = (char*)workspace;
  cudaStream_t st = (cudaStream_t)stream;

  // With the default schedule, a batch too small to give the resident narrow
  // lanes about one and a half extensions each would occupy few warps on few
  // SMs and be bound by one lane's walk through its longest extension: route it
  // to the warp-per-extension forms, whose antidiagonal latency is far lower.
  // Above X = 10 the narrow lanes also hand every extension whose band passes
  // the cap to the wide form, which can start only after the narrow launch
  // ends, so the narrow launch must not be held up by one lane's long walk:
  // keys above 20000 (above 5000 unless the batch gives each lane 7 or more
  // extensions) go straight to the wide form.  An explicit schedule is
  // followed as given.
  if (sched == nullptr) {
    const int wt = sch.narrow_band_cap;
    const long long narrow_lanes =
        (long long)D->sms *
        D->narrow_blocks[narrow_kind(scoring.xdrop)][wt == 32 ? 0 : (wt == 48 ? 1 : 2)]
                        [narrow_variant(sch.narrow_unroll == 0 ? 16 : sch.narrow_unroll, sch.narrow_track,
                                        scoring.xdrop)] *
        kBlockThreads;
    if (2 * 2 * n_pairs < 3 * narrow_lanes) sch.narrow_max_xdrop = -1;
    else if (scoring.xdrop > 10)
      sch.narrow_max_len = min(sch.narrow_max_len, 2 * n_pairs < 7 * narrow_lanes ? 5000 : 20000);
  }
  g_launches = 0;
  record(st, 0);
  set_store_extent(read_word_offsets, read_lengths, n_reads, st);
  rc = expand_and_queue(packed_words, read_word_offsets, read_lengths, n_reads, pairs, n_pairs, k,
                        scoring, results, ws, L, sch, st);
  if (rc != DIBELLA_OK) return rc;
  record(st, 1);
  if (n_pairs == 0) return DIBELLA_OK;

  ExtendParams ep;
  ep.words = packed_words;
  ep.items = (const Item*)(ws + L.items);
  ep.ext = (ExtOut*)(ws + L.ext);
  ep.cnt = (Counters*)(ws + L.counters);
  ep.sc = {scoring.match, scoring.mismatch, scoring.gap, scoring.xdrop};
  ep.gband = (int*)(ws + L.gband);
  ep.gcap = gcap;
  ep.forward_max = 0;
  ep.cells_idx = 1;
  ep.wclock = nullptr;
  ep.q_cap = 2 * n_pairs;
  ep.narrow_max_d = 0;
  ep.long_q = nullptr;
  int* q[kNumQ];
  for (int i = 0; i < kNumQ; ++i) q[i] = (int*)(ws + L.queue[i]);
  rc = launch_extensions(*D, sch, scoring.xdrop, ep, q, st);
  if (rc != DIBELLA_OK) return rc;
  rc = finish(read_lengths, pairs, n_pairs, k, results, ep.ext, st);
  record(st, 8);
  return rc;
}

int dibella_staging_bytes(int64_t n_pairs, int64_t* bytes_out) {
  if (!bytes_out || n_pairs < 0 || n_pairs > (1ll << 29)) return DIBELLA_EINVAL;
  *bytes_out = (int64_t)(align256(sizeof(dibella_pair_t) * (size_t)n_pairs) +
                         align256(sizeof(dibella_result_t) * (size_t)n_pairs));
  return DIBELLA_OK;
}

int dibella_xdrop_batch_noalloc(const uint32_t* packed_words, const int64_t* read_word_offsets,
                                const int32_t* read_lengths, int64_t n_reads, const dibella_pair_t* pairs,
                                int64_t n_pairs, int32_t k, dibella_scoring_t scoring,
                                dibella_result_t* results, void* stream) {
  if (n_pairs > kNoAllocMaxPairs) {
    g_last_error = "dibella_xdrop_batch_noalloc: " + std::to_string((long long)n_pairs) +
                   " seeds exceed the no-allocation maximum of " + std::to_string(kNoAllocMaxPairs);
    return DIBELLA_ENOMEM;
  }
  int rc = validate_common(n_reads, n_pairs, k, scoring);
  if (rc != DIBELLA_OK) return rc;
  void* scratch = nullptr;
  rc = noalloc_scratch(&scratch);
  if (rc != DIBELLA_OK) return rc;
  // The batch path clears the counters it needs zeroed on every call.
  return dibella_xdrop_batch(packed_words, read_word_offsets, read_lengths, n_reads, pairs, n_pairs, k, scoring,
                             results, scratch, (int64_t)kNoAllocBytes, stream, nullptr);
}

int dibella_xdrop_batch_host(const uint32_t* packed_words, const int64_t* read_word_offsets,
                             const int32_t* read_lengths, int64_t n_reads,
                             const dibella_pair_t* host_pairs, int64_t n_pairs, int32_t k,
                             dibella_scoring_t scoring, dibella_result_t* host_results, void* staging,
                             void* workspace, int64_t workspace_bytes, void* stream,
                             const dibella_schedule_t* sched) {
  int rc = validate_common(n_reads, n_pairs, k, scoring);
  if (rc != DIBELLA_OK) return rc;
  if (n_pairs > 0 && (!host_pairs || !host_results || !staging)) return DIBELLA_EINVAL;
  if (staging && ((uintptr_t)staging & 255)) return DIBELLA_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  dibella_pair_t* dpairs = (dibella_pair_t*)staging;
  dibella_result_t* dres = (dibella_result_t*)((char*)staging + align256(sizeof(dibella_pair_t) * (size_t)n_pairs));
  if (n_pairs > 0) {
    cudaError_t e = cudaMemcpyAsync(dpairs, host_pairs, sizeof(dibella_pair_t) * n_pairs,
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync H2D");
  }
  rc = dibella_xdrop_batch(packed_words, read_word_offsets, read_lengths, n_reads, dpairs, n_pairs, k,
                           scoring, dres, workspace, workspace_bytes, stream, sched);
  if (rc != DIBELLA_OK) return rc;
  if (n_pairs > 0) {
    cudaError_t e = cudaMemcpyAsync(host_results, dres, sizeof(dibella_result_t) * n_pairs,
                                    cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync D2H");
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  return DIBELLA_OK;
}

int dibella_xdrop_stream(const uint32_t* packed_words, const int64_t* read_word_offsets,
                         const int32_t* read_lengths, int64_t n_reads, const dibella_pair_t* host_pairs,
                         int64_t n_pairs, int64_t chunk_pairs, int32_t k, dibella_scoring_t scoring,
                         dibella_result_t* host_results, void* const* staging, void* const* workspace,
                         int64_t workspace_bytes, void* const* streams, const dibella_schedule_t* sched,
                         int64_t* n_chunks_out) {
  int rc = validate_common(n_reads, n_pairs, k, scoring);
  if (rc != DIBELLA_OK) return rc;
  if (chunk_pairs < 1 || chunk_pairs > (1ll << 29) || !staging || !workspace || !streams) return DIBELLA_EINVAL;
  if (n_pairs > 0 && (!host_pairs || !host_results)) return DIBELLA_EINVAL;
  for (int s = 0; s < 2; ++s)
    if (!staging[s] || ((uintptr_t)staging[s] & 255) || !workspace[s]) return DIBELLA_EINVAL;
  int64_t start = 0, chunks = 0;
  while (start < n_pairs) {
    int64_t end = std::min(n_pairs, start + chunk_pairs);
    if (end < n_pairs) {  // never split the seed records of one candidate pair
      int64_t e2 = end;
      while (e2 > start && host_pairs[e2].read_a == host_pairs[e2 - 1].read_a &&
             host_pairs[e2].read_b == host_pairs[e2 - 1].read_b)
        --e2;
      if (e2 == start) return DIBELLA_EINVAL;  // one candidate pair has more seeds than a chunk holds
      end = e2;
    }
    const int slot = (int)(chunks & 1);
    cudaStream_t st = (cudaStream_t)streams[slot];
    const int64_t n = end - start;
    dibella_pair_t* dpairs = (dibella_pair_t*)staging[slot];
    dibella_result_t* dres =
        (dibella_result_t*)((char*)staging[slot] + align256(sizeof(dibella_pair_t) * (size_t)chunk_pairs));
    cudaError_t e = cudaMemcpyAsync(dpairs, host_pairs + start, sizeof(dibella_pair_t) * n,
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync H2D");
    rc = dibella_xdrop_batch(packed_words, read_word_offsets, read_lengths, n_reads, dpairs, n, k, scoring, dres,
                             workspace[slot], workspace_bytes, streams[slot], sched);
    if (rc != DIBELLA_OK) return rc;
    e = cudaMemcpyAsync(host_results + start, dres, sizeof(dibella_result_t) * n, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync D2H");
    start = end;
    ++chunks;
  }
  for (int s = 0; s < 2; ++s) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)streams[s]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  }
  if (n_chunks_out) *n_chunks_out = chunks;
  return DIBELLA_OK;
}

int dibella_xdrop_per_pair(const uint32_t* packed_words, const int64_t* read_word_offsets,
                           const int32_t* read_lengths, int64_t n_reads, const dibella_pair_t* pairs,
                           int64_t n_pairs, int32_t k, dibella_scoring_t scoring,
                           dibella_result_t* results, void* workspace, int64_t workspace_bytes,
                           void* stream) {
  int rc = validate_common(n_reads, n_pairs, k, scoring);
  if (rc != DIBELLA_OK) return rc;
  if (n_pairs > 0 && (!packed_words || !read_word_offsets || !read_lengths || !pairs || !results))
    return DIBELLA_EINVAL;
  if (!workspace || ((uintptr_t)workspace & 255)) return DIBELLA_EINVAL;
  const int gcap = gcap_from_workspace(n_pairs, workspace_bytes);
  if (gcap < 64) return DIBELLA_ENOMEM;
  const Layout L = layout_for(n_pairs, gcap);
  char* ws = (char*)workspace;
  cudaStream_t st = (cudaStream_t)stream;
  dibella_schedule_t sch;
  dibella_get_default_schedule(&sch);
  set_store_extent(read_word_offsets, read_lengths, n_reads, st);
  rc = expand_and_queue(packed_words, read_word_offsets, read_lengths, n_reads, pairs, n_pairs, k,
                        scoring, results, ws, L, sch, st);
  if (rc != DIBELLA_OK) return rc;
  const Scoring sc = {scoring.match, scoring.mismatch, scoring.gap, scoring.xdrop};
  // The candidate pairs' boundaries (runs of equal read_a, read_b) come from
  // a host copy of the records, read once before the launches.
  std::vector<dibella_pair_t> hp((size_t)n_pairs);
  cudaError_t e = cudaMemcpyAsync(hp.data(), pairs, sizeof(dibella_pair_t) * (size_t)n_pairs,
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "per-pair record copy");
  for (long long t0 = 0; t0 < n_pairs;) {
    long long t1 = t0 + 1;
    while (t1 < n_pairs && hp[t1].read_a == hp[t0].read_a && hp[t1].read_b == hp[t0].read_b) ++t1;
    per_pair_kernel<<<1, 32, 0, st>>>(packed_words, (const Item*)(ws + L.items), (ExtOut*)(ws + L.ext), t0, t1,
                                      sc, (int*)(ws + L.gband), gcap);
    t0 = t1;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "per-pair launch");
  return finish(read_lengths, pairs, n_pairs, k, results, (const ExtOut*)(ws + L.ext), st);
}

int dibella_autotune(const uint32_t* packed_words, const int64_t* read_word_offsets,
                     const int32_t* read_lengths, int64_t n_reads, const dibella_pair_t* pairs,
                     int64_t n_pairs, int32_t k, dibella_scoring_t scoring, dibella_result_t* results,
                     void* workspace, int64_t workspace_bytes, void* stream, int32_t repeats,
                     dibella_schedule_t* best_out, float* best_ms_out, int32_t* n_tried_out) {
  int rc = validate_common(n_reads, n_pairs, k, scoring);
  if (rc != DIBELLA_OK) return rc;
  if (!best_out || repeats < 1 || n_pairs < 1) return DIBELLA_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return DIBELLA_EINVAL;  // timing needs a live stream
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
  int tried = 0;
  // Median of `repeats` timed runs (after one untimed run) of one schedule.
  auto time_one = [&](const dibella_schedule_t& cand, float* ms_out) -> int {
    float best = 0;
    std::vector<float> t;
    for (int r = 0; r <= repeats; ++r) {
      cudaEventRecord(e0, st);
      int rr = dibella_xdrop_batch(packed_words, read_word_offsets, read_lengths, n_reads, pairs, n_pairs, k,
                                   scoring, results, workspace, workspace_bytes, stream, &cand);
      if (rr != DIBELLA_OK) return rr;
      cudaEventRecord(e1, st);
      cudaError_t ee = cudaEventSynchronize(e1);
      if (ee != cudaSuccess) return cuda_fail(ee, "cudaEventSynchronize");
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    best = t[t.size() / 2];
    *ms_out = best;
    ++tried;
    return DIBELLA_OK;
  };
  dibella_schedule_t cur;
  dibella_get_default_schedule(&cur);
  float cur_ms = 0;
  rc = time_one(cur, &cur_ms);
  auto consider = [&](const dibella_schedule_t& cand) -> int {
    if (validate_schedule(cand) != DIBELLA_OK) return DIBELLA_OK;
    float ms = 0;
    int rr = time_one(cand, &ms);
    if (rr != DIBELLA_OK) return rr;
    if (ms < cur_ms) {
      cur = cand;
      cur_ms = ms;
    }
    return DIBELLA_OK;
  };
  // Stage 1: routing (thread- vs warp-per-extension) x per-thread band chunk.
  const int lens[5] = {-1, 2000, 8000, 32000, 1 << 30};
  const int caps[3] = {32, 48, 64};
  const dibella_schedule_t base1 = cur;
  for (int li = 0; li < 5 && rc == DIBELLA_OK; ++li)
    for (int ci = 0; ci < 3 && rc == DIBELLA_OK; ++ci) {
      dibella_schedule_t c = base1;
      c.narrow_max_xdrop = lens[li] < 0 ? -1 : DIBELLA_XDROP_INF;
      c.narrow_max_len = lens[li] < 0 ? 0 : lens[li];
      c.narrow_band_cap = caps[ci];
      if (li == 0 && ci > 0) continue;  // all-wide ignores the narrow chunk
      rc = consider(c);
    }
  // Stage 1b: the mid form's band (none, 128, 192 or 256 cells per lane).
  {
    const dibella_schedule_t base1b = cur;
    const int mids[4] = {0, 128, 192, 256};
    for (int mi = 0; mi < 4 && rc == DIBELLA_OK; ++mi) {
      if (mids[mi] == base1b.mid_band_cap) continue;
      dibella_schedule_t c = base1b;
      c.mid_band_cap = mids[mi];
      rc = consider(c);
    }
  }
  // Stage 1c: the split of the narrow launch (none, or a first pass of 64, 128 or 256 antidiagonals).
  {
    const dibella_schedule_t base1c = cur;
    const int splits[4] = {0, 64, 128, 256};
    for (int si = 0; si < 4 && rc == DIBELLA_OK; ++si) {
      if (splits[si] == base1c.narrow_split_d) continue;
      dibella_schedule_t c = base1c;
      c.narrow_split_d = splits[si];
      rc = consider(c);
    }
  }
  // Stage 1d: the narrow form's band walk: groups of 4, 8 or 16 cells with the
  // live range found by scans of the new row, or 16 with it tracked in registers.
  {
    const dibella_schedule_t base1d = cur;
    const int unrolls[4] = {4, 8, 16, 16}, tracks[4] = {0, 0, 0, 1};
    const int cur_u = base1d.narrow_unroll == 0 ? 16 : base1d.narrow_unroll;
    for (int vi = 0; vi < 4 && rc == DIBELLA_OK; ++vi) {
      if (tracks[vi] == base1d.narrow_track && (tracks[vi] != 0 || unrolls[vi] == cur_u)) continue;
      dibella_schedule_t c = base1d;
      c.narrow_unroll = unrolls[vi];
      c.narrow_track = tracks[vi];
      rc = consider(c);
    }
  }
  // Stage 2: lanes per extension (warp or 16/8-lane groups) x register slots of the wide form.
  {
    const dibella_schedule_t base2 = cur;
    const int lanes[3] = {32, 16, 8};
    for (int li = 0; li < 3 && rc == DIBELLA_OK; ++li)
      for (int ws = 8; ws <= 32 && rc == DIBELLA_OK; ws += 8) {
        dibella_schedule_t c = base2;
        c.wide_group_lanes = lanes[li];
        c.wide_slots = ws;
        rc = consider(c);
      }
  }
  // Stage 3: resident blocks per SM (occupancy maximum, or capped).
  for (int b = 1; b <= 3 && rc == DIBELLA_OK; ++b) {
    dibella_schedule_t c = cur;
    c.wide_blocks_per_sm = b;
    c.narrow_blocks_per_sm = b;
    rc = consider(c);
  }
  // Stage 4: length buckets that order the queues (longest first).
  const int sets[3][DIBELLA_MAX_BUCKETS + 1] = {
      {2, 5000, 0, 0, 0, 0, 0, 0, 0},
      {6, 500, 2000, 5000, 10000, 20000, 0, 0, 0},
      {8, 300, 1000, 2500, 5000, 10000, 20000, 40000, 0}};
  for (int si = 0; si < 3 && rc == DIBELLA_OK; ++si) {
    dibella_schedule_t c = cur;
    c.n_buckets = sets[si][0];
    for (int b = 0; b < DIBELLA_MAX_BUCKETS; ++b) c.bucket_bounds[b] = sets[si][1 + b];
    rc = consider(c);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != DIBELLA_OK) return rc;
  *best_out = cur;
  if (best_ms_out) *best_ms_out = cur_ms;
  if (n_tried_out) *n_tried_out = tried;
  return DIBELLA_OK;
}

int dibella_enable_phase_timing(int enable) {
  if (enable) {
    for (int i = 0; i < 10; ++i) {
      if (g_ev[i] != nullptr) continue;
      cudaError_t e = cudaEventCreate(&g_ev[i]);
      if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    }
  }
  g_timing = enable != 0;
  g_ev_count = 0;
  return DIBELLA_OK;
}

int dibella_phase_times(float* ms_out, int n_max) {
  if (!ms_out || n_max < 0) return DIBELLA_EINVAL;
  if (g_ev_count < 2) return 0;
  cudaError_t e = cudaEventSynchronize(g_ev[g_ev_count - 1]);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
  int n = 0;
  for (int i = 0; i + 1 < g_ev_count && n < n_max; ++i) {
    float ms = 0;
    e = cudaEventElapsedTime(&ms, g_ev[i], g_ev[i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    ms_out[n++] = ms;
  }
  return n;
}

int dibella_batch_counters(const void* workspace, void* stream, int64_t* out, int n_max) {
  if (!workspace || !out || n_max < 0) return DIBELLA_EINVAL;
  Counters c;
  cudaError_t e = cudaMemcpyAsync(&c, workspace, sizeof(c), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync counters");
  e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  const int64_t v[16] = {c.stat[0], c.stat[1], c.stat[2], c.stat[3], c.stat[4], c.stat[5],
                         (int64_t)c.cells[0], (int64_t)(c.cells[1] + c.cells[4] + c.cells[5]),
                         (int64_t)c.cells[2], (int64_t)c.cells[3], (int64_t)c.cells[4],
                         (int64_t)c.cells[5], (int64_t)c.cells[6], c.stat[6], (int64_t)c.cells[7], c.stat[7]};
  int n = std::min(n_max, 16);
  for (int i = 0; i < n; ++i) out[i] = v[i];
  return n;
}

int dibella_last_launch_count(void) { return g_launches; }

int dibella_bounds_check(int64_t* out, int reset) {
  if (!out) return DIBELLA_EINVAL;
  for (int i = 0; i < 4; ++i) out[i] = 0;
#ifdef DIBELLA_BOUNDS_CHECK
  unsigned long long v[4] = {0, 0, 0, 0};
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(v, g_bounds_fault, sizeof(v));
  if (e == cudaSuccess && reset) {
    const unsigned long long z[4] = {0, 0, 0, 0};
    e = cudaMemcpyToSymbol(g_bounds_fault, z, sizeof(z));
  }
  if (e != cudaSuccess) return cuda_fail(e, "bounds record");
  for (int i = 0; i < 4; ++i) out[i] = (int64_t)v[i];
  return 1;
#else
  (void)reset;
  return 0;
#endif
}

int dibella_enable_warp_clock(int launch) {
  if (launch < 0 || launch > 5) return DIBELLA_EINVAL;
  g_clock_launch = launch;
  g_clocked_warps = 0;
  return DIBELLA_OK;
}

int dibella_warp_clock(uint64_t* out, int max_warps) {
  if (!out || max_warps < 0) return DIBELLA_EINVAL;
  const int n = std::min(max_warps, g_clocked_warps);
  if (n == 0) return 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(out, g_warp_clock, sizeof(unsigned long long) * 2 * (size_t)n);
  if (e != cudaSuccess) return cuda_fail(e, "warp clock read");
  return n;
}

const char* dibella_last_error(void) { return g_last_error.c_str(); }

const char* dibella_version(void) {
#ifdef DIBELLA_BOUNDS_CHECK
  return "dibella-gb300 0.2.0 (sm_103a, bounds-checked debug build)";
#else
  return "dibella-gb300 0.2.0 (sm_103a)";
#endif
}

}  // extern "C"
