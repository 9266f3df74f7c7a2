// Candidate pairs on the GPU: the steps diBELLA runs before alignment.
//
//   Sec. 3      every k-mer occurrence of every read, in canonical orientation
//               (the smaller 2-bit code of the k-mer and of its reverse
//               complement), counted over all occurrences;
//   Sec. 3-4    a k-mer is retained when its multiplicity is in [mult_lo, mult_hi];
//   Sec. 8      (overlap detection, Algorithm 1) every pair of distinct reads that
//               share a retained k-mer, once per pair of occurrences, with both
//               positions and the strand (1 when the orientations differ);
//   Sec. 8, 5   seed constraints: per read pair, occurrences sorted by (pos_a,
//               pos_b, strand); seed 0 is the first, each next seed the first
//               whose pos_a is at least min_seed_gap (0 = k) past the last one,
//               up to max_seeds.
//
// GPU design (one pass over the read store per hash step, everything else
// linear in the retained occurrences):
//   count    a warp per read, a lane per position: the canonical code from the
//            2-bit store, inserted into an open-addressing table (16-byte slots
//            of key + 1, count and cursor, so that one probe touches one
//            sector; linear probing, bounded probes) that counts occurrences;
//   allocate each lane takes 16 slots: retained slots get a segment of the
//            occurrence array (one warp-aggregated atomic per 512 slots) and
//            join the retained list;
//   fill     the same walk as count: each retained occurrence takes the next
//            place of its k-mer's segment (an atomic on the slot's cursor) as
//            (read << 32 | pos << 1 | orientation);
//   emit     a thread per retained k-mer sorts its (at most mult_hi)
//            occurrences and appends one 64-bit key per occurrence pair:
//            read_a | read_b | pos_a | pos_b | strand, packed most significant
//            first with bit widths from the read count and the longest read;
//   sort     LSD radix sort of those keys (8-bit digits, stable: per-tile
//            digit histograms, one scan, warp-match ranking in the scatter);
//   select   a thread per run start (a new (read_a, read_b)) applies the
//            greedy seed rule along its run;
//   compact  a scan of the selection flags writes the 24-byte pair records,
//            sorted by (read_a, read_b, seed_id).
// Nothing here waits on another block; every probe loop is bounded.

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/dibella.h"

namespace {

constexpr unsigned kFullMask = 0xFFFFFFFFu;
constexpr unsigned long long kEmptyKey = 0ull;  // slots hold canonical code + 1 (see canonical)
constexpr int kMaxProbe = 1 << 14;
constexpr int kMaxMult = 32;
constexpr int kScanThreads = 1024;  // 32 warps: block_sum and the warp-total scan rely on it
constexpr int kScanBlocks = 256;    // at most kScanThreads
constexpr int kSortThreads = 256;
constexpr int kSortItems = 32;
constexpr int kAllocPerLane = 16;
constexpr int kTile = kSortThreads * kSortItems;  // keys per sort / scan tile

// Device counters of one call (also copied to the caller's counts array).
struct CandState {
  unsigned long long instances;   // k-mer occurrences
  unsigned long long retained;    // retained k-mers
  unsigned long long inst_cursor; // retained occurrences placed
  unsigned long long occ_pairs;   // occurrence pairs emitted
  unsigned long long n_keys;      // occurrence-pair keys held (occ_pairs, capped at the capacity)
  unsigned long long candidates;  // distinct (read_a, read_b)
  unsigned long long seeds;       // seed records written
  unsigned int status;            // bit 0 table full, bit 1 pair capacity, bit 2 output
                                  // capacity, bit 3 occurrence capacity, bit 4 sort inconsistency
  unsigned int pad;
  unsigned long long pass_count;  // partitioned count: occurrences appended in this pass
  unsigned long long pass_held;   // ... capped at the pass capacity
  unsigned long long max_pass;    // ... the largest pass
};

// Warp-aggregated atomicAdd: every lane of the warp calls it (v = 0 allowed);
// each lane gets the old value plus the sum of v over the lanes below it.
__device__ __forceinline__ unsigned long long warp_atomic_add(unsigned long long* addr, unsigned long long v) {
  const int lane = threadIdx.x & 31;
  unsigned long long incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += t;
  }
  const unsigned long long total = __shfl_sync(0xFFFFFFFFu, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && total) base = atomicAdd(addr, total);
  base = __shfl_sync(0xFFFFFFFFu, base, 31);
  return base + incl - v;
}

struct KeyLayout {  // bit positions of the packed occurrence-pair key
  int sh_ra, sh_rb, sh_pa, sh_pb;
  unsigned long long m_read, m_pos;
};

// Occurrence-pair keys that do not fit one word (the partitioned path): hi =
// read_a << rbits | read_b, lo = pos_a << (pbits + 1) | pos_b << 1 | strand;
// sorted by (hi, lo).
struct __align__(16) Key2 {
  unsigned long long lo, hi;
};

// Per key type: the sort tile (keys per block iteration of the radix passes)
// and the 8-bit digit at bit `shift` (shift in [0, 64) for one word, [0, 128)
// for two, never straddling a word: the passes run at multiples of 8 per word).
template <typename K>
struct KeyOps;
template <>
struct KeyOps<unsigned long long> {
  static constexpr int kTile = 8192;
  __device__ static unsigned digit(const unsigned long long& k, int shift) { return (unsigned)((k >> shift) & 255u); }
};
template <>
struct KeyOps<Key2> {
  static constexpr int kTile = 4096;
  __device__ static unsigned digit(const Key2& k, int shift) {
    return shift < 64 ? (unsigned)((k.lo >> shift) & 255u) : (unsigned)((k.hi >> (shift - 64)) & 255u);
  }
};

// Fields of an occurrence-pair key (one word: the bit layout of KeyLayout; two
// words: Key2 above with sh_pa / sh_pb in lo and sh_ra / sh_rb in hi).
__device__ __forceinline__ unsigned long long make_key(const KeyLayout& kl, unsigned long long ra,
                                                       unsigned long long rb, unsigned long long pa,
                                                       unsigned long long pb, unsigned long long strand,
                                                       unsigned long long*) {
  return (ra << kl.sh_ra) | (rb << kl.sh_rb) | (pa << kl.sh_pa) | (pb << kl.sh_pb) | strand;
}
__device__ __forceinline__ Key2 make_key(const KeyLayout& kl, unsigned long long ra, unsigned long long rb,
                                         unsigned long long pa, unsigned long long pb, unsigned long long strand,
                                         Key2*) {
  Key2 k;
  k.lo = (pa << kl.sh_pa) | (pb << kl.sh_pb) | strand;
  k.hi = (ra << kl.sh_ra) | (rb << kl.sh_rb);
  return k;
}
__device__ __forceinline__ unsigned long long run_of(const KeyLayout& kl, const unsigned long long& k) {
  return k >> kl.sh_rb;
}
__device__ __forceinline__ unsigned long long run_of(const KeyLayout&, const Key2& k) { return k.hi; }
__device__ __forceinline__ unsigned long long lo_word(const unsigned long long& k) { return k; }
__device__ __forceinline__ unsigned long long lo_word(const Key2& k) { return k.lo; }
__device__ __forceinline__ unsigned long long hi_word(const unsigned long long& k) { return k; }
__device__ __forceinline__ unsigned long long hi_word(const Key2& k) { return k.hi; }

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

// k bases of the forward copy starting at base index idx, base t at bits 2t.
__device__ __forceinline__ unsigned long long bases_le(const uint32_t* __restrict__ words, long long idx,
                                                       int k) {
  const long long w = idx >> 4;
  const int sh = (int)(idx & 15) * 2;
  const unsigned long long lo = (unsigned long long)__ldg(words + w) | ((unsigned long long)__ldg(words + w + 1) << 32);
  unsigned long long x = lo >> sh;
  if (sh > 0 && sh + 2 * k > 64) x |= (unsigned long long)__ldg(words + w + 2) << (64 - sh);
  return k == 32 ? x : (x & ((1ull << (2 * k)) - 1ull));
}

// Canonical code and orientation of the k-mer whose bases (first at bits 0-1)
// are x: the forward code has the first base most significant; the reverse
// complement code is the complement of x (its first base is the complement of
// the k-mer's last).  A code of all ones would need fw = rc = 2^64-1, i.e.
// x = 0 and fw = 0: so code + 1 never wraps to the empty key 0.
__device__ __forceinline__ unsigned long long canonical(unsigned long long x, int k, unsigned* orient) {
  unsigned long long y = __brevll(x);
  y = ((y >> 1) & 0x5555555555555555ull) | ((y & 0x5555555555555555ull) << 1);
  const unsigned long long fw = k == 32 ? y : (y >> (64 - 2 * k));
  const unsigned long long rc = k == 32 ? ~x : (x ^ ((1ull << (2 * k)) - 1ull));
  *orient = fw > rc ? 1u : 0u;
  return fw <= rc ? fw : rc;
}

// One table slot: canonical code + 1 (0 = empty), occurrence count, and the
// cursor into the k-mer's occurrence segment (set by allocate, advanced by fill).
struct __align__(16) Slot {
  unsigned long long key;
  unsigned int count;
  unsigned int cursor;
};

struct TableRef {
  Slot* slots;
  unsigned long long mask;  // slots - 1
};

__device__ long long table_insert(const TableRef& t, unsigned long long key, CandState* st) {
  unsigned long long s = mix64(key) & t.mask;
  for (int i = 0; i < kMaxProbe; ++i) {
    const unsigned long long cur = t.slots[s].key;
    if (cur == key) return (long long)s;
    if (cur == kEmptyKey) {
      const unsigned long long prev = atomicCAS(&t.slots[s].key, kEmptyKey, key);
      if (prev == kEmptyKey || prev == key) return (long long)s;
    }
    s = (s + 1) & t.mask;
  }
  atomicOr(&st->status, 1u);
  return -1;
}

__device__ long long table_find(const TableRef& t, unsigned long long key) {
  unsigned long long s = mix64(key) & t.mask;
  for (int i = 0; i < kMaxProbe; ++i) {
    const unsigned long long cur = t.slots[s].key;
    if (cur == key) return (long long)s;
    if (cur == kEmptyKey) return -1;
    s = (s + 1) & t.mask;
  }
  return -1;
}

struct StoreRef {
  const uint32_t* words;
  const int64_t* word_offsets;
  const int32_t* lengths;
  long long n_reads;
  int k;
};

// Pass 1 (count) and pass 3 (fill) share the walk over every k-mer occurrence.
template <bool kFill>
__global__ void kmer_walk_kernel(StoreRef sr, TableRef t, unsigned long long* inst, unsigned long long inst_cap,
                                 int mult_lo, int mult_hi, CandState* st) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = warp; r < sr.n_reads; r += n_warps) {
    const long long len = sr.lengths[r];
    const long long first = sr.word_offsets[r] * 16;
    for (long long p = lane; p + sr.k <= len; p += 32) {
      unsigned orient;
      const unsigned long long c = canonical(bases_le(sr.words, first + p, sr.k), sr.k, &orient) + 1ull;
      if (!kFill) {
        const long long s = table_insert(t, c, st);
        if (s >= 0) atomicAdd(&t.slots[s].count, 1u);
      } else {
        const long long s = table_find(t, c);
        if (s < 0) continue;
        const int cnt = (int)t.slots[s].count;
        if (cnt < mult_lo || cnt > mult_hi) continue;
        const unsigned long long at = atomicAdd(&t.slots[s].cursor, 1u);
        if (at >= inst_cap) {
          atomicOr(&st->status, 8u);
          continue;
        }
        inst[at] = ((unsigned long long)r << 32) | ((unsigned long long)p << 1) | orient;
      }
    }
  }
}

// Pass 2: retained slots get their occurrence segment.  Each lane takes
// kAllocPerLane consecutive slots; one warp-aggregated atomic per counter
// serves the warp's 32 x kAllocPerLane slots.
__global__ void allocate_kernel(TableRef t, unsigned long long n_slots, int mult_lo, int mult_hi,
                                unsigned int* retained_list, CandState* st) {
  const unsigned long long lane = threadIdx.x & 31;
  constexpr unsigned long long kWarpSpan = 32ull * kAllocPerLane;
  const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
  const unsigned long long n_warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long w0 = warp * kWarpSpan; w0 < n_slots; w0 += n_warps * kWarpSpan) {
    const unsigned long long s0 = w0 + lane * kAllocPerLane;
    unsigned long long occ_sum = 0, keep_occ = 0, keep_n = 0;
    for (int j = 0; j < kAllocPerLane; ++j) {
      const unsigned long long s = s0 + j;
      if (s >= n_slots || t.slots[s].key == kEmptyKey) continue;
      const int c = (int)t.slots[s].count;
      occ_sum += c;
      if (c >= mult_lo && c <= mult_hi) {
        keep_occ += c;
        keep_n += 1;
      }
    }
    warp_atomic_add(&st->instances, occ_sum);
    unsigned long long b = warp_atomic_add(&st->inst_cursor, keep_occ);
    unsigned long long r = warp_atomic_add(&st->retained, keep_n);
    for (int j = 0; j < kAllocPerLane && keep_n; ++j) {
      const unsigned long long s = s0 + j;
      if (s >= n_slots || t.slots[s].key == kEmptyKey) continue;
      const int c = (int)t.slots[s].count;
      if (c < mult_lo || c > mult_hi) continue;
      t.slots[s].cursor = (unsigned int)b;
      retained_list[r++] = (unsigned int)s;
      b += c;
    }
  }
}

// Pass 4: occurrence pairs of every retained k-mer, as packed keys.
__global__ void emit_pairs_kernel(TableRef t, const unsigned int* retained_list, const unsigned long long* inst,
                                  unsigned long long inst_cap, KeyLayout kl, unsigned long long* keys_out,
                                  unsigned long long capacity, CandState* st) {
  const unsigned long long n = st->retained;
  const unsigned long long lane = threadIdx.x & 31;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long w0 = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) - lane; w0 < n;
       w0 += stride) {
    const unsigned long long i = w0 + lane;
    unsigned long long v[kMaxMult];
    int c = 0, n_pairs = 0;
    if (i < n) {
      const unsigned s = retained_list[i];
      c = (int)t.slots[s].count;
      const unsigned long long b = (unsigned long long)t.slots[s].cursor - c;  // fill advanced it by c
      if (b + c > inst_cap) c = 0;  // its occurrences did not fit (status bit 3 is set)
      for (int x = 0; x < c; ++x) v[x] = inst[b + x];
      for (int x = 1; x < c; ++x) {  // insertion sort by (read, pos, orientation)
        const unsigned long long e = v[x];
        int y = x - 1;
        while (y >= 0 && v[y] > e) {
          v[y + 1] = v[y];
          --y;
        }
        v[y + 1] = e;
      }
      for (int x = 0; x < c; ++x)
        for (int y = x + 1; y < c; ++y) n_pairs += (v[x] >> 32) != (v[y] >> 32);
    }
    const unsigned long long at = warp_atomic_add(&st->occ_pairs, (unsigned long long)n_pairs);
    if (n_pairs == 0) continue;
    if (at + n_pairs > capacity) {
      atomicOr(&st->status, 2u);
      continue;
    }
    unsigned long long o = at;
    for (int x = 0; x < c; ++x)
      for (int y = x + 1; y < c; ++y) {
        const unsigned long long ra = v[x] >> 32, rb = v[y] >> 32;
        if (ra == rb) continue;
        const unsigned long long pa = (v[x] >> 1) & 0x7FFFFFFFull, pb = (v[y] >> 1) & 0x7FFFFFFFull;
        const unsigned long long strand = (v[x] ^ v[y]) & 1ull;
        keys_out[o++] = (ra << kl.sh_ra) | (rb << kl.sh_rb) | (pa << kl.sh_pa) | (pb << kl.sh_pb) | strand;
      }
  }
}

// The keys held: the pairs emitted, capped at the capacity (a capped run is
// flagged in status bit 1 and its results are incomplete).
__global__ void cap_keys_kernel(CandState* st, unsigned long long capacity) {
  st->n_keys = st->occ_pairs < capacity ? st->occ_pairs : capacity;
}

// ---- LSD radix sort of 64-bit keys (8-bit digits) ------------------------

template <typename K>
__global__ void digit_hist_kernel(const K* __restrict__ keys, const unsigned long long* n_ptr, int shift,
                                  unsigned int* hist, unsigned long long n_tiles_max) {
  constexpr int kT = KeyOps<K>::kTile;
  __shared__ unsigned int h[256];
  const unsigned long long n = *n_ptr;
  const unsigned long long n_tiles = (n + kT - 1) / kT;
  for (unsigned long long tile = blockIdx.x; tile < n_tiles && tile < n_tiles_max; tile += gridDim.x) {
    h[threadIdx.x] = 0;
    __syncthreads();
    const unsigned long long t0 = tile * kT;
    for (int j = 0; j < kT / kSortThreads; ++j) {
      const unsigned long long i = t0 + (unsigned long long)j * kSortThreads + threadIdx.x;
      if (i < n) atomicAdd(&h[KeyOps<K>::digit(keys[i], shift)], 1u);
    }
    __syncthreads();
    hist[(unsigned long long)threadIdx.x * n_tiles + tile] = h[threadIdx.x];
    __syncthreads();
  }
}

// Exclusive scan of len u32 counts into u64 offsets; len is fixed_len, or from
// *n_ptr: 256 digit counts per sort tile of `tile` keys (mode 1), one per
// kTile keys (mode 2).  Two
// launches of kScanBlocks blocks: each block sums its contiguous segment
// (scan_reduce_kernel), then scans it from the sum of the segments before it
// (scan_apply_kernel).  Both read the counts coalesced.
__device__ __forceinline__ unsigned long long scan_len(const unsigned long long* n_ptr, int mode,
                                                       unsigned long long fixed_len) {
  // mode 1: fixed_len holds the sort tile
  if (mode == 1) return 256ull * ((*n_ptr + fixed_len - 1) / fixed_len);
  if (mode == 2) return (*n_ptr + kTile - 1) / kTile;
  return fixed_len;
}

// Sum over the block (kScanThreads threads); every thread gets the result.
__device__ __forceinline__ unsigned long long block_sum(unsigned long long v, unsigned long long* wsum) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  v = wsum[threadIdx.x & 31];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
  __syncthreads();
  return v;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const unsigned int* counts,
                                                                   const unsigned long long* n_ptr, int mode,
                                                                   unsigned long long fixed_len,
                                                                   unsigned long long* part) {
  __shared__ unsigned long long wsum[32];
  const unsigned long long len = scan_len(n_ptr, mode, fixed_len);
  const unsigned long long seg = (len + gridDim.x - 1) / gridDim.x;
  const unsigned long long lo = blockIdx.x * seg;
  const unsigned long long hi = lo + seg < len ? lo + seg : len;
  unsigned long long s = 0;
  for (unsigned long long i = lo + threadIdx.x; i < hi; i += kScanThreads) s += counts[i];
  s = block_sum(s, wsum);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const unsigned int* counts,
                                                                  unsigned long long* offsets,
                                                                  const unsigned long long* n_ptr, int mode,
                                                                  unsigned long long fixed_len,
                                                                  const unsigned long long* part) {
  __shared__ unsigned long long wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long len = scan_len(n_ptr, mode, fixed_len);
  const unsigned long long seg = (len + gridDim.x - 1) / gridDim.x;
  const unsigned long long lo = blockIdx.x * seg;
  const unsigned long long hi = lo + seg < len ? lo + seg : len;
  // gridDim.x <= kScanThreads: thread t holds the sum of segment t.
  unsigned long long base = block_sum(threadIdx.x < blockIdx.x ? part[threadIdx.x] : 0ull, wsum);
  for (unsigned long long c = lo; c < hi; c += kScanThreads) {  // uniform over the block
    const unsigned long long i = c + threadIdx.x;
    const unsigned long long v = i < hi ? counts[i] : 0ull;
    unsigned long long x = v;  // inclusive scan within the warp
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(kFullMask, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {  // inclusive scan of the 32 warp totals
      unsigned long long w = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFullMask, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    if (i < hi) offsets[i] = base + (warp > 0 ? wsum[warp - 1] : 0ull) + x - v;
    base += wsum[31];
    __syncthreads();
  }
}

void scan_counts(const unsigned int* counts, unsigned long long* offsets, const unsigned long long* n_ptr, int mode,
                 unsigned long long fixed_len, unsigned long long* part, cudaStream_t st) {
  scan_reduce_kernel<<<kScanBlocks, kScanThreads, 0, st>>>(counts, n_ptr, mode, fixed_len, part);
  scan_apply_kernel<<<kScanBlocks, kScanThreads, 0, st>>>(counts, offsets, n_ptr, mode, fixed_len, part);
}

// One stable pass of the LSD sort, a tile of kTile keys per block iteration:
// the tile is copied into shared memory (16-byte asynchronous copies), each
// warp ranks its contiguous kWarpKeys keys by digit (counts, then a prefix over
// warps and digits, then ranks in input order), the permutation that sorts the
// tile by digit is built in shared memory, and the tile is written out in that
// order so that each digit's keys go to consecutive addresses.  A destination
// outside [0, n) (counts that disagree with the histogram) is skipped and
// flagged in status bit 4.
constexpr int kScatterThreads = 256;
constexpr int kScatterBlocksPerSM = 2;
constexpr int kScatterWarps = kScatterThreads / 32;
template <typename K>
constexpr size_t scatter_smem() {
  return (size_t)KeyOps<K>::kTile * sizeof(K) + (size_t)KeyOps<K>::kTile * 2 + (size_t)kScatterWarps * 256 * 4 +
         256 * 8 + 256 * 4;
}
static_assert(KeyOps<unsigned long long>::kTile <= 65536 && KeyOps<Key2>::kTile <= 65536, "tile indices are 16-bit");
static_assert(kScatterBlocksPerSM * (scatter_smem<unsigned long long>() + 1024) <= 228 * 1024 &&
                  kScatterBlocksPerSM * (scatter_smem<Key2>() + 1024) <= 228 * 1024,
              "scatter tiles do not fit shared memory");

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src, unsigned src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gmem_src), "r"(src_bytes)
               : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename K>
__global__ void __launch_bounds__(kScatterThreads, kScatterBlocksPerSM)
    digit_scatter_kernel(const K* __restrict__ in, K* __restrict__ out, const unsigned long long* n_ptr, int shift,
                         const unsigned long long* offsets, unsigned int* status) {
  constexpr int kT = KeyOps<K>::kTile;
  constexpr int kWarpKeys = kT / kScatterWarps;
  constexpr int kPerChunk = 16 / (int)sizeof(K);  // keys per 16-byte copy
  extern __shared__ __align__(16) unsigned char smem[];
  K* skey = (K*)smem;                                                              // the tile, input order
  unsigned short* inv = (unsigned short*)(smem + (size_t)kT * sizeof(K));          // sorted slot -> input index
  unsigned int* wcnt = (unsigned int*)(smem + (size_t)kT * (sizeof(K) + 2));       // [warp][digit]
  unsigned long long* gbase = (unsigned long long*)(wcnt + kScatterWarps * 256);  // digit's first output slot
  unsigned int* lstart = (unsigned int*)(gbase + 256);                           // digit's first slot in the tile
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const unsigned long long n = *n_ptr;
  const unsigned long long n_tiles = (n + kT - 1) / kT;
  const int w0 = warp * kWarpKeys;
  for (unsigned long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const unsigned long long t0 = tile * kT;
    const int m = n - t0 < (unsigned long long)kT ? (int)(n - t0) : kT;
    for (int c = threadIdx.x; c < kT / kPerChunk; c += kScatterThreads) {
      const int e = kPerChunk * c;  // a 16-byte chunk: keys e .. e + kPerChunk - 1, zero-filled past the tile's end
      const int valid = m - e < kPerChunk ? (m - e > 0 ? m - e : 0) : kPerChunk;
      const unsigned bytes = (unsigned)valid * (unsigned)sizeof(K);
      cp_async16(skey + e, bytes ? (const void*)(in + t0 + e) : (const void*)in, bytes);
    }
    for (int x = threadIdx.x; x < kScatterWarps * 256; x += kScatterThreads) wcnt[x] = 0;
    cp_async_wait_all();
    __syncthreads();
    for (int r = 0; r < kWarpKeys; r += 32) {
      const int i = w0 + r + lane;
      if (i < m) atomicAdd(&wcnt[warp * 256 + KeyOps<K>::digit(skey[i], shift)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 256) {  // thread d: prefix of digit d over the warps, and its tile count
      unsigned tot = 0;
      for (int w = 0; w < kScatterWarps; ++w) {
        const unsigned v = wcnt[w * 256 + threadIdx.x];
        wcnt[w * 256 + threadIdx.x] = tot;
        tot += v;
      }
      lstart[threadIdx.x] = tot;
      gbase[threadIdx.x] = offsets[(unsigned long long)threadIdx.x * n_tiles + tile];
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the 256 tile counts, 8 digits per lane
      unsigned v[8], sum = 0;
      for (int q = 0; q < 8; ++q) {
        v[q] = lstart[lane * 8 + q];
        sum += v[q];
      }
      unsigned x = sum;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(kFullMask, x, o);
        if (lane >= o) x += y;
      }
      unsigned acc = x - sum;
      for (int q = 0; q < 8; ++q) {
        lstart[lane * 8 + q] = acc;
        acc += v[q];
      }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < kScatterWarps * 256; x += kScatterThreads) wcnt[x] += lstart[x & 255];
    __syncthreads();
    unsigned int* next = wcnt + warp * 256;  // this warp's next slot per digit
    for (int r = 0; r < kWarpKeys; r += 32) {
      const int i = w0 + r + lane;
      const bool ok = i < m;
      const unsigned d = ok ? KeyOps<K>::digit(skey[i], shift) : 256u;
      const unsigned peers = __match_any_sync(kFullMask, d);
      const unsigned rank = __popc(peers & lt);
      const unsigned c = ok ? next[d] : 0u;
      __syncwarp();
      if (ok && rank == 0) next[d] = c + __popc(peers);
      __syncwarp();
      if (ok && c + rank < (unsigned)kT) inv[c + rank] = (unsigned short)i;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < m; q += kScatterThreads) {
      const K key = skey[inv[q] & (kT - 1)];
      const unsigned d = KeyOps<K>::digit(key, shift);
      const unsigned long long g = gbase[d] + (unsigned long long)(q - (int)lstart[d]);
      if (g < n)
        out[g] = key;
      else
        atomicOr(status, 16u);
    }
    __syncthreads();  // the next tile reuses shared memory
  }
}

cudaError_t set_scatter_smem() {
  cudaError_t e = cudaFuncSetAttribute(digit_scatter_kernel<unsigned long long>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)scatter_smem<unsigned long long>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(digit_scatter_kernel<Key2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)scatter_smem<Key2>());
  return e;
}

// One stable LSD pass by the digit at `shift`: histogram, scan, scatter.
template <typename K>
void radix_pass(const K* src, K* dst, const unsigned long long* n_ptr, int shift, unsigned int* hist,
                unsigned long long* hoff, unsigned long long tiles_max, unsigned long long* part,
                unsigned int* status, int sms, cudaStream_t st) {
  digit_hist_kernel<K><<<sms * 8, 256, 0, st>>>(src, n_ptr, shift, hist, tiles_max);
  scan_counts(hist, hoff, n_ptr, 1, (unsigned long long)KeyOps<K>::kTile, part, st);
  digit_scatter_kernel<K><<<sms * kScatterBlocksPerSM, kScatterThreads, scatter_smem<K>(), st>>>(
      src, dst, n_ptr, shift, hoff, status);
}

// ---- sort-based count (when code and occurrence index share 64 bits) ----------

__global__ void occ_count_kernel(StoreRef sr, unsigned int* cnt) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < sr.n_reads;
       r += (long long)gridDim.x * blockDim.x) {
    const int len = sr.lengths[r];
    cnt[r] = len >= sr.k ? (unsigned)(len - sr.k + 1) : 0u;
  }
}

// The occurrence total; above the capacity (n_bases understated) it is capped
// for the sort and status bit 3 marks the results incomplete.
__global__ void occ_total_kernel(const unsigned int* cnt, const unsigned long long* off, long long n_reads,
                                 unsigned long long cap, CandState* st) {
  unsigned long long total = n_reads > 0 ? off[n_reads - 1] + cnt[n_reads - 1] : 0ull;
  if (total > cap) {
    total = cap;
    st->status |= 8u;
  }
  st->instances = total;
}

// Every occurrence as (canonical code << ib | occurrence index), and its read,
// position and orientation under that index.
__global__ void extract_kernel(StoreRef sr, const unsigned long long* off, int ib, unsigned long long cap,
                               unsigned long long* keys, unsigned long long* info) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = warp; r < sr.n_reads; r += n_warps) {
    const long long len = sr.lengths[r];
    const long long first = sr.word_offsets[r] * 16;
    const unsigned long long o = off[r];
    for (long long p = lane; p + sr.k <= len; p += 32) {
      unsigned orient;
      const unsigned long long c = canonical(bases_le(sr.words, first + p, sr.k), sr.k, &orient);
      const unsigned long long idx = o + (unsigned long long)p;
      if (idx >= cap) break;  // n_bases understated (status bit 3)
      keys[idx] = (c << ib) | idx;
      info[idx] = ((unsigned long long)r << 32) | ((unsigned long long)p << 1) | orient;
    }
  }
}

// A thread per run of equal codes in the sorted occurrences (n_ptr of them):
// the multiplicity, and for a retained k-mer its occurrence pairs (as in
// emit_pairs_kernel), as one-word or two-word keys.
template <typename K>
__global__ void run_emit_kernel(const unsigned long long* __restrict__ sorted, const unsigned long long* info, int ib,
                                int mult_lo, int mult_hi, KeyLayout kl, K* keys_out,
                                unsigned long long capacity, const unsigned long long* n_ptr, CandState* st) {
  const unsigned long long n = *n_ptr;
  const unsigned long long imask = (1ull << ib) - 1ull;
  const unsigned long long lane = threadIdx.x & 31;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long w0 = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) - lane; w0 < n;
       w0 += stride) {
    const unsigned long long i = w0 + lane;
    bool keep = false;
    int c = 0;
    if (i < n && (i == 0 || (sorted[i - 1] >> ib) != (sorted[i] >> ib))) {
      const unsigned long long code = sorted[i] >> ib;
      unsigned long long e = i + 1;
      while (e < n && (sorted[e] >> ib) == code && e - i <= (unsigned long long)mult_hi) ++e;
      const unsigned long long mult = e - i;  // capped at mult_hi + 1: enough to reject
      keep = mult >= (unsigned long long)mult_lo && mult <= (unsigned long long)mult_hi;
      c = keep ? (int)mult : 0;
    }
    warp_atomic_add(&st->retained, keep ? 1u : 0u);
    unsigned long long v[kMaxMult];
    int n_pairs = 0;
    if (keep) {
      for (int x = 0; x < c; ++x) v[x] = info[sorted[i + x] & imask];
      for (int x = 1; x < c; ++x) {
        const unsigned long long t = v[x];
        int y = x - 1;
        while (y >= 0 && v[y] > t) {
          v[y + 1] = v[y];
          --y;
        }
        v[y + 1] = t;
      }
      for (int x = 0; x < c; ++x)
        for (int y = x + 1; y < c; ++y) n_pairs += (v[x] >> 32) != (v[y] >> 32);
    }
    const unsigned long long at = warp_atomic_add(&st->occ_pairs, (unsigned long long)n_pairs);
    if (n_pairs == 0) continue;
    if (at + n_pairs > capacity) {
      atomicOr(&st->status, 2u);
      continue;
    }
    unsigned long long o = at;
    for (int x = 0; x < c; ++x)
      for (int y = x + 1; y < c; ++y) {
        const unsigned long long ra = v[x] >> 32, rb = v[y] >> 32;
        if (ra == rb) continue;
        const unsigned long long pa = (v[x] >> 1) & 0x7FFFFFFFull, pb = (v[y] >> 1) & 0x7FFFFFFFull;
        const unsigned long long strand = (v[x] ^ v[y]) & 1ull;
        keys_out[o++] = make_key(kl, ra, rb, pa, pb, strand, (K*)nullptr);
      }
  }
}

// The partitioned count: one pass per hash part of the canonical codes.  Every
// occurrence whose code falls in part `part` of n_parts is appended (one
// warp-aggregated atomic per 32 positions) as (code << ib | slot) with its
// read, position and orientation under that slot; the order within a pass is
// free, since each run is ordered by (read, position) before its pairs are
// formed and the pairs are sorted afterwards.
__device__ __forceinline__ unsigned part_of(unsigned long long code, unsigned n_parts) {
  return (unsigned)__umul64hi(mix64(code + 0x9E3779B97F4A7C15ull), (unsigned long long)n_parts);
}

__global__ void extract_part_kernel(StoreRef sr, unsigned part, unsigned n_parts, int ib, unsigned long long cap,
                                    unsigned long long* keys, unsigned long long* info, CandState* st) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = warp; r < sr.n_reads; r += n_warps) {
    const long long len = sr.lengths[r];
    const long long first = sr.word_offsets[r] * 16;
    for (long long p0 = 0; p0 + sr.k <= len; p0 += 32) {  // uniform over the warp
      const long long p = p0 + lane;
      unsigned orient = 0;
      unsigned long long c = 0;
      bool mine = false;
      if (p + sr.k <= len) {
        c = canonical(bases_le(sr.words, first + p, sr.k), sr.k, &orient);
        mine = part_of(c, n_parts) == part;
      }
      const unsigned bal = __ballot_sync(kFullMask, mine);
      if (!bal) continue;
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(&st->pass_count, (unsigned long long)__popc(bal));
      base = __shfl_sync(kFullMask, base, 0);
      if (!mine) continue;
      const unsigned long long idx = base + __popc(bal & lt);
      if (idx >= cap) {
        atomicOr(&st->status, 8u);
        continue;
      }
      keys[idx] = (c << ib) | idx;
      info[idx] = ((unsigned long long)r << 32) | ((unsigned long long)p << 1) | orient;
    }
  }
}

// Per pass: the occurrences it holds (capped at the capacity, flagged in
// status bit 3), their running total, and the largest pass so far.
__global__ void pass_begin_kernel(CandState* st) { st->pass_count = 0; }
__global__ void pass_end_kernel(CandState* st, unsigned long long cap) {
  const unsigned long long c = st->pass_count;
  st->instances += c;
  if (c > st->max_pass) st->max_pass = c;
  st->pass_held = c < cap ? c : cap;
}

// ---- seed selection and compaction -----------------------------------------

// A thread per run start walks its run: selection flags and seed ids.
template <typename K>
__global__ void select_kernel(const K* __restrict__ keys, CandState* st, KeyLayout kl,
                              int max_seeds, int gap, unsigned int* flags, unsigned int* sid) {
  const unsigned long long n = st->n_keys;
  const unsigned long long lane = threadIdx.x & 31;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long w0 = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) - lane; w0 < n;
       w0 += stride) {
    const unsigned long long i = w0 + lane;
    const bool start = i < n && (i == 0 || run_of(kl, keys[i - 1]) != run_of(kl, keys[i]));
    warp_atomic_add(&st->candidates, start ? 1u : 0u);
    if (!start) continue;
    const unsigned long long run = run_of(kl, keys[i]);
    int taken = 0;
    long long last = 0;
    for (unsigned long long u = i; u < n && run_of(kl, keys[u]) == run; ++u) {
      const long long pa = (long long)((lo_word(keys[u]) >> kl.sh_pa) & kl.m_pos);
      const bool take = taken < max_seeds && (taken == 0 || pa >= last + gap);
      flags[u] = take ? 1u : 0u;
      sid[u] = take ? (unsigned)taken : 0u;
      if (take) {
        last = pa;
        ++taken;
      }
    }
  }
}

// Per-tile sums of the flags.
__global__ void tile_sum_kernel(const unsigned int* flags, const CandState* st, unsigned int* sums) {
  __shared__ unsigned int s[kSortThreads];
  const unsigned long long n = st->n_keys;
  const unsigned long long n_tiles = (n + kTile - 1) / kTile;
  for (unsigned long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    unsigned int v = 0;
    for (int j = 0; j < kSortItems; ++j) {
      const unsigned long long i = tile * kTile + (unsigned long long)threadIdx.x * kSortItems + j;
      if (i < n) v += flags[i];
    }
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = kSortThreads / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) sums[tile] = s[0];
    __syncthreads();
  }
}

template <typename K>
__global__ void compact_kernel(const K* __restrict__ keys, const unsigned int* flags,
                               const unsigned int* sid, const unsigned long long* tile_off, CandState* st,
                               KeyLayout kl, dibella_pair_t* out, unsigned long long capacity) {
  __shared__ unsigned int s[kSortThreads];
  const unsigned long long n = st->n_keys;
  const unsigned long long n_tiles = (n + kTile - 1) / kTile;
  for (unsigned long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const unsigned long long i0 = tile * kTile + (unsigned long long)threadIdx.x * kSortItems;
    unsigned int v = 0;
    for (int j = 0; j < kSortItems; ++j)
      if (i0 + j < n) v += flags[i0 + j];
    s[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x == 0) {  // exclusive scan of the 256 thread sums
      unsigned int acc = 0;
      for (int t = 0; t < kSortThreads; ++t) {
        const unsigned int x = s[t];
        s[t] = acc;
        acc += x;
      }
    }
    __syncthreads();
    unsigned long long o = tile_off[tile] + s[threadIdx.x];
    for (int j = 0; j < kSortItems; ++j) {
      const unsigned long long i = i0 + j;
      if (i >= n || !flags[i]) continue;
      if (o >= capacity) {
        atomicOr(&st->status, 4u);
        ++o;
        continue;
      }
      const K key = keys[i];
      const unsigned long long hw = hi_word(key), lw = lo_word(key);
      dibella_pair_t r;
      r.read_a = (uint32_t)((hw >> kl.sh_ra) & kl.m_read);
      r.read_b = (uint32_t)((hw >> kl.sh_rb) & kl.m_read);
      r.pos_a = (uint32_t)((lw >> kl.sh_pa) & kl.m_pos);
      r.pos_b = (uint32_t)((lw >> kl.sh_pb) & kl.m_pos);
      r.strand = (uint8_t)(lw & 1ull);
      r.pad[0] = r.pad[1] = r.pad[2] = 0;
      r.seed_id = sid[i];
      out[o++] = r;
    }
    __syncthreads();
  }
}

__global__ void finish_kernel(CandState* st, const unsigned long long* tile_off, const unsigned int* tile_sums,
                              int64_t* counts_out) {
  const unsigned long long n = st->n_keys;
  const unsigned long long n_tiles = (n + kTile - 1) / kTile;
  st->seeds = n_tiles ? tile_off[n_tiles - 1] + tile_sums[n_tiles - 1] : 0;
  counts_out[0] = (int64_t)st->seeds;
  counts_out[1] = (int64_t)st->candidates;
  counts_out[2] = (int64_t)st->instances;
  counts_out[3] = (int64_t)st->retained;
  counts_out[4] = (int64_t)st->occ_pairs;
  counts_out[5] = (int64_t)st->status;
}

// Partitioned path: counts_out[6] = the occurrences of the largest pass.
__global__ void max_pass_kernel(const CandState* st, int64_t* counts_out) {
  counts_out[6] = (int64_t)st->max_pass;
}

int bits_for(unsigned long long v) {  // bits needed for values 0..v
  int b = 1;
  while (b < 63 && (v >> b) != 0) ++b;
  return b;
}

// The sort-based count keys each occurrence by (canonical code << ib |
// occurrence index), ib = bits(n_bases): it applies while both fit 64 bits
// (k = 17 up to 2^30 bases); otherwise the hash table counts.
bool use_sort(long long n_bases, int k) { return 2 * k + bits_for(n_bases > 0 ? n_bases : 1) <= 64; }

struct CandLayout {
  bool sort;                 // sort-based count (else the hash table)
  unsigned long long slots;  // hash table slots (power of two; 0 on the sort path)
  unsigned long long inst;   // occurrence capacity
  unsigned long long pairs;  // occurrence-pair capacity
  unsigned long long tiles;  // sort tiles (the larger of the two sorts)
  size_t state, table, retained, inst_arr, occ_cnt, occ_off, okeys0, okeys1, info, pk0, pk1, hist, hoff, flags,
      sid, tsum, toff, part, total;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

CandLayout cand_layout(long long n_reads, long long n_bases, int k, int mult_hi) {
  CandLayout L;
  const unsigned long long inst = (unsigned long long)(n_bases > 0 ? n_bases : 1);
  const unsigned long long reads = (unsigned long long)(n_reads > 0 ? n_reads : 1);
  L.sort = use_sort(n_bases, k);
  unsigned long long slots = 0;
  if (!L.sort) {
    slots = 1024;
    while (slots < inst + inst / 2) slots <<= 1;  // load factor below 2/3
  }
  L.slots = slots;
  L.inst = inst;
  L.pairs = inst * (unsigned long long)(mult_hi > 1 ? mult_hi - 1 : 1) / 2 + 1;
  const unsigned long long ptiles = (L.pairs + kTile - 1) / kTile, otiles = (inst + kTile - 1) / kTile;
  L.tiles = ptiles > otiles ? ptiles : otiles;
  size_t off = 0;
  L.state = off;    off = align256(off + sizeof(CandState));
  L.table = off;    off = align256(off + sizeof(Slot) * slots);
  L.retained = off; off = align256(off + 4 * slots);
  L.inst_arr = off; off = align256(off + (L.sort ? 0 : 8 * inst));
  L.occ_cnt = off;  off = align256(off + (L.sort ? 4 * reads : 0));
  L.occ_off = off;  off = align256(off + (L.sort ? 8 * reads : 0));
  L.okeys0 = off;   off = align256(off + (L.sort ? 8 * inst : 0));
  L.okeys1 = off;   off = align256(off + (L.sort ? 8 * inst : 0));
  L.info = off;     off = align256(off + (L.sort ? 8 * inst : 0));
  L.pk0 = off;      off = align256(off + 8 * L.pairs);
  L.pk1 = off;      off = align256(off + 8 * L.pairs);
  L.hist = off;     off = align256(off + 4 * 256 * L.tiles);
  L.hoff = off;     off = align256(off + 8 * 256 * L.tiles);
  L.flags = off;    off = align256(off + 4 * L.pairs);
  L.sid = off;      off = align256(off + 4 * L.pairs);
  L.tsum = off;     off = align256(off + 4 * L.tiles);
  L.toff = off;     off = align256(off + 8 * L.tiles);
  L.part = off;     off = align256(off + 8 * kScanBlocks);
  L.total = off;
  return L;
}

// Workspace of the partitioned path: one pass's occurrence keys (two
// buffers) and words, the occurrence-pair keys (two-word when they do not fit
// one word; two buffers), selection flags and seed ids, and the sort and scan
// scratch.  pass_cap = occurrences one pass holds: n_bases / n_parts with a
// quarter more for the unevenness of the hash parts, plus 2^16.
struct PartLayout {
  unsigned long long pass_cap, pairs, tiles;
  bool wide;  // two-word occurrence-pair keys
  size_t state, okeys0, okeys1, info, pk0, pk1, hist, hoff, flags, sid, tsum, toff, part, total;
};

unsigned long long part_capacity(long long n_bases, int n_parts) {
  const unsigned long long per = ((unsigned long long)(n_bases > 0 ? n_bases : 1) + n_parts - 1) / n_parts;
  return per + per / 4 + 65536;
}

PartLayout part_layout(long long n_bases, int n_parts, long long occ_pair_capacity, bool wide) {
  PartLayout L;
  L.pass_cap = part_capacity(n_bases, n_parts);
  L.pairs = (unsigned long long)(occ_pair_capacity > 0 ? occ_pair_capacity : 1);
  L.wide = wide;
  const size_t ksz = wide ? sizeof(Key2) : 8;
  const unsigned long long ktile = wide ? KeyOps<Key2>::kTile : KeyOps<unsigned long long>::kTile;
  const unsigned long long otiles = (L.pass_cap + kTile - 1) / kTile, ptiles = (L.pairs + ktile - 1) / ktile;
  L.tiles = otiles > ptiles ? otiles : ptiles;
  const unsigned long long ctiles = (L.pairs + kTile - 1) / kTile;  // compaction tiles
  size_t off = 0;
  L.state = off;  off = align256(off + sizeof(CandState));
  L.okeys0 = off; off = align256(off + 8 * L.pass_cap);
  L.okeys1 = off; off = align256(off + 8 * L.pass_cap);
  L.info = off;   off = align256(off + 8 * L.pass_cap);
  L.pk0 = off;    off = align256(off + ksz * L.pairs);
  L.pk1 = off;    off = align256(off + ksz * L.pairs);
  L.hist = off;   off = align256(off + 4 * 256 * L.tiles);
  L.hoff = off;   off = align256(off + 8 * 256 * L.tiles);
  L.flags = off;  off = align256(off + 4 * L.pairs);
  L.sid = off;    off = align256(off + 4 * L.pairs);
  L.tsum = off;   off = align256(off + 4 * ctiles);
  L.toff = off;   off = align256(off + 8 * ctiles);
  L.part = off;   off = align256(off + 8 * kScanBlocks);
  L.total = off;
  return L;
}

// Occurrence-pair keys are two words when read, read, position, position and
// strand need more than 64 bits.
bool wide_pair_keys(long long n_reads, int max_read_len) {
  const int rbits = bits_for(n_reads > 0 ? (unsigned long long)(n_reads - 1) : 0);
  const int pbits = bits_for(max_read_len > 0 ? (unsigned long long)max_read_len : 0);
  return 2 * rbits + 2 * pbits + 1 > 64;
}

// Selection, compaction and counts over the sorted occurrence-pair keys.
template <typename K>
void select_and_compact(const K* keys, CandState* state, const KeyLayout& kl, int max_seeds, int gap,
                        unsigned int* flags, unsigned int* sid, unsigned int* tsum, unsigned long long* toff,
                        unsigned long long* part, dibella_pair_t* pairs_out, long long pairs_capacity,
                        int64_t* counts_out, int sms, cudaStream_t st) {
  const int sort_blocks = sms * 8;
  select_kernel<K><<<sms * 8, 256, 0, st>>>(keys, state, kl, max_seeds, gap, flags, sid);
  tile_sum_kernel<<<sort_blocks, kSortThreads, 0, st>>>(flags, state, tsum);
  scan_counts(tsum, toff, &state->n_keys, 2, 0, part, st);
  compact_kernel<K><<<sort_blocks, kSortThreads, 0, st>>>(keys, flags, sid, toff, state, kl, pairs_out,
                                                          (unsigned long long)pairs_capacity);
  finish_kernel<<<1, 1, 0, st>>>(state, toff, tsum, counts_out);
}

}  // namespace

extern "C" {

int dibella_candidate_workspace_bytes_parts(int64_t n_reads, int64_t n_bases, int32_t max_read_len, int32_t k,
                                            int32_t n_parts, int64_t occ_pair_capacity, int64_t* bytes_out) {
  if (!bytes_out || n_reads < 0 || n_bases < 0 || k < 1 || k > 32 || n_parts < 1 || n_parts > 4096 ||
      occ_pair_capacity < 0 || occ_pair_capacity > (1ll << 40) || max_read_len < 0 ||
      max_read_len > DIBELLA_MAX_READ_LEN)
    return DIBELLA_EINVAL;
  *bytes_out = (int64_t)part_layout(n_bases, n_parts, occ_pair_capacity, wide_pair_keys(n_reads, max_read_len)).total;
  return DIBELLA_OK;
}

int dibella_candidate_pairs_parts(const uint32_t* packed_words, const int64_t* read_word_offsets,
                                  const int32_t* read_lengths, int64_t n_reads, int64_t n_bases, int32_t max_read_len,
                                  int32_t k, int32_t mult_lo, int32_t mult_hi, int32_t max_seeds,
                                  int32_t min_seed_gap, int32_t n_parts, int64_t occ_pair_capacity,
                                  dibella_pair_t* pairs_out, int64_t pairs_capacity, int64_t* counts_out,
                                  void* workspace, int64_t workspace_bytes, void* stream) {
  if (n_reads < 0 || n_bases < 0 || k < 1 || k > 32 || mult_lo < 1 || mult_hi < mult_lo || mult_hi > kMaxMult ||
      max_seeds < 1 || min_seed_gap < 0 || max_read_len < 0 || max_read_len > DIBELLA_MAX_READ_LEN ||
      n_parts < 1 || n_parts > 4096 || occ_pair_capacity < 0 || occ_pair_capacity > (1ll << 40) ||
      pairs_capacity < 0 || !counts_out || !workspace || ((uintptr_t)workspace & 255))
    return DIBELLA_EINVAL;
  if (n_reads > 0 && (!packed_words || !read_word_offsets || !read_lengths)) return DIBELLA_EINVAL;
  if (pairs_capacity > 0 && !pairs_out) return DIBELLA_EINVAL;
  if (n_reads > (1ll << 32)) return DIBELLA_EINVAL;  // read ids are 32-bit
  const int rbits = bits_for(n_reads > 0 ? (unsigned long long)(n_reads - 1) : 0);
  const int pbits = bits_for(max_read_len > 0 ? (unsigned long long)max_read_len : 0);
  const bool wide = 2 * rbits + 2 * pbits + 1 > 64;
  const PartLayout L = part_layout(n_bases, n_parts, occ_pair_capacity, wide);
  // a pass keys each occurrence by (code << ib | slot): both must fit 64 bits
  const int ib = bits_for(L.pass_cap);
  if (2 * k + ib > 64) return DIBELLA_EINVAL;
  if ((unsigned long long)workspace_bytes < L.total) return DIBELLA_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  CandState* state = (CandState*)(ws + L.state);
  unsigned long long* ok0 = (unsigned long long*)(ws + L.okeys0);
  unsigned long long* ok1 = (unsigned long long*)(ws + L.okeys1);
  unsigned long long* info = (unsigned long long*)(ws + L.info);
  unsigned int* hist = (unsigned int*)(ws + L.hist);
  unsigned long long* hoff = (unsigned long long*)(ws + L.hoff);
  unsigned int* flags = (unsigned int*)(ws + L.flags);
  unsigned int* sid = (unsigned int*)(ws + L.sid);
  unsigned int* tsum = (unsigned int*)(ws + L.tsum);
  unsigned long long* toff = (unsigned long long*)(ws + L.toff);
  unsigned long long* part = (unsigned long long*)(ws + L.part);

  KeyLayout kl;
  kl.sh_pb = 1;
  kl.sh_pa = 1 + pbits;
  kl.m_read = (1ull << rbits) - 1ull;
  kl.m_pos = (1ull << pbits) - 1ull;
  if (wide) {  // lo = pa | pb | strand, hi = ra | rb
    kl.sh_rb = 0;
    kl.sh_ra = rbits;
  } else {
    kl.sh_rb = 1 + 2 * pbits;
    kl.sh_ra = 1 + 2 * pbits + rbits;
  }
  cudaError_t e;
  if ((e = set_scatter_smem()) != cudaSuccess) return DIBELLA_ECUDA;
  if ((e = cudaMemsetAsync(state, 0, sizeof(CandState), st)) != cudaSuccess) return DIBELLA_ECUDA;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  StoreRef sr{packed_words, read_word_offsets, read_lengths, (long long)n_reads, k};
  for (int p = 0; p < n_parts && n_reads > 0; ++p) {
    pass_begin_kernel<<<1, 1, 0, st>>>(state);
    extract_part_kernel<<<sms * 16, 256, 0, st>>>(sr, (unsigned)p, (unsigned)n_parts, ib, L.pass_cap, ok0, info,
                                                  state);
    pass_end_kernel<<<1, 1, 0, st>>>(state, L.pass_cap);
    unsigned long long* osrc = ok0;
    unsigned long long* odst = ok1;
    for (int j = 0; j < (2 * k + 7) / 8; ++j) {
      radix_pass(osrc, odst, &state->pass_held, ib + 8 * j, hist, hoff, L.tiles, part, &state->status, sms, st);
      unsigned long long* tmp = osrc;
      osrc = odst;
      odst = tmp;
    }
    if (wide)
      run_emit_kernel<Key2><<<sms * 8, 256, 0, st>>>(osrc, info, ib, mult_lo, mult_hi, kl, (Key2*)(ws + L.pk0),
                                                     L.pairs, &state->pass_held, state);
    else
      run_emit_kernel<unsigned long long><<<sms * 8, 256, 0, st>>>(osrc, info, ib, mult_lo, mult_hi, kl,
                                                                   (unsigned long long*)(ws + L.pk0), L.pairs,
                                                                   &state->pass_held, state);
  }
  cap_keys_kernel<<<1, 1, 0, st>>>(state, L.pairs);
  const int gap = min_seed_gap > 0 ? min_seed_gap : k;
  if (wide) {
    Key2* src = (Key2*)(ws + L.pk0);
    Key2* dst = (Key2*)(ws + L.pk1);
    const int lo_bits = 1 + 2 * pbits, hi_bits = 2 * rbits;
    for (int j = 0; j < (lo_bits + 7) / 8 + (hi_bits + 7) / 8; ++j) {
      const int shift = j < (lo_bits + 7) / 8 ? 8 * j : 64 + 8 * (j - (lo_bits + 7) / 8);
      radix_pass(src, dst, &state->n_keys, shift, hist, hoff, L.tiles, part, &state->status, sms, st);
      Key2* tmp = src;
      src = dst;
      dst = tmp;
    }
    select_and_compact(src, state, kl, max_seeds, gap, flags, sid, tsum, toff, part, pairs_out, pairs_capacity,
                       counts_out, sms, st);
  } else {
    unsigned long long* src = (unsigned long long*)(ws + L.pk0);
    unsigned long long* dst = (unsigned long long*)(ws + L.pk1);
    const int passes = (kl.sh_ra + rbits + 7) / 8;
    for (int j = 0; j < passes; ++j) {
      radix_pass(src, dst, &state->n_keys, 8 * j, hist, hoff, L.tiles, part, &state->status, sms, st);
      unsigned long long* tmp = src;
      src = dst;
      dst = tmp;
    }
    select_and_compact(src, state, kl, max_seeds, gap, flags, sid, tsum, toff, part, pairs_out, pairs_capacity,
                       counts_out, sms, st);
  }
  max_pass_kernel<<<1, 1, 0, st>>>(state, counts_out);
  e = cudaGetLastError();
  return e == cudaSuccess ? DIBELLA_OK : DIBELLA_ECUDA;
}

int dibella_candidate_workspace_bytes(int64_t n_reads, int64_t n_bases, int32_t k, int32_t mult_hi,
                                      int64_t* bytes_out) {
  if (!bytes_out || n_reads < 0 || n_bases < 0 || k < 1 || k > 32 || mult_hi < 1 || mult_hi > kMaxMult)
    return DIBELLA_EINVAL;
  *bytes_out = (int64_t)cand_layout(n_reads, n_bases, k, mult_hi).total;
  return DIBELLA_OK;
}

int dibella_candidate_pairs(const uint32_t* packed_words, const int64_t* read_word_offsets,
                            const int32_t* read_lengths, int64_t n_reads, int64_t n_bases, int32_t max_read_len,
                            int32_t k, int32_t mult_lo, int32_t mult_hi, int32_t max_seeds, int32_t min_seed_gap,
                            dibella_pair_t* pairs_out, int64_t pairs_capacity, int64_t* counts_out,
                            void* workspace, int64_t workspace_bytes, void* stream) {
  if (n_reads < 0 || n_bases < 0 || k < 1 || k > 32 || mult_lo < 1 || mult_hi < mult_lo || mult_hi > kMaxMult ||
      max_seeds < 1 || min_seed_gap < 0 || max_read_len < 0 || max_read_len > DIBELLA_MAX_READ_LEN ||
      pairs_capacity < 0 || !counts_out || !workspace || ((uintptr_t)workspace & 255))
    return DIBELLA_EINVAL;
  if (n_reads > 0 && (!packed_words || !read_word_offsets || !read_lengths)) return DIBELLA_EINVAL;
  if (n_bases >= (int64_t)0xFFFFFFFFll) return DIBELLA_EINVAL;  // occurrence cursors are 32-bit
  if (pairs_capacity > 0 && !pairs_out) return DIBELLA_EINVAL;
  const int rbits = bits_for(n_reads > 0 ? (unsigned long long)(n_reads - 1) : 0);
  const int pbits = bits_for(max_read_len > 0 ? (unsigned long long)max_read_len : 0);
  if (2 * rbits + 2 * pbits + 1 > 64) return DIBELLA_EINVAL;
  const CandLayout L = cand_layout(n_reads, n_bases, k, mult_hi);
  if ((unsigned long long)workspace_bytes < L.total) return DIBELLA_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  CandState* state = (CandState*)(ws + L.state);
  TableRef t;
  t.slots = (Slot*)(ws + L.table);
  t.mask = L.slots - 1;
  unsigned int* retained = (unsigned int*)(ws + L.retained);
  unsigned long long* inst = (unsigned long long*)(ws + L.inst_arr);
  unsigned long long* pk0 = (unsigned long long*)(ws + L.pk0);
  unsigned long long* pk1 = (unsigned long long*)(ws + L.pk1);
  unsigned int* hist = (unsigned int*)(ws + L.hist);
  unsigned long long* hoff = (unsigned long long*)(ws + L.hoff);
  unsigned int* flags = (unsigned int*)(ws + L.flags);
  unsigned int* sid = (unsigned int*)(ws + L.sid);
  unsigned int* tsum = (unsigned int*)(ws + L.tsum);
  unsigned long long* toff = (unsigned long long*)(ws + L.toff);
  unsigned long long* part = (unsigned long long*)(ws + L.part);

  KeyLayout kl;
  kl.sh_pb = 1;
  kl.sh_pa = 1 + pbits;
  kl.sh_rb = 1 + 2 * pbits;
  kl.sh_ra = 1 + 2 * pbits + rbits;
  kl.m_read = (1ull << rbits) - 1ull;
  kl.m_pos = (1ull << pbits) - 1ull;

  cudaError_t e;
  if ((e = set_scatter_smem()) != cudaSuccess) return DIBELLA_ECUDA;
  if ((e = cudaMemsetAsync(state, 0, sizeof(CandState), st)) != cudaSuccess) return DIBELLA_ECUDA;
  if (!L.sort && (e = cudaMemsetAsync(t.slots, 0, sizeof(Slot) * L.slots, st)) != cudaSuccess) return DIBELLA_ECUDA;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  StoreRef sr{packed_words, read_word_offsets, read_lengths, (long long)n_reads, k};
  const int walk_blocks = sms * 16;
  const int sort_blocks = sms * 8;
  if (n_reads > 0 && L.sort) {
    // Occurrence keys (code << ib | index), sorted by the code digits only: the
    // stable passes keep each k-mer's occurrences in index order.
    unsigned int* occ_cnt = (unsigned int*)(ws + L.occ_cnt);
    unsigned long long* occ_off = (unsigned long long*)(ws + L.occ_off);
    unsigned long long* ok0 = (unsigned long long*)(ws + L.okeys0);
    unsigned long long* ok1 = (unsigned long long*)(ws + L.okeys1);
    unsigned long long* info = (unsigned long long*)(ws + L.info);
    const int ib = bits_for((unsigned long long)n_bases);
    occ_count_kernel<<<sms * 4, 256, 0, st>>>(sr, occ_cnt);
    scan_counts(occ_cnt, occ_off, &state->instances, 0, (unsigned long long)n_reads, part, st);
    occ_total_kernel<<<1, 1, 0, st>>>(occ_cnt, occ_off, (long long)n_reads, L.inst, state);
    extract_kernel<<<walk_blocks, 256, 0, st>>>(sr, occ_off, ib, L.inst, ok0, info);
    unsigned long long* osrc = ok0;
    unsigned long long* odst = ok1;
    for (int j = 0; j < (2 * k + 7) / 8; ++j) {
      radix_pass(osrc, odst, &state->instances, ib + 8 * j, hist, hoff, L.tiles, part, &state->status, sms, st);
      unsigned long long* tmp = osrc;
      osrc = odst;
      odst = tmp;
    }
    run_emit_kernel<<<sms * 8, 256, 0, st>>>(osrc, info, ib, mult_lo, mult_hi, kl, pk0, L.pairs, &state->instances,
                                             state);
  } else if (n_reads > 0) {
    kmer_walk_kernel<false><<<walk_blocks, 256, 0, st>>>(sr, t, inst, L.inst, mult_lo, mult_hi, state);
    allocate_kernel<<<sms * 8, 256, 0, st>>>(t, L.slots, mult_lo, mult_hi, retained, state);
    kmer_walk_kernel<true><<<walk_blocks, 256, 0, st>>>(sr, t, inst, L.inst, mult_lo, mult_hi, state);
    emit_pairs_kernel<<<sms * 8, 256, 0, st>>>(t, retained, inst, L.inst, kl, pk0, L.pairs, state);
  }
  cap_keys_kernel<<<1, 1, 0, st>>>(state, L.pairs);
  // Radix sort by the whole key (read_a, read_b, pos_a, pos_b, strand).
  const int key_bits = kl.sh_ra + rbits;
  const int passes = (key_bits + 7) / 8;
  unsigned long long* src = pk0;
  unsigned long long* dst = pk1;
  for (int pss = 0; pss < passes; ++pss) {
    radix_pass(src, dst, &state->n_keys, 8 * pss, hist, hoff, L.tiles, part, &state->status, sms, st);
    unsigned long long* tmp = src;
    src = dst;
    dst = tmp;
  }
  select_kernel<<<sms * 8, 256, 0, st>>>(src, state, kl, max_seeds, min_seed_gap > 0 ? min_seed_gap : k, flags, sid);
  tile_sum_kernel<<<sort_blocks, kSortThreads, 0, st>>>(flags, state, tsum);
  scan_counts(tsum, toff, &state->n_keys, 2, 0, part, st);
  compact_kernel<<<sort_blocks, kSortThreads, 0, st>>>(src, flags, sid, toff, state, kl, pairs_out,
                                                         (unsigned long long)pairs_capacity);
  finish_kernel<<<1, 1, 0, st>>>(state, toff, tsum, counts_out);
  e = cudaGetLastError();
  return e == cudaSuccess ? DIBELLA_OK : DIBELLA_ECUDA;
}

}  // extern "C"
