/* dibella.h — C ABI of the GB300 seed-and-extend X-drop library (libdibella.so).
 *
 * The library aligns candidate long-read pairs from shared k-mer seeds with
 * X-drop extension, the per-pair work of diBELLA (Ellis et al., ICPP 2019):
 *   - alignment and its score: Sec. 2 ("Read-to-Read Alignment"), the
 *     definition of a pairwise alignment of s and t and its scoring;
 *   - X-drop: Sec. 2, the paragraph replacing full dynamic programming by a
 *     banded search that stops once the score drops X below the best
 *     (after Zhang et al. 2000); SeqAn's implementation in the paper;
 *   - seeds: Sec. 2 (shared k-mers, Fig. 1) and Sec. 8 (retained k-mer
 *     positions per overlapping pair; seed count / spacing constraints);
 *   - the per-pair alignment stage: Sec. 9 ("Alignment").
 * The paper fixes no recurrence, band rule or tie-break; this library
 * implements the reading documented on dibella_xdrop_batch below.
 *
 * All entry points return 0 (DIBELLA_OK) on success or a negative status;
 * on an argument error nothing has been written and no work was enqueued
 * (dibella_pack_reads may have written part of packed_words before it finds
 * a bad base).
 * Thread safety: calls may run concurrently on different streams with
 * distinct workspaces.  No entry point allocates device memory.
 */
#ifndef DIBELLA_H_
#define DIBELLA_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
enum {
  DIBELLA_OK = 0,
  DIBELLA_EINVAL = -1,   /* bad scalar argument, null pointer or size       */
  DIBELLA_EBASE = -2,    /* a read holds a byte other than A, C, G, T       */
  DIBELLA_ENOMEM = -3,   /* caller-provided workspace too small             */
  DIBELLA_ECUDA = -4,    /* a CUDA runtime call failed (see last_error)     */
  DIBELLA_ETIMEOUT = -5  /* reserved: a bounded device wait ran out         */
};

/* Per-result status bits (dibella_result_t.status). */
#define DIBELLA_RES_SEED_MISMATCH 1  /* the k seed bases are not identical   */
#define DIBELLA_RES_INVALID_SEED 2   /* read id / seed position out of range  */
#define DIBELLA_RES_BEST_OF_PAIR 4   /* best seed of its candidate pair       */
#define DIBELLA_RES_BAND_OVERFLOW 8  /* band wider than the workspace allows;
                                        score/coordinates/cells not computed  */

/* X values at or above this act as "no drop-off" for reads whose path scores
 * stay above -2^30 (every read accepted here when |gap| * length < 2^30). */
#define DIBELLA_XDROP_INF (1 << 30)

/* Limits checked on the host (EINVAL otherwise). */
#define DIBELLA_MAX_K 32
#define DIBELLA_MAX_SCORE 64         /* |match|, |mismatch|, |gap| <= 64      */
#define DIBELLA_MAX_READ_LEN (1 << 24)

/* ---- records ---------------------------------------------------------- */

/* Linear-gap scoring (Sec. 2: matches rewarded; mismatches, insertions and
 * deletions penalised).  Requires match > 0, mismatch <= 0, gap < 0, each of
 * magnitude <= DIBELLA_MAX_SCORE, and 0 <= xdrop <= DIBELLA_XDROP_INF. */
typedef struct {
  int32_t match, mismatch, gap, xdrop;
} dibella_scoring_t;

/* One seed of a candidate pair (24 bytes).  The seed is the shared k-mer at
 * pos_a in read_a and at pos_b in read_b, both in FORWARD coordinates;
 * strand = 1 when the occurrences have opposite orientation, i.e. read_b is
 * aligned reverse-complemented.  A candidate pair with several seeds is a run
 * of consecutive records with equal (read_a, read_b); seed_id is the caller's
 * label and is not interpreted. */
typedef struct {
  uint32_t read_a, read_b, pos_a, pos_b;
  uint8_t strand;
  uint8_t pad[3];
  uint32_t seed_id;
} dibella_pair_t;

/* Result of one seed (40 bytes).  Coordinates are half-open; [begin_b, end_b)
 * is in forward coordinates of read_b whatever the strand.  cells = evaluated
 * DP cells of both extensions (the work behind GCUPS). */
typedef struct {
  int32_t score, score_left, score_right;
  uint32_t begin_a, end_a, begin_b, end_b;
  int32_t status;
  int64_t cells;
} dibella_result_t;

/* ---- packed read store ------------------------------------------------ */
/* Layout (Sec. 3: 2 bits per base; A=0 C=1 G=2 T=3, complement = 3 - code):
 * 32-bit words, 16 bases per word, base q of a copy at bits 2*(q%16).
 * The store opens with 8 zero words; then, per read r, its forward copy at
 * word read_word_offsets[r] (a multiple of 4, i.e. 16-byte aligned) followed
 * immediately by its reverse-complement copy; each copy takes
 * 4*ceil(ceil(len/16)/4) words; the store closes with 8 zero words (the
 * kernels read up to 128 bases past either end of a copy and ignore them).
 * Holding both orientations lets every extension read both sequences in
 * ascending word order, reverse complement included. */

/* Words needed for n_reads reads whose ASCII spans are given by the n_reads+1
 * entries of ascii_offsets (non-decreasing).  Host pointers.  EINVAL on a
 * negative count, a decreasing offset or a read longer than
 * DIBELLA_MAX_READ_LEN. */
int dibella_packed_words(const int64_t* ascii_offsets, int64_t n_reads,
                         int64_t* n_words_out);

/* Pack reads to the store layout above.  All pointers are HOST pointers and
 * the caller owns every buffer: packed_words holds dibella_packed_words()
 * words, read_word_offsets and read_lengths hold n_reads entries each.
 * Bytes A/C/G/T (either case) are accepted; any other byte returns EBASE
 * with *bad_index = its position in `ascii` (bad_index may be NULL).
 * n_threads <= 0 uses every hardware thread. */
int dibella_pack_reads(const char* ascii, const int64_t* ascii_offsets, int64_t n_reads,
                       uint32_t* packed_words, int64_t* read_word_offsets,
                       int32_t* read_lengths, int64_t* bad_index, int32_t n_threads);

/* ---- scheduling ------------------------------------------------------- */
/* How a batch is split across the extension kernels.  Results never depend
 * on the schedule; only speed does.  Every extension first goes to one of:
 *   narrow  one thread per extension, band in per-thread shared memory of
 *           narrow_band_cap cells (32, 48 or 64);
 *   wide    a warp (or a group of 16 or 8 lanes) per extension, band in
 *           registers: wide_slots chunks (16, 24 or 32), of which
 *           wide_slots - 2 hold the band; a chunk is 2 cells per lane
 *           packed as int16 pairs when wide_packed is set and
 *           xdrop <= 8000 (exact: scores are kept relative to a moving base),
 *           else 32 int32 cells of one warp;
 *   split   with narrow_split_d > 0 the narrow form runs in two passes: the
 *           first stops every extension at antidiagonal narrow_split_d,
 *           the second re-runs the unfinished ones from the origin, so that
 *           long extensions share warps with long ones only;
 *   mid     the narrow form's escalations first go, when mid_band_cap > 0
 *           and xdrop <= 8000, to a second one-thread-per-extension form
 *           whose per-thread band holds mid_band_cap int16 cells (one warp
 *           per block); its own escalations go to the wide form;
 * an extension whose band outgrows its form is re-run from the start by the
 * next wider form: the narrow form's by the mid (else the wide) form, the wide form's by
 * the next rung of 8 -> 16 -> 24 -> 32 slots, then by a block of 8 warps
 * per extension with an 8192-cell band in shared memory (the CTA form), and
 * beyond that by a warp whose band lives in the workspace (sized by
 * max_read_len: it cannot overflow).
 * An extension is routed to narrow when xdrop <= narrow_max_xdrop and
 * min(remaining A, remaining B) <= narrow_max_len.  When a call passes no
 * schedule, batches with fewer than 1.5 extensions per resident narrow lane
 * go entirely to the wide form (they would wait on one lane's longest
 * extension), and for xdrop > 10 keys above 20000 (above 5000 in batches
 * with fewer than 7 extensions per lane) go to the wide form (a narrow lane
 * would otherwise hold up the escalations behind its long extension); an
 * explicit schedule is followed as given.  Work is ordered by
 * n_buckets length buckets (longest first); bucket b holds keys below
 * bucket_bounds[b] (ascending), the last bucket everything else. */
#define DIBELLA_MAX_BUCKETS 8
typedef struct {
  int32_t narrow_max_xdrop;
  int32_t narrow_max_len;
  int32_t narrow_band_cap;
  int32_t wide_slots;             /* 8 (packed, one warp only), 16, 24, 32,   */
                                  /* or 0 = 8 if xdrop <= 30 else 24          */
                                  /* else 24                                  */
  int32_t wide_packed;            /* 1: int16-pair cells when xdrop <= 8000   */
  int32_t wide_group_lanes;       /* packed wide form: lanes per extension,   */
                                  /* 32 (one warp), 16 or 8 (2 or 4 per warp, */
                                  /* chunks of 2 cells per lane); 0 = 32      */
  int32_t wide_blocks_per_sm;     /* 0 = occupancy maximum                   */
  int32_t narrow_blocks_per_sm;   /* 0 = occupancy maximum                   */
  int32_t n_buckets;              /* 1..DIBELLA_MAX_BUCKETS                  */
  int32_t bucket_bounds[DIBELLA_MAX_BUCKETS];
  int32_t mid_band_cap;           /* mid form: 0 (none), 128, 192 or 256      */
  int32_t narrow_split_d;         /* > 0: narrow form in two passes, the      */
                                  /* first stopping at this antidiagonal      */
  int32_t narrow_unroll;          /* narrow form: cells per unrolled group of */
                                  /* its band walk, 4, 8 or 16 (0 = 16)       */
  int32_t narrow_track;           /* 1 (the default's): narrow form keeps its */
                                  /* live range and maximum in registers while*/
                                  /* it walks the band (16-cell groups, int16 */
                                  /* rows; narrow_unroll is then ignored), 0: */
                                  /* finds them by scans of the new row       */
} dibella_schedule_t;

/* The schedule used when a call passes NULL.  set() validates (EINVAL). */
int dibella_get_default_schedule(dibella_schedule_t* out);
int dibella_set_default_schedule(const dibella_schedule_t* sched);

/* ---- X-drop batch ----------------------------------------------------- */

/* Device workspace bytes for a batch of n_pairs seeds over reads of at most
 * max_read_len bases (a bound, used to size the global-memory band of the
 * widest kernel so that it can never overflow). */
int dibella_xdrop_workspace_bytes(int64_t n_pairs, int32_t max_read_len,
                                  int64_t* bytes_out);

/* Align every seed record.  DEVICE pointers: packed_words, read_word_offsets,
 * read_lengths (the store above, n_reads reads), pairs (n_pairs records),
 * results (n_pairs records, written in input order), workspace
 * (workspace_bytes, at least dibella_xdrop_workspace_bytes(n_pairs, ...);
 * 256-byte aligned).  `stream` is a cudaStream_t (NULL = legacy default).
 * `sched` may be NULL.  Asynchronous: argument errors return synchronously,
 * per-seed problems go to result.status, and no host synchronisation or
 * allocation happens, so the call can be captured in a CUDA graph.
 *
 * Semantics, per seed (Sec. 2 and Sec. 8-9, with these readings):
 *   B' = read_b if strand = 0, else its reverse complement; the seed sits at
 *   pos_a in A and at pos_b' = (strand ? len_b - pos_b - k : pos_b) in B'.
 *   seed score = sum over the k seed columns of match/mismatch.
 *   Left extension: reversed A[0,pos_a) against reversed B'[0,pos_b');
 *   right extension: A[pos_a+k, len_a) against B'[pos_b'+k, len_b).
 *   Each extension runs the antidiagonal X-drop DP H(i,j) = max(H(i-1,j-1) +
 *   s(a_i,b_j), H(i-1,j) + gap, H(i,j-1) + gap) from H(0,0) = 0, where:
 *     band of antidiagonal d = [lo(d-1), hi(d-1)+1] clipped to the matrix,
 *       lo/hi = smallest/largest i of the LIVE cells of d-1;
 *     a cell is live iff H >= best(<d) - xdrop; dead cells are -infinity;
 *     best improves on a strictly larger value; on the improving
 *       antidiagonal the live cell of smallest i wins;
 *     the extension stops at the first antidiagonal without a live cell.
 *   score = seed + left best + right best; begin/end from the winning cells;
 *   cells = evaluated band cells of both extensions (antidiagonals >= 1).
 *   Invalid seeds (read id >= n_reads, strand > 1, pos + k beyond the read)
 *   get status DIBELLA_RES_INVALID_SEED and zero fields.  In each run of
 *   records with equal (read_a, read_b) the valid record with the highest
 *   score (earliest on ties) gets DIBELLA_RES_BEST_OF_PAIR.
 * Requires 1 <= k <= DIBELLA_MAX_K and the scoring limits above. */
int dibella_xdrop_batch(const uint32_t* packed_words, const int64_t* read_word_offsets,
                        const int32_t* read_lengths, int64_t n_reads,
                        const dibella_pair_t* pairs, int64_t n_pairs, int32_t k,
                        dibella_scoring_t scoring, dibella_result_t* results,
                        void* workspace, int64_t workspace_bytes, void* stream,
                        const dibella_schedule_t* sched);

/* Callers that cannot allocate device memory: for example a host runtime
 * whose own pool owns all of the GPU's memory, a latency-critical loop in
 * which an allocation might block or synchronise the device, or plug-in code
 * that may not hold allocations of its own.  This entry point runs the same
 * alignment as dibella_xdrop_batch (same arguments, results and semantics,
 * default schedule) without any workspace from the caller and without
 * allocating.  Its scratch is one fixed array inside the library, 9,568,768
 * bytes (about 9.1 MiB), which every GPU that loads the library keeps until
 * the process exits.
 * Limits: at most DIBELLA_NOALLOC_MAX_PAIRS seed records per call (more
 * returns DIBELLA_ENOMEM, with the reason in dibella_last_error(), and does
 * nothing); an extension whose band (the cells of one antidiagonal between
 * its first and last live cell, plus one) grows beyond
 * DIBELLA_NOALLOC_MAX_BAND cells gets DIBELLA_RES_BAND_OVERFLOW and zero
 * fields, where dibella_xdrop_batch with a workspace sized for the longest
 * read computes it (such bands need X far above the read's error budget:
 * about X >= 8000 with unit scores, or reads that agree over 8 kb or more at
 * X = DIBELLA_XDROP_INF).
 * Every call looks up the array's device address with cudaGetSymbolAddress
 * (the first lookup on a device loads the library's module there), so make
 * the first call on each device before any stream capture.
 * All calls share the one array and each leaves its contents behind; the
 * parts that must start at zero are cleared by every call, but calls whose
 * work overlaps on the GPU (other streams, other threads) race on it, so
 * serialise them.
 * The paper has no counterpart: this is an interface for integration, not
 * part of the method. */
#define DIBELLA_NOALLOC_MAX_PAIRS 16384
#define DIBELLA_NOALLOC_MAX_BAND 8189
int dibella_xdrop_batch_noalloc(const uint32_t* packed_words, const int64_t* read_word_offsets,
                                const int32_t* read_lengths, int64_t n_reads, const dibella_pair_t* pairs,
                                int64_t n_pairs, int32_t k, dibella_scoring_t scoring,
                                dibella_result_t* results, void* stream);

/* The same alignment with HOST pairs and results: copies the pairs in, runs
 * dibella_xdrop_batch, copies the results out and synchronises `stream`.
 * The store and the workspace are device memory; pairs/results should be
 * pinned host memory for full copy speed.  staging is device memory of at
 * least dibella_staging_bytes(n_pairs) bytes, 256-byte aligned. */
int dibella_staging_bytes(int64_t n_pairs, int64_t* bytes_out);
int dibella_xdrop_batch_host(const uint32_t* packed_words, const int64_t* read_word_offsets,
                             const int32_t* read_lengths, int64_t n_reads,
                             const dibella_pair_t* host_pairs, int64_t n_pairs, int32_t k,
                             dibella_scoring_t scoring, dibella_result_t* host_results,
                             void* staging, void* workspace, int64_t workspace_bytes,
                             void* stream, const dibella_schedule_t* sched);

/* Stream a host-resident seed set through the GPU in chunks of at most
 * chunk_pairs records, with the read store resident in HBM (the paper's
 * streaming of bounded phases, Sec. 4, applied to the alignment tasks).
 * Chunk ends move back to the previous change of (read_a, read_b), so no
 * candidate pair is split (EINVAL if one pair has more seeds than a chunk).
 * Two slots alternate: staging[s] (device, dibella_staging_bytes(chunk_pairs)
 * bytes, 256-byte aligned), workspace[s] (device, workspace_bytes each, sized
 * for chunk_pairs) and streams[s]; each chunk's H2D copy, batch and D2H copy
 * are queued on its slot's stream, so the copies of one chunk overlap the
 * kernels of the other.  host_pairs / host_results should be pinned.
 * Synchronises both streams; *n_chunks_out (may be NULL) gets the count. */
int dibella_xdrop_stream(const uint32_t* packed_words, const int64_t* read_word_offsets,
                         const int32_t* read_lengths, int64_t n_reads, const dibella_pair_t* host_pairs,
                         int64_t n_pairs, int64_t chunk_pairs, int32_t k, dibella_scoring_t scoring,
                         dibella_result_t* host_results, void* const* staging, void* const* workspace,
                         int64_t workspace_bytes, void* const* streams, const dibella_schedule_t* sched,
                         int64_t* n_chunks_out);

/* Baseline form of the same computation: one kernel launch per candidate
 * pair (one warp runs the left then the right extension of each of the
 * pair's seed records, with the batched path's packed register form and its
 * escalations; no queues, no persistent kernels, no graph), all on `stream`.
 * Same arguments and results as dibella_xdrop_batch; used to measure what
 * batching buys.  Requires the same workspace.  Reads the records back to
 * the host once (a synchronisation) to find the candidate pairs. */
int dibella_xdrop_per_pair(const uint32_t* packed_words, const int64_t* read_word_offsets,
                           const int32_t* read_lengths, int64_t n_reads,
                           const dibella_pair_t* pairs, int64_t n_pairs, int32_t k,
                           dibella_scoring_t scoring, dibella_result_t* results,
                           void* workspace, int64_t workspace_bytes, void* stream);

/* ---- candidate pairs --------------------------------------------------- */

/* The steps before alignment, on the GPU: every k-mer occurrence of every read
 * in canonical orientation (Sec. 3: the smaller 2-bit code, A<C<G<T, of the
 * k-mer and of its reverse complement; orientation 1 when the reverse
 * complement is the smaller), its multiplicity over all occurrences, the
 * k-mers retained for mult_lo <= multiplicity <= mult_hi (Sec. 3-4), every
 * pair of distinct reads sharing a retained k-mer once per pair of
 * occurrences (Sec. 8, Algorithm 1; read_a < read_b, positions in forward
 * coordinates, strand = XOR of the orientations), and per read pair the seeds
 * (Sec. 8 seed constraints, Sec. 5 options): occurrences sorted by (pos_a,
 * pos_b, strand), seed 0 the first, each next seed the first whose pos_a is
 * at least min_seed_gap (0 = k) past the previous seed's, up to max_seeds.
 *
 * Workspace bytes for reads of n_bases bases in total (a hash table of 1.5 to
 * 3 slots per base, the retained occurrences and room for n_bases x
 * (mult_hi - 1) / 2 occurrence pairs: about 50 to 92 + 12 x (mult_hi - 1)
 * bytes per base).  EINVAL outside 1 <= k <= 32,
 * 1 <= mult_hi <= 32. */
int dibella_candidate_workspace_bytes(int64_t n_reads, int64_t n_bases, int32_t k, int32_t mult_hi,
                                      int64_t* bytes_out);

/* DEVICE pointers: the store (packed_words, read_word_offsets, read_lengths
 * of n_reads reads, n_bases bases in total, none longer than max_read_len),
 * pairs_out (pairs_capacity records), counts_out (6 int64), workspace
 * (256-byte aligned, workspace_bytes >= the size above).  Asynchronous on
 * `stream` (a cudaStream_t); nothing is allocated.  Writes the seed records
 * sorted by (read_a, read_b, seed_id) and counts_out = {seed records,
 * candidate pairs, k-mer occurrences, retained k-mers, occurrence pairs,
 * status}; status 0 = complete, else bit 0 the hash table filled, bit 1 more
 * occurrence pairs than the workspace holds, bit 2 more seed records than
 * pairs_capacity, bit 3 more occurrences than n_bases, bit 4 a radix pass
 * whose counts disagreed with its histogram (the records are then
 * incomplete).  Synchronous EINVAL: k outside 1..32, 1 <= mult_lo <= mult_hi
 * <= 32 violated, max_seeds < 1, min_seed_gap < 0, max_read_len outside
 * 0..DIBELLA_MAX_READ_LEN, null or misaligned buffers, or read and position
 * fields that do not pack into one 64-bit sort key (2 x bits(n_reads - 1) +
 * 2 x bits(max_read_len) + 1 > 64); ENOMEM when the workspace is too small. */
int dibella_candidate_pairs(const uint32_t* packed_words, const int64_t* read_word_offsets,
                            const int32_t* read_lengths, int64_t n_reads, int64_t n_bases, int32_t max_read_len,
                            int32_t k, int32_t mult_lo, int32_t mult_hi, int32_t max_seeds, int32_t min_seed_gap,
                            dibella_pair_t* pairs_out, int64_t pairs_capacity, int64_t* counts_out,
                            void* workspace, int64_t workspace_bytes, void* stream);

/* The same candidate pairs for read sets too large for one sort key
 * (dibella_candidate_pairs refuses more than 2^32 - 2 bases and occurrence-pair
 * fields wider than 64 bits).  The k-mer count runs in n_parts passes, the
 * paper's streaming of memory-limited phases (Sec. 4; Sec. 6-7 count the
 * k-mers in passes bounded by memory): pass p takes every occurrence whose
 * canonical code hashes to part p, so each k-mer is counted whole in one
 * pass, and keys it by (code << b | slot) with b = bits of the pass capacity
 * (n_bases / n_parts plus a quarter, plus 2^16 occurrences; 2k + b must not
 * exceed 64, else EINVAL: for k = 17, at least n_bases / 2^29 parts).  The
 * occurrence pairs of every pass (read_a, read_b, pos_a, pos_b, strand) are
 * kept in occ_pair_capacity slots, one 64-bit key each, or two 64-bit words
 * each (read_a | read_b, then pos_a | pos_b | strand) when the fields need
 * more than 64 bits; then they are sorted and the seeds selected as above.
 * Results are identical to dibella_candidate_pairs whenever both apply.
 * Workspace bytes for n_bases bases in n_parts passes and occ_pair_capacity
 * occurrence pairs (about 24 x 1.25 x n_bases / n_parts + 40 x
 * occ_pair_capacity bytes with two-word keys).  EINVAL outside 1 <= k <= 32,
 * 1 <= n_parts <= 4096, 0 <= occ_pair_capacity <= 2^40, 0 <= max_read_len <=
 * DIBELLA_MAX_READ_LEN. */
int dibella_candidate_workspace_bytes_parts(int64_t n_reads, int64_t n_bases, int32_t max_read_len, int32_t k,
                                            int32_t n_parts, int64_t occ_pair_capacity, int64_t* bytes_out);

/* Arguments as for dibella_candidate_pairs, plus n_parts and
 * occ_pair_capacity as above (the workspace must be sized for them with the
 * same n_reads, n_bases and max_read_len).  counts_out holds 7 int64: the six
 * of dibella_candidate_pairs, then the occurrences of the largest pass; status
 * bit 3 now means a pass held more occurrences than its capacity (use more
 * parts), bit 1 more occurrence pairs than occ_pair_capacity.  Asynchronous on
 * `stream`, allocates nothing.  Synchronous EINVAL on the argument limits of
 * dibella_candidate_pairs (the 64-bit key limits excepted), n_reads > 2^32,
 * or 2k + bits(pass capacity) > 64; ENOMEM when the workspace is too small. */
int dibella_candidate_pairs_parts(const uint32_t* packed_words, const int64_t* read_word_offsets,
                                  const int32_t* read_lengths, int64_t n_reads, int64_t n_bases, int32_t max_read_len,
                                  int32_t k, int32_t mult_lo, int32_t mult_hi, int32_t max_seeds,
                                  int32_t min_seed_gap, int32_t n_parts, int64_t occ_pair_capacity,
                                  dibella_pair_t* pairs_out, int64_t pairs_capacity, int64_t* counts_out,
                                  void* workspace, int64_t workspace_bytes, void* stream);

/* ---- traceback ---------------------------------------------------------- */
/* The edits of each seed's best alignment (Sec. 1: an alignment is the list
 * of edits that makes two overlapping regions identical; Sec. 2: the columns
 * of an alignment pair two characters or a character with a gap).  Each seed
 * is aligned as by dibella_xdrop_batch (same band, prune and tie rules) while
 * every evaluated cell keeps the move that gave its value, the diagonal
 * first, then the step in A, then the step in B' on equal values; the walk
 * from each extension's best cell back to the seed follows those moves.
 * Columns run from (begin_a, begin_b') to (end_a, end_b') in A and B' (B
 * reverse complemented when strand = 1): the left extension's, the k seed
 * columns, the right extension's.  They are written run-length encoded, one
 * 32-bit word per run: run length << 4 | op, with the SAM/BAM op numbers
 * below ('I' = a base of B' against a gap, 'D' = a base of A against a gap). */
#define DIBELLA_OP_INS 1
#define DIBELLA_OP_DEL 2
#define DIBELLA_OP_EQ 7
#define DIBELLA_OP_DIFF 8

/* Workspace for dibella_xdrop_traceback: n_lanes slots of
 * 3 x (max_read_len + 2) int32 (H rows) + moves_words 32-bit words (the moves
 * of every evaluated antidiagonal up to the best one: 3 words per
 * antidiagonal plus 2 bits per cell), rounded up to 256 bytes.  EINVAL for
 * n_lanes outside 1..2^24, moves_words outside 2..2^34, max_read_len outside
 * 0..DIBELLA_MAX_READ_LEN. */
int dibella_traceback_workspace_bytes(int64_t n_lanes, int32_t max_read_len, int64_t moves_words,
                                      int64_t* bytes_out);

/* DEVICE pointers: the store (as for dibella_xdrop_batch; no read longer than
 * max_read_len), pairs (n_pairs records), results (n_pairs records, written
 * as dibella_xdrop_batch writes them but without DIBELLA_RES_BEST_OF_PAIR),
 * ops (n_pairs x ops_per_seed words: seed t's runs at t * ops_per_seed) and
 * n_ops (n_pairs int32: seed t's run count; 0 for an invalid seed; -1 when
 * more than ops_per_seed runs were needed, nothing claimed; -2 when an
 * extension's moves up to its best cell exceeded moves_words; -3 when a read
 * is longer than max_read_len, the result then carries
 * DIBELLA_RES_BAND_OVERFLOW and zero fields).  Asynchronous on `stream`
 * (a cudaStream_t); allocates nothing.  A warp per seed (n_lanes warps,
 * each with one workspace slot, taking seeds t = w, w + n_lanes, ...)
 * re-runs both extensions with the band across its lanes, then one lane walks
 * back: meant for the seeds whose edits are wanted (accepted overlaps).
 * Sizing: a warp walking one seed is latency bound, so give it occupancy:
 * 24 warps per SM (3,648 on 152 SMs; 80 registers per thread) traced twice
 * as many seeds per second as 8; moves_words must hold, per extension, 3 words per antidiagonal up
 * to the best one plus 2 bits per evaluated cell, about (m + n) x (3 + band /
 * 16) words for an m x n extension (2^18 words cover a 30 kb overlap at a
 * 40-cell band).  EINVAL on the scoring limits of
 * dibella_xdrop_batch, k outside 1..32, ops_per_seed < 1, null or
 * misaligned (256-byte) pointers or a size outside the limits above; ENOMEM
 * when workspace_bytes is below dibella_traceback_workspace_bytes. */
int dibella_xdrop_traceback(const uint32_t* packed_words, const int64_t* read_word_offsets,
                            const int32_t* read_lengths, int64_t n_reads, int32_t max_read_len,
                            const dibella_pair_t* pairs, int64_t n_pairs, int32_t k, dibella_scoring_t scoring,
                            dibella_result_t* results, uint32_t* ops, int32_t ops_per_seed, int32_t* n_ops,
                            int64_t n_lanes, int64_t moves_words, void* workspace, int64_t workspace_bytes,
                            void* stream);

/* ---- autotuning -------------------------------------------------------- */
/* Pick a schedule for batches like this one: runs dibella_xdrop_batch on the
 * given (sample) batch with candidate schedules and returns the fastest in
 * *best_out (median of `repeats` timed runs each, CUDA events on `stream`).
 * The search is staged: routing threshold between the one-thread and the
 * wide forms x per-thread band chunk (32/48/64), then the mid form's band
 * (none/128/192/256), the split of the narrow form (none/64/128/256
 * antidiagonals), its band walk (cell groups of 4/8/16 with scans of the
 * new row, or 16 with the live range tracked), then lanes per extension
 * (32/16/8) x register slots (16/24/32) of the wide form, then resident
 * blocks per SM, then length-bucket bounds; each stage keeps the best so
 * far.  Same arguments as
 * dibella_xdrop_batch; results hold the last run's output.  Synchronises
 * `stream`; refused (EINVAL) while `stream` is capturing.  *best_ms_out and
 * *n_tried_out (either may be NULL) receive the winner's time and the number
 * of schedules timed.  The paper has no tuner; its Sec. 9 names the cost
 * differences (read length, X-drop early exit) this one adapts to. */
int dibella_autotune(const uint32_t* packed_words, const int64_t* read_word_offsets,
                     const int32_t* read_lengths, int64_t n_reads, const dibella_pair_t* pairs,
                     int64_t n_pairs, int32_t k, dibella_scoring_t scoring, dibella_result_t* results,
                     void* workspace, int64_t workspace_bytes, void* stream, int32_t repeats,
                     dibella_schedule_t* best_out, float* best_ms_out, int32_t* n_tried_out);

/* ---- diagnostics ------------------------------------------------------ */
/* Phase timing: when enabled, dibella_xdrop_batch records CUDA events on
 * `stream` at nine points around its phases.  Under
 * stream capture they are recorded as external events, so a replayed CUDA
 * graph records them too.  dibella_phase_times() synchronises on the last
 * event and writes up to n_max phase durations in ms: queueing (expand, scan,
 * scatter), narrow form (first pass), second narrow pass (0 without one),
 * first wide launch, mid form (0 without one), the wide launch on the
 * escalations, the slot ladder with the CTA and global forms, combine;
 * returns the count written (8 after a batch).  Enable it before any capture
 * (it creates the events). */
int dibella_enable_phase_timing(int enable);
int dibella_phase_times(float* ms_out, int n_max);

/* Counters of the last batch run with `workspace` (synchronises `stream`):
 * out[0] extensions routed narrow, out[1] routed wide, out[2..4] extensions
 * that outgrew the narrow / wide / CTA (shared-memory) form, out[5] band
 * overflows, out[6..9] evaluated cells of the extensions finished by the
 * narrow, wide (register or packed, all launches), CTA and global-band
 * forms, out[10] and out[11] the part of out[7] finished by the wide launch
 * on the escalations and by the slot-ladder rungs, out[12] the cells of the
 * extensions finished by the mid form, out[13] extensions that outgrew the
 * mid form, out[14] the cells the narrow and mid forms evaluated for the
 * extensions they handed on (restarted from the origin by the wider form or
 * the second narrow pass, so evaluated twice; not part of the cells of any
 * result), out[15] the extensions the first narrow pass handed to the
 * second.  Returns the number written (<= n_max, at most 16), or a negative
 * status. */
int dibella_batch_counters(const void* workspace, void* stream, int64_t* out, int n_max);

/* Number of kernels the calling thread's last dibella_xdrop_batch (or _host /
 * _noalloc) launched: queueing, every extension form (launched even when its
 * queue is empty) and combine.  Host-side count; no device work, no errors.
 * The paper has no counterpart: it reports the GPU work of a batch. */
int dibella_last_launch_count(void);

/* Per-warp clock of one extension launch, for the load balance of the
 * persistent queues (the paper measures the same imbalance as max/avg time
 * over ranks, Sec. 9): after dibella_enable_warp_clock(launch) with launch =
 * 1 narrow form, 2 first wide launch, 3 mid form, 4 wide launch on the
 * escalations (0 = off), every later batch has each warp of that launch write
 * the GPU's global timer (ns) when it starts and when it finds its queue
 * empty and leaves (launch 5: the second narrow pass).  dibella_warp_clock synchronises the device and copies
 * the last clocked launch's (start, end) pairs, 2 x uint64 per warp, for at
 * most max_warps warps (65536 at most are clocked); returns the number of
 * warps written, or a negative status.  One clock array serves the process:
 * clock one batch at a time.  The paper has no counterpart: a measurement. */
int dibella_enable_warp_clock(int launch);
int dibella_warp_clock(uint64_t* out, int max_warps);

/* Measured integer throughput of one instruction class, the ceiling the
 * extension kernels' cell rates are compared with: every thread of a grid
 * that fills each SM to its occupancy limit runs 8 independent chains of
 * op_class for `iters` iterations (one untimed launch first, then one timed
 * with CUDA events on `stream`).  Classes: 0 integer add (two dependent
 * adds, 2 ops), 1 IMNMX (max then min, 2 ops), 2 int16x2 add-then-max (DPX,
 * 2 instructions x 2 halves x 2 ops), 3 int16x2 three-way min and max (same
 * count), 4 one int32 DP cell with the 8 ops of the cell convention
 * (diagonal compare, select, add; gap max, add; final max; prune compare,
 * select).  Writes lane-ops per second to *ops_per_s_out and the timed
 * launch's duration to *ms_out (may be NULL).  Synchronous; EINVAL outside
 * 0 <= op_class <= 4, 1 <= iters <= 2^30, or while `stream` is capturing.
 * The paper has no counterpart: this is measurement infrastructure. */
int dibella_int_peak(int32_t op_class, int64_t iters, double* ops_per_s_out, double* ms_out, void* stream);

/* Bounds record of the debug build (libdibella_debug.so, compiled with
 * DIBELLA_BOUNDS_CHECK): its X-drop kernels check every packed-store word
 * they read, every per-thread shared-memory slot, queue push, item index and
 * global-band slot; a failed check is recorded (the first one's code, index
 * and limit, and a count) and the access skipped, never trapped.  Writes
 * out[0..3] = code (0 = clean; 1 shared slot, 2 queue push, 3 item index,
 * 4 store word, 5 global band slot), index, limit, count; clears the record
 * when reset != 0.  Synchronises the device.  Returns 1 in the debug build,
 * 0 (and zeros) in the release build, or a negative status. */
int dibella_bounds_check(int64_t* out, int reset);

/* Text of the last CUDA error seen by this thread's calls ("" if none). */
const char* dibella_last_error(void);
/* Library version string. */
const char* dibella_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DIBELLA_H_ */
