// Host-side read packer: ASCII reads -> 2-bit dual-orientation store.
//
// diBELLA Sec. 3 encodes every base of the four-letter alphabet in 2 bits.
// The store keeps, per read, a forward copy and a reverse-complement copy so
// that the extension kernels read every sequence in ascending word order
// (the layout is specified in include/dibella.h).

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/dibella.h"

namespace {

constexpr int64_t kPadWords = 8;

inline int64_t copy_words(int64_t len) { return ((len + 15) / 16 + 3) / 4 * 4; }

// 2-bit code of an ASCII base, or -1.
inline int code_of(unsigned char c) {
  switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
  }
}

}  // namespace

extern "C" int dibella_packed_words(const int64_t* ascii_offsets, int64_t n_reads,
                                    int64_t* n_words_out) {
  if (n_reads < 0 || n_words_out == nullptr || (n_reads > 0 && ascii_offsets == nullptr))
    return DIBELLA_EINVAL;
  int64_t words = kPadWords;
  for (int64_t r = 0; r < n_reads; ++r) {
    const int64_t len = ascii_offsets[r + 1] - ascii_offsets[r];
    if (len < 0 || len > DIBELLA_MAX_READ_LEN) return DIBELLA_EINVAL;
    words += 2 * copy_words(len);
  }
  *n_words_out = words + kPadWords;
  return DIBELLA_OK;
}

extern "C" int dibella_pack_reads(const char* ascii, const int64_t* ascii_offsets,
                                  int64_t n_reads, uint32_t* packed_words,
                                  int64_t* read_word_offsets, int32_t* read_lengths,
                                  int64_t* bad_index, int32_t n_threads) {
  int64_t total = 0;
  const int rc = dibella_packed_words(ascii_offsets, n_reads, &total);
  if (rc != DIBELLA_OK) return rc;
  if (packed_words == nullptr || (n_reads > 0 && (ascii == nullptr || read_word_offsets == nullptr ||
                                                  read_lengths == nullptr)))
    return DIBELLA_EINVAL;

  std::vector<int64_t> offs((size_t)n_reads);
  int64_t w = kPadWords;
  for (int64_t r = 0; r < n_reads; ++r) {
    offs[(size_t)r] = w;
    w += 2 * copy_words(ascii_offsets[r + 1] - ascii_offsets[r]);
  }

  std::atomic<int64_t> first_bad(INT64_MAX);
  std::atomic<int64_t> next(0);
  auto worker = [&]() {
    for (;;) {
      const int64_t r = next.fetch_add(1);
      if (r >= n_reads) return;
      const char* s = ascii + ascii_offsets[r];
      const int64_t len = ascii_offsets[r + 1] - ascii_offsets[r];
      const int64_t cw = copy_words(len);
      uint32_t* fwd = packed_words + offs[(size_t)r];
      uint32_t* rev = fwd + cw;
      std::memset(fwd, 0, (size_t)(2 * cw) * sizeof(uint32_t));
      for (int64_t q = 0; q < len; ++q) {
        const int c = code_of((unsigned char)s[q]);
        if (c < 0) {
          int64_t cur = first_bad.load();
          const int64_t idx = ascii_offsets[r] + q;
          while (idx < cur && !first_bad.compare_exchange_weak(cur, idx)) {
          }
          break;
        }
        fwd[q >> 4] |= (uint32_t)c << (2 * (q & 15));
        const int64_t rq = len - 1 - q;  // position in the reverse complement
        rev[rq >> 4] |= (uint32_t)(3 - c) << (2 * (rq & 15));
      }
    }
  };
  int threads = n_threads > 0 ? n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
  threads = (int)std::min<int64_t>(threads, std::max<int64_t>(1, n_reads));
  if (threads <= 1) {
    worker();
  } else {
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t) pool.emplace_back(worker);
    for (auto& th : pool) th.join();
  }
  if (first_bad.load() != INT64_MAX) {
    if (bad_index) *bad_index = first_bad.load();
    return DIBELLA_EBASE;
  }
  std::memset(packed_words, 0, kPadWords * sizeof(uint32_t));
  std::memset(packed_words + total - kPadWords, 0, kPadWords * sizeof(uint32_t));
  for (int64_t r = 0; r < n_reads; ++r) {
    read_word_offsets[r] = offs[(size_t)r];
    read_lengths[r] = (int32_t)(ascii_offsets[r + 1] - ascii_offsets[r]);
  }
  return DIBELLA_OK;
}
