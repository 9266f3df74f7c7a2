// Seeded synthetic long-read workloads: genome, reads, candidate pairs, seeds.
//
// This module produces INPUTS only; it contains none of the alignment
// arithmetic.  Both the CUDA path and the CPU oracle consume what it writes.
//
// Shapes follow the paper's long-read workloads (diBELLA Sec. 5: PacBio
// E. coli at 30x, mean read length ~10 kb; Sec. 1: long reads of 1-100 kb
// with 5-35% error) with these generation rules:
//   * genome: uniform random ACGT; optionally repeat families (each copy the
//     family consensus with a given substitution divergence) and exact tandem
//     arrays, all placed without overlap;
//   * reads: template length from the configured distribution (capped at the
//     genome length), uniform start (no wrap), fair-coin strand; per template
//     base with probability e an error: substitution (to one of the 3 other
//     bases), insertion (emit the base, then one uniform random base) or
//     deletion (skip the base), in the configured proportions; reads are drawn
//     until the template bases reach coverage x genome length;
//   * candidate pairs (Sec. 4 stages 1-3 done exactly on the CPU): canonical
//     k-mers (min of the 2-bit code and its reverse complement's, A<C<G<T),
//     multiplicity counted over all read positions, k-mers with multiplicity
//     in [mult_lo, mult_hi] retained (Sec. 3 filtering), every pair of
//     distinct reads sharing a retained k-mer becomes a candidate (Sec. 8,
//     Algorithm 1 without the multi-node owner rule); strand = XOR of the two
//     occurrences' orientations;
//   * seeds per pair (Sec. 8 seed constraints; Sec. 5 options: one seed, all
//     seeds at least k apart, seeds at least 1,000 bp apart): sorted by
//     (pos_a, pos_b), the first is seed 0, each next seed is the first whose
//     pos_a is at least min_seed_gap (0 = k) past the previous seed's, up to
//     max_seeds.
// All random draws come from std::mt19937_64: the master stream draws read
// lengths/starts/strands/error rates; each read's bases use their own stream
// seeded from (seed, read index), so output does not depend on thread count.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <set>
#include <string>
#include <thread>
#include <vector>

extern "C" {

typedef struct {
  uint64_t seed;
  int64_t genome_len;
  int32_t repeat_families;     // number of repeat families (0 = none)
  int32_t repeat_unit_len;     // length of each family consensus
  int32_t repeat_copies;       // copies placed per family
  int32_t tandem_period_lo;    // tandem unit period range
  int32_t tandem_period_hi;
  int32_t tandem_array_lo;     // tandem array length range
  int32_t tandem_array_hi;
  int32_t len_dist;            // 0 uniform int [len_a, len_b]; 1 lognormal(mean, sd)
                               // clipped to [len_a, len_b]; 2 log-uniform [len_a, len_b]
  int64_t tandem_bases;        // total bases of tandem arrays (0 = none)
  double repeat_divergence;    // substitution rate of each copy vs its consensus
  double coverage;
  double len_a, len_b, len_mean, len_sd;
  double err_lo, err_hi;       // per-read error rate ~ U[err_lo, err_hi]
  double p_sub, p_ins, p_del;  // error type proportions (sum to 1)
  int32_t k;
  int32_t mult_lo, mult_hi;
  int32_t max_seeds;
  int32_t n_threads;
  int32_t min_seed_gap;        // least pos_a distance between seeds of a pair (0 = k)
  int32_t pairs_mode;          // 0 every candidate pair; 1 none (reads only); 2 the candidate
                               // pairs whose read_a lies in one of the ranges below
  int64_t n_ranges;            // pairs_mode 2: number of half-open read-id ranges
  const int64_t* ranges;       // pairs_mode 2: lo0, hi0, lo1, hi1, ... (ascending, disjoint)
} wl_config_t;

typedef struct {
  uint32_t read_a, read_b, pos_a, pos_b;
  uint8_t strand;
  uint8_t pad[3];
  uint32_t seed_id;
} wl_pair_t;

}  // extern "C"

static_assert(sizeof(wl_pair_t) == 24, "pair record layout");

namespace {

const char kBases[4] = {'A', 'C', 'G', 'T'};

uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

int base_code(char c) {
  switch (c) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    default: return 3;
  }
}

char comp(char c) { return kBases[3 - base_code(c)]; }

struct Workload {
  std::string genome;
  std::string reads;               // concatenated ASCII
  std::vector<int64_t> offsets;    // n_reads + 1
  std::vector<int64_t> tmpl_start; // template start in the genome
  std::vector<int32_t> tmpl_len;
  std::vector<uint8_t> tmpl_strand;
  std::vector<wl_pair_t> pairs;
  int64_t n_instances = 0;
  int64_t n_retained_kmers = 0;
  int64_t n_candidate_pairs = 0;
};

int n_workers(const wl_config_t& c) {
  int t = c.n_threads;
  if (t <= 0) t = (int)std::max(1u, std::thread::hardware_concurrency());
  return t;
}

template <class F>
void parallel_for(int64_t n, int threads, F&& f) {
  if (threads <= 1 || n < 2) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t)
    pool.emplace_back([&]() {
      for (;;) {
        int64_t i = next.fetch_add(1);
        if (i >= n) return;
        f(i);
      }
    });
  for (auto& th : pool) th.join();
}

void make_genome(const wl_config_t& c, Workload& w) {
  std::mt19937_64 rng(splitmix64(c.seed ^ 0x47454E4F4D45ull));
  w.genome.resize((size_t)c.genome_len);
  for (auto& ch : w.genome) ch = kBases[rng() & 3];

  // Repeat families and tandem arrays, placed without overlap.
  struct Element { int64_t len; int kind; int family; };
  std::vector<Element> elems;
  std::vector<std::string> consensus;
  for (int f = 0; f < c.repeat_families; ++f) {
    std::string s((size_t)c.repeat_unit_len, 'A');
    for (auto& ch : s) ch = kBases[rng() & 3];
    consensus.push_back(s);
    for (int cp = 0; cp < c.repeat_copies; ++cp) elems.push_back({c.repeat_unit_len, 0, f});
  }
  int64_t tandem_total = 0;
  while (tandem_total < c.tandem_bases) {
    std::uniform_int_distribution<int64_t> alen(c.tandem_array_lo, c.tandem_array_hi);
    int64_t L = alen(rng);
    elems.push_back({L, 1, -1});
    tandem_total += L;
  }
  std::set<std::pair<int64_t, int64_t>> placed;  // [start, end)
  std::uniform_real_distribution<double> u01(0.0, 1.0);
  for (const Element& e : elems) {
    if (e.len >= c.genome_len) continue;
    std::uniform_int_distribution<int64_t> pos(0, c.genome_len - e.len);
    for (int attempt = 0; attempt < 1000; ++attempt) {
      int64_t s = pos(rng), t = s + e.len;
      auto it = placed.lower_bound({s, INT64_MIN});
      bool clash = false;
      if (it != placed.end() && it->first < t) clash = true;
      if (it != placed.begin()) {
        auto prev = std::prev(it);
        if (prev->second > s) clash = true;
      }
      if (clash) continue;
      placed.insert({s, t});
      if (e.kind == 0) {
        const std::string& cons = consensus[(size_t)e.family];
        for (int64_t q = 0; q < e.len; ++q) {
          char ch = cons[(size_t)q];
          if (u01(rng) < c.repeat_divergence) {
            int other = (base_code(ch) + 1 + (int)(rng() % 3)) & 3;
            ch = kBases[other];
          }
          w.genome[(size_t)(s + q)] = ch;
        }
      } else {
        std::uniform_int_distribution<int> per(c.tandem_period_lo, c.tandem_period_hi);
        int p = per(rng);
        std::string unit((size_t)p, 'A');
        for (auto& ch : unit) ch = kBases[rng() & 3];
        for (int64_t q = 0; q < e.len; ++q) w.genome[(size_t)(s + q)] = unit[(size_t)(q % p)];
      }
      break;
    }
  }
}

void make_reads(const wl_config_t& c, Workload& w) {
  std::mt19937_64 rng(splitmix64(c.seed ^ 0x52454144ull));
  std::uniform_real_distribution<double> u01(0.0, 1.0);
  const double target = c.coverage * (double)c.genome_len;
  double total = 0;
  std::vector<double> err;
  const double sigma2 = std::log(1.0 + (c.len_sd / std::max(c.len_mean, 1.0)) * (c.len_sd / std::max(c.len_mean, 1.0)));
  const double mu = std::log(std::max(c.len_mean, 1.0)) - sigma2 / 2.0;
  std::lognormal_distribution<double> lognorm(mu, std::sqrt(sigma2));
  while (total < target) {
    int64_t L;
    if (c.len_dist == 0) {
      std::uniform_int_distribution<int64_t> ud((int64_t)c.len_a, (int64_t)c.len_b);
      L = ud(rng);
    } else if (c.len_dist == 1) {
      double x = lognorm(rng);
      x = std::min(std::max(x, c.len_a), c.len_b);
      L = (int64_t)std::llround(x);
    } else {
      double x = std::exp(std::log(c.len_a) + u01(rng) * (std::log(c.len_b) - std::log(c.len_a)));
      L = (int64_t)std::llround(x);
    }
    L = std::min<int64_t>(std::max<int64_t>(L, 1), c.genome_len);
    std::uniform_int_distribution<int64_t> sd(0, c.genome_len - L);
    const int64_t start = sd(rng);
    const uint8_t strand = (uint8_t)(rng() & 1);
    const double e = c.err_lo + (c.err_hi - c.err_lo) * u01(rng);
    w.tmpl_start.push_back(start);
    w.tmpl_len.push_back((int32_t)L);
    w.tmpl_strand.push_back(strand);
    err.push_back(e);
    total += (double)L;
  }
  const int64_t n = (int64_t)w.tmpl_len.size();
  std::vector<std::string> seqs((size_t)n);
  parallel_for(n, n_workers(c), [&](int64_t r) {
    std::mt19937_64 g(splitmix64(c.seed * 0x9E3779B97F4A7C15ull + (uint64_t)r + 1));
    std::uniform_real_distribution<double> uu(0.0, 1.0);
    const int64_t L = w.tmpl_len[(size_t)r];
    std::string tmpl = w.genome.substr((size_t)w.tmpl_start[(size_t)r], (size_t)L);
    if (w.tmpl_strand[(size_t)r]) {
      std::reverse(tmpl.begin(), tmpl.end());
      for (auto& ch : tmpl) ch = comp(ch);
    }
    const double e = err[(size_t)r];
    const double ps = e * c.p_sub, pi = e * (c.p_sub + c.p_ins);
    std::string out;
    out.reserve((size_t)(L + L / 4 + 8));
    for (char ch : tmpl) {
      const double x = uu(g);
      if (x < ps) {
        int other = (base_code(ch) + 1 + (int)(g() % 3)) & 3;
        out.push_back(kBases[other]);
      } else if (x < pi) {
        out.push_back(ch);
        out.push_back(kBases[g() & 3]);
      } else if (x < e) {
        // deletion: skip the template base
      } else {
        out.push_back(ch);
      }
    }
    seqs[(size_t)r] = std::move(out);
  });
  w.offsets.assign((size_t)n + 1, 0);
  for (int64_t r = 0; r < n; ++r) w.offsets[(size_t)r + 1] = w.offsets[(size_t)r] + (int64_t)seqs[(size_t)r].size();
  w.reads.resize((size_t)w.offsets[(size_t)n]);
  parallel_for(n, n_workers(c), [&](int64_t r) {
    std::memcpy(&w.reads[(size_t)w.offsets[(size_t)r]], seqs[(size_t)r].data(), seqs[(size_t)r].size());
  });
}

struct Instance {
  uint64_t canon;
  uint32_t rid;
  uint32_t pos_orient;  // pos | orientation << 31
};

struct RawPair {
  uint32_t ra, rb, pa, pb;
  uint8_t strand;
};

void select_seeds(const wl_config_t& c, Workload& w, std::vector<std::vector<RawPair>>& emitted);

void make_pairs(const wl_config_t& c, Workload& w) {
  const int k = c.k;
  const int threads = n_workers(c);
  const int64_t n = (int64_t)w.offsets.size() - 1;
  const uint64_t mask = (k == 32) ? ~0ull : ((1ull << (2 * k)) - 1);
  const int kParts = 1024;
  auto part_of = [&](uint64_t canon) { return (int)(splitmix64(canon) % kParts); };

  // Pass 1: count instances per partition, per read (so pass 2 can scatter in parallel).
  std::vector<std::vector<int64_t>> cnt((size_t)n);
  parallel_for(n, threads, [&](int64_t r) {
    std::vector<int64_t> local(kParts, 0);
    const char* s = w.reads.data() + w.offsets[(size_t)r];
    const int64_t L = w.offsets[(size_t)r + 1] - w.offsets[(size_t)r];
    uint64_t fw = 0, rc = 0;
    for (int64_t p = 0; p < L; ++p) {
      const uint64_t b = (uint64_t)base_code(s[p]);
      fw = ((fw << 2) | b) & mask;
      rc = (rc >> 2) | ((3 - b) << (2 * (k - 1)));
      if (p + 1 >= k) local[(size_t)part_of(std::min(fw, rc))] += 1;
    }
    cnt[(size_t)r] = std::move(local);
  });
  std::vector<int64_t> part_start(kParts + 1, 0);
  for (int64_t r = 0; r < n; ++r)
    for (int q = 0; q < kParts; ++q) part_start[(size_t)q + 1] += cnt[(size_t)r][(size_t)q];
  for (int q = 0; q < kParts; ++q) part_start[(size_t)q + 1] += part_start[(size_t)q];
  const int64_t total = part_start[kParts];
  w.n_instances = total;
  // Per-read write cursors into each partition.
  std::vector<int64_t> cursor(kParts);
  for (int q = 0; q < kParts; ++q) cursor[(size_t)q] = part_start[(size_t)q];
  for (int64_t r = 0; r < n; ++r)
    for (int q = 0; q < kParts; ++q) {
      const int64_t v = cnt[(size_t)r][(size_t)q];
      cnt[(size_t)r][(size_t)q] = cursor[(size_t)q];
      cursor[(size_t)q] += v;
    }
  std::vector<Instance> inst((size_t)total);
  parallel_for(n, threads, [&](int64_t r) {
    std::vector<int64_t>& cur = cnt[(size_t)r];
    const char* s = w.reads.data() + w.offsets[(size_t)r];
    const int64_t L = w.offsets[(size_t)r + 1] - w.offsets[(size_t)r];
    uint64_t fw = 0, rc = 0;
    for (int64_t p = 0; p < L; ++p) {
      const uint64_t b = (uint64_t)base_code(s[p]);
      fw = ((fw << 2) | b) & mask;
      rc = (rc >> 2) | ((3 - b) << (2 * (k - 1)));
      if (p + 1 >= k) {
        const uint64_t canon = std::min(fw, rc);
        const uint32_t orient = fw <= rc ? 0u : 1u;
        const uint32_t pos = (uint32_t)(p + 1 - k);
        inst[(size_t)cur[(size_t)part_of(canon)]++] = {canon, (uint32_t)r, pos | (orient << 31)};
      }
    }
  });
  cnt.clear();
  cnt.shrink_to_fit();

  // Pass 2: per partition sort, multiplicity filter, pair emission.
  std::vector<std::vector<RawPair>> emitted((size_t)kParts);
  std::vector<int64_t> retained((size_t)kParts, 0);
  parallel_for(kParts, threads, [&](int64_t q) {
    Instance* b = inst.data() + part_start[(size_t)q];
    Instance* e = inst.data() + part_start[(size_t)q + 1];
    std::sort(b, e, [](const Instance& x, const Instance& y) {
      if (x.canon != y.canon) return x.canon < y.canon;
      if (x.rid != y.rid) return x.rid < y.rid;
      return x.pos_orient < y.pos_orient;
    });
    std::vector<RawPair>& out = emitted[(size_t)q];
    for (Instance* run = b; run < e;) {
      Instance* end = run + 1;
      while (end < e && end->canon == run->canon) ++end;
      const int64_t mult = end - run;
      if (mult >= c.mult_lo && mult <= c.mult_hi) {
        retained[(size_t)q] += 1;
        for (Instance* x = run; x < end; ++x)
          for (Instance* y = x + 1; y < end; ++y) {
            if (x->rid == y->rid) continue;
            // sorted by rid: x->rid < y->rid
            RawPair p;
            p.ra = x->rid;
            p.rb = y->rid;
            p.pa = x->pos_orient & 0x7FFFFFFFu;
            p.pb = y->pos_orient & 0x7FFFFFFFu;
            p.strand = (uint8_t)((x->pos_orient >> 31) ^ (y->pos_orient >> 31));
            out.push_back(p);
          }
      }
      run = end;
    }
  });
  inst.clear();
  inst.shrink_to_fit();
  for (int q = 0; q < kParts; ++q) w.n_retained_kmers += retained[(size_t)q];

  select_seeds(c, w, emitted);
}

// Group the occurrence pairs by read pair and apply the seed rule (Sec. 8 seed
// constraints, Sec. 5 options); appends the records to w.pairs, sorted by
// (read_a, read_b, seed_id).  Consumes `emitted`.
void select_seeds(const wl_config_t& c, Workload& w, std::vector<std::vector<RawPair>>& emitted) {
  const int k = c.k;
  const int threads = n_workers(c);
  const int kParts = 1024;
  // Group by read pair: partition pairs by read_a so each group sorts independently.
  std::vector<std::vector<RawPair>> by_a((size_t)kParts);
  for (auto& v : emitted) {
    for (const RawPair& p : v) by_a[(size_t)(p.ra % kParts)].push_back(p);
    std::vector<RawPair>().swap(v);
  }
  std::vector<std::vector<wl_pair_t>> chosen((size_t)kParts);
  std::vector<int64_t> n_cand((size_t)kParts, 0);
  parallel_for(kParts, threads, [&](int64_t q) {
    auto& v = by_a[(size_t)q];
    std::sort(v.begin(), v.end(), [](const RawPair& x, const RawPair& y) {
      if (x.ra != y.ra) return x.ra < y.ra;
      if (x.rb != y.rb) return x.rb < y.rb;
      if (x.pa != y.pa) return x.pa < y.pa;
      if (x.pb != y.pb) return x.pb < y.pb;
      return x.strand < y.strand;
    });
    for (size_t s = 0; s < v.size();) {
      size_t t = s + 1;
      while (t < v.size() && v[t].ra == v[s].ra && v[t].rb == v[s].rb) ++t;
      n_cand[(size_t)q] += 1;
      int taken = 0;
      int64_t last_pa = -1;
      const int64_t gap = c.min_seed_gap > 0 ? c.min_seed_gap : k;
      for (size_t u = s; u < t && taken < c.max_seeds; ++u) {
        if (taken > 0 && (int64_t)v[u].pa < last_pa + gap) continue;
        wl_pair_t out;
        std::memset(&out, 0, sizeof(out));
        out.read_a = v[u].ra;
        out.read_b = v[u].rb;
        out.pos_a = v[u].pa;
        out.pos_b = v[u].pb;
        out.strand = v[u].strand;
        out.seed_id = (uint32_t)taken;
        chosen[(size_t)q].push_back(out);
        last_pa = v[u].pa;
        ++taken;
      }
      s = t;
    }
    std::vector<RawPair>().swap(v);
  });
  for (int q = 0; q < kParts; ++q) w.n_candidate_pairs += n_cand[(size_t)q];
  for (auto& v : chosen) w.pairs.insert(w.pairs.end(), v.begin(), v.end());
  std::sort(w.pairs.begin(), w.pairs.end(), [](const wl_pair_t& x, const wl_pair_t& y) {
    if (x.read_a != y.read_a) return x.read_a < y.read_a;
    if (x.read_b != y.read_b) return x.read_b < y.read_b;
    return x.seed_id < y.seed_id;
  });
}

// The candidate pairs whose read_a lies in the configured read-id ranges,
// without indexing every k-mer of the read set: the same pairs and seeds as
// make_pairs, restricted to those read_a (memory grows with the ranges' k-mers,
// not with the whole read set; the multiplicities still count every read).
//   1. the canonical codes of the range reads, sorted and unique (the set S);
//   2. a 2^32-bit filter of S by hash; every occurrence of every read whose
//      code passes the filter and is found in S counts towards its code;
//   3. the occurrences of the retained codes of S (multiplicity in
//      [mult_lo, mult_hi]) are collected and sorted by (code, read, position);
//   4. per code, every occurrence pair of distinct reads whose smaller read
//      lies in a range becomes an occurrence pair; seed selection as before.
bool in_ranges(const wl_config_t& c, uint32_t r) {
  for (int64_t q = 0; q < c.n_ranges; ++q)
    if ((int64_t)r >= c.ranges[2 * q] && (int64_t)r < c.ranges[2 * q + 1]) return true;
  return false;
}

template <class F>
void for_each_kmer(const Workload& w, int64_t r, int k, F&& f) {
  const uint64_t mask = (k == 32) ? ~0ull : ((1ull << (2 * k)) - 1);
  const char* s = w.reads.data() + w.offsets[(size_t)r];
  const int64_t L = w.offsets[(size_t)r + 1] - w.offsets[(size_t)r];
  uint64_t fw = 0, rc = 0;
  for (int64_t p = 0; p < L; ++p) {
    const uint64_t b = (uint64_t)base_code(s[p]);
    fw = ((fw << 2) | b) & mask;
    rc = (rc >> 2) | ((3 - b) << (2 * (k - 1)));
    if (p + 1 >= k) f(std::min(fw, rc), fw <= rc ? 0u : 1u, (uint32_t)(p + 1 - k));
  }
}

void make_pairs_ranges(const wl_config_t& c, Workload& w) {
  const int k = c.k;
  const int threads = n_workers(c);
  const int64_t n = (int64_t)w.offsets.size() - 1;
  std::vector<int64_t> rlist;
  for (int64_t q = 0; q < c.n_ranges; ++q)
    for (int64_t r = std::max<int64_t>(0, c.ranges[2 * q]); r < std::min<int64_t>(n, c.ranges[2 * q + 1]); ++r)
      rlist.push_back(r);
  // 1. codes of the range reads
  std::vector<std::vector<uint64_t>> local((size_t)rlist.size());
  parallel_for((int64_t)rlist.size(), threads, [&](int64_t i) {
    std::vector<uint64_t>& v = local[(size_t)i];
    for_each_kmer(w, rlist[(size_t)i], k, [&](uint64_t code, uint32_t, uint32_t) { v.push_back(code); });
  });
  std::vector<uint64_t> S;
  for (auto& v : local) {
    S.insert(S.end(), v.begin(), v.end());
    std::vector<uint64_t>().swap(v);
  }
  std::sort(S.begin(), S.end());
  S.erase(std::unique(S.begin(), S.end()), S.end());
  // 2. filter, then count every occurrence of the codes of S over all reads
  const int kFilterBits = 32;
  std::vector<uint64_t> filter((size_t)1 << (kFilterBits - 6), 0);
  auto fbit = [&](uint64_t code) { return splitmix64(code) >> (64 - kFilterBits); };
  for (uint64_t code : S) {
    const uint64_t b = fbit(code);
    filter[(size_t)(b >> 6)] |= 1ull << (b & 63);
  }
  auto find = [&](uint64_t code) -> int64_t {
    const uint64_t b = fbit(code);
    if (!((filter[(size_t)(b >> 6)] >> (b & 63)) & 1ull)) return -1;
    auto it = std::lower_bound(S.begin(), S.end(), code);
    return (it != S.end() && *it == code) ? (int64_t)(it - S.begin()) : -1;
  };
  std::vector<uint32_t> cnt(S.size(), 0);
  std::atomic<int64_t> total(0);
  parallel_for(n, threads, [&](int64_t r) {
    int64_t here = 0;
    for_each_kmer(w, r, k, [&](uint64_t code, uint32_t, uint32_t) {
      ++here;
      const int64_t i = find(code);
      if (i >= 0) __atomic_fetch_add(&cnt[(size_t)i], 1u, __ATOMIC_RELAXED);
    });
    total.fetch_add(here);
  });
  w.n_instances = total.load();
  // 3. occurrences of the retained codes of S
  auto retained = [&](int64_t i) { return cnt[(size_t)i] >= (uint32_t)c.mult_lo && cnt[(size_t)i] <= (uint32_t)c.mult_hi; };
  for (size_t i = 0; i < S.size(); ++i) w.n_retained_kmers += retained((int64_t)i) ? 1 : 0;
  std::vector<std::vector<Instance>> found((size_t)n);
  parallel_for(n, threads, [&](int64_t r) {
    for_each_kmer(w, r, k, [&](uint64_t code, uint32_t orient, uint32_t pos) {
      const int64_t i = find(code);
      if (i >= 0 && retained(i)) found[(size_t)r].push_back({code, (uint32_t)r, pos | (orient << 31)});
    });
  });
  std::vector<Instance> inst;
  for (auto& v : found) {
    inst.insert(inst.end(), v.begin(), v.end());
    std::vector<Instance>().swap(v);
  }
  std::sort(inst.begin(), inst.end(), [](const Instance& x, const Instance& y) {
    if (x.canon != y.canon) return x.canon < y.canon;
    if (x.rid != y.rid) return x.rid < y.rid;
    return x.pos_orient < y.pos_orient;
  });
  // 4. occurrence pairs whose smaller read is in a range
  std::vector<std::vector<RawPair>> emitted(1);
  for (size_t a = 0; a < inst.size();) {
    size_t e = a + 1;
    while (e < inst.size() && inst[e].canon == inst[a].canon) ++e;
    for (size_t x = a; x < e; ++x) {
      if (!in_ranges(c, inst[x].rid)) continue;
      for (size_t y = x + 1; y < e; ++y) {
        if (inst[x].rid == inst[y].rid) continue;
        RawPair p;
        p.ra = inst[x].rid;
        p.rb = inst[y].rid;
        p.pa = inst[x].pos_orient & 0x7FFFFFFFu;
        p.pb = inst[y].pos_orient & 0x7FFFFFFFu;
        p.strand = (uint8_t)((inst[x].pos_orient >> 31) ^ (inst[y].pos_orient >> 31));
        emitted[0].push_back(p);
      }
    }
    a = e;
  }
  select_seeds(c, w, emitted);
}

}  // namespace

extern "C" {

void* wl_generate(const wl_config_t* cfg) {
  if (cfg->pairs_mode < 0 || cfg->pairs_mode > 2) return nullptr;
  if (cfg->pairs_mode == 2 && (cfg->n_ranges < 0 || (cfg->n_ranges > 0 && !cfg->ranges))) return nullptr;
  Workload* w = new Workload();
  make_genome(*cfg, *w);
  make_reads(*cfg, *w);
  if (cfg->pairs_mode == 0)
    make_pairs(*cfg, *w);
  else if (cfg->pairs_mode == 2)
    make_pairs_ranges(*cfg, *w);
  return w;
}

int64_t wl_genome_len(void* h) { return (int64_t)static_cast<Workload*>(h)->genome.size(); }
const char* wl_genome(void* h) { return static_cast<Workload*>(h)->genome.data(); }
int64_t wl_n_reads(void* h) { return (int64_t)static_cast<Workload*>(h)->tmpl_len.size(); }
int64_t wl_n_bases(void* h) { return (int64_t)static_cast<Workload*>(h)->reads.size(); }
const char* wl_reads(void* h) { return static_cast<Workload*>(h)->reads.data(); }
const int64_t* wl_offsets(void* h) { return static_cast<Workload*>(h)->offsets.data(); }
const int64_t* wl_tmpl_start(void* h) { return static_cast<Workload*>(h)->tmpl_start.data(); }
const int32_t* wl_tmpl_len(void* h) { return static_cast<Workload*>(h)->tmpl_len.data(); }
const uint8_t* wl_tmpl_strand(void* h) { return static_cast<Workload*>(h)->tmpl_strand.data(); }
int64_t wl_n_pairs(void* h) { return (int64_t)static_cast<Workload*>(h)->pairs.size(); }
const wl_pair_t* wl_pairs(void* h) { return static_cast<Workload*>(h)->pairs.data(); }
int64_t wl_stat(void* h, int which) {
  Workload* w = static_cast<Workload*>(h);
  switch (which) {
    case 0: return w->n_instances;
    case 1: return w->n_retained_kmers;
    case 2: return w->n_candidate_pairs;
    default: return -1;
  }
}
void wl_free(void* h) { delete static_cast<Workload*>(h); }

}  // extern "C"
