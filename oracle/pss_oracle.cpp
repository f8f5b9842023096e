// pss_oracle.cpp — CPU oracle for Parallel Space Saving.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// CPU-baseline leg of bench.py may load this library.  It shares no code with
// the CUDA path; the one module both include is the seeded input generator
// (paper_1606_04669_gb300/gen/pss_zipf.h), which holds none of the method.
//
// Plain, slow, obviously correct, single-threaded.  Every function follows
// the paper (M. Cafaro, M. Pulimeno, I. Epicoco, G. Aloisio, "Parallel Space
// Saving on Multi and Many-Core Processors", arXiv:1606.04669):
//
//   * block decomposition of the input: Algorithm 1 (bounds left/right);
//   * sequential Space Saving per block: Section 3 (the k-counter update
//     rule) and Algorithm 1 (SpaceSaving call);
//   * combine of two summaries, including Prune(k): Algorithm 2;
//   * ParallelReduction as a binary tree over adjacent pairs: Algorithm 1;
//   * Pruned(global, n, k): Algorithm 1 with the k-majority threshold of
//     Section 3 (frequency >= floor(n/k) + 1, i.e. count * k > n).
//
// Readings of points the paper leaves open:
//   * every counter also carries an error err (Metwally et al.'s Space
//     Saving): on eviction err := the evicted count; combine adds to err the
//     same quantity it adds to the count;
//   * the evicted counter is the minimum of (count, touch) where touch is the
//     position (within the block) of the counter's last update, i.e. the
//     least recently updated counter among those with the minimum count;
//   * a summary with fewer than k counters in use has minimum m = 0;
//   * Prune(k) keeps the k largest by (count descending, item ascending);
//   * the reduction tree pairs adjacent summaries level by level and carries
//     an odd last summary up unchanged.
//
// Parity: pinned by the tests under tests/ (brute-force histograms, the
// error bounds, the counter-sum invariant, a naive scan twin of the heap,
// closed-form special cases and hand-derived examples).

#include <algorithm>
#include <cstdint>
#include <thread>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "../paper_1606_04669_gb300/gen/pss_zipf.h"

namespace {

struct Entry {
  uint64_t item, count, err;
};

// A stream summary in canonical order: count descending, item ascending.
struct Summary {
  std::vector<Entry> e;
  uint64_t m = 0;          // minimum count if k counters are in use, else 0
  uint64_t n_covered = 0;  // number of stream items the summary describes
};

bool canonical_less(const Entry& a, const Entry& b) {
  if (a.count != b.count) return a.count > b.count;
  return a.item < b.item;
}

void canonicalize(Summary& s, uint32_t k) {
  std::sort(s.e.begin(), s.e.end(), canonical_less);
  if (s.e.size() > k) s.e.resize(k);
  s.m = (s.e.size() == k) ? s.e.back().count : 0;
}

// Algorithm 1: process r owns [floor(r n / p), floor((r + 1) n / p) - 1].
uint64_t block_left(uint64_t r, uint64_t n, uint64_t p) {
  return (uint64_t)(((unsigned __int128)r * n) / p);
}

uint64_t load_item(const void* items, int width, uint64_t i) {
  if (width == 4) return ((const uint32_t*)items)[i];
  return ((const uint64_t*)items)[i];
}

// Sequential Space Saving with k counters (Section 3).  The minimum counter
// is found with an indexed binary min-heap keyed by (count, touch).
class SpaceSaving {
 public:
  explicit SpaceSaving(uint32_t k) : k_(k) {
    c_.reserve(k);
    heap_.reserve(k);
    pos_.reserve(k);
    where_.reserve(2 * (size_t)k);
  }

  // Item x at position t of the block.
  void offer(uint64_t x, uint64_t t) {
    auto it = where_.find(x);
    if (it != where_.end()) {
      // Monitored: its estimated frequency is incremented by one.
      Counter& c = c_[it->second];
      c.count += 1;
      c.touch = t;
      sift_down(pos_[it->second]);
      return;
    }
    if (c_.size() < k_) {
      // A counter is available: it monitors x with frequency one.
      uint32_t id = (uint32_t)c_.size();
      c_.push_back(Counter{x, 1, 0, t});
      pos_.push_back((uint32_t)heap_.size());
      heap_.push_back(id);
      sift_up(pos_[id]);
      where_[x] = id;
      return;
    }
    // All counters are occupied: the counter with minimum frequency is
    // incremented by one and its item is replaced by x.
    uint32_t id = heap_[0];
    Counter& v = c_[id];
    where_.erase(v.item);
    v.err = v.count;
    v.count += 1;
    v.item = x;
    v.touch = t;
    where_[x] = id;
    sift_down(0);
  }

  Summary summary(uint64_t len) const {
    Summary s;
    s.e.reserve(c_.size());
    for (const Counter& c : c_) s.e.push_back(Entry{c.item, c.count, c.err});
    s.n_covered = len;
    canonicalize(s, k_);
    return s;
  }

 private:
  struct Counter {
    uint64_t item, count, err, touch;
  };

  bool key_less(uint32_t a, uint32_t b) const {
    if (c_[a].count != c_[b].count) return c_[a].count < c_[b].count;
    return c_[a].touch < c_[b].touch;
  }
  void swap_at(size_t i, size_t j) {
    std::swap(heap_[i], heap_[j]);
    pos_[heap_[i]] = (uint32_t)i;
    pos_[heap_[j]] = (uint32_t)j;
  }
  void sift_up(size_t i) {
    while (i > 0) {
      size_t parent = (i - 1) / 2;
      if (!key_less(heap_[i], heap_[parent])) break;
      swap_at(i, parent);
      i = parent;
    }
  }
  void sift_down(size_t i) {
    const size_t n = heap_.size();
    for (;;) {
      size_t l = 2 * i + 1, r = l + 1, best = i;
      if (l < n && key_less(heap_[l], heap_[best])) best = l;
      if (r < n && key_less(heap_[r], heap_[best])) best = r;
      if (best == i) return;
      swap_at(i, best);
      i = best;
    }
  }

  uint32_t k_;
  std::vector<Counter> c_;
  std::vector<uint32_t> heap_;  // counter ids, heap-ordered by (count, touch)
  std::vector<uint32_t> pos_;   // counter id -> index in heap_
  std::unordered_map<uint64_t, uint32_t> where_;
};

Summary space_saving(const void* items, int width, uint64_t left, uint64_t len, uint32_t k) {
  SpaceSaving ss(k);
  for (uint64_t t = 0; t < len; ++t) ss.offer(load_item(items, width, left + t), t);
  return ss.summary(len);
}

// Algorithm 2: combine(S1, S2, k).
Summary combine(const Summary& s1, const Summary& s2, uint32_t k) {
  const uint64_t m1 = s1.m, m2 = s2.m;
  std::unordered_map<uint64_t, size_t> in2;
  in2.reserve(2 * s2.e.size() + 1);
  for (size_t j = 0; j < s2.e.size(); ++j) in2[s2.e[j].item] = j;
  std::vector<bool> removed(s2.e.size(), false);
  Summary sc;
  sc.e.reserve(s1.e.size() + s2.e.size());
  for (const Entry& c1 : s1.e) {
    auto it = in2.find(c1.item);
    if (it != in2.end()) {
      const Entry& c2 = s2.e[it->second];
      sc.e.push_back(Entry{c1.item, c1.count + c2.count, c1.err + c2.err});
      removed[it->second] = true;
    } else {
      sc.e.push_back(Entry{c1.item, c1.count + m2, c1.err + m2});
    }
  }
  for (size_t j = 0; j < s2.e.size(); ++j) {
    if (removed[j]) continue;
    const Entry& c2 = s2.e[j];
    sc.e.push_back(Entry{c2.item, c2.count + m1, c2.err + m1});
  }
  sc.n_covered = s1.n_covered + s2.n_covered;
  canonicalize(sc, k);  // Prune(k)
  return sc;
}

// Algorithm 1's ParallelReduction as a binary tree over adjacent pairs;
// returns every level, level 0 being the p block summaries.
std::vector<std::vector<Summary>> reduction_tree(std::vector<Summary> level0, uint32_t k) {
  std::vector<std::vector<Summary>> levels;
  levels.push_back(std::move(level0));
  while (levels.back().size() > 1) {
    const std::vector<Summary>& cur = levels.back();
    std::vector<Summary> next;
    next.reserve((cur.size() + 1) / 2);
    for (size_t i = 0; i + 1 < cur.size(); i += 2) next.push_back(combine(cur[i], cur[i + 1], k));
    if (cur.size() % 2) next.push_back(cur.back());
    levels.push_back(std::move(next));
  }
  return levels;
}

// Pruned(global, n, k): the entries whose count exceeds n / k.
Summary pruned(const Summary& s, uint64_t n, uint32_t k) {
  Summary out;
  out.m = s.m;
  out.n_covered = s.n_covered;
  for (const Entry& e : s.e)
    if ((unsigned __int128)e.count * k > (unsigned __int128)n) out.e.push_back(e);
  return out;
}

void write_summary(const Summary& s, uint64_t* item, uint64_t* count, uint64_t* err) {
  for (size_t i = 0; i < s.e.size(); ++i) {
    item[i] = s.e[i].item;
    count[i] = s.e[i].count;
    err[i] = s.e[i].err;
  }
}

Summary read_summary(const uint64_t* item, const uint64_t* count, const uint64_t* err,
                     uint32_t size, uint64_t m, uint64_t n_covered) {
  Summary s;
  s.e.resize(size);
  for (uint32_t i = 0; i < size; ++i) s.e[i] = Entry{item[i], count[i], err[i]};
  s.m = m;
  s.n_covered = n_covered;
  return s;
}

}  // namespace

extern "C" {

int oracle_abi_version(void) { return 1; }

// Algorithm 1 block bounds: [*left, *right_excl) for rank r of p over n items.
void oracle_block_bounds(uint64_t n, uint64_t p, uint64_t r, uint64_t* left, uint64_t* right_excl) {
  *left = block_left(r, n, p);
  *right_excl = block_left(r + 1, n, p);
}

// Sequential Space Saving over items[0, len) (width 4 or 8 bytes per item).
// Writes the canonical summary (up to k entries) and returns its size.
uint32_t oracle_space_saving(const void* items, uint64_t len, int width, uint32_t k,
                             uint64_t* item, uint64_t* count, uint64_t* err, uint64_t* m) {
  Summary s = space_saving(items, width, 0, len, k);
  write_summary(s, item, count, err);
  *m = s.m;
  return (uint32_t)s.e.size();
}

// Algorithm 2 on two canonical summaries; returns the size of the result.
uint32_t oracle_combine(const uint64_t* ai, const uint64_t* ac, const uint64_t* ae, uint32_t an,
                        uint64_t am, uint64_t a_cov, const uint64_t* bi, const uint64_t* bc,
                        const uint64_t* be, uint32_t bn, uint64_t bm, uint64_t b_cov, uint32_t k,
                        uint64_t* item, uint64_t* count, uint64_t* err, uint64_t* m,
                        uint64_t* n_covered) {
  Summary a = read_summary(ai, ac, ae, an, am, a_cov);
  Summary b = read_summary(bi, bc, be, bn, bm, b_cov);
  Summary c = combine(a, b, k);
  write_summary(c, item, count, err);
  *m = c.m;
  *n_covered = c.n_covered;
  return (uint32_t)c.e.size();
}

// Number of nodes of the reduction tree over p leaves (all levels).
uint64_t oracle_tree_nodes(uint64_t p) {
  uint64_t total = 0;
  for (uint64_t w = p;; w = (w + 1) / 2) {
    total += w;
    if (w <= 1) break;
  }
  return total;
}

// The whole hot path: p block summaries (Algorithm 1), the binary reduction
// tree (Algorithm 2 at every node).  Node j of the flattened output is level
// 0 nodes first, then level 1, ...; node j's entries live at [j*k, j*k+size[j]).
// Returns the number of levels.
int oracle_pss_tree(const void* items, uint64_t n, int width, uint32_t k, uint32_t p,
                    uint64_t* item, uint64_t* count, uint64_t* err, uint32_t* size, uint64_t* m,
                    uint64_t* n_covered) {
  std::vector<Summary> level0;
  level0.reserve(p);
  for (uint32_t r = 0; r < p; ++r) {
    uint64_t left = block_left(r, n, p), right = block_left(r + 1, n, p);
    level0.push_back(space_saving(items, width, left, right - left, k));
  }
  std::vector<std::vector<Summary>> levels = reduction_tree(std::move(level0), k);
  size_t node = 0;
  for (const auto& level : levels) {
    for (const Summary& s : level) {
      write_summary(s, item + node * (size_t)k, count + node * (size_t)k, err + node * (size_t)k);
      size[node] = (uint32_t)s.e.size();
      m[node] = s.m;
      n_covered[node] = s.n_covered;
      ++node;
    }
  }
  return (int)levels.size();
}

// Only the summary of block r of p (Algorithm 1 bounds), for sampled checks.
uint32_t oracle_block_summary(const void* items, uint64_t n, int width, uint32_t k, uint32_t p,
                              uint32_t r, uint64_t* item, uint64_t* count, uint64_t* err,
                              uint64_t* m) {
  uint64_t left = block_left(r, n, p), right = block_left(r + 1, n, p);
  Summary s = space_saving(items, width, left, right - left, k);
  write_summary(s, item, count, err);
  *m = s.m;
  return (uint32_t)s.e.size();
}

// Pruned(global, n, k) on a canonical summary; returns the number reported.
uint32_t oracle_query(const uint64_t* si, const uint64_t* sc, const uint64_t* se, uint32_t sn,
                      uint64_t n, uint32_t k, uint64_t* item, uint64_t* count, uint64_t* err) {
  Summary s = read_summary(si, sc, se, sn, 0, 0);
  Summary q = pruned(s, n, k);
  write_summary(q, item, count, err);
  return (uint32_t)q.e.size();
}

// ---- seeded input generator (host side of the shared module) ----

}  // extern "C"

namespace {
// The sampler's tables, built once by the shared module's own functions.
const pssg_tables* gen_tables() {
  static const pssg_tables tb = [] {
    pssg_tables t;
    pssg_tables_init(&t);
    return t;
  }();
  return &tb;
}
}  // namespace

extern "C" {

void oracle_philox4x32_10(uint32_t* ctr, uint32_t k0, uint32_t k1) { pssg_philox4x32_10(ctr, k0, k1); }

// Items [start, start + count) of the stream (seed, stream, s, U = 2^log2u).
void oracle_gen_zipf(void* out, uint64_t start, uint64_t count, int width, uint64_t seed,
                     uint32_t stream, double s, int log2u) {
  const pssg_tables* tb = gen_tables();
  pssg_zipf z;
  pssg_zipf_init(&z, tb, s, (log2u >= 64) ? ~0ull : (1ull << log2u));
  for (uint64_t i = 0; i < count; ++i) {
    uint64_t x = pssg_zipf_item(&z, tb, log2u, seed, stream, start + i);
    if (width == 4)
      ((uint32_t*)out)[i] = (uint32_t)x;
    else
      ((uint64_t*)out)[i] = x;
  }
}

// The same items, generated by `threads` host threads (input preparation for
// large oracle runs; the oracle's own computation stays single-threaded).
void oracle_gen_zipf_mt(void* out, uint64_t start, uint64_t count, int width, uint64_t seed,
                        uint32_t stream, double s, int log2u, int threads) {
  if (threads < 1) threads = 1;
  std::vector<std::thread> pool;
  const uint64_t per = (count + threads - 1) / threads;
  for (int t = 0; t < threads; ++t) {
    const uint64_t lo = per * t, hi = std::min(count, lo + per);
    if (lo >= hi) break;
    char* base = (char*)out + lo * (uint64_t)width;
    pool.emplace_back(oracle_gen_zipf, (void*)base, start + lo, hi - lo, width, seed, stream, s, log2u);
  }
  for (auto& th : pool) th.join();
}

// Ranks only (no bijection), for distribution tests of the generator.
void oracle_gen_zipf_ranks(uint64_t* out, uint64_t start, uint64_t count, uint64_t seed,
                           uint32_t stream, double s, uint64_t n_ranks) {
  const pssg_tables* tb = gen_tables();
  pssg_zipf z;
  pssg_zipf_init(&z, tb, s, n_ranks);
  for (uint64_t i = 0; i < count; ++i) out[i] = pssg_zipf_rank(&z, tb, seed, stream, start + i);
}

uint64_t oracle_rank_to_item(uint64_t r, int log2u) { return pssg_rank_to_item(r, log2u); }

double oracle_gen_log(double x) { return pssg_log(x); }
double oracle_gen_exp(double x) { return pssg_exp(x); }
double oracle_gen_log_t(double x) { return pssg_log_t(gen_tables(), x); }
double oracle_gen_exp_t(double x) { return pssg_exp_t(gen_tables(), x); }

}  // extern "C"
