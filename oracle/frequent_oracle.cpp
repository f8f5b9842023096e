// frequent_oracle.cpp — CPU oracle for the Frequent (Misra–Gries) summary and
// its merge, the second counter-based summary the paper discusses (Section 2)
// next to Space Saving.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// CPU-baseline leg of bench.py may load this library.  It shares no code with
// the CUDA path.
//
// The paper names the algorithm (Misra and Gries; Frequent of Demaine et al.;
// Karp et al.) and the parallel merge of Frequent summaries only through the
// works it cites, so this file follows those published definitions:
//   * J. Misra and D. Gries, "Finding repeated elements", Science of Computer
//     Programming 2(2), 1982: with k - 1 counters, an item already counted
//     adds 1 to its counter; an item not counted takes a free counter with
//     count 1; when no counter is free, every counter loses 1, counters that
//     reach 0 are freed, and the item is not stored.  Every item whose
//     frequency exceeds n / k keeps a counter.
//   * P. K. Agarwal, G. Cormode, Z. Huang, J. M. Phillips, Z. Wei and K. Yi,
//     "Mergeable summaries", PODS 2012, the merge of two such summaries: add
//     the counts of equal items (an absent item counts 0); when more than
//     k - 1 items remain, subtract the k-th largest count from every counter
//     and drop the counters that are not positive.
// The blocks, the binary reduction tree and the canonical order (count
// descending, item ascending) are those of the Space Saving path
// (Algorithm 1).  Readings:
//   * Delta = floor((n_covered - sum of counts) / k) bounds what every count
//     misses: count <= f <= count + Delta for a stored item, f <= Delta for
//     any other (for one block (n - sum) is exactly k times the number of
//     decrement steps);
//   * the query reports the entries whose upper bound count + Delta exceeds
//     n / k ((count + Delta) * k > n: no k-majority item is missed), each with
//     err = Delta; the guaranteed query reports count * k > n.
//
// Parity: pinned by the tests under tests/ (the Boyer–Moore majority vote,
// which is this algorithm with one counter; exact histograms when k exceeds
// the distinct items; the Delta invariants against brute-force counts; merge
// bounds and symmetry; a hand-traced example).
#include <algorithm>
#include <cstdint>
#include <map>
#include <vector>

namespace {

struct FEntry {
  uint64_t item, count;
};

struct FSummary {
  std::vector<FEntry> e;  // canonical order: count descending, item ascending
  uint64_t n_covered = 0;
};

void f_canonicalize(FSummary& s) {
  std::sort(s.e.begin(), s.e.end(), [](const FEntry& a, const FEntry& b) {
    if (a.count != b.count) return a.count > b.count;
    return a.item < b.item;
  });
}

uint64_t f_block_left(uint64_t r, uint64_t n, uint64_t p) {
  return (uint64_t)(((unsigned __int128)r * n) / p);
}

uint64_t f_load(const void* items, int width, uint64_t i) {
  return width == 4 ? ((const uint32_t*)items)[i] : ((const uint64_t*)items)[i];
}

// Misra–Gries with k - 1 counters over items [left, left + len).
FSummary misra_gries(const void* items, int width, uint64_t left, uint64_t len, uint32_t k) {
  const size_t counters = k - 1;
  std::map<uint64_t, uint64_t> c;
  for (uint64_t t = 0; t < len; ++t) {
    const uint64_t x = f_load(items, width, left + t);
    auto it = c.find(x);
    if (it != c.end()) {
      it->second += 1;
    } else if (c.size() < counters) {
      c[x] = 1;
    } else {
      // no free counter: every counter loses 1; x is not stored
      for (auto i = c.begin(); i != c.end();) {
        i->second -= 1;
        if (i->second == 0) i = c.erase(i);
        else ++i;
      }
    }
  }
  FSummary s;
  for (const auto& kv : c) s.e.push_back(FEntry{kv.first, kv.second});
  s.n_covered = len;
  f_canonicalize(s);
  return s;
}

// The merge of two summaries with k - 1 counters each.
FSummary f_combine(const FSummary& a, const FSummary& b, uint32_t k) {
  std::map<uint64_t, uint64_t> sum;
  for (const FEntry& e : a.e) sum[e.item] += e.count;
  for (const FEntry& e : b.e) sum[e.item] += e.count;
  FSummary out;
  out.n_covered = a.n_covered + b.n_covered;
  if (sum.size() <= (size_t)(k - 1)) {
    for (const auto& kv : sum) out.e.push_back(FEntry{kv.first, kv.second});
  } else {
    std::vector<uint64_t> counts;
    for (const auto& kv : sum) counts.push_back(kv.second);
    std::sort(counts.begin(), counts.end(), [](uint64_t x, uint64_t y) { return x > y; });
    const uint64_t ck = counts[k - 1];  // the k-th largest count
    for (const auto& kv : sum)
      if (kv.second > ck) out.e.push_back(FEntry{kv.first, kv.second - ck});
  }
  f_canonicalize(out);
  return out;
}

uint64_t f_delta(const FSummary& s, uint32_t k) {
  uint64_t total = 0;
  for (const FEntry& e : s.e) total += e.count;
  return (s.n_covered - total) / k;
}

FSummary f_read(const uint64_t* item, const uint64_t* count, uint32_t size, uint64_t n_covered) {
  FSummary s;
  for (uint32_t i = 0; i < size; ++i) s.e.push_back(FEntry{item[i], count[i]});
  s.n_covered = n_covered;
  return s;
}

void f_write(const FSummary& s, uint64_t* item, uint64_t* count) {
  for (size_t i = 0; i < s.e.size(); ++i) {
    item[i] = s.e[i].item;
    count[i] = s.e[i].count;
  }
}

}  // namespace

extern "C" {

// Misra–Gries (k - 1 counters) over items[0, len); canonical entries; returns
// the number of entries.
uint32_t oracle_frequent(const void* items, uint64_t len, int width, uint32_t k, uint64_t* item,
                         uint64_t* count) {
  FSummary s = misra_gries(items, width, 0, len, k);
  f_write(s, item, count);
  return (uint32_t)s.e.size();
}

// The merge of two canonical summaries; returns the size of the result.
uint32_t oracle_frequent_combine(const uint64_t* ai, const uint64_t* ac, uint32_t an,
                                 uint64_t a_cov, const uint64_t* bi, const uint64_t* bc,
                                 uint32_t bn, uint64_t b_cov, uint32_t k, uint64_t* item,
                                 uint64_t* count, uint64_t* n_covered) {
  FSummary c = f_combine(f_read(ai, ac, an, a_cov), f_read(bi, bc, bn, b_cov), k);
  f_write(c, item, count);
  *n_covered = c.n_covered;
  return (uint32_t)c.e.size();
}

// p block summaries (Algorithm 1 bounds) and the binary reduction tree of
// merges.  Node j of the flattened output (level 0 first) holds its entries
// at [j * (k - 1), j * (k - 1) + size[j]).  Returns the number of levels.
int oracle_frequent_tree(const void* items, uint64_t n, int width, uint32_t k, uint32_t p,
                         uint64_t* item, uint64_t* count, uint32_t* size, uint64_t* n_covered) {
  std::vector<std::vector<FSummary>> levels(1);
  for (uint32_t r = 0; r < p; ++r) {
    const uint64_t left = f_block_left(r, n, p), right = f_block_left(r + 1, n, p);
    levels[0].push_back(misra_gries(items, width, left, right - left, k));
  }
  while (levels.back().size() > 1) {
    const std::vector<FSummary>& cur = levels.back();
    std::vector<FSummary> next;
    for (size_t i = 0; i + 1 < cur.size(); i += 2) next.push_back(f_combine(cur[i], cur[i + 1], k));
    if (cur.size() % 2) next.push_back(cur.back());
    levels.push_back(std::move(next));
  }
  const size_t stride = k - 1;
  size_t node = 0;
  for (const auto& level : levels) {
    for (const FSummary& s : level) {
      f_write(s, item + node * stride, count + node * stride);
      size[node] = (uint32_t)s.e.size();
      n_covered[node] = s.n_covered;
      ++node;
    }
  }
  return (int)levels.size();
}

// The query on a canonical summary: guaranteed = 0 reports (count + Delta) *
// k > n, guaranteed = 1 reports count * k > n; err = Delta on every entry.
// Returns the number reported.
uint32_t oracle_frequent_query(const uint64_t* si, const uint64_t* sc, uint32_t sn,
                               uint64_t n_covered, uint64_t n, uint32_t k, int guaranteed,
                               uint64_t* item, uint64_t* count, uint64_t* err) {
  const FSummary s = f_read(si, sc, sn, n_covered);
  const uint64_t delta = f_delta(s, k);
  uint32_t out = 0;
  for (const FEntry& e : s.e) {
    const uint64_t bound = guaranteed ? e.count : e.count + delta;
    if ((unsigned __int128)bound * k > (unsigned __int128)n) {
      item[out] = e.item;
      count[out] = e.count;
      err[out] = delta;
      ++out;
    }
  }
  return out;
}

}  // extern "C"
