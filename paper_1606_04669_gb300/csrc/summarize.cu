// summarize.cu — per-block Space Saving (Section 3 update rule; Algorithm 1's
// SpaceSaving call on the block bounds of Algorithm 1), one CTA per block.
//
// The sequential rule, with k counters (item, count, err, touch):
//   x monitored          -> count += 1, touch = t
//   a counter is free    -> (x, 1, 0, t)
//   else victim v = argmin (count, touch) -> err = count, count += 1,
//                                            item = x, touch = t
// is reproduced exactly while the CTA consumes a window of W = BS * IPT items
// per step.  Definitions for one window, all relative to its start state:
//
//   * bucket list: the counters of minimum count m ordered by touch (oldest
//     first).  Evictions take them in that order; a counter leaves the bucket
//     when it is hit.  The list is rebuilt when the bucket runs out (an
//     "epoch" ends): from the older members, sorted by touch, followed by the
//     log of counters that reached count m + 1 during the epoch, which is in
//     time order by construction.
//   * events: the first occurrence of each item missing from the table
//     ("misses"), plus "conversions": the first occurrence of a bucket
//     member's item after that member was evicted in this window.  A missed
//     item claims a "pending" cell of the table in the lookup pass itself,
//     keyed by the window position of the occurrence that claimed it; its
//     counter is written into that cell once its victim is known.
//   * event e (in time order) evicts the (e + s)-th bucket member, s being the
//     number of members before it that were "skipped" (hit before their turn).
//     Only members hit inside the window can be skipped or converted; one warp
//     decides just those, in list order, each with the time of the event that
//     reaches it (32 at once where bounds on that time settle every one of
//     them, else one at a time).  Every other assignment is arithmetic.
//   * the window is cut only where the bucket runs out (or a fill or a
//     per-window capacity ends): everything before the cut is exact, the rest
//     is processed again from the new state.  In miss-heavy streams, where
//     that happens soon after every start, windows are sized to the bucket's
//     expected end instead (the window body is compiled for both kinds).
//
// Table: item -> counter slot in buckets of four 32-bit cells (16-bit tag,
// slot + 1) read with one 128-bit shared load.  Each item has two buckets
// (two hashes); it goes to the first unless that one is full, and a bit per
// bucket records that some item of the first bucket lives in its second.
// Deletions clear the cell (no tombstones); the bits are recounted at every
// bucket-list rebuild, so they stay close to exact.
//
// Items: the next window is copied into shared memory (cp.async) as soon as
// the cut fixes where it starts, while the window's last phases run.  Each
// counter's err is written once, at insertion, into the block's output node.
// Above SS_SMEM_MAX_K counters the least-touched per-counter arrays live in a
// per-CTA slice of HBM scratch instead of shared memory.
//
// Output: the block's summary sorted by item ascending, with size, minimum m
// (the minimum count if k counters are in use, else 0) and the block length.
#include <atomic>
#include <type_traits>

#include "pss_internal.cuh"
#include "pss_kernels.cuh"

namespace pss {

namespace {

constexpr uint32_t NONE32 = 0xFFFFFFFFu;
constexpr uint16_t NONE16 = 0xFFFFu;
constexpr uint32_t PEND = 0x8000u;  // cell reference of a pending item: PEND | window position
constexpr int HMAX = 256;     // skipped members tracked per window
constexpr int CONVMAX = 32;   // conversions tracked per window (one per lane)
constexpr uint32_t EVR_HEAVY = 512;  // events per 1024 items of a miss-heavy stream

template <typename ItemT>
struct ItemOps;
template <>
struct ItemOps<uint32_t> {
  __device__ static __forceinline__ uint32_t h1(uint32_t x) { return x * 0x9E3779B1u; }
  __device__ static __forceinline__ uint32_t h3(uint32_t x) { return x * 0xC2B2AE35u; }
  __device__ static __forceinline__ u64 sort_key(uint32_t x, uint32_t slot) {
    return ((u64)x << 16) | slot;
  }
};
template <>
struct ItemOps<u64> {
  __device__ static __forceinline__ uint32_t h1(u64 x) {
    return (uint32_t)((x * 0x9E3779B97F4A7C15ull) >> 32);
  }
  __device__ static __forceinline__ uint32_t h3(u64 x) {
    return (uint32_t)((x * 0xD6E8FEB86659FD93ull) >> 32);
  }
  __device__ static __forceinline__ u64 sort_key(u64 x, uint32_t) { return x; }
};

struct SSState {
  uint32_t m;            // count of the minimum bucket (valid once full)
  uint32_t head;         // next unread index of the bucket list
  uint32_t list_len;
  uint32_t log_len;      // entries of the next-bucket log
  uint32_t used;         // counters in use
  uint32_t full;         // used == k
  uint32_t epoch_start;  // position at which the current bucket list was built
  uint32_t nvalid, nhit;  // candidate compaction
  uint32_t nskip, nconv, astop;
  uint32_t cut;          // exact prefix of the window
  uint32_t norig;        // events (not conversions) before the cut
  uint32_t exhausted;
  uint32_t maxdisp;      // largest distance of an item past its second bucket
  uint32_t evn, evc;     // the last cut window: events before its cut, and the cut (0: none)
  uint32_t status;
};

template <typename ItemT>
struct SSSmem {
  uint32_t NB, nbshift, NBW, CMAX, SORTN;
  // persistent state
  ItemT* item;
  uint32_t* cnt;
  uint32_t* touch;
  uint32_t* cell;     // NB * 4 cells: (tag << 16) | ref, 0 = empty; ref = slot + 1 or
                      // PEND | window position of a pending item
  uint32_t* ovf;      // 2 * NBW words: bit b set when an item of first bucket b lives
                      // outside it; second half: past its second bucket
  uint32_t* hfirst;   // per slot: first hit position in the window (members only)
  uint16_t* cellof;   // per slot: its cell
  uint16_t* list;
  uint16_t* logq;
  // window scratch (aliased by the rebuild sort)
  ItemT* wbuf;        // the window's items
  uint32_t* ppos;     // per claiming position: first occurrence of its item
  uint16_t* pslot;    // per claiming position: the counter its item gets
  uint16_t* pcell;    // per claiming position: the claimed cell
  uint16_t* rankpos;  // per event (time order): its position
  uint16_t* evpid;    // per event: the claiming position of its item
  uint16_t* logpos;
  uint16_t* cand;
  uint16_t* candidx;
  uint16_t* hitc;
  uint16_t* skipl;
  uint16_t* convt;
  uint16_t* convlo;
  uint16_t* convsrc;
  uint16_t* convfrom;  // per conversion: the evicted member's slot
  uint16_t* convto;    // per conversion: the slot its item gets (NONE16 past the cut)
  uint32_t* wsum;
  uint32_t* rkey;     // rebuild sort (over the window scratch)
  uint16_t* rpay;
  u64* fkey;          // final sort (over everything after touch)
  uint16_t* fpay;
  uint32_t* ferr;
};

__host__ __device__ inline uint32_t ilog2c(uint32_t x) {
  uint32_t r = 0;
  while ((1u << r) < x) ++r;
  return r;
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared-memory layout of one CTA (returns its bytes).  BIG (k above what
// fits): the bucket list, its log, each slot's cell, the first-hit positions
// and the large rebuild sort live in a per-CTA slice of global memory
// (gbase; the bytes go to *gbytes), the table is sized for <= 3/4 load, and
// the candidate list holds one chunk less.
template <typename ItemT, int BS, int IPT, bool BIG>
__host__ __device__ inline size_t ss_carve(uint32_t k, unsigned char* base, unsigned char* gbase,
                                           SSSmem<ItemT>* out, size_t* gbytes = nullptr) {
  constexpr uint32_t W = BS * IPT;
  SSSmem<ItemT> L;
  // room for k counters and a window of pending items at <= 1/2 load (3/4 BIG)
  const uint32_t nbk = BIG ? (k + W + 2) / 3 : (k + W + 1) / 2;
  L.NB = next_pow2(nbk < 16 ? 16 : nbk);
  L.nbshift = 32 - ilog2c(L.NB);
  L.NBW = (L.NB + 31) / 32;
  L.CMAX = BIG ? W + BS : W + 2 * BS;
  L.SORTN = next_pow2(k);
  size_t off = 0, goff = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align16(off + bytes);
    return base + o;
  };
  auto gtake = [&](size_t bytes) {
    size_t o = goff;
    goff = align16(goff + bytes);
    return gbase + o;
  };
  L.item = (ItemT*)take(sizeof(ItemT) * k);
  L.cnt = (uint32_t*)take(4ull * k);
  L.touch = (uint32_t*)take(4ull * k);
  const size_t after_touch = off;
  L.wsum = (uint32_t*)take(4ull * 2 * (BS / 32 + 1));
  L.cell = (uint32_t*)take(16ull * L.NB);
  L.ovf = (uint32_t*)take(8ull * L.NBW);
  if (BIG) {
    L.hfirst = (uint32_t*)gtake(4ull * k);
    L.cellof = (uint16_t*)gtake(2ull * k);
    L.list = (uint16_t*)gtake(2ull * k);
    L.logq = (uint16_t*)gtake(2ull * k);
  } else {
    L.hfirst = (uint32_t*)take(4ull * k);
    L.cellof = (uint16_t*)take(2ull * k);
    L.list = (uint16_t*)take(2ull * k);
    L.logq = (uint16_t*)take(2ull * k);
  }
  const size_t u0 = off;
  L.wbuf = (ItemT*)take(sizeof(ItemT) * W);
  L.ppos = (uint32_t*)take(4ull * W);
  L.pslot = (uint16_t*)take(2ull * W);
  L.pcell = (uint16_t*)take(2ull * W);
  L.rankpos = (uint16_t*)take(2ull * W);
  L.evpid = (uint16_t*)take(2ull * W);
  L.logpos = (uint16_t*)take(2ull * W);
  L.cand = (uint16_t*)take(2ull * L.CMAX);
  L.candidx = (uint16_t*)take(2ull * L.CMAX);
  L.hitc = (uint16_t*)take(2ull * L.CMAX);
  L.skipl = (uint16_t*)take(2ull * HMAX);
  L.convt = (uint16_t*)take(2ull * CONVMAX);
  L.convlo = (uint16_t*)take(2ull * CONVMAX);
  L.convsrc = (uint16_t*)take(2ull * CONVMAX);
  L.convfrom = (uint16_t*)take(2ull * CONVMAX);
  L.convto = (uint16_t*)take(2ull * CONVMAX);
  // The rebuild sort reuses the window scratch
  // (after wbuf, which holds the next window's items, copied in during the
  // window's last phases)
  if (BIG) {
    L.rkey = (uint32_t*)gtake(4ull * L.SORTN);
    L.rpay = (uint16_t*)gtake(2ull * L.SORTN);
  } else {
    const size_t s0 = u0 + align16(sizeof(ItemT) * W);
    L.rkey = (uint32_t*)(base + s0);
    L.rpay = (uint16_t*)(base + s0 + align16(4ull * L.SORTN));
    const size_t sort_end = s0 + align16(4ull * L.SORTN) + align16(2ull * L.SORTN);
    if (sort_end > off) off = sort_end;
  }
  // The final sort reuses everything after touch (the state is dead by then).
  L.fkey = (u64*)(base + after_touch);
  L.fpay = (uint16_t*)(base + after_touch + 8ull * L.SORTN);
  size_t final_end = align16(after_touch + 8ull * L.SORTN + align16(2ull * L.SORTN));
  if (BIG) {
    L.ferr = (uint32_t*)gtake(4ull * k);
  } else {
    L.ferr = (uint32_t*)(base + final_end);
    final_end = align16(final_end + 4ull * k);
  }
  if (final_end > off) off = final_end;
  if (out) *out = L;
  if (gbytes) *gbytes = goff;
  return off;
}

template <int BS>
__device__ __forceinline__ uint32_t block_min_u32(uint32_t v, uint32_t* scratch) {
  v = __reduce_min_sync(0xffffffffu, v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  uint32_t r = 0xFFFFFFFFu;
#pragma unroll
  for (int w = 0; w < BS / 32; ++w) r = min(r, scratch[w]);
  __syncthreads();
  return r;
}

// Number of entries of the sorted arr[0..n) smaller than x (n <= 1024), by
// one warp: a search over 32 segments, then inside the segment found.
__device__ __forceinline__ uint32_t warp_lower_bound(const uint16_t* arr, uint32_t n, uint32_t x) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t seg = (n + 31) / 32;
  bool p = false;
  if (seg && lane * seg < n) p = arr[min((lane + 1) * seg, n) - 1] < x;
  const uint32_t nfull = __popc(__ballot_sync(0xffffffffu, p));
  const uint32_t base = min(nfull * seg, n);  // the last segment may be partial
  const uint32_t j = base + lane;
  const bool q = lane < seg && j < n && arr[j] < x;
  return base + __popc(__ballot_sync(0xffffffffu, q));
}

template <typename ItemT, int BS, int IPT>
struct SSBlock {
  SSSmem<ItemT> s;
  SSState* S;
  uint32_t k;
  uint32_t par;  // scan scratch parity

  // Exclusive block scan with one barrier: every warp scans the warp totals
  // itself.  Consecutive scans alternate two buffers, so the barrier of the
  // next scan separates a buffer's reads from its next writes.
  __device__ __forceinline__ uint32_t scan(uint32_t v, uint32_t* total) {
    uint32_t* buf = s.wsum + (par ? (BS / 32 + 1) : 0);
    par ^= 1;
    constexpr int NW = BS / 32;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) buf[warp] = x;
    __syncthreads();
    uint32_t w = lane < (uint32_t)NW ? buf[lane] : 0u;
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= (uint32_t)o) w += y;
    }
    const uint32_t before = __shfl_sync(0xffffffffu, w, (warp + 31) & 31);
    *total = __shfl_sync(0xffffffffu, w, NW - 1);
    return (warp ? before : 0u) + x - v;
  }

  // The same scan for values made of single-bit fields (BITS marks the bit
  // positions used): the warp part is one ballot per field.
  template <uint32_t BITS>
  __device__ __forceinline__ uint32_t scan_bits(uint32_t v, uint32_t* total) {
    uint32_t* buf = s.wsum + (par ? (BS / 32 + 1) : 0);
    par ^= 1;
    constexpr int NW = BS / 32;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    uint32_t x = 0, wt = 0;
#pragma unroll
    for (int b = 0; b < 32; ++b) {
      if (!((BITS >> b) & 1u)) continue;
      const unsigned bal = __ballot_sync(0xffffffffu, (v >> b) & 1u);
      x += (uint32_t)__popc(bal & below) << b;
      wt += (uint32_t)__popc(bal) << b;
    }
    if (lane == 0) buf[warp] = wt;
    __syncthreads();
    uint32_t w = lane < (uint32_t)NW ? buf[lane] : 0u;
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= (uint32_t)o) w += y;
    }
    const uint32_t before = __shfl_sync(0xffffffffu, w, (warp + 31) & 31);
    *total = __shfl_sync(0xffffffffu, w, NW - 1);
    return (warp ? before : 0u) + x;
  }

  __device__ __forceinline__ bool ovf_bit(uint32_t half, uint32_t b) const {
    return (s.ovf[half * s.NBW + (b >> 5)] >> (b & 31)) & 1u;
  }

  // Result of a table match: slot >= 0, -2 - pid for the pending item of
  // claiming position pid, -1 for none.
  // Tags are never 0, so an empty cell never matches.
  static __device__ __forceinline__ uint32_t tag_of(uint32_t h) {
    const uint32_t t = h & 0xFFFFu;
    return t ? t : 1u;
  }

  __device__ __forceinline__ int ref_match(uint32_t ref, ItemT x) const {
    if (ref & PEND) {
      const uint32_t pid = ref & (PEND - 1);
      return s.wbuf[pid] == x ? -2 - (int)pid : -1;
    }
    return s.item[ref - 1] == x ? (int)(ref - 1) : -1;
  }

  __device__ __forceinline__ int cell_match(uint32_t c, uint32_t tag, ItemT x) const {
    if ((c >> 16) != tag) return -1;
    return ref_match(c & 0xFFFFu, x);
  }

  // The cells of one bucket with x's tag, checked in cell order.
  __device__ __forceinline__ int match4(const uint4& c, uint32_t tag, ItemT x) const {
    unsigned mm = ((c.x >> 16) == tag ? 1u : 0u) | ((c.y >> 16) == tag ? 2u : 0u) |
                  ((c.z >> 16) == tag ? 4u : 0u) | ((c.w >> 16) == tag ? 8u : 0u);
    while (mm) {
      const int i = __ffs(mm) - 1;
      const uint32_t cv = i == 0 ? c.x : (i == 1 ? c.y : (i == 2 ? c.z : c.w));
      const int r = ref_match(cv & 0xFFFFu, x);
      if (r != -1) return r;
      mm &= mm - 1;
    }
    return -1;
  }

  __device__ __forceinline__ int find_in(uint32_t bb, uint32_t tag, ItemT x) const {
    const uint4 c = *(const uint4*)&s.cell[bb * 4];
    return match4(c, tag, x);
  }

  // x outside its first bucket b: in its second bucket or past it, where the
  // overflow bits of b say so
  __device__ __forceinline__ int find_overflow(ItemT x, uint32_t b, uint32_t tag) const {
    if (!ovf_bit(0, b)) return -1;
    const uint32_t b2 = ItemOps<ItemT>::h3(x) >> s.nbshift, mask = s.NB - 1;
    const uint32_t d = ovf_bit(1, b) ? *(volatile uint32_t*)&S->maxdisp : 0u;
    for (uint32_t dd = 0; dd <= d; ++dd) {
      const int r = find_in((b2 + dd) & mask, tag, x);
      if (r != -1) return r;
    }
    return -1;
  }

  // x (occurring at window position rel) in the table, or else a pending cell
  // claimed for it.  Claims run concurrently and nothing leaves the table
  // meanwhile: every claimant of one item walks the same cells in the same
  // order, and compares each filled cell with x, so they agree on one cell.
  __device__ int find_or_claim(ItemT x, uint32_t rel, uint32_t& status) {
    const uint32_t h = ItemOps<ItemT>::h1(x);
    const uint32_t b = h >> s.nbshift, tag = tag_of(h), mask = s.NB - 1;
    int r = find_overflow(x, b, tag);
    if (r != -1) return r;
    const uint32_t val = (tag << 16) | PEND | rel;
    const uint32_t b2 = ItemOps<ItemT>::h3(x) >> s.nbshift;
    for (uint32_t step = 0; step <= s.NB; ++step) {
      const uint32_t bb = step == 0 ? b : ((b2 + step - 1) & mask);
      // the overflow bits go up before any claim they describe
      if (step == 1) atomicOr(&s.ovf[b >> 5], 1u << (b & 31));
      if (step == 2) atomicOr(&s.ovf[s.NBW + (b >> 5)], 1u << (b & 31));
      const uint4 cv = *(const uint4*)&s.cell[bb * 4];
      const uint32_t cs[4] = {cv.x, cv.y, cv.z, cv.w};
      for (int i = 0; i < 4; ++i) {
        uint32_t c = cs[i];
        if (c == 0u) {
          c = atomicCAS(&s.cell[bb * 4 + i], 0u, val);
          if (c == 0u) {
            s.pcell[rel] = (uint16_t)(bb * 4 + i);
            if (step >= 2) atomicMax(&S->maxdisp, step - 1);
            return -2 - (int)rel;
          }
        }
        r = cell_match(c, tag, x);
        if (r != -1) return r;
      }
    }
    status |= ST_PROBE;  // cannot happen: the table has room for k + W items
    s.pcell[rel] = NONE16;
    return -2 - (int)rel;
  }

  // Claims an empty cell of bucket bb for val (a cell seen taken is skipped).
  __device__ __forceinline__ bool claim(uint32_t bb, uint32_t val, uint32_t slot) {
    const uint4 cv = *(const uint4*)&s.cell[bb * 4];
    const uint32_t cs[4] = {cv.x, cv.y, cv.z, cv.w};
    for (int i = 0; i < 4; ++i) {
      if (cs[i] == 0u && atomicCAS(&s.cell[bb * 4 + i], 0u, val) == 0u) {
        s.cellof[slot] = (uint16_t)(bb * 4 + i);
        return true;
      }
    }
    return false;
  }

  __device__ __forceinline__ void insert(ItemT x, uint32_t slot, uint32_t& status) {
    const uint32_t h = ItemOps<ItemT>::h1(x);
    const uint32_t b = h >> s.nbshift, mask = s.NB - 1;
    const uint32_t val = (tag_of(h) << 16) | (slot + 1);
    if (claim(b, val, slot)) return;
    atomicOr(&s.ovf[b >> 5], 1u << (b & 31));
    const uint32_t b2 = ItemOps<ItemT>::h3(x) >> s.nbshift;
    for (uint32_t dd = 0; dd < s.NB; ++dd) {
      if (claim((b2 + dd) & mask, val, slot)) {
        if (dd) {
          atomicOr(&s.ovf[s.NBW + (b >> 5)], 1u << (b & 31));
          atomicMax(&S->maxdisp, dd);
        }
        return;
      }
    }
    status |= ST_PROBE;
  }

  // One occurrence at position t for counter tgt (NONE32: none).
  __device__ __forceinline__ void add_occurrence(uint32_t tgt, uint32_t t) {
    if (tgt != NONE32) {
      atomicAdd(&s.cnt[tgt], 1u);
      atomicMax(&s.touch[tgt], t);
    }
  }

  // Window scratch that must start clear (the rebuild sort writes over it).
  __device__ void reset_window_scratch() {
    constexpr uint32_t W = BS * IPT;
    for (uint32_t i = threadIdx.x; i < W; i += BS) {
      s.ppos[i] = NONE32;
      s.logpos[i] = 0;
    }
  }

  __device__ void rebuild_table(uint32_t& status) {
    for (uint32_t c = threadIdx.x; c < 4 * s.NB; c += BS) s.cell[c] = 0;
    for (uint32_t w = threadIdx.x; w < 2 * s.NBW; w += BS) s.ovf[w] = 0;
    if (threadIdx.x == 0) S->maxdisp = 0;
    __syncthreads();
    const uint32_t used = S->used;
    for (uint32_t i = threadIdx.x; i < used; i += BS) insert(s.item[i], i, status);
    __syncthreads();
  }

  // Build the bucket list of the minimum count, oldest touch first.  `now` is
  // the position of the next item to process.  Returns true when the large
  // sort wrote over the window scratch (which must then be reset).
  __device__ bool rebuild_list(bool full_scan, uint32_t now) {
    // thread-contiguous ranges of counters: [c0, c1)
    const uint32_t per = (k + BS - 1) / BS;
    const uint32_t c0 = min(threadIdx.x * per, k), c1 = min(c0 + per, k);
    uint32_t mn = 0xFFFFFFFFu;
    for (uint32_t i = c0; i < c1; ++i) mn = min(mn, s.cnt[i]);
    for (uint32_t w = threadIdx.x; w < 2 * s.NBW; w += BS) s.ovf[w] = 0;
    if (threadIdx.x == 0) S->maxdisp = 0;
    // in the half of the scan buffer the window's last scan did not use: no
    // barrier separates that scan's reads of its own half from these writes
    mn = block_min_u32<BS>(mn, s.wsum + (par ? (BS / 32 + 1) : 0));
    // overflow bits and distances of the counters as they are placed now
    for (uint32_t i = c0; i < c1; ++i) {
      const ItemT x = s.item[i];
      const uint32_t b = ItemOps<ItemT>::h1(x) >> s.nbshift;
      const uint32_t cb = (uint32_t)s.cellof[i] >> 2;
      if (cb != b) {
        atomicOr(&s.ovf[b >> 5], 1u << (b & 31));
        const uint32_t dd = (cb - (ItemOps<ItemT>::h3(x) >> s.nbshift)) & (s.NB - 1);
        if (dd) {
          atomicOr(&s.ovf[s.NBW + (b >> 5)], 1u << (b & 31));
          atomicMax(&S->maxdisp, dd);
        }
      }
    }
    const bool incremental = !full_scan && mn == S->m + 1;
    const uint32_t epoch = S->epoch_start;
    // (a) members to sort by touch: all of them, or those older than the epoch
    uint32_t nloc = 0;
    for (uint32_t i = c0; i < c1; ++i)
      nloc += (s.cnt[i] == mn && (!incremental || s.touch[i] < epoch)) ? 1u : 0u;
    uint32_t n1;
    uint32_t o = scan(nloc, &n1);
    const bool small = n1 <= (uint32_t)BS;
    uint32_t* key = small ? (uint32_t*)s.cand : s.rkey;   // cand holds >= 2 * BS u16 = BS u32
    uint16_t* pay = small ? s.candidx : s.rpay;
    for (uint32_t i = c0; i < c1; ++i) {
      if (s.cnt[i] == mn && (!incremental || s.touch[i] < epoch)) {
        key[o] = s.touch[i];
        pay[o] = (uint16_t)i;
        ++o;
      }
    }
    __syncthreads();
    if (small) {
      // touches of distinct counters differ: rank = number of smaller keys
      if (threadIdx.x < n1) {
        const uint32_t my = key[threadIdx.x];
        uint32_t rk = 0;
        for (uint32_t j = 0; j < n1; ++j) rk += key[j] < my ? 1u : 0u;
        s.list[rk] = pay[threadIdx.x];
      }
    } else {
      const uint32_t n2p = next_pow2(n1);
      for (uint32_t i = n1 + threadIdx.x; i < n2p; i += BS) {
        key[i] = 0xFFFFFFFFu;
        pay[i] = 0xFFFF;
      }
      __syncthreads();
      for (uint32_t size = 2; size <= n2p; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
          for (uint32_t i = threadIdx.x; i < (n2p >> 1); i += BS) {
            const uint32_t lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
            const bool asc = (lo & size) == 0;
            const uint32_t a = key[lo], b = key[hi];
            if ((a > b) == asc) {
              key[lo] = b; key[hi] = a;
              const uint16_t t = pay[lo]; pay[lo] = pay[hi]; pay[hi] = t;
            }
          }
          __syncthreads();
        }
      }
      for (uint32_t i = threadIdx.x; i < n1; i += BS) s.list[i] = pay[i];
    }
    // (b) the log: members that reached count mn during the epoch, in time order
    uint32_t n = n1;
    if (incremental) {
      const uint32_t ll = S->log_len;
      const uint32_t lper = (ll + BS - 1) / BS;
      const uint32_t l0 = min(threadIdx.x * lper, ll), l1 = min(l0 + lper, ll);
      uint32_t lc = 0;
      for (uint32_t j = l0; j < l1; ++j) lc += s.cnt[s.logq[j]] == mn ? 1u : 0u;
      uint32_t tot;
      uint32_t lo = n1 + scan(lc, &tot);
      for (uint32_t j = l0; j < l1; ++j) {
        const uint16_t q = s.logq[j];
        if (s.cnt[q] == mn) {
          if (lo < k) s.list[lo] = q;
          ++lo;
        }
      }
      n += tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      S->m = mn;
      S->head = 0;
      S->list_len = n < k ? n : k;
      S->log_len = 0;
      S->epoch_start = now;
    }
    __syncthreads();
    return !small;
  }
};

// Asynchronous copy of items [t, t + W) of xs (those below len; zeros past it)
// into wbuf, one element per copy (a window may start at any item).  Every
// thread issues its share; cp_wait() + a barrier make the window visible.
template <typename ItemT, int BS, int IPT>
__device__ __forceinline__ void copy_window(ItemT* wbuf, const ItemT* __restrict__ xs, uint32_t t,
                                            uint32_t len) {
  constexpr uint32_t W = BS * IPT;
  for (uint32_t i = threadIdx.x; i < W; i += BS) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(wbuf + i);
    const bool in = t + i < len;
    const ItemT* src = xs + (in ? t + i : 0u);
    const uint32_t n = in ? (uint32_t)sizeof(ItemT) : 0u;
    if (sizeof(ItemT) == 4)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(n)
                   : "memory");
    else
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(n)
                   : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// The summary of block r of p (Algorithm 1 bounds over n items) into node
// `node` of `out`; called by all threads of the CTA.
template <typename ItemT, int BS, int IPT, bool BIG>
__device__ void summarize_block(const ItemT* __restrict__ items, u64 n, uint32_t p, uint32_t r,
                                const SetView<ItemT>& out, uint32_t node, unsigned char* smem,
                                unsigned char* gslice, SSState& S_) {
  constexpr uint32_t W = BS * IPT;
  // bit fields of a per-thread count in [0, IPT]
  constexpr uint32_t kCountBits = IPT < 2 ? 1u : (IPT < 4 ? 3u : (IPT < 8 ? 7u : 15u));
  SSBlock<ItemT, BS, IPT> B;
  B.k = out.k;
  B.S = &S_;
  B.par = 0;
  ss_carve<ItemT, BS, IPT, BIG>(B.k, smem, gslice, &B.s);
  SSState& S = S_;
  auto& s = B.s;
  const uint32_t k = B.k;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u64 left = block_bound(r, n, p), right = block_bound((u64)r + 1, n, p);
  const size_t obase = (size_t)node * k;
  if (right - left >= (1ull << 32)) {
    if (tid == 0) {
      out.size[node] = 0;
      out.m[node] = 0;
      out.ncov[node] = right - left;
      atomicOr(out.status, (uint32_t)ST_CHUNK);
    }
    return;
  }
  const uint32_t len = (uint32_t)(right - left);
  const ItemT* __restrict__ xs = items + left;
  uint32_t status = 0;

  for (uint32_t i = tid; i < 4 * s.NB; i += BS) s.cell[i] = 0;
  for (uint32_t i = tid; i < 2 * s.NBW; i += BS) s.ovf[i] = 0;
  // counters start at 0 (a fresh slot is never written before it counts)
  for (uint32_t i = tid; i < k; i += BS) {
    s.hfirst[i] = NONE32;
    s.cnt[i] = 0;
    s.touch[i] = 0;
  }
  // err of slot q is kept in the output node (written once per insertion)
  u64* __restrict__ gerr = out.err + obase;
  B.reset_window_scratch();
  if (tid == 0) {
    S.m = 0; S.head = 0; S.list_len = 0; S.log_len = 0; S.used = 0; S.full = 0;
    S.epoch_start = 0; S.maxdisp = 0; S.status = 0; S.evn = 0; S.evc = 0;
  }
  __syncthreads();

  // The window's items sit in wbuf (pending cells name them by position);
  // the next window is copied in as soon as its start is known.
  uint32_t t0 = 0, stall = 0;
  if (len) copy_window<ItemT, BS, IPT>(s.wbuf, xs, 0, len);
  // One window; false when the block makes no progress.  It is compiled
  // twice: HEAVY for windows of miss-heavy streams (EVR_HEAVY or more events
  // per 1024 items), where windows end soon after they start because the
  // bucket list runs out, and the plain form for the rest, which then carries
  // none of the miss-heavy code.  In HEAVY windows the window is sized to the
  // items the list's remaining entries last at that rate, with an eighth to
  // spare (any length gives the same result; items looked up past the cut
  // would be looked up again), and missing items claim cells at once.
  auto window = [&](auto mode) -> bool {
    constexpr bool HEAVY = decltype(mode)::value;
    uint32_t nact = min(W, len - t0);
    if constexpr (HEAVY) {
      const uint32_t want = (S.list_len - S.head) * S.evc * 9u / (S.evn * 8u) + 32u;
      nact = min(nact, max(want, W / 4));
    }
    ItemT x[IPT];
#pragma unroll
    for (int j = 0; j < IPT; ++j) x[j] = s.wbuf[tid * IPT + j];
    const uint32_t full = S.full, m = S.m;
    // per-window state: written here, first read after the lookup's barrier
    if (tid == 0) {
      S.cut = nact;
      S.exhausted = 0;
      S.nvalid = 0;
      S.nhit = 0;
      S.nskip = 0;
      S.nconv = 0;
      S.astop = NONE32;
      S.norig = 0;
    }

    // ---- P1: look up or claim; first hit of bucket members; first occurrence of misses
    int sl[IPT];                  // slot, or -2 - pid for a pending item
    uint32_t miss = 0, mhit = 0;  // bit j: item j missed / hit a bucket member
    {
      // first buckets of all items first (independent loads), then resolve
      uint4 hc[IPT];
      uint32_t tg[IPT];
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const uint32_t h = ItemOps<ItemT>::h1(x[j]);
        tg[j] = B.tag_of(h);
        hc[j] = *(const uint4*)&s.cell[(h >> s.nbshift) * 4];
      }
#pragma unroll
      for (int j = 0; j < IPT; ++j) sl[j] = B.match4(hc[j], tg[j], x[j]);
      // In a HEAVY window a missing item whose first bucket has a free cell,
      // and none of whose items lives outside it, claims there at once:
      // the first step of find_or_claim's walk (a cell seen free and since
      // claimed fails the CAS and is compared, as in the walk).  Elsewhere
      // the packed walk below runs the few missing lanes on full warps.
      if constexpr (HEAVY) {
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
          const uint32_t rel = tid * IPT + j;
          if (sl[j] != -1 || rel >= nact) continue;
          const uint32_t h = ItemOps<ItemT>::h1(x[j]), b = h >> s.nbshift;
          if (B.ovf_bit(0, b)) continue;
          const uint32_t tag = B.tag_of(h), val = (tag << 16) | PEND | rel;
          const uint4 cv = *(const uint4*)&s.cell[b * 4];
          const uint32_t c4[4] = {cv.x, cv.y, cv.z, cv.w};
          for (int i = 0; i < 4; ++i) {
            uint32_t c = c4[i];
            if (c == 0u) {
              c = atomicCAS(&s.cell[b * 4 + i], 0u, val);
              if (c == 0u) {
                s.pcell[rel] = (uint16_t)(b * 4 + i);
                sl[j] = -2 - (int)rel;
                break;
              }
            }
            const int r = B.cell_match(c, tag, x[j]);
            if (r != -1) {
              sl[j] = r;
              break;
            }
          }
        }
      }
      // the rest (past the first bucket, or not in the table), packed onto
      // the warp's lanes; results by position in evpid (free until P2):
      // slot, or PEND | pid
      {
        unsigned bal[IPT];
        uint32_t base[IPT], tot = 0;
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
          bal[j] = __ballot_sync(0xffffffffu, sl[j] == -1 && tid * IPT + j < nact);
          base[j] = tot;
          tot += __popc(bal[j]);
        }
        for (uint32_t g0 = 0; g0 < tot; g0 += 32) {
          const uint32_t g = g0 + lane;
          if (g < tot) {
            int jj = 0;
#pragma unroll
            for (int j = 1; j < IPT; ++j) jj += g >= base[j] ? 1 : 0;
            unsigned bj = bal[0];
#pragma unroll
            for (int j = 1; j < IPT; ++j)
              if (jj == j) bj = bal[j];
            const uint32_t src = __fns(bj, 0, (int)(g - base[jj]) + 1);
            const uint32_t rel = ((warp << 5) + src) * IPT + (uint32_t)jj;
            const int r = B.find_or_claim(s.wbuf[rel], rel, status);
            s.evpid[rel] = (uint16_t)(r >= 0 ? (uint32_t)r : (PEND | (uint32_t)(-2 - r)));
          }
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
          if (bal[j] >> lane & 1) {
            const uint32_t v = s.evpid[tid * IPT + j];
            sl[j] = (v & PEND) ? -2 - (int)(v & (PEND - 1)) : (int)v;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const uint32_t rel = tid * IPT + j;
        const int r = sl[j];
        if (rel < nact) {
          if (r < 0) {
            miss |= 1u << j;
            atomicMin(&s.ppos[-2 - r], rel);
          } else if (full && s.cnt[r] == m) {
            mhit |= 1u << j;
            atomicMin(&s.hfirst[r], rel);
          }
        }
      }
    }
    // Hits on counters outside the minimum bucket commute with everything:
    // a window of those only just adds its occurrences.
    if (!__syncthreads_or((miss | mhit) != 0)) {
      if (t0 + nact < len) copy_window<ItemT, BS, IPT>(s.wbuf, xs, t0 + nact, len);
      // Skewed windows hit a few counters over and over: the warp adds its
      // occurrences of one of them (lane 0's first) with a single atomic pair.
      const uint32_t hot = __shfl_sync(0xffffffffu, tid * IPT < nact ? (uint32_t)sl[0] : NONE32, 0);
      uint32_t hot_n = 0, hot_t = 0;
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const uint32_t rel = tid * IPT + j;
        const uint32_t tgt = rel < nact ? (uint32_t)sl[j] : NONE32;
        const bool h = tgt == hot && hot != NONE32;
        const unsigned bal = __ballot_sync(0xffffffffu, h);
        if (bal) {
          hot_n += __popc(bal);
          hot_t = max(hot_t, t0 + (((uint32_t)warp << 5) + 31u - __clz(bal)) * IPT + j);
        }
        if (!h) B.add_occurrence(tgt, t0 + rel);
      }
      if (lane == 0 && hot_n) {
        atomicAdd(&s.cnt[hot], hot_n);
        atomicMax(&s.touch[hot], hot_t);
      }
      t0 += nact;
      return true;
    }

    // ---- P2: first occurrences of the misses (the events), ranked by position
    uint32_t first = 0;
#pragma unroll
    for (int j = 0; j < IPT; ++j)
      if ((miss >> j & 1) && s.ppos[-2 - sl[j]] == tid * IPT + j) first |= 1u << j;
    uint32_t M;
    const uint32_t rbase = B.template scan_bits<kCountBits>(__popc(first), &M);
    {
      uint32_t rr = rbase;
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        if (first >> j & 1) {
          s.rankpos[rr] = (uint16_t)(tid * IPT + j);
          s.evpid[rr] = (uint16_t)(-2 - sl[j]);
          ++rr;
        }
      }
    }

    // ---- P3: the bucket members still at count m, in list order (the scan
    // totals give every thread the running counts)
    bool list_end = false;
    if (full && M > 0) {
      uint32_t nv = 0, nh = 0, j0 = S.head;
      const uint32_t ll = S.list_len;
      for (;;) {
        if (nv >= M + 2 * nh + 1) break;
        if (j0 >= ll) {
          list_end = true;
          break;
        }
        if (nv + BS > s.CMAX) break;
        const uint32_t j = j0 + tid;
        bool valid = false, hit = false;
        uint16_t q = 0;
        if (j < ll) {
          q = s.list[j];
          valid = s.cnt[q] == m;
          hit = valid && s.hfirst[q] != NONE32;
        }
        uint32_t tt;
        const uint32_t ex =
            B.template scan_bits<0x10001u>((valid ? 1u : 0u) | (hit ? 0x10000u : 0u), &tt);
        if (valid) {
          const uint32_t a = nv + (ex & 0xFFFFu);
          s.cand[a] = q;
          s.candidx[a] = (uint16_t)j;
          if (hit) s.hitc[nh + (ex >> 16)] = (uint16_t)a;
        }
        nv += tt & 0xFFFFu;
        nh += tt >> 16;
        j0 += BS;
      }
      if (tid == 0) {
        S.nvalid = nv;
        S.nhit = nh;
      }
    }
    __syncthreads();

    // ---- P4: one warp decides the members hit in this window (skips, conversions).
    // Member j (in list order, candidate index a, first hit at h) is reached by
    // the merged event e = a - s, s the skips before it; each earlier member was
    // skipped or converted, so exactly j - s conversions precede e.  Hence it is
    // reached iff a - j < M, and its event time lies in [T[a - j], T[a]] (T the
    // original events' times; the upper end needs a < M).  A member whose h lies
    // below that range is skipped, above it converted, whatever came before; a
    // batch of 32 members with none in between is decided at once.  Otherwise the
    // batch (and the rest) takes the walk one member at a time.
    if (full && M > 0 && warp == 0) {
      const uint32_t nv = S.nvalid, nh = S.nhit;
      const unsigned below = (1u << lane) - 1u;
      uint32_t nskip = 0, nconv = 0, astop = nv;
      uint32_t ct = NONE32, clo = 0, cs = 0;  // walk: conversion held by this lane, sorted by time
      bool done = false, walk = false;
      for (uint32_t hb = 0; hb < nh && !done; hb += 32) {
       // this batch's hit members, one per lane
       uint32_t a_l = 0, hq_l = 0;
       if (hb + lane < nh) {
         a_l = s.hitc[hb + lane];
         hq_l = s.hfirst[s.cand[a_l]];
       }
       if (!walk && nh - hb >= 2u) {  // a lone member: the walk costs less
         const uint32_t nb0 = min(32u, nh - hb), j = hb + lane;
         const unsigned ub = __ballot_sync(0xffffffffu, lane < nb0 && a_l - j >= M);
         const uint32_t lim = ub ? (uint32_t)__ffs(ub) - 1u : nb0;  // reached members
         bool amb = false, skp = false;
         if (lane < lim) {
           if (a_l >= M) {
             amb = true;
           } else {
             const uint32_t tlo = s.rankpos[a_l - j], thi = s.rankpos[a_l];
             skp = hq_l < tlo;
             amb = !skp && hq_l <= thi;
           }
         }
         const unsigned bskip = __ballot_sync(0xffffffffu, lane < lim && skp);
         const unsigned bconv = __ballot_sync(0xffffffffu, lane < lim && !skp && !amb);
         const uint32_t ns = __popc(bskip), nc = __popc(bconv);
         if (!__any_sync(0xffffffffu, amb) && nskip + ns <= (uint32_t)HMAX &&
             nconv + nc <= (uint32_t)CONVMAX) {
           if ((bskip >> lane) & 1u) s.skipl[nskip + __popc(bskip & below)] = (uint16_t)a_l;
           nskip += ns;
           if (nc) {
             const bool cv = (bconv >> lane) & 1u;
             uint32_t lo = 0, rk = 0;
             if (cv) {  // original events before the conversion's time
               uint32_t hi = M;
               while (lo < hi) {
                 const uint32_t mid = (lo + hi) >> 1;
                 if (s.rankpos[mid] < hq_l) lo = mid + 1;
                 else hi = mid;
               }
             }
             for (unsigned mm = bconv; mm; mm &= mm - 1) {  // time order among the new ones
               const uint32_t t2 = __shfl_sync(0xffffffffu, hq_l, __ffs(mm) - 1);
               rk += t2 < hq_l ? 1u : 0u;
             }
             // merge with the conversions of earlier batches (time order)
             uint32_t ot = NONE32, olo = 0, osrc = 0, ork = lane;
             if (lane < nconv) {
               ot = s.convt[lane];
               olo = s.convlo[lane];
               osrc = s.convsrc[lane];
             }
             for (uint32_t c = 0; c < nconv; ++c) {
               const uint32_t t2 = __shfl_sync(0xffffffffu, ot, c);
               rk += t2 < hq_l ? 1u : 0u;
             }
             for (unsigned mm = bconv; mm; mm &= mm - 1) {
               const uint32_t t2 = __shfl_sync(0xffffffffu, hq_l, __ffs(mm) - 1);
               ork += t2 < ot ? 1u : 0u;
             }
             __syncwarp();
             if (lane < nconv) {
               s.convt[ork] = (uint16_t)ot;
               s.convlo[ork] = (uint16_t)olo;
               s.convsrc[ork] = (uint16_t)osrc;
             }
             if (cv) {
               s.convt[rk] = (uint16_t)hq_l;
               s.convlo[rk] = (uint16_t)lo;
               s.convsrc[rk] = (uint16_t)a_l;
             }
             __syncwarp();
             nconv += nc;
           }
           if (ub) done = true;  // later members are not reached either
           continue;
         }
       }
       if (!walk) {  // the walk from here: this lane's conversion of the list so far
         walk = true;
         if (lane < nconv) {
           ct = s.convt[lane];
           clo = s.convlo[lane];
           cs = s.convsrc[lane];
         }
       }
       const uint32_t nb_ = min(32u, nh - hb);
       for (uint32_t ii = 0; ii < nb_; ++ii) {
        const uint32_t a = __shfl_sync(0xffffffffu, a_l, ii);
        const uint32_t hq = __shfl_sync(0xffffffffu, hq_l, ii);
        const uint32_t e = a - nskip;  // the event that reaches this member
        const uint32_t mi = lane < nconv ? lane + clo : NONE32;
        const unsigned bc = __ballot_sync(0xffffffffu, mi == e);
        uint32_t tau;
        if (bc) {
          tau = __shfl_sync(0xffffffffu, ct, __ffs(bc) - 1);
        } else {
          const uint32_t nb = __popc(__ballot_sync(0xffffffffu, mi < e));
          const uint32_t i = e - nb;
          if (i >= M) {  // no event reaches this member, nor any later one
            done = true;
            break;
          }
          tau = s.rankpos[i];
        }
        if (hq < tau) {  // hit before its turn: it leaves the bucket
          if (nskip == HMAX) {
            astop = a;
            done = true;
            break;
          }
          if (lane == 0) s.skipl[nskip] = (uint16_t)a;
          ++nskip;
        } else {  // evicted at tau; its item comes back at hq
          if (nconv == CONVMAX) {
            astop = a;
            done = true;
            break;
          }
          const uint32_t lo = warp_lower_bound(s.rankpos, M, hq);
          const uint32_t pos = __popc(__ballot_sync(0xffffffffu, lane < nconv && ct < hq));
          const uint32_t pct = __shfl_up_sync(0xffffffffu, ct, 1);
          const uint32_t pclo = __shfl_up_sync(0xffffffffu, clo, 1);
          const uint32_t pcs = __shfl_up_sync(0xffffffffu, cs, 1);
          if (lane > pos && lane <= nconv) {
            ct = pct;
            clo = pclo;
            cs = pcs;
          }
          if (lane == pos) {
            ct = hq;
            clo = lo;
            cs = a;
          }
          ++nconv;
        }
       }
      }
      if (walk && lane < nconv) {
        s.convt[lane] = (uint16_t)ct;
        s.convlo[lane] = (uint16_t)clo;
        s.convsrc[lane] = (uint16_t)cs;
      }
      if (lane == 0) {
        S.nskip = nskip;
        S.nconv = nconv;
        S.astop = astop;
      }
    }
    __syncthreads();

    // ---- P5: every event's victim (or the cut), one thread per event; the
    // victim of a miss is kept by its claiming position
    const uint32_t nconv = S.nconv, nskip = S.nskip;
    const uint32_t limit = full ? min(S.nvalid, S.astop) : 0u;
    const bool can_exhaust = full && list_end && S.astop >= S.nvalid;
    const uint32_t nfree = full ? 0u : k - S.used;
    const uint32_t used0 = S.used;
    // event e passes skipped member i iff skipl[i] - i <= e (non-decreasing in i)
    auto assign = [&](uint32_t e) {
      uint32_t lo = 0, hi = nskip;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s.skipl[mid] - mid <= e) lo = mid + 1;
        else hi = mid;
      }
      return e + lo;
    };
    for (uint32_t r = tid; r < M; r += BS) {
      const uint32_t pid = s.evpid[r];
      if (!full) {
        if (r < nfree) s.pslot[pid] = (uint16_t)(used0 + r);
        else atomicMin(&S.cut, (uint32_t)s.rankpos[r]);
        continue;
      }
      // conversions merged before this event: convlo is non-decreasing
      uint32_t lo = 0, hi = nconv;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s.convlo[mid] <= r) lo = mid + 1;
        else hi = mid;
      }
      const uint32_t a = assign(r + lo);
      if (a < limit) {
        s.pslot[pid] = s.cand[a];
      } else {
        atomicMin(&S.cut, (uint32_t)s.rankpos[r]);
        if (can_exhaust) S.exhausted = 1;
      }
    }
    // conversion events: thread c handles conversion c
    uint32_t cvict = 0, ctime = NONE32, csrc = 0;
    ItemT citem = (ItemT)0;
    if (tid < nconv) {
      ctime = s.convt[tid];
      csrc = s.cand[s.convsrc[tid]];
      citem = s.item[csrc];
      const uint32_t a = assign(tid + s.convlo[tid]);
      if (a < limit) {
        cvict = s.cand[a];
      } else {
        atomicMin(&S.cut, ctime);
        if (can_exhaust) S.exhausted = 1;
      }
      // occurrences of the evicted member's item go to the new slot
      s.convfrom[tid] = (uint16_t)csrc;
      s.convto[tid] = a < limit ? (uint16_t)cvict : NONE16;
    }
    __syncthreads();
    const uint32_t cut = S.cut;

    // ---- P6: commit the events before the cut and count every occurrence
    // before it.  A victim's counter is already at m (it was not hit before
    // its eviction, or it would have been skipped) and every new item occurs
    // before the cut, which raises its touch above the victim's, so the
    // commit writes neither count nor touch and the counting needs no
    // barrier after it.  Each victim's cell is freed and the event's claimed
    // cell names the victim; claims past the cut are dropped.  Every cell has
    // one writer; conversions claim cells that are free.
    for (uint32_t r = tid; r < M; r += BS) {
      const uint32_t pid = s.evpid[r], rel = s.rankpos[r];
      const uint32_t pc = s.pcell[pid];
      // the last event before the cut records how many there are
      if (rel < cut && (r + 1 == M || s.rankpos[r + 1] >= cut)) S.norig = r + 1;
      if (rel >= cut) {
        if (pc != NONE16) s.cell[pc] = 0u;
        continue;
      }
      const uint32_t v = s.pslot[pid];
      if (full) s.cell[s.cellof[v]] = 0u;
      if (pc != NONE16) {
        s.cell[pc] = (s.cell[pc] & 0xFFFF0000u) | (v + 1);
        s.cellof[v] = (uint16_t)pc;
      }
      s.item[v] = s.wbuf[pid];
      gerr[v] = full ? m : 0u;
      if (full) s.logpos[rel] = (uint16_t)(v + 1);
    }
    if (tid < nconv && ctime < cut) {
      s.cell[s.cellof[cvict]] = 0u;
      B.insert(citem, cvict, status);
      s.item[cvict] = citem;
      gerr[cvict] = m;
      s.logpos[ctime] = (uint16_t)(cvict + 1);
    }
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const uint32_t rel = tid * IPT + j;
      uint32_t tgt = NONE32;
      if (rel < cut) {
        if (miss >> j & 1) {
          tgt = s.pslot[-2 - sl[j]];
        } else {
          tgt = (uint32_t)sl[j];
          if (mhit >> j & 1) {
            uint32_t f = NONE16;  // the member was evicted: its item was re-inserted
            for (uint32_t c = 0; c < nconv; ++c)
              if (s.convfrom[c] == tgt && s.convt[c] < cut) f = s.convto[c];
            if (f != NONE16) tgt = f;
            else if (s.hfirst[tgt] == rel) s.logpos[rel] = (uint16_t)(tgt + 1);  // m -> m + 1
          }
        }
      }
      B.add_occurrence(tgt, t0 + rel);
    }
    __syncthreads();
    // the next window starts at the cut: its items come in while the
    // remaining phases run (nothing reads wbuf from here on)
    if (t0 + cut < len) copy_window<ItemT, BS, IPT>(s.wbuf, xs, t0 + cut, len);

    // ---- P7: log in time order, reset the window scratch, advance
    const uint32_t log0 = S.log_len;  // read before the scan's barrier: warp 0 rewrites it
    uint32_t nl = 0;
    uint16_t lg[IPT];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const uint32_t rel = tid * IPT + j;
      lg[j] = s.logpos[rel];
      if (lg[j] && rel < cut) ++nl;
      s.logpos[rel] = 0;
    }
    uint32_t ltot;
    const uint32_t lbase = B.template scan_bits<kCountBits>(nl, &ltot);
    {
      uint32_t o = log0 + lbase;
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        if (lg[j] && tid * IPT + j < cut) {
          if (o < k) s.logq[o] = (uint16_t)(lg[j] - 1);
          ++o;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      if (mhit >> j & 1) s.hfirst[sl[j]] = NONE32;
      s.ppos[tid * IPT + j] = NONE32;
    }
    // The applied events are the prefix of the merged sequence before the cut.
    // Every thread derives the rebuild decision itself (no barrier here; the
    // rebuild's own barriers order warp 0's state updates before their use).
    const uint32_t norig = S.norig;
    const uint32_t need = full ? ((S.exhausted && cut < nact) ? 1u : 0u)
                               : (used0 + norig == k ? 2u : 0u);
    if (warp == 0) {
      const uint32_t nc = __popc(__ballot_sync(0xffffffffu, lane < nconv && s.convt[lane] < cut));
      const uint32_t nev = norig + nc;
      if (lane == 0) {
        const uint32_t nlog = log0 + ltot;
        S.log_len = nlog < k ? nlog : k;
        if (full) {
          if (nev) S.head = s.candidx[assign(nev - 1)] + 1u;
        } else {
          S.used = used0 + norig;
          if (S.used == k) S.full = 1;
        }
      }
    }
    stall = cut ? 0u : stall + 1u;
    if (tid == 0 && cut) {
      S.evn = norig;
      S.evc = cut;
    }
    if (need) {
      const bool clobbered = B.rebuild_list(need == 2, t0 + cut);
      if (S.maxdisp > 2) B.rebuild_table(status);
      if (clobbered) B.reset_window_scratch();
    }
    if (stall >= 3) {
      status |= ST_NOPROGRESS;
      return false;
    }
    t0 += cut;
    return true;
  };
  while (t0 < len) {
    cp_wait();
    __syncthreads();
    const bool heavy = S.full && S.evc && S.evn * 1024u >= EVR_HEAVY * S.evc;
    if (!(heavy ? window(std::true_type{}) : window(std::false_type{}))) break;
  }
  cp_wait();  // a copy may be in flight after an error exit


  // ---- output: the summary sorted by item ascending
  if (status) atomicOr(&S.status, status);
  __syncthreads();
  const uint32_t used = S.used;
  uint32_t mn = 0xFFFFFFFFu;
  for (uint32_t i = tid; i < used; i += BS) mn = min(mn, s.cnt[i]);
  mn = block_min_u32<BS>(mn, s.wsum);  // before the sort keys overwrite wsum
  const uint32_t n2p = next_pow2(used ? used : 1);
  for (uint32_t i = tid; i < used; i += BS) s.ferr[i] = (uint32_t)gerr[i];
  for (uint32_t i = tid; i < n2p; i += BS) {
    if (i < used) {
      s.fkey[i] = ItemOps<ItemT>::sort_key(s.item[i], i);
      s.fpay[i] = (uint16_t)i;
    } else {
      s.fkey[i] = ~0ull;
      s.fpay[i] = 0xFFFF;
    }
  }
  __syncthreads();
  block_bitonic_sort<BS, uint16_t>(s.fkey, s.fpay, n2p);
  for (uint32_t i = tid; i < used; i += BS) {
    const uint32_t q = s.fpay[i];
    out.item[obase + i] = s.item[q];
    out.count[obase + i] = s.cnt[q];
    out.err[obase + i] = s.ferr[q];
  }
  if (tid == 0) {
    out.size[node] = used;
    out.m[node] = (used == k) ? (u64)mn : 0ull;
    out.ncov[node] = len;
    if (S.status) atomicOr(out.status, S.status);
  }
}

// Register budget for 1024 threads per SM: two CTAs of 512 or four of 256.
template <typename ItemT, int BS, int IPT, bool BIG>
__global__ void __launch_bounds__(BS, 1024 / BS)
    ss_block_kernel(const ItemT* __restrict__ items, u64 n, uint32_t p, uint32_t r0,
                    SetView<ItemT> out, uint32_t node0, unsigned char* gscratch, size_t gslice) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SSState S;
  summarize_block<ItemT, BS, IPT, BIG>(items, n, p, r0 + blockIdx.x, out, node0 + blockIdx.x,
                                       smem, BIG ? gscratch + (size_t)blockIdx.x * gslice : nullptr,
                                       S);
}

// Persistent form for many streams: each CTA takes (stream, block) tasks from
// a shared counter until the list is exhausted.  Tasks are listed longest
// block first so that the last wave is short.
template <typename ItemT, int BS, int IPT>
__global__ void __launch_bounds__(BS, 1024 / BS)
    ss_batch_kernel(const BatchStream* __restrict__ streams, const BatchTask* __restrict__ tasks,
                    uint32_t ntasks, uint32_t* counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SSState S;
  __shared__ uint32_t next;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t t = next;
    __syncthreads();
    if (t >= ntasks) break;
    const BatchTask task = tasks[t];
    const BatchStream st = streams[task.stream];
    const SetView<ItemT> out = set_view_dev<ItemT>(st.level0, st.p, st.k);
    summarize_block<ItemT, BS, IPT, false>((const ItemT*)st.items, st.n, st.p, task.index, out,
                                           task.index, smem, nullptr, S);
    __syncthreads();
  }
}

}  // namespace

namespace {
std::atomic<uint32_t> g_warp_kmax{WARP_SS_DEFAULT_K};
std::atomic<uint32_t> g_round_kmax{ROUND_SS_DEFAULT_K};
std::atomic<int> g_sms{0};

// Whether a launch of `count` blocks with k counters runs on the round
// kernel: k up to round_kmax(), and enough blocks to fill half the warps
// the round kernel keeps resident (with fewer, the CTA kernel's 256 or 512
// threads per block win; measured at 2^28 and 2^30 items).
template <typename ItemT>
bool use_round_kernel(uint32_t k, uint32_t count) {
  if (k > round_kmax()) return false;
  int sms = g_sms.load(std::memory_order_relaxed);
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return false;
    g_sms.store(sms, std::memory_order_relaxed);
  }
  const uint32_t per_sm = round_resident_warps<ItemT>(k);
  return per_sm > 0 && 2ull * count >= (uint64_t)sms * per_sm;
}
}  // namespace

uint32_t warp_kmax() { return g_warp_kmax.load(); }
uint32_t round_kmax() { return g_round_kmax.load(); }

template <typename ItemT>
size_t ss_smem_bytes(uint32_t k) {
  return k > SS_SMEM_MAX_K ? ss_carve<ItemT, SS_BS, SS_IPT, true>(k, nullptr, nullptr, nullptr)
                           : ss_carve<ItemT, SS_BS, SS_IPT, false>(k, nullptr, nullptr, nullptr);
}

namespace {

// Resident CTAs per SM of one kernel shape (0 if it cannot run).
int resident_ctas(const void* kern, int bs, size_t smem) {
  if (ensure_kernel_attrs(kern) != cudaSuccess) return 0;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, bs, smem) != cudaSuccess)
    return 0;
  return blocks;
}

template <typename ItemT>
size_t shape_smem(uint32_t k, int shape) {
  switch (shape) {
    case SS_SHAPE_NARROW:
      return ss_carve<ItemT, SS_BS_NARROW, SS_IPT_NARROW, false>(k, nullptr, nullptr, nullptr);
    case SS_SHAPE_SMALL:
      return ss_carve<ItemT, SS_BS_SMALL, SS_IPT_SMALL, false>(k, nullptr, nullptr, nullptr);
    default:
      return ss_smem_bytes<ItemT>(k);
  }
}

inline int shape_threads(int shape) {
  return shape == SS_SHAPE_NARROW ? SS_BS_NARROW : shape == SS_SHAPE_SMALL ? SS_BS_SMALL : SS_BS;
}

inline int shape_items_per_thread(int shape) {
  return shape == SS_SHAPE_NARROW ? SS_IPT_NARROW : shape == SS_SHAPE_SMALL ? SS_IPT_SMALL : SS_IPT;
}

template <typename ItemT>
const void* block_kernel_of(int shape) {
  switch (shape) {
    case SS_SHAPE_NARROW:
      return (const void*)ss_block_kernel<ItemT, SS_BS_NARROW, SS_IPT_NARROW, false>;
    case SS_SHAPE_SMALL:
      return (const void*)ss_block_kernel<ItemT, SS_BS_SMALL, SS_IPT_SMALL, false>;
    default:
      return (const void*)ss_block_kernel<ItemT, SS_BS, SS_IPT, false>;
  }
}

template <typename ItemT>
const void* batch_kernel_of(int shape) {
  switch (shape) {
    case SS_SHAPE_NARROW:
      return (const void*)ss_batch_kernel<ItemT, SS_BS_NARROW, SS_IPT_NARROW>;
    case SS_SHAPE_SMALL:
      return (const void*)ss_batch_kernel<ItemT, SS_BS_SMALL, SS_IPT_SMALL>;
    default:
      return (const void*)ss_batch_kernel<ItemT, SS_BS, SS_IPT>;
  }
}

}  // namespace

template <typename ItemT>
int ss_shape(uint32_t k, bool batch) {
  if (k > SS_SMEM_MAX_K) return SS_SHAPE_WIDE;
  // shape + 1, 0 = not decided yet; decided on the first device that asks
  // (one kind of GPU per process), so that later launches and stream captures
  // only read it
  static std::atomic<int> memo[2][SS_SMEM_MAX_K + 1];
  std::atomic<int>& m = memo[batch ? 1 : 0][k];
  const int known = m.load(std::memory_order_relaxed);
  if (known) return known - 1;
  int best = SS_SHAPE_WIDE, best_threads = -1;
  // in order of preference on a tie
  for (int shape : {SS_SHAPE_NARROW, SS_SHAPE_SMALL, SS_SHAPE_WIDE}) {
    const void* kern = batch ? batch_kernel_of<ItemT>(shape) : block_kernel_of<ItemT>(shape);
    const int t = resident_ctas(kern, shape_threads(shape), shape_smem<ItemT>(k, shape)) *
                  shape_threads(shape);
    if (t > best_threads) {
      best = shape;
      best_threads = t;
    }
  }
  m.store(best + 1, std::memory_order_relaxed);
  return best;
}

namespace {

// The shape a launch of `count` blocks runs: the occupancy choice, except
// that the small shape gives way to the wide shape when every
// block of the launch fits on the SMs at once in the wide shape.  Then no
// block waits for a slot, the launch takes as long as one block, and 512
// threads finish a block sooner (measured on the served workload, whose
// ticks summarize a few blocks each).
template <typename ItemT>
int ss_launch_shape(uint32_t k, bool batch, uint64_t count) {
  const int shape = ss_shape<ItemT>(k, batch);
  if (shape != SS_SHAPE_SMALL) return shape;
  int sms = g_sms.load(std::memory_order_relaxed);
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return shape;
    g_sms.store(sms, std::memory_order_relaxed);
  }
  // wide CTAs per SM at this k, + 1 (0 = not known yet)
  static std::atomic<int> memo[2][SS_SMEM_MAX_K + 1];
  std::atomic<int>& m = memo[batch ? 1 : 0][k];
  int wide = m.load(std::memory_order_relaxed) - 1;
  if (wide < 0) {
    const void* kern = batch ? batch_kernel_of<ItemT>(SS_SHAPE_WIDE) : block_kernel_of<ItemT>(SS_SHAPE_WIDE);
    wide = resident_ctas(kern, SS_BS, shape_smem<ItemT>(k, SS_SHAPE_WIDE));
    m.store(wide + 1, std::memory_order_relaxed);
  }
  return count <= (uint64_t)sms * (uint64_t)wide ? SS_SHAPE_WIDE : shape;
}

}  // namespace

// Whether a launch with k counters (k <= SS_SMEM_MAX_K) runs the large-k
// form (part of the state in global scratch, table at <= 3/4 load): for
// 2048 < k <= 3072, where it keeps two 512-thread CTAs per SM instead of one
// (measured at n = 2^30, k = 3000: 15-28% less time at s = 0.5-2.0, equal
// results; at k = 4000 it lost 15% at s = 0.5, so the range stops short).
template <typename ItemT>
bool use_large_k_form(uint32_t k) {
  if (k <= 2048 || k > 3072) return false;
  static std::atomic<int> memo[3072 - 2048 + 1];  // 1 + decision, 0 = not decided yet
  std::atomic<int>& m = memo[k - 2049];
  const int known = m.load(std::memory_order_relaxed);
  if (known) return known == 2;
  const int std_ctas = resident_ctas((const void*)ss_block_kernel<ItemT, SS_BS, SS_IPT, false>,
                                     SS_BS, ss_smem_bytes<ItemT>(k));
  const int big_ctas =
      resident_ctas((const void*)ss_block_kernel<ItemT, SS_BS, SS_IPT, true>, SS_BS,
                    ss_carve<ItemT, SS_BS, SS_IPT, true>(k, nullptr, nullptr, nullptr));
  const bool big = big_ctas > std_ctas;
  m.store(big ? 2 : 1, std::memory_order_relaxed);
  return big;
}

template <typename ItemT>
cudaError_t launch_summarize_blocks(const ItemT* items, u64 n, uint32_t p, uint32_t r0,
                                    uint32_t count, SetView<ItemT> out, uint32_t node0,
                                    cudaStream_t stream, bool may_allocate) {
  if (out.k <= warp_kmax())
    return launch_summarize_warp_blocks<ItemT>(items, n, p, r0, count, out, node0, stream);
  if (use_round_kernel<ItemT>(out.k, count))
    return launch_summarize_round_blocks<ItemT>(items, n, p, r0, count, out, node0, stream);
  if (out.k <= SS_SMEM_MAX_K && !(may_allocate && use_large_k_form<ItemT>(out.k))) {
    const int shape = ss_launch_shape<ItemT>(out.k, false, count);
    const void* kern = block_kernel_of<ItemT>(shape);
    cudaError_t e = ensure_kernel_attrs(kern);
    if (e != cudaSuccess) return e;
    if (count == 0) return cudaSuccess;
    const size_t smem = shape_smem<ItemT>(out.k, shape);
    if (shape == SS_SHAPE_NARROW)
      ss_block_kernel<ItemT, SS_BS_NARROW, SS_IPT_NARROW, false>
          <<<count, SS_BS_NARROW, smem, stream>>>(items, n, p, r0, out, node0, nullptr, 0);
    else if (shape == SS_SHAPE_SMALL)
      ss_block_kernel<ItemT, SS_BS_SMALL, SS_IPT_SMALL, false>
          <<<count, SS_BS_SMALL, smem, stream>>>(items, n, p, r0, out, node0, nullptr, 0);
    else
      ss_block_kernel<ItemT, SS_BS, SS_IPT, false>
          <<<count, SS_BS, smem, stream>>>(items, n, p, r0, out, node0, nullptr, 0);
    return cudaGetLastError();
  }
  // large k: a slice of global scratch per CTA, ordered on the stream
  const size_t smem = ss_carve<ItemT, SS_BS, SS_IPT, true>(out.k, nullptr, nullptr, nullptr);
  auto kern = ss_block_kernel<ItemT, SS_BS, SS_IPT, true>;
  cudaError_t e = ensure_kernel_attrs((const void*)kern);
  if (e != cudaSuccess) return e;
  if (count == 0) return cudaSuccess;
  size_t gslice = 0;
  ss_carve<ItemT, SS_BS, SS_IPT, true>(out.k, nullptr, nullptr, nullptr, &gslice);
  void* g = nullptr;
  e = cudaMallocAsync(&g, gslice * count, stream);
  if (e != cudaSuccess) return e;
  kern<<<count, SS_BS, smem, stream>>>(items, n, p, r0, out, node0, (unsigned char*)g, gslice);
  e = cudaGetLastError();
  cudaError_t f = cudaFreeAsync(g, stream);
  return e != cudaSuccess ? e : f;
}

template <typename ItemT>
cudaError_t launch_summarize_batch(const BatchStream* streams, const BatchTask* tasks,
                                   uint32_t ntasks, uint32_t* counter, uint32_t k, uint32_t grid,
                                   cudaStream_t stream) {
  if (k > SS_SMEM_MAX_K) return cudaErrorInvalidValue;  // the batch keeps k in shared memory
  const int shape = ss_launch_shape<ItemT>(k, true, ntasks);
  cudaError_t e = ensure_kernel_attrs(batch_kernel_of<ItemT>(shape));
  if (e != cudaSuccess) return e;
  if (ntasks == 0 || grid == 0) return cudaSuccess;
  const size_t smem = shape_smem<ItemT>(k, shape);
  if (shape == SS_SHAPE_NARROW)
    ss_batch_kernel<ItemT, SS_BS_NARROW, SS_IPT_NARROW>
        <<<grid, SS_BS_NARROW, smem, stream>>>(streams, tasks, ntasks, counter);
  else if (shape == SS_SHAPE_SMALL)
    ss_batch_kernel<ItemT, SS_BS_SMALL, SS_IPT_SMALL>
        <<<grid, SS_BS_SMALL, smem, stream>>>(streams, tasks, ntasks, counter);
  else
    ss_batch_kernel<ItemT, SS_BS, SS_IPT>
        <<<grid, SS_BS, smem, stream>>>(streams, tasks, ntasks, counter);
  return cudaGetLastError();
}

template <typename ItemT>
int summarize_ctas_per_sm(uint32_t k, uint64_t ntasks) {
  if (k > SS_SMEM_MAX_K) return 0;
  const int shape = ss_launch_shape<ItemT>(k, true, ntasks);
  return resident_ctas(batch_kernel_of<ItemT>(shape), shape_threads(shape),
                       shape_smem<ItemT>(k, shape));
}

template cudaError_t launch_summarize_batch<uint32_t>(const BatchStream*, const BatchTask*, uint32_t,
                                                      uint32_t*, uint32_t, uint32_t, cudaStream_t);
template cudaError_t launch_summarize_batch<u64>(const BatchStream*, const BatchTask*, uint32_t,
                                                 uint32_t*, uint32_t, uint32_t, cudaStream_t);
template int summarize_ctas_per_sm<uint32_t>(uint32_t, uint64_t);
template int summarize_ctas_per_sm<u64>(uint32_t, uint64_t);
template size_t ss_smem_bytes<uint32_t>(uint32_t);
template size_t ss_smem_bytes<u64>(uint32_t);
template int ss_shape<uint32_t>(uint32_t, bool);
template int ss_shape<u64>(uint32_t, bool);
template cudaError_t launch_summarize_blocks<uint32_t>(const uint32_t*, u64, uint32_t, uint32_t,
                                                       uint32_t, SetView<uint32_t>, uint32_t,
                                                       cudaStream_t, bool);
template cudaError_t launch_summarize_blocks<u64>(const u64*, u64, uint32_t, uint32_t, uint32_t,
                                                  SetView<u64>, uint32_t, cudaStream_t, bool);

}  // namespace pss

extern "C" int pss_plan_kernel(uint32_t k, uint32_t count, int item_bytes) {
  if (k < 2 || (item_bytes != 4 && item_bytes != 8)) return -1;
  if (k <= pss::warp_kmax()) return PSS_KERNEL_WARP;
  const bool round = item_bytes == 4 ? pss::use_round_kernel<uint32_t>(k, count)
                                     : pss::use_round_kernel<pss::u64>(k, count);
  return round ? PSS_KERNEL_ROUND : PSS_KERNEL_CTA;
}

extern "C" int pss_plan_cta_shape(uint32_t k, int item_bytes, int batch, int* threads,
                                  int* items_per_thread) {
  if (k < 2 || k > PSS_MAX_K || (item_bytes != 4 && item_bytes != 8) || !threads ||
      !items_per_thread)
    return PSS_EINVAL;
  const int shape = item_bytes == 4 ? pss::ss_shape<uint32_t>(k, batch != 0)
                                    : pss::ss_shape<pss::u64>(k, batch != 0);
  *threads = pss::shape_threads(shape);
  *items_per_thread = pss::shape_items_per_thread(shape);
  return PSS_OK;
}

extern "C" uint32_t pss_set_round_kmax(uint32_t kmax) {
  return pss::g_round_kmax.exchange(kmax < PSS_MAX_K_RESIDENT ? kmax : PSS_MAX_K_RESIDENT);
}

extern "C" uint32_t pss_set_warp_kmax(uint32_t kmax) {
  return pss::g_warp_kmax.exchange(kmax < pss::WARP_SS_MAX_K ? kmax : pss::WARP_SS_MAX_K);
}
