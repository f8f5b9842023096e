// summarize_round.cu — per-block Space Saving (Section 3 update rule on the
// block bounds of Algorithm 1) for small and mid k: one warp per block, the
// block's items taken 32 at a time (lane i holds item t0 + i) in rounds.
//
// The counters (item, u32 count, u32 touch = position of the last update,
// u32 err) and a linear-probe table of 16-bit cells (slot + 1; 0 empty,
// 0xFFFF a freed cell) at most 3/4 taken live in the warp's slice of shared
// memory.  Evictions follow the minimum of (count, touch): the counters at the
// minimum count m wait in a queue in touch order; a counter that reaches
// m + 1 during the queue's epoch is appended to a log in time order, so when
// the queue runs out the next one is the counters at m + 1 from before the
// epoch (sorted by touch) followed by the log (already in touch order).
//
// A round probes every lane's item and applies at once the longest prefix of
// the lanes whose effects commute:
//   * hits add to their counters with shared-memory atomics (count + 1,
//     touch = max of the positions); the occurrences of one missing item form
//     a group (__match_any_sync) led by its lowest lane, which applies them
//     all;
//   * while counters are free, each missing item's leader takes one;
//   * on a full table each missing item's leader is an event: events take
//     victims from the queue in order, skipping entries no longer at m and
//     entries hit earlier in the round (they left the minimum before the
//     event); a victim hit later in the round ends the prefix before that
//     lane (its probe is stale), as does an event that finds the queue empty
//     (the queue is rebuilt and the round resumes).
// Each victim's cell is freed, the new item takes a cell from the first free
// one its probe found, err = m, count = m + its occurrences.  When freed cells
// make the table more than 3/4 taken it is rebuilt.  The output node is
// sorted by item, the layout the combine kernel reads.
#include <algorithm>
#include <atomic>

#include "pss_internal.cuh"
#include "pss_kernels.cuh"

namespace pss {

namespace {

constexpr uint32_t RFULL = 0xffffffffu;
constexpr uint32_t R_EMPTY = 0u, R_FREED = 0xFFFFu;
constexpr uint16_t R_NOSLOT = 0xFFFF;
constexpr uint32_t R_NONE = 0xFFFFFFFFu;
constexpr int R_MAX_WPC = 8;

template <typename ItemT>
struct RHash;
template <>
struct RHash<uint32_t> {
  __device__ static __forceinline__ uint32_t h(uint32_t x) {
    x ^= x >> 16;
    x *= 0x21f0aaadu;
    x ^= x >> 15;
    x *= 0x735a2d97u;
    x ^= x >> 15;
    return x;
  }
};
template <>
struct RHash<u64> {
  __device__ static __forceinline__ uint32_t h(u64 x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return (uint32_t)x;
  }
};

// One warp's slice.
struct RLayout {
  uint32_t cap, nb, shift;
  size_t cnt, touch, err, cellof, queue, logq, hitl, cell, bytes;
};

__host__ __device__ inline RLayout r_layout(uint32_t k, int item_bytes) {
  RLayout L;
  L.cap = next_pow2(k < 32 ? 32 : k);
  L.nb = next_pow2(2 * k < 64 ? 64 : 2 * k);
  uint32_t lg = 0;
  while ((1u << lg) < L.nb) ++lg;
  L.shift = 32 - lg;
  auto up = [](size_t x) { return (x + 15) & ~(size_t)15; };
  size_t off = up((size_t)item_bytes * L.cap);
  L.cnt = off;    off += up(4ull * L.cap);
  L.touch = off;  off += up(4ull * L.cap);
  L.err = off;    off += up(4ull * L.cap);
  L.cellof = off; off += up(2ull * L.cap);
  L.queue = off;  off += up(2ull * L.cap);
  L.logq = off;   off += up(2ull * L.cap);
  L.hitl = off;   off += up((size_t)L.cap);
  L.cell = off;   off += up(2ull * L.nb);
  L.bytes = off;
  return L;
}

template <typename ItemT>
struct RWarp {
  ItemT* item;
  uint32_t* cnt;
  uint32_t* touch;
  uint32_t* err;
  uint16_t* cellof;
  uint16_t* queue;
  uint16_t* logq;
  uint8_t* hitl;
  unsigned short* cell;
  uint32_t k, cap, nbmask, shift, lane;
  // warp-uniform state
  uint32_t used, m, qh, qlen, loglen, epoch, taken;  // taken: cells not empty
  bool full;
  uint32_t status;  // this lane's ST_* bits

  __device__ __forceinline__ uint32_t home(uint32_t h) const { return h >> shift; }

  // This lane's probe for x: its slot, or -1 with *fpos = the first free
  // (empty or freed) cell of its run.  Freed cells do not end a run.
  __device__ __forceinline__ int find(ItemT x, uint32_t h, uint32_t* fpos) {
    uint32_t pos = home(h);
    uint32_t fp = R_NONE;
    for (uint32_t step = 0; step <= nbmask; ++step) {
      const uint32_t c = cell[pos];
      if (c == R_EMPTY) {
        *fpos = fp == R_NONE ? pos : fp;
        return -1;
      }
      if (c == R_FREED) {
        if (fp == R_NONE) fp = pos;
      } else if (item[c - 1] == x) {
        return (int)c - 1;
      }
      pos = (pos + 1) & nbmask;
    }
    *fpos = fp;
    if (fp == R_NONE) status |= ST_PROBE;  // cannot happen: the table is at most 3/4 taken
    return -1;
  }

  // Claims the first free cell from pos for slot s (lanes claim concurrently:
  // a 32-bit compare-and-swap on the word holding the cell; a swap that fails
  // because the other cell of the word changed retries).  Returns whether the
  // claimed cell was empty (not a freed one).
  __device__ __forceinline__ bool insert(uint32_t s, uint32_t pos) {
    uint32_t* words = reinterpret_cast<uint32_t*>(cell);
    pos &= nbmask;
    for (uint32_t tries = 0; tries <= 3 * nbmask + 3; ++tries) {
      const uint32_t sh = (pos & 1u) * 16u;
      uint32_t* wp = &words[pos >> 1];
      const uint32_t old = *(volatile uint32_t*)wp;
      const uint32_t half = (old >> sh) & 0xFFFFu;
      if (half != R_EMPTY && half != R_FREED) {
        pos = (pos + 1) & nbmask;
        continue;
      }
      const uint32_t nw = (old & ~(0xFFFFu << sh)) | ((s + 1) << sh);
      if (atomicCAS(wp, old, nw) == old) {
        cellof[s] = (uint16_t)pos;
        return half == R_EMPTY;
      }
    }
    status |= ST_PROBE;
    return false;
  }

  // A fresh table of the used counters.
  __device__ void rebuild_table() {
    for (uint32_t i = lane; i <= nbmask; i += 32) cell[i] = (unsigned short)R_EMPTY;
    __syncwarp();
    for (uint32_t i = lane; i < used; i += 32) insert(i, home(RHash<ItemT>::h(item[i])));
    __syncwarp();
    taken = used;
  }

  // queue[0 .. n) sorted by touch ascending (n <= cap; entries past n unused).
  __device__ void sort_queue_by_touch(uint32_t n) {
    const uint32_t n2 = next_pow2(n < 2 ? 2 : n);
    for (uint32_t i = n + lane; i < n2; i += 32) queue[i] = R_NOSLOT;
    __syncwarp();
    for (uint32_t size = 2; size <= n2; size <<= 1) {
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t i = lane; i < (n2 >> 1); i += 32) {
          const uint32_t lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
          const bool asc = (lo & size) == 0;
          const uint16_t a = queue[lo], b = queue[hi];
          const u64 ka = a == R_NOSLOT ? ~0ull : (u64)touch[a];
          const u64 kb = b == R_NOSLOT ? ~0ull : (u64)touch[b];
          if ((ka > kb) == asc) {
            queue[lo] = b;
            queue[hi] = a;
          }
        }
        __syncwarp();
      }
    }
  }

  // The queue of the new minimum count, from position `now` on.
  // incremental: the previous queue ran out, so every count is above m; if
  // the new minimum is m + 1 the queue is the counters at m + 1 from before
  // the epoch (sorted by touch) followed by the log's entries still at m + 1.
  __device__ void rebuild_queue(bool incremental, uint32_t now) {
    uint32_t mn = 0xFFFFFFFFu;
    for (uint32_t i = lane; i < used; i += 32) mn = min(mn, cnt[i]);
    mn = __reduce_min_sync(RFULL, mn);
    const bool inc = incremental && mn == m + 1;
    const unsigned below = (1u << lane) - 1u;
    uint32_t n = 0;
    for (uint32_t b0 = 0; b0 < used; b0 += 32) {
      const uint32_t i = b0 + lane;
      const bool in = i < used && cnt[i] == mn && (!inc || touch[i] < epoch);
      const unsigned bm = __ballot_sync(RFULL, in);
      if (in) queue[n + (uint32_t)__popc(bm & below)] = (uint16_t)i;
      n += (uint32_t)__popc(bm);
    }
    __syncwarp();
    sort_queue_by_touch(n);
    if (inc) {
      for (uint32_t b0 = 0; b0 < loglen; b0 += 32) {
        const uint32_t i = b0 + lane;
        const uint16_t q = i < loglen ? logq[i] : R_NOSLOT;
        const bool in = q != R_NOSLOT && cnt[q] == mn;
        const unsigned bm = __ballot_sync(RFULL, in);
        if (in) queue[n + (uint32_t)__popc(bm & below)] = q;
        n += (uint32_t)__popc(bm);
      }
    }
    __syncwarp();
    m = mn;
    qh = 0;
    qlen = n;
    loglen = 0;
    epoch = now;
  }

  // Slots [0, used) in item order in queue[0 .. used).
  __device__ void sort_by_item() {
    const uint32_t n2 = next_pow2(used < 2 ? 2 : used);
    for (uint32_t i = lane; i < n2; i += 32) queue[i] = i < used ? (uint16_t)i : R_NOSLOT;
    __syncwarp();
    for (uint32_t size = 2; size <= n2; size <<= 1) {
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t i = lane; i < (n2 >> 1); i += 32) {
          const uint32_t lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
          const bool asc = (lo & size) == 0;
          const uint16_t a = queue[lo], b = queue[hi];
          const bool greater = a == R_NOSLOT ? b != R_NOSLOT : (b != R_NOSLOT && item[a] > item[b]);
          if (greater == asc) {
            queue[lo] = b;
            queue[hi] = a;
          }
        }
        __syncwarp();
      }
    }
  }
};

template <typename ItemT>
__device__ void round_block(const ItemT* __restrict__ xs, uint32_t len, uint32_t k,
                            unsigned char* slice, const SetView<ItemT>& out, uint32_t node) {
  const RLayout L = r_layout(k, (int)sizeof(ItemT));
  RWarp<ItemT> W;
  W.item = (ItemT*)slice;
  W.cnt = (uint32_t*)(slice + L.cnt);
  W.touch = (uint32_t*)(slice + L.touch);
  W.err = (uint32_t*)(slice + L.err);
  W.cellof = (uint16_t*)(slice + L.cellof);
  W.queue = (uint16_t*)(slice + L.queue);
  W.logq = (uint16_t*)(slice + L.logq);
  W.hitl = (uint8_t*)(slice + L.hitl);
  W.cell = (unsigned short*)(slice + L.cell);
  W.k = k;
  W.cap = L.cap;
  W.nbmask = L.nb - 1;
  W.shift = L.shift;
  W.lane = threadIdx.x & 31;
  W.used = W.m = W.qh = W.qlen = W.loglen = W.epoch = W.taken = 0;
  W.full = false;
  W.status = 0;
  for (uint32_t i = W.lane; i < L.nb; i += 32) W.cell[i] = (unsigned short)R_EMPTY;
  for (uint32_t i = W.lane; i < L.cap; i += 32) W.hitl[i] = 0xFF;
  __syncwarp();
  const uint32_t lane = W.lane;
  const unsigned below = (1u << lane) - 1u;
  const uint32_t taken_max = (L.nb >> 2) * 3;

  ItemT nxt = lane < len ? xs[lane] : (ItemT)0;
  for (uint32_t t0 = 0; t0 < len; t0 += 32) {
    const ItemT x = nxt;
    const uint32_t here = min(32u, len - t0);
    if (t0 + 32 + lane < len) nxt = xs[t0 + 32 + lane];
    const uint32_t h = RHash<ItemT>::h(x);
    uint32_t start = 0;
    // every round applies at least one lane, or rebuilds the queue and then
    // applies one: at most 2 * 32 rounds
    for (uint32_t guard = 0; start < here; ++guard) {
      if (guard > 2 * 32 + 2) {
        W.status |= ST_NOPROGRESS;
        break;
      }
      const bool act = lane >= start && lane < here;
      int s = -1;
      uint32_t fpos = R_NONE;
      if (act) s = W.find(x, h, &fpos);
      const bool miss = act && s < 0;
      const bool hit = act && !miss;
      // hits add with shared-memory atomics; the occurrences of one missing
      // item form a group led by its lowest lane
      const unsigned mm = __ballot_sync(RFULL, miss);
      unsigned grp = 0;
      if (miss) grp = __match_any_sync(mm, x);
      const bool leader = miss && (grp & below) == 0;
      uint32_t end;
      if (!W.full) {
        // free counters: each missing item's leader takes one; the round
        // ends at the first leader that finds none
        const unsigned lead = __ballot_sync(RFULL, leader);
        const uint32_t free_n = k - W.used;
        end = (uint32_t)__popc(lead) <= free_n ? here : (uint32_t)__fns(lead, 0, (int)free_n + 1);
        const unsigned before = end >= 32 ? RFULL : (1u << end) - 1u;
        bool fresh = false;
        if (leader && lane < end) {
          const unsigned g = grp & before;
          const uint32_t slot = W.used + (uint32_t)__popc(lead & below);
          W.item[slot] = x;
          W.cnt[slot] = (uint32_t)__popc(g);
          W.touch[slot] = t0 + 31u - (uint32_t)__clz(g);
          W.err[slot] = 0;
          fresh = W.insert(slot, fpos);
        }
        if (hit && lane < end) {
          atomicAdd(&W.cnt[s], 1u);
          atomicMax(&W.touch[s], t0 + lane);
        }
        W.taken += (uint32_t)__popc(__ballot_sync(RFULL, fresh));
        W.used += (uint32_t)__popc(lead & before);
        __syncwarp();
        if (W.used == k) {
          W.full = true;
          W.rebuild_queue(false, t0 + end);
        }
      } else {
        // full table: events take victims from the queue
        const uint32_t ch = hit ? W.cnt[s] : 0u;
        const bool minhit = hit && ch == W.m;
        const unsigned mh = __ballot_sync(RFULL, minhit);
        const unsigned em = __ballot_sync(RFULL, leader);
        const uint32_t ne = (uint32_t)__popc(em);
        end = here;
        uint32_t v = R_NOSLOT;  // this event's victim
        bool exhausted = false;
        if (ne) {
          if (!mh) {
            // no counter of the minimum is hit in the round: the j-th event
            // takes the j-th entry still at m
            const uint32_t rank = (uint32_t)__popc(em & below);
            uint32_t assigned = 0, qp = W.qh;
            for (uint32_t iter = 0; assigned < ne && qp < W.qlen && iter <= W.qlen; ++iter) {
              const uint32_t pos = qp + lane;
              const uint16_t q = pos < W.qlen ? W.queue[pos] : R_NOSLOT;
              const bool valid = q != R_NOSLOT && W.cnt[q] == W.m;
              const unsigned vm = __ballot_sync(RFULL, valid);
              const uint32_t nv = (uint32_t)__popc(vm);
              const uint32_t tk = min(nv, ne - assigned);
              const bool mine = leader && rank >= assigned && rank < assigned + tk;
              const int src = mine ? (int)__fns(vm, 0, (int)(rank - assigned) + 1) : (int)lane;
              const uint16_t got = __shfl_sync(RFULL, q, src);
              if (mine) v = got;
              qp += tk < nv ? (uint32_t)__fns(vm, 0, (int)tk) + 1 : 32u;
              assigned += tk;
            }
            W.qh = min(qp, W.qlen);
            if (assigned < ne) {
              end = (uint32_t)__fns(em, 0, (int)assigned + 1);
              exhausted = true;
            }
          } else {
            // some minimum counters are hit: the earliest hit of each goes to
            // hitl, then a warp-uniform walk of the events in order
            unsigned mg = 0;
            if (minhit) mg = __match_any_sync(mh, s);
            const bool mlead = minhit && (mg & below) == 0;
            if (mlead) W.hitl[s] = (uint8_t)lane;
            __syncwarp();
            uint32_t e = 0, qp = W.qh;
            for (uint32_t iter = 0; e < ne && iter <= W.qlen + 32; ++iter) {
              const uint32_t lam = (uint32_t)__fns(em, 0, (int)e + 1);
              if (lam >= end) break;
              if (qp >= W.qlen) {
                end = lam;
                exhausted = true;
                break;
              }
              const uint16_t q = W.queue[qp];
              ++qp;
              if (W.cnt[q] != W.m) continue;  // left the minimum in an earlier round
              const uint32_t l = W.hitl[q];
              if (l != 0xFF && l < lam) continue;  // hit before this event
              if (lane == lam) v = q;
              if (l != 0xFF && l < end) end = l;  // its later hit is stale
              ++e;
            }
            W.qh = min(qp, W.qlen);
            __syncwarp();
            if (mlead) W.hitl[s] = 0xFF;
          }
        }
        const unsigned before = end >= 32 ? RFULL : (1u << end) - 1u;
        const bool ev = leader && lane < end;
        // victims' cells are freed before the new items claim cells
        if (ev) W.cell[W.cellof[v]] = (unsigned short)R_FREED;
        __syncwarp();
        bool fresh = false;
        bool logged = false;
        uint16_t logslot = R_NOSLOT;
        if (ev) {
          const unsigned g = grp & before;
          const uint32_t c = (uint32_t)__popc(g);
          W.item[v] = x;
          W.err[v] = W.m;
          W.cnt[v] = W.m + c;
          W.touch[v] = t0 + 31u - (uint32_t)__clz(g);
          fresh = W.insert(v, fpos);
          logged = c == 1;
          logslot = (uint16_t)v;
        }
        uint32_t old = 0;
        const bool apply_hit = hit && lane < end;
        if (apply_hit) {
          old = atomicAdd(&W.cnt[s], 1u);
          atomicMax(&W.touch[s], t0 + lane);
        }
        __syncwarp();
        // a minimum counter hit exactly once in the prefix reached m + 1 there
        if (apply_hit && old == W.m && W.cnt[s] == W.m + 1) {
          logged = true;
          logslot = (uint16_t)s;
        }
        // counters that reached m + 1 in the round, in time order
        const unsigned lm = __ballot_sync(RFULL, logged);
        if (logged) W.logq[W.loglen + (uint32_t)__popc(lm & below)] = logslot;
        W.loglen += (uint32_t)__popc(lm);
        W.taken += (uint32_t)__popc(__ballot_sync(RFULL, fresh));
        __syncwarp();
        if (exhausted) W.rebuild_queue(true, t0 + end);
      }
      if (W.taken > taken_max) W.rebuild_table();
      start = end;
    }
    __syncwarp();
  }

  // output: the summary in item order, minimum m (k counters in use, else 0)
  uint32_t mn = 0xFFFFFFFFu;
  for (uint32_t i = lane; i < W.used; i += 32) mn = min(mn, W.cnt[i]);
  mn = __reduce_min_sync(RFULL, mn);
  W.sort_by_item();
  const size_t base = (size_t)node * out.k;
  for (uint32_t i = lane; i < W.used; i += 32) {
    const uint16_t q = W.queue[i];
    out.item[base + i] = W.item[q];
    out.count[base + i] = W.cnt[q];
    out.err[base + i] = W.err[q];
  }
  const uint32_t st = __reduce_or_sync(RFULL, W.status);
  if (lane == 0) {
    out.size[node] = W.used;
    out.m[node] = W.used == k ? (u64)mn : 0ull;
    out.ncov[node] = len;
    if (st) atomicOr(out.status, st);
  }
}

template <typename ItemT>
__device__ __forceinline__ void round_task(const ItemT* items, u64 n, uint32_t p, uint32_t r,
                                           const SetView<ItemT>& out, uint32_t node,
                                           unsigned char* slice) {
  const u64 left = block_bound(r, n, p), right = block_bound((u64)r + 1, n, p);
  if (right - left >= (1ull << 32)) {
    if ((threadIdx.x & 31) == 0) {
      out.size[node] = 0;
      out.m[node] = 0;
      out.ncov[node] = right - left;
      atomicOr(out.status, (uint32_t)ST_CHUNK);
    }
    return;
  }
  round_block<ItemT>(items + left, (uint32_t)(right - left), out.k, slice, out, node);
}

// Warp w of CTA b summarizes block r0 + b * warps + w into node node0 + ...
template <typename ItemT>
__global__ void __launch_bounds__(32 * R_MAX_WPC) ssr_block_kernel(const ItemT* __restrict__ items,
                                                                   u64 n, uint32_t p, uint32_t r0,
                                                                   uint32_t count,
                                                                   SetView<ItemT> out,
                                                                   uint32_t node0, uint32_t wbytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t j = blockIdx.x * (blockDim.x >> 5) + warp;
  if (j >= count) return;  // the whole warp
  round_task<ItemT>(items, n, p, r0 + j, out, node0 + j, smem + (size_t)warp * wbytes);
}

// Persistent form for many streams: each warp takes (stream, block) tasks
// from a shared counter (the tasks of one launch share k).
template <typename ItemT>
__global__ void __launch_bounds__(32 * R_MAX_WPC) ssr_batch_kernel(const BatchStream* __restrict__ streams,
                                                                   const BatchTask* __restrict__ tasks,
                                                                   uint32_t ntasks, uint32_t* counter,
                                                                   uint32_t wbytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* slice = smem + (size_t)warp * wbytes;
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(counter, 1u);
    t = __shfl_sync(RFULL, t, 0);
    if (t >= ntasks) break;
    const BatchTask task = tasks[t];
    const BatchStream st = streams[task.stream];
    const SetView<ItemT> out = set_view_dev<ItemT>(st.level0, st.p, st.k);
    round_task<ItemT>((const ItemT*)st.items, st.n, st.p, task.index, out, task.index, slice);
    __syncwarp();
  }
}

// Warps per CTA with the most warps resident per SM (ties: fewer), per k.
template <typename ItemT>
int round_warps_per_cta(uint32_t k, bool batch) {
  static std::atomic<int> memo[2][PSS_MAX_K_RESIDENT + 1];
  if (k < 2 || k > PSS_MAX_K_RESIDENT) return 0;
  std::atomic<int>& mm = memo[batch ? 1 : 0][k];
  int v = mm.load(std::memory_order_relaxed);
  if (v) return v;
  const void* kern = batch ? (const void*)ssr_batch_kernel<ItemT> : (const void*)ssr_block_kernel<ItemT>;
  if (ensure_kernel_attrs(kern) != cudaSuccess) return 0;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  const size_t wb = r_layout(k, (int)sizeof(ItemT)).bytes;
  int best = 0, best_warps = 0;
  for (int wpc = 1; wpc <= R_MAX_WPC; wpc *= 2) {
    if ((size_t)wpc * wb > (size_t)optin) break;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, 32 * wpc, (size_t)wpc * wb) !=
        cudaSuccess)
      return 0;
    if (blocks * wpc > best_warps) {
      best_warps = blocks * wpc;
      best = wpc;
    }
  }
  if (best) mm.store(best, std::memory_order_relaxed);
  return best;
}

}  // namespace

size_t round_warp_bytes(uint32_t k, int item_bytes) { return r_layout(k, item_bytes).bytes; }

template <typename ItemT>
uint32_t round_resident_warps(uint32_t k) {
  static std::atomic<uint32_t> memo[PSS_MAX_K_RESIDENT + 1];
  if (k < 2 || k > PSS_MAX_K_RESIDENT) return 0;
  uint32_t v = memo[k].load(std::memory_order_relaxed);
  if (v) return v;
  const int wpc = round_warps_per_cta<ItemT>(k, false);
  if (wpc <= 0) return 0;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, (const void*)ssr_block_kernel<ItemT>,
                                                    32 * wpc,
                                                    (size_t)wpc * r_layout(k, (int)sizeof(ItemT)).bytes) !=
      cudaSuccess)
    return 0;
  v = (uint32_t)(blocks * wpc);
  memo[k].store(v, std::memory_order_relaxed);
  return v;
}

template uint32_t round_resident_warps<uint32_t>(uint32_t);
template uint32_t round_resident_warps<u64>(uint32_t);

template <typename ItemT>
cudaError_t launch_summarize_round_blocks(const ItemT* items, u64 n, uint32_t p, uint32_t r0,
                                          uint32_t count, SetView<ItemT> out, uint32_t node0,
                                          cudaStream_t stream) {
  const uint32_t k = out.k;
  const int wpc = round_warps_per_cta<ItemT>(k, false);
  if (wpc <= 0) return cudaErrorInvalidConfiguration;
  if (count == 0) return cudaSuccess;
  const size_t wb = r_layout(k, (int)sizeof(ItemT)).bytes;
  const uint32_t grid = (count + (uint32_t)wpc - 1) / (uint32_t)wpc;
  ssr_block_kernel<ItemT><<<grid, 32 * wpc, (size_t)wpc * wb, stream>>>(items, n, p, r0, count, out,
                                                                        node0, (uint32_t)wb);
  return cudaGetLastError();
}

template <typename ItemT>
uint32_t round_batch_grid(uint32_t k, uint32_t ntasks, int sms) {
  const int wpc = round_warps_per_cta<ItemT>(k, true);
  if (wpc <= 0) return 0;
  const void* kern = (const void*)ssr_batch_kernel<ItemT>;
  const size_t wb = r_layout(k, (int)sizeof(ItemT)).bytes;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, 32 * wpc, (size_t)wpc * wb) !=
          cudaSuccess ||
      blocks <= 0)
    return 0;
  const uint64_t need = (ntasks + (uint32_t)wpc - 1) / (uint32_t)wpc;
  return (uint32_t)std::min<uint64_t>((uint64_t)sms * (uint64_t)blocks, need ? need : 1);
}

template <typename ItemT>
cudaError_t launch_summarize_round_batch(const BatchStream* streams, const BatchTask* tasks,
                                         uint32_t ntasks, uint32_t* counter, uint32_t k,
                                         uint32_t grid, cudaStream_t stream) {
  const int wpc = round_warps_per_cta<ItemT>(k, true);
  if (wpc <= 0) return cudaErrorInvalidConfiguration;
  if (ntasks == 0 || grid == 0) return cudaSuccess;
  const size_t wb = r_layout(k, (int)sizeof(ItemT)).bytes;
  ssr_batch_kernel<ItemT><<<grid, 32 * wpc, (size_t)wpc * wb, stream>>>(streams, tasks, ntasks,
                                                                        counter, (uint32_t)wb);
  return cudaGetLastError();
}

template cudaError_t launch_summarize_round_blocks<uint32_t>(const uint32_t*, u64, uint32_t,
                                                             uint32_t, uint32_t,
                                                             SetView<uint32_t>, uint32_t,
                                                             cudaStream_t);
template cudaError_t launch_summarize_round_blocks<u64>(const u64*, u64, uint32_t, uint32_t,
                                                        uint32_t, SetView<u64>, uint32_t,
                                                        cudaStream_t);
template uint32_t round_batch_grid<uint32_t>(uint32_t, uint32_t, int);
template uint32_t round_batch_grid<u64>(uint32_t, uint32_t, int);
template cudaError_t launch_summarize_round_batch<uint32_t>(const BatchStream*, const BatchTask*,
                                                            uint32_t, uint32_t*, uint32_t, uint32_t,
                                                            cudaStream_t);
template cudaError_t launch_summarize_round_batch<u64>(const BatchStream*, const BatchTask*,
                                                       uint32_t, uint32_t*, uint32_t, uint32_t,
                                                       cudaStream_t);

}  // namespace pss
