// frequent.cu — Frequent (Misra–Gries) block summaries, the second
// counter-based summary the paper discusses next to Space Saving (Section 2).
//
// With k - 1 counters (the k-majority problem): an item already counted adds
// 1 to its counter; an item not counted takes a free counter with count 1;
// when no counter is free every counter loses 1, the counters that reach 0
// are freed, and the item is not stored (Misra and Gries, 1982).  Unlike
// Space Saving the result is a set with no tie to break: which free counter
// an item takes does not change it.
//
// One warp per block of Algorithm 1.  The warp's k - 1 counters (item, u32
// count) and a linear-probe hash table of 16-bit cells (slot + 1) at most
// half full live in its own slice of shared memory (24 KB at k = 2000, so
// that 9 warps share an SM).  The warp
// takes 32 items at a time, one per lane, in stream order, in rounds: every
// lane probes its item, and the round applies at once the longest prefix
// whose effects commute (additions to counters, by shared-memory atomics;
// new items taking free counters, the first occurrence of each found with
// __match_any_sync; decrement steps that cannot bring a count to 0); the
// lanes after the prefix probe again in the next round.
// A decrement step is one pass of the lanes over the counters; when it frees
// counters the warp compacts the live ones to the front and rebuilds the
// table (freed counters leave no holes in the probe runs).  There are at most
// n / k decrement steps in a block of n items, so this work adds O(1) per
// item.  The output node is sorted by item (a bitonic sort over
// the warp's slice), the layout the combine kernel reads; err and m are 0.
#include <algorithm>
#include <atomic>

#include "pss_internal.cuh"
#include "pss_kernels.cuh"

namespace pss {

namespace {

constexpr uint32_t FULL_MASK = 0xffffffffu;

template <typename ItemT>
struct FHash;
template <>
struct FHash<uint32_t> {
  __device__ static __forceinline__ uint32_t h(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
  }
};
template <>
struct FHash<u64> {
  __device__ static __forceinline__ uint32_t h(u64 x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return (uint32_t)x;
  }
};

// One warp's slice: key[cap], cnt[cap], cell[nb].
struct FLayout {
  uint32_t cap, nb, shift;
  size_t cnt, cell, bytes;
};

__host__ __device__ inline FLayout f_layout(uint32_t kc, int item_bytes) {
  FLayout L;
  L.cap = next_pow2(kc < 32 ? 32 : kc);
  L.nb = next_pow2(2 * kc < 64 ? 64 : 2 * kc);
  uint32_t lg = 0;
  while ((1u << lg) < L.nb) ++lg;
  L.shift = 32 - lg;
  auto up = [](size_t x) { return (x + 15) & ~(size_t)15; };
  L.cnt = up((size_t)item_bytes * L.cap);
  L.cell = L.cnt + up(4ull * L.cap);
  L.bytes = L.cell + up(2ull * L.nb);
  return L;
}

template <typename ItemT>
struct FWarp {
  ItemT* key;
  uint32_t* sc;      // stored counts: count + base
  unsigned short* cell;  // slot + 1, 0 = empty
  uint32_t kc, cap, nbmask, shift, lane;
  uint32_t used;     // counters in use, slots [0, used) (warp-uniform)
  uint32_t base;     // decrement steps so far (warp-uniform)
  uint32_t minc;     // full table: a lower bound on the smallest count (warp-uniform)
  uint32_t status;   // ST_* bits seen by this lane

  __device__ __forceinline__ uint32_t home(uint32_t h) const { return h >> shift; }

  // This lane's probe for x: its slot, or -1 with *epos = the first empty
  // cell of its probe run.  Cells are only added between rebuilds, so a
  // stored x sits before the first empty cell from its home.
  __device__ __forceinline__ int find(ItemT x, uint32_t h, uint32_t* epos) {
    uint32_t pos = home(h);
    for (uint32_t step = 0; step <= nbmask; ++step) {
      const uint32_t c = cell[pos];
      if (c == 0u) {
        *epos = pos;
        return -1;
      }
      if (key[c - 1] == x) return (int)c - 1;
      pos = (pos + 1) & nbmask;
    }
    status |= ST_PROBE;  // cannot happen: the table is at most half full
    *epos = 0xFFFFFFFFu;
    return -1;
  }

  // Table insert of slot s (lanes insert concurrently), walking its probe
  // run from cell pos (its home, or the first empty cell a probe of this
  // table found): a 32-bit compare-and-swap on the word holding a cell claims
  // it when empty (a failed swap because the other cell of the word changed
  // retries).
  __device__ __forceinline__ void insert(uint32_t s, uint32_t pos) {
    uint32_t* words = reinterpret_cast<uint32_t*>(cell);
    pos &= nbmask;
    for (uint32_t tries = 0; tries <= 3 * nbmask + 3; ++tries) {
      const uint32_t sh = (pos & 1u) * 16u;
      uint32_t* wp = &words[pos >> 1];
      const uint32_t old = *(volatile uint32_t*)wp;
      if ((old >> sh) & 0xFFFFu) {
        pos = (pos + 1) & nbmask;  // taken: next cell
        continue;
      }
      if (atomicCAS(wp, old, old | ((s + 1) << sh)) == old) return;
    }
    status |= ST_PROBE;
  }

  // The smallest count of the used counters (all lanes; warp-uniform result).
  __device__ uint32_t min_count() const {
    uint32_t mn = 0xFFFFFFFFu;
    for (uint32_t i = lane; i < used; i += 32) mn = min(mn, sc[i] - base);
    return __reduce_min_sync(FULL_MASK, mn);
  }

  // After a decrement step that may have brought counts to 0: free those
  // counters (live ones compacted to the front in slot order, then a fresh
  // table), else tighten the bound on the smallest count.
  __device__ void settle() {
    bool zero = false;
    for (uint32_t i = lane; i < used; i += 32) zero |= sc[i] == base;
    if (!__any_sync(FULL_MASK, zero)) {
      minc = min_count();
      return;
    }
    uint32_t live = 0;
    for (uint32_t b0 = 0; b0 < used; b0 += 32) {
      const uint32_t i = b0 + lane;
      const uint32_t c = i < used ? sc[i] : base;
      const ItemT kx = i < used ? key[i] : (ItemT)0;
      const unsigned bl = __ballot_sync(FULL_MASK, c != base);
      __syncwarp();  // every lane has read its slot before any write
      if (c != base) {
        const uint32_t d = live + (uint32_t)__popc(bl & ((1u << lane) - 1u));
        key[d] = kx;
        sc[d] = c;
      }
      live += (uint32_t)__popc(bl);
      __syncwarp();
    }
    used = live;
    for (uint32_t i = lane; i <= nbmask; i += 32) cell[i] = 0;
    __syncwarp();
    for (uint32_t i = lane; i < used; i += 32) insert(i, home(FHash<ItemT>::h(key[i])));
    __syncwarp();
  }

  // Slots [0, cap) in item order, the used ones first with their counts
  // (unused: count 0).
  __device__ void sort_by_item() {
    for (uint32_t i = lane; i < cap; i += 32) sc[i] = i < used ? sc[i] - base : 0u;
    __syncwarp();
    for (uint32_t size = 2; size <= cap; size <<= 1) {
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t i = lane; i < (cap >> 1); i += 32) {
          const uint32_t lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
          const bool asc = (lo & size) == 0;
          const ItemT ka = key[lo], kb = key[hi];
          const uint32_t ca = sc[lo], cb = sc[hi];
          const bool greater = ca == 0u ? cb != 0u : (cb != 0u && ka > kb);
          if (greater == asc) {
            key[lo] = kb; key[hi] = ka;
            sc[lo] = cb; sc[hi] = ca;
          }
        }
        __syncwarp();
      }
    }
  }
};

template <typename ItemT>
__device__ void frequent_block(const ItemT* __restrict__ xs, uint32_t len, uint32_t kc,
                               unsigned char* slice, const SetView<ItemT>& out, uint32_t node) {
  const FLayout L = f_layout(kc, (int)sizeof(ItemT));
  FWarp<ItemT> W;
  W.key = (ItemT*)slice;
  W.sc = (uint32_t*)(slice + L.cnt);
  W.cell = (unsigned short*)(slice + L.cell);
  W.kc = kc;
  W.cap = L.cap;
  W.nbmask = L.nb - 1;
  W.shift = L.shift;
  W.lane = threadIdx.x & 31;
  W.used = 0;
  W.base = 0;
  W.minc = 0;
  W.status = 0;
  for (uint32_t i = W.lane; i < L.nb; i += 32) W.cell[i] = 0;
  __syncwarp();
  const unsigned below = (1u << W.lane) - 1u;

  // 32 items per coalesced load (lane i holds item t0 + i), the next 32 in
  // flight meanwhile.  Lanes [start, here) are still to be applied; each
  // round applies a prefix of them whose effects commute and probes the rest
  // again.
  ItemT nxt = W.lane < len ? xs[W.lane] : (ItemT)0;
  for (uint32_t t0 = 0; t0 < len; t0 += 32) {
    const ItemT x = nxt;
    const uint32_t here = min(32u, len - t0);
    if (t0 + 32 + W.lane < len) nxt = xs[t0 + 32 + W.lane];
    const uint32_t h = FHash<ItemT>::h(x);
    uint32_t start = 0;
    while (start < here) {
      const bool act = W.lane >= start && W.lane < here;
      int s = -1;
      uint32_t epos = 0xFFFFFFFFu;
      if (act) s = W.find(x, h, &epos);
      const bool miss = act && s < 0;
      const unsigned mm = __ballot_sync(FULL_MASK, miss);
      uint32_t end;
      if (W.used < kc) {
        // Free counters: the first occurrence (leader) of each missing item
        // takes one, its later occurrences in the round add to it.  The round
        // ends at the first leader that finds no free counter.
        unsigned grp = 0;
        if (miss) grp = __match_any_sync(mm, x);
        const bool leader = miss && (grp & below) == 0;
        const unsigned lead = __ballot_sync(FULL_MASK, leader);
        const uint32_t free_n = kc - W.used;
        end = (uint32_t)__popc(lead) <= free_n ? here : (uint32_t)__fns(lead, 0, (int)free_n + 1);
        if (leader && W.lane < end) {
          const uint32_t slot = W.used + (uint32_t)__popc(lead & below);
          W.key[slot] = x;
          W.sc[slot] = W.base + 1u;
          W.insert(slot, epos);  // cells before it in the run stay taken
        }
        __syncwarp();
        if (W.lane < end) {
          if (act && !miss) {
            atomicAdd(&W.sc[s], 1u);
          } else if (miss && !leader) {
            const uint32_t lo = (uint32_t)__ffs(grp) - 1;
            atomicAdd(&W.sc[W.used + (uint32_t)__popc(lead & ((1u << lo) - 1u))], 1u);
          }
        }
        W.used += (uint32_t)__popc(lead & (end >= 32 ? FULL_MASK : (1u << end) - 1u));
        if (W.used == kc) W.minc = 1;  // new counters hold 1
      } else {
        // Full table: every missing occurrence is a decrement step.  While
        // fewer steps than the smallest count have run, no count reaches 0,
        // so the table's membership is fixed and hits and steps commute.
        const uint32_t nm = (uint32_t)__popc(mm);
        const uint32_t take = nm < W.minc ? nm : W.minc;  // steps applied now
        end = nm < W.minc ? here : (uint32_t)__fns(mm, 0, (int)W.minc) + 1;
        if (act && !miss && W.lane < end) atomicAdd(&W.sc[s], 1u);
        W.base += take;
        W.minc -= take;
      }
      __syncwarp();
      if (W.used == kc && W.minc == 0) W.settle();
      start = end;
    }
    __syncwarp();
  }

  W.sort_by_item();
  const size_t base = (size_t)node * out.k;
  for (uint32_t i = W.lane; i < W.used; i += 32) {
    out.item[base + i] = W.key[i];
    out.count[base + i] = W.sc[i];
    out.err[base + i] = 0ull;
  }
  const uint32_t st = __reduce_or_sync(FULL_MASK, W.status);
  if (W.lane == 0) {
    out.size[node] = W.used;
    out.m[node] = 0ull;
    out.ncov[node] = len;
    if (st) atomicOr(out.status, st);
  }
}

// Warp w of CTA b summarizes block r0 + b * warps + w of p into node
// node0 + b * warps + w; each warp owns `wbytes` of shared memory.
template <typename ItemT>
__global__ void __launch_bounds__(256) frequent_block_kernel(const ItemT* __restrict__ items,
                                                             u64 n, uint32_t p, uint32_t r0,
                                                             uint32_t count, SetView<ItemT> out,
                                                             uint32_t node0, uint32_t kc,
                                                             uint32_t wbytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t j = blockIdx.x * (blockDim.x >> 5) + warp;
  if (j >= count) return;  // the whole warp
  const uint32_t r = r0 + j, node = node0 + j;
  const u64 left = block_bound(r, n, p), right = block_bound((u64)r + 1, n, p);
  if (right - left >= (1ull << 32)) {
    if (lane == 0) {
      out.size[node] = 0;
      out.m[node] = 0;
      out.ncov[node] = right - left;
      atomicOr(out.status, (uint32_t)ST_CHUNK);
    }
    return;
  }
  frequent_block<ItemT>(items + left, (uint32_t)(right - left), kc, smem + (size_t)warp * wbytes,
                        out, node);
}

// Persistent form for many streams: each warp takes (stream, block) tasks
// from a shared counter until the list is exhausted (the tasks of one launch
// share kc, so every warp's slice has one layout).
template <typename ItemT>
__global__ void __launch_bounds__(256) frequent_batch_kernel(const BatchStream* __restrict__ streams,
                                                             const BatchTask* __restrict__ tasks,
                                                             uint32_t ntasks, uint32_t* counter,
                                                             uint32_t wbytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* slice = smem + (size_t)warp * wbytes;
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(counter, 1u);
    t = __shfl_sync(FULL_MASK, t, 0);
    if (t >= ntasks) break;
    const BatchTask task = tasks[t];
    const BatchStream st = streams[task.stream];
    const SetView<ItemT> out = set_view_dev<ItemT>(st.level0, st.p, st.k);
    const u64 left = block_bound(task.index, st.n, st.p);
    const u64 right = block_bound((u64)task.index + 1, st.n, st.p);
    if (right - left >= (1ull << 32)) {
      if (lane == 0) {
        out.size[task.index] = 0;
        out.m[task.index] = 0;
        out.ncov[task.index] = right - left;
        atomicOr(out.status, (uint32_t)ST_CHUNK);
      }
      continue;
    }
    frequent_block<ItemT>((const ItemT*)st.items + left, (uint32_t)(right - left), st.k, slice,
                          out, task.index);
    __syncwarp();
  }
}

// Warps per CTA with the most warps resident per SM (ties: fewer), per k.
template <typename ItemT>
int frequent_warps_per_cta(uint32_t kc) {
  static std::atomic<int> memo[PSS_MAX_K_RESIDENT + 1];
  if (kc > PSS_MAX_K_RESIDENT) return 0;
  int v = memo[kc].load(std::memory_order_relaxed);
  if (v) return v;
  const void* kern = (const void*)frequent_block_kernel<ItemT>;
  if (ensure_kernel_attrs(kern) != cudaSuccess) return 0;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  const size_t wb = f_layout(kc, (int)sizeof(ItemT)).bytes;
  int best = 0, best_warps = 0;
  for (int wpc = 1; wpc <= 8; wpc *= 2) {
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
  if (best) memo[kc].store(best, std::memory_order_relaxed);
  return best;
}

}  // namespace

size_t frequent_warp_bytes(uint32_t kc, int item_bytes) { return f_layout(kc, item_bytes).bytes; }

template <typename ItemT>
cudaError_t launch_frequent_blocks(const ItemT* items, u64 n, uint32_t p, uint32_t r0,
                                   uint32_t count, SetView<ItemT> out, uint32_t node0,
                                   cudaStream_t stream) {
  const uint32_t kc = out.k;
  const int wpc = frequent_warps_per_cta<ItemT>(kc);
  if (wpc <= 0) return cudaErrorInvalidConfiguration;
  if (count == 0) return cudaSuccess;
  const size_t wb = f_layout(kc, (int)sizeof(ItemT)).bytes;
  const uint32_t grid = (count + (uint32_t)wpc - 1) / (uint32_t)wpc;
  frequent_block_kernel<ItemT><<<grid, 32 * wpc, (size_t)wpc * wb, stream>>>(
      items, n, p, r0, count, out, node0, kc, (uint32_t)wb);
  return cudaGetLastError();
}

template <typename ItemT>
uint32_t frequent_batch_grid(uint32_t kc, uint32_t ntasks, int sms) {
  if (kc == 0 || kc > PSS_MAX_K_RESIDENT) return 0;
  const int wpc = frequent_warps_per_cta<ItemT>(kc);
  if (wpc <= 0) return 0;
  const void* kern = (const void*)frequent_batch_kernel<ItemT>;
  if (ensure_kernel_attrs(kern) != cudaSuccess) return 0;
  const size_t wb = f_layout(kc, (int)sizeof(ItemT)).bytes;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, 32 * wpc, (size_t)wpc * wb) !=
          cudaSuccess ||
      blocks <= 0)
    return 0;
  const uint64_t need = (ntasks + (uint32_t)wpc - 1) / (uint32_t)wpc;
  return (uint32_t)std::min<uint64_t>((uint64_t)sms * (uint64_t)blocks, need ? need : 1);
}

template <typename ItemT>
cudaError_t launch_frequent_batch(const BatchStream* streams, const BatchTask* tasks,
                                  uint32_t ntasks, uint32_t* counter, uint32_t kc, uint32_t grid,
                                  cudaStream_t stream) {
  const int wpc = frequent_warps_per_cta<ItemT>(kc);
  if (wpc <= 0) return cudaErrorInvalidConfiguration;
  cudaError_t e = ensure_kernel_attrs((const void*)frequent_batch_kernel<ItemT>);
  if (e != cudaSuccess) return e;
  if (ntasks == 0 || grid == 0) return cudaSuccess;
  const size_t wb = f_layout(kc, (int)sizeof(ItemT)).bytes;
  frequent_batch_kernel<ItemT><<<grid, 32 * wpc, (size_t)wpc * wb, stream>>>(streams, tasks, ntasks,
                                                                            counter, (uint32_t)wb);
  return cudaGetLastError();
}

template uint32_t frequent_batch_grid<uint32_t>(uint32_t, uint32_t, int);
template uint32_t frequent_batch_grid<u64>(uint32_t, uint32_t, int);
template cudaError_t launch_frequent_batch<uint32_t>(const BatchStream*, const BatchTask*, uint32_t,
                                                     uint32_t*, uint32_t, uint32_t, cudaStream_t);
template cudaError_t launch_frequent_batch<u64>(const BatchStream*, const BatchTask*, uint32_t,
                                                uint32_t*, uint32_t, uint32_t, cudaStream_t);
template cudaError_t launch_frequent_blocks<uint32_t>(const uint32_t*, u64, uint32_t, uint32_t,
                                                      uint32_t, SetView<uint32_t>, uint32_t,
                                                      cudaStream_t);
template cudaError_t launch_frequent_blocks<u64>(const u64*, u64, uint32_t, uint32_t, uint32_t,
                                                 SetView<u64>, uint32_t, cudaStream_t);

}  // namespace pss
