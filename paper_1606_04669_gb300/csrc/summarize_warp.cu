// summarize_warp.cu — per-block Space Saving for small k (Section 3 update
// rule on the block bounds of Algorithm 1): one warp per block, the k <= 256
// counters held in the warp's registers, CPL per lane (slot q lives in lane
// q % 32 at index q / 32).
//
// With few counters nearly every item of a weakly skewed stream is a miss,
// so the bucket of minimum count runs out every few dozen items and a
// window-parallel CTA would cut its windows almost at once.  Here the rule
// is applied one item at a time, as written:
//   * hit: one ballot over the lanes' comparisons; the owning lane adds one
//     and stamps the position;
//   * fill: the next free slot takes the item (count 1, err 0);
//   * miss on a full summary: the victim is the minimum of (count, touch) over
//     all counters — each lane keeps the minimum of its own CPL counters, two
//     warp min-reductions (count, then touch among the minimum counts) find
//     the lane; touches of distinct counters differ, so the victim is unique.
//     In a block of fewer than 2^16 items every count and touch fits in 16
//     bits, so (count << 16 | touch) orders the counters the same way and one
//     reduction of that key finds the victim (PACK).
// Output: the block's summary sorted by item ascending (rank of each entry =
// number of smaller items), minimum m (if k counters are in use, else 0) and
// the block length.
#include "pss_internal.cuh"
#include "pss_kernels.cuh"

namespace pss {

namespace {

constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr int WS_WPB = 4;  // warps (blocks in flight) per CTA

template <typename ItemT, int CPL, bool PACK>
__device__ void warp_summarize(const ItemT* __restrict__ items, u64 n, uint32_t p, uint32_t r,
                               const SetView<ItemT>& out, uint32_t node) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t k = out.k;
  const size_t obase = (size_t)node * k;
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
  const uint32_t len = (uint32_t)(right - left);
  const ItemT* __restrict__ xs = items + left;

  ItemT it[CPL];
  uint32_t cn[CPL], tc[CPL], er[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    it[c] = (ItemT)0;
    cn[c] = 0;  // 0: slot not in use
    tc[c] = 0;
    er[c] = 0;
  }
  uint32_t used = 0;
  // this lane's minimum (count, touch) over its slots in use, and its index
  uint32_t lc = NONE, lt = NONE;
  int li = 0;
  auto local_min = [&]() {
    lc = NONE;
    lt = NONE;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      if constexpr (PACK) {  // lc holds the packed key
        const uint32_t key = cn[c] ? (cn[c] << 16) | tc[c] : NONE;
        if (key < lc) {
          lc = key;
          li = c;
        }
      } else if (cn[c] && (cn[c] < lc || (cn[c] == lc && tc[c] < lt))) {
        lc = cn[c];
        lt = tc[c];
        li = c;
      }
    }
  };

  ItemT v = lane < len ? xs[lane] : (ItemT)0;
  for (uint32_t base = 0; base < len; base += 32) {
    const uint32_t nb = min(32u, len - base);
    const ItemT cur = v;
    if (base + 32 + lane < len) v = xs[base + 32 + lane];
    for (uint32_t i = 0; i < nb; ++i) {
      const ItemT x = __shfl_sync(0xffffffffu, cur, i);
      const uint32_t t = base + i;
      int hc = -1;
#pragma unroll
      for (int c = 0; c < CPL; ++c)
        if (cn[c] && it[c] == x) hc = c;
      if (__ballot_sync(0xffffffffu, hc >= 0)) {
        if (hc >= 0) {
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            if (c == hc) {
              cn[c] += 1;
              tc[c] = t;
            }
          }
          if (used == k && hc == li) local_min();
        }
      } else if (used < k) {
        if (lane == (used & 31)) {
          const int cq = (int)(used >> 5);
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            if (c == cq) {
              it[c] = x;
              cn[c] = 1;
              tc[c] = t;
              er[c] = 0;
            }
          }
        }
        ++used;
        if (used == k) local_min();
      } else {
        bool victim;
        if constexpr (PACK) {
          victim = lc == __reduce_min_sync(0xffffffffu, lc);
        } else {
          const uint32_t mc = __reduce_min_sync(0xffffffffu, lc);
          const uint32_t mt = __reduce_min_sync(0xffffffffu, lc == mc ? lt : NONE);
          victim = lc == mc && lt == mt;
        }
        if (victim) {
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            if (c == li) {
              er[c] = cn[c];
              cn[c] += 1;
              it[c] = x;
              tc[c] = t;
            }
          }
          local_min();
        }
      }
    }
  }

  // ---- output: rank of each entry among the items in use
  uint32_t rank[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) rank[c] = 0;
  for (int src = 0; src < 32; ++src) {
#pragma unroll
    for (int c2 = 0; c2 < CPL; ++c2) {
      const ItemT y = __shfl_sync(0xffffffffu, it[c2], src);
      const uint32_t yc = __shfl_sync(0xffffffffu, cn[c2], src);
#pragma unroll
      for (int c = 0; c < CPL; ++c) rank[c] += (yc && y < it[c]) ? 1u : 0u;
    }
  }
  uint32_t mn = NONE;
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    if (cn[c]) {
      out.item[obase + rank[c]] = it[c];
      out.count[obase + rank[c]] = cn[c];
      out.err[obase + rank[c]] = er[c];
      mn = min(mn, cn[c]);
    }
  }
  mn = __reduce_min_sync(0xffffffffu, mn);
  if (lane == 0) {
    out.size[node] = used;
    out.m[node] = (used == k) ? (u64)mn : 0ull;
    out.ncov[node] = len;
  }
}

// Block r with the packed keys when it holds fewer than 2^16 items.
template <typename ItemT, int CPL>
__device__ __forceinline__ void summarize_one(const ItemT* __restrict__ items, u64 n, uint32_t p,
                                              uint32_t r, const SetView<ItemT>& out, uint32_t node) {
  if (block_bound((u64)r + 1, n, p) - block_bound(r, n, p) < (1ull << 16))
    warp_summarize<ItemT, CPL, true>(items, n, p, r, out, node);
  else
    warp_summarize<ItemT, CPL, false>(items, n, p, r, out, node);
}

template <typename ItemT, int CPL>
__global__ void __launch_bounds__(32 * WS_WPB) ssw_block_kernel(const ItemT* __restrict__ items,
                                                                 u64 n, uint32_t p, uint32_t r0,
                                                                 uint32_t count,
                                                                 SetView<ItemT> out,
                                                                 uint32_t node0) {
  const uint32_t w = blockIdx.x * WS_WPB + (threadIdx.x >> 5);
  if (w >= count) return;
  summarize_one<ItemT, CPL>(items, n, p, r0 + w, out, node0 + w);
}

// Persistent form: each warp takes (stream, block) tasks from the counter.
template <typename ItemT, int CPL>
__global__ void __launch_bounds__(32 * WS_WPB) ssw_batch_kernel(const BatchStream* __restrict__ streams,
                                                                 const BatchTask* __restrict__ tasks,
                                                                 uint32_t ntasks, uint32_t* counter) {
  const uint32_t lane = threadIdx.x & 31;
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= ntasks) break;
    const BatchTask task = tasks[t];
    const BatchStream st = streams[task.stream];
    const SetView<ItemT> out = set_view_dev<ItemT>(st.level0, st.p, st.k);
    summarize_one<ItemT, CPL>((const ItemT*)st.items, st.n, st.p, task.index, out, task.index);
  }
}

template <typename ItemT, int CPL>
cudaError_t launch_blocks_cpl(const ItemT* items, u64 n, uint32_t p, uint32_t r0, uint32_t count,
                              SetView<ItemT> out, uint32_t node0, cudaStream_t stream) {
  const uint32_t grid = (count + WS_WPB - 1) / WS_WPB;
  ssw_block_kernel<ItemT, CPL><<<grid, 32 * WS_WPB, 0, stream>>>(items, n, p, r0, count, out, node0);
  return cudaGetLastError();
}

template <typename ItemT, int CPL>
cudaError_t launch_batch_cpl(const BatchStream* streams, const BatchTask* tasks, uint32_t ntasks,
                             uint32_t* counter, uint32_t grid, cudaStream_t stream) {
  ssw_batch_kernel<ItemT, CPL><<<grid, 32 * WS_WPB, 0, stream>>>(streams, tasks, ntasks, counter);
  return cudaGetLastError();
}

template <typename ItemT, int CPL>
int ctas_cpl() {
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ssw_batch_kernel<ItemT, CPL>,
                                                    32 * WS_WPB, 0) != cudaSuccess)
    return 0;
  return blocks;
}

}  // namespace

template <typename ItemT>
cudaError_t launch_summarize_warp_blocks(const ItemT* items, u64 n, uint32_t p, uint32_t r0,
                                         uint32_t count, SetView<ItemT> out, uint32_t node0,
                                         cudaStream_t stream) {
  if (count == 0) return cudaSuccess;
  if (out.k <= 64) return launch_blocks_cpl<ItemT, 2>(items, n, p, r0, count, out, node0, stream);
  if (out.k <= 128) return launch_blocks_cpl<ItemT, 4>(items, n, p, r0, count, out, node0, stream);
  if (out.k <= 256) return launch_blocks_cpl<ItemT, 8>(items, n, p, r0, count, out, node0, stream);
  return cudaErrorInvalidValue;
}

template <typename ItemT>
cudaError_t launch_summarize_warp_batch(const BatchStream* streams, const BatchTask* tasks,
                                        uint32_t ntasks, uint32_t* counter, uint32_t k,
                                        uint32_t grid, cudaStream_t stream) {
  if (ntasks == 0 || grid == 0) return cudaSuccess;
  if (k <= 64) return launch_batch_cpl<ItemT, 2>(streams, tasks, ntasks, counter, grid, stream);
  if (k <= 128) return launch_batch_cpl<ItemT, 4>(streams, tasks, ntasks, counter, grid, stream);
  if (k <= 256) return launch_batch_cpl<ItemT, 8>(streams, tasks, ntasks, counter, grid, stream);
  return cudaErrorInvalidValue;
}

template <typename ItemT>
int summarize_warp_ctas_per_sm(uint32_t k) {
  if (k <= 64) return ctas_cpl<ItemT, 2>();
  if (k <= 128) return ctas_cpl<ItemT, 4>();
  if (k <= 256) return ctas_cpl<ItemT, 8>();
  return 0;
}

template cudaError_t launch_summarize_warp_blocks<uint32_t>(const uint32_t*, u64, uint32_t,
                                                            uint32_t, uint32_t, SetView<uint32_t>,
                                                            uint32_t, cudaStream_t);
template cudaError_t launch_summarize_warp_blocks<u64>(const u64*, u64, uint32_t, uint32_t,
                                                       uint32_t, SetView<u64>, uint32_t,
                                                       cudaStream_t);
template cudaError_t launch_summarize_warp_batch<uint32_t>(const BatchStream*, const BatchTask*,
                                                           uint32_t, uint32_t*, uint32_t,
                                                           uint32_t, cudaStream_t);
template cudaError_t launch_summarize_warp_batch<u64>(const BatchStream*, const BatchTask*,
                                                      uint32_t, uint32_t*, uint32_t, uint32_t,
                                                      cudaStream_t);
template int summarize_warp_ctas_per_sm<uint32_t>(uint32_t);
template int summarize_warp_ctas_per_sm<u64>(uint32_t);

}  // namespace pss
