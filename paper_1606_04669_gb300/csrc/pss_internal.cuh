// pss_internal.cuh — device data layout and block-level helpers of libpss.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pss.h"

namespace pss {

typedef unsigned long long u64;

// Status bits a kernel records in the summaries it produces.
enum : uint32_t {
  ST_PROBE = 1u << 0,     // a hash probe sequence ran past the table size
  ST_NOPROGRESS = 1u << 1,  // the window loop made no progress twice in a row
  ST_CHUNK = 1u << 2,     // a block held 2^32 items or more
  ST_LAYOUT = 1u << 3,    // inconsistent launch parameters
};

// A set of `nodes` summaries of capacity k each, structure of arrays:
// node j's entries are item/count/err[j*k, j*k + size[j]), sorted by item.
template <typename ItemT>
struct SetView {
  ItemT* item;
  u64* count;
  u64* err;
  uint32_t* size;
  u64* m;
  u64* ncov;
  uint32_t* status;  // one word per set: OR of ST_* bits of every producer
  uint32_t nodes;
  uint32_t k;
};

// Byte layout of one set allocation.
struct SetLayout {
  size_t item, count, err, size, m, ncov, status, total;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline SetLayout set_layout(uint32_t nodes, uint32_t k, int item_bytes) {
  SetLayout L;
  size_t e = (size_t)nodes * k;
  size_t off = 0;
  L.item = off;   off = align_up(off + e * item_bytes, 256);
  L.count = off;  off = align_up(off + e * 8, 256);
  L.err = off;    off = align_up(off + e * 8, 256);
  L.size = off;   off = align_up(off + (size_t)nodes * 4, 256);
  L.m = off;      off = align_up(off + (size_t)nodes * 8, 256);
  L.ncov = off;   off = align_up(off + (size_t)nodes * 8, 256);
  L.status = off; off = align_up(off + 4, 256);
  L.total = off;
  return L;
}

template <typename ItemT>
inline SetView<ItemT> set_view(void* base, uint32_t nodes, uint32_t k) {
  SetLayout L = set_layout(nodes, k, (int)sizeof(ItemT));
  char* b = (char*)base;
  SetView<ItemT> v;
  v.item = (ItemT*)(b + L.item);
  v.count = (u64*)(b + L.count);
  v.err = (u64*)(b + L.err);
  v.size = (uint32_t*)(b + L.size);
  v.m = (u64*)(b + L.m);
  v.ncov = (u64*)(b + L.ncov);
  v.status = (uint32_t*)(b + L.status);
  v.nodes = nodes;
  v.k = k;
  return v;
}

// Device-side view of a set allocation (same layout as set_layout).
template <typename ItemT>
__device__ __forceinline__ SetView<ItemT> set_view_dev(void* base, uint32_t nodes, uint32_t k) {
  const size_t e = (size_t)nodes * k;
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  char* b = (char*)base;
  size_t off = 0;
  SetView<ItemT> v;
  v.item = (ItemT*)(b + off);    off = up(off + e * sizeof(ItemT));
  v.count = (u64*)(b + off);     off = up(off + e * 8);
  v.err = (u64*)(b + off);       off = up(off + e * 8);
  v.size = (uint32_t*)(b + off); off = up(off + (size_t)nodes * 4);
  v.m = (u64*)(b + off);         off = up(off + (size_t)nodes * 8);
  v.ncov = (u64*)(b + off);      off = up(off + (size_t)nodes * 8);
  v.status = (uint32_t*)(b + off);
  v.nodes = nodes;
  v.k = k;
  return v;
}

// One stream of a batch (device-resident descriptor).
struct BatchStream {
  const void* items;  // device items of the stream
  u64 n;              // its length
  uint32_t p, k;      // blocks and counters
  void* level0;       // set of p block summaries (set_layout(p, k, w))
};

// One unit of work of a batch: block `index` of stream `stream`, or (merge)
// node `index` of the next level of stream `stream`.
struct BatchTask {
  uint32_t stream, index;
};

// One stream's step of the reduction tree in a batch: level `in` (in_nodes
// summaries) into level `out` (ceil(in_nodes / 2) summaries).
struct MergeDesc {
  void* in;
  void* out;
  uint32_t in_nodes, k;
};

// One stream's query in a batch: Pruned(root, n, kq) written at out_off;
// k is the root's capacity, filter the query of launch_canon (1: Space
// Saving candidates, 3: Frequent candidates).
struct QueryDesc {
  void* root;
  u64 n;
  uint32_t k, out_off;
  uint32_t kq;
  int32_t filter;
};

// floor(r * n / p) without overflow (r <= p, p < 2^32): 128-bit product,
// long division by 32-bit digits.  Algorithm 1's block bound.
__host__ __device__ inline u64 block_bound(u64 r, u64 n, uint32_t p) {
#if defined(__CUDA_ARCH__)
  u64 hi = __umul64hi(r, n);
#else
  u64 hi = (u64)(((unsigned __int128)r * n) >> 64);
#endif
  u64 lo = r * n;
  uint32_t d[4] = {(uint32_t)(hi >> 32), (uint32_t)hi, (uint32_t)(lo >> 32), (uint32_t)lo};
  u64 rem = 0, q = 0;
  for (int i = 0; i < 4; ++i) {
    u64 cur = (rem << 32) | d[i];
    u64 qd = cur / p;
    rem = cur - qd * p;
    q = (q << 32) | qd;  // the top two quotient digits are zero (result < 2^64)
  }
  return q;
}

// ---------------------------------------------------------------- block scan

// Exclusive prefix sum of v over the block (BS threads, BS a multiple of
// 32).  `warp_sums` holds BS/32 + 1 words of shared scratch.  Returns the
// exclusive prefix; *total receives the block sum.  Contains two barriers.
template <int BS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums,
                                                         uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    constexpr int NW = BS / 32;
    uint32_t w = lane < NW ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NW) warp_sums[lane] = w;  // inclusive
    if (lane == NW - 1) warp_sums[NW] = w;
  }
  __syncthreads();
  uint32_t before = warp ? warp_sums[warp - 1] : 0;
  *total = warp_sums[BS / 32];
  return before + x - v;
}

// ------------------------------------------------------------- bitonic sort

// Sort n2 (a power of two) pairs (key, pay) ascending by (key, pay) in
// shared memory; all threads of the block call it.  Ends with a barrier.
template <int BS, typename PayT>
__device__ void block_bitonic_sort(u64* key, PayT* pay, uint32_t n2) {
  for (uint32_t size = 2; size <= n2; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < (n2 >> 1); i += BS) {
        uint32_t lo = 2 * i - (i & (stride - 1));
        uint32_t hi = lo + stride;
        bool asc = (lo & size) == 0;
        u64 ka = key[lo], kb = key[hi];
        PayT pa = pay[lo], pb = pay[hi];
        bool greater = (ka > kb) || (ka == kb && pa > pb);
        if (greater == asc) {
          key[lo] = kb; key[hi] = ka;
          pay[lo] = pb; pay[hi] = pa;
        }
      }
      __syncthreads();
    }
  }
}

__host__ __device__ inline uint32_t next_pow2(uint32_t x) {
  uint32_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace pss
