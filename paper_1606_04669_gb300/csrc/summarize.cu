// summarize.cu — per-block Space Saving (Section 3 update rule; Algorithm 1's
// SpaceSaving call on the block bounds of Algorithm 1), one CTA per block.
//
// The sequential rule, with k counters (item, count, err, touch):
//   x monitored            -> count += 1, touch = t
//   a counter is free      -> (x, 1, 0, t)
//   else, victim v = argmin (count, touch) -> err = count, count += 1,
//                                              item = x, touch = t
// is reproduced exactly while the CTA consumes a window of BS items at once:
//
//   1. every thread looks its item up in a shared-memory open-addressing
//      table (item -> counter slot); hits commute with one another, so a
//      window of hits only is applied with atomics;
//   2. missing items are de-duplicated inside the window (first occurrence by
//      position), ranked by position, and the r-th one is given the r-th
//      oldest counter of the minimum-count bucket.  That bucket is kept as a
//      list sorted by touch (the FIFO of the counters that reached the
//      minimum count, oldest first); entries invalidated by a later hit are
//      skipped lazily (their count is no longer the minimum);
//   3. the assignment is exact for the window prefix in which no hit lands on
//      a counter that a miss of that prefix evicts, the bucket does not run
//      out and the table does not fill up; the window is cut at the first
//      position where one of these fails, the prefix is applied, and the next
//      window starts there;
//   4. when the bucket runs out, the next one is built from (a) the counters
//      already at that count before the current epoch, sorted by touch, and
//      (b) the log of counters that reached it during the epoch, which is
//      already in time order.
//
// Output: the block's summary sorted by item ascending, with size, minimum m
// (the minimum count if k counters are in use, else 0) and the block length.
#include "pss_internal.cuh"
#include "pss_kernels.cuh"

namespace pss {

namespace {

constexpr uint16_t CELL_EMPTY = 0;
constexpr uint16_t CELL_TOMB = 0xFFFF;

template <typename ItemT>
struct ItemOps;
template <>
struct ItemOps<uint32_t> {
  static constexpr uint32_t SENT = 0xFFFFFFFFu;
  __device__ static __forceinline__ uint32_t h1(uint32_t x) { return x * 0x9E3779B1u; }
  __device__ static __forceinline__ uint32_t h2(uint32_t x) { return x * 0x85EBCA77u; }
  __device__ static __forceinline__ u64 sort_key(uint32_t x, uint32_t slot) {
    return ((u64)x << 16) | slot;
  }
};
template <>
struct ItemOps<u64> {
  static constexpr u64 SENT = ~0ull;
  __device__ static __forceinline__ uint32_t h1(u64 x) {
    return (uint32_t)((x * 0x9E3779B97F4A7C15ull) >> 32);
  }
  __device__ static __forceinline__ uint32_t h2(u64 x) {
    return (uint32_t)((x * 0xC2B2AE3D27D4EB4Full) >> 32);
  }
  __device__ static __forceinline__ u64 sort_key(u64 x, uint32_t) { return x; }
};

struct SSState {
  uint32_t m;            // count of the minimum bucket (valid once full)
  uint32_t head;         // next unread index of the bucket list
  uint32_t list_len;
  uint32_t log_len;      // entries of the next-bucket log
  uint32_t log_over;     // log overflowed: next rebuild scans everything
  uint32_t used;         // counters in use
  uint32_t full;         // used == k
  uint32_t tombs;        // tombstones in the hash table
  uint32_t tomb_reuse;   // tombstones re-used by this window's inserts
  uint32_t epoch_start;  // position at which the current bucket list was built
  uint32_t P;            // exact prefix of the current window
  uint32_t found, j0;    // victim gathering cursor
  uint32_t need_rebuild; // 0 none, 1 incremental, 2 full scan
  uint32_t stall;
  uint32_t status;
  uint32_t red;          // reduction scratch
};

template <typename ItemT, int BS>
struct SSSmem {
  uint32_t C, cshift, WT, wshift, LOGCAP, SORTN;
  u64* skey;
  ItemT* item;
  uint32_t* cnt;
  uint32_t* err;
  uint32_t* touch;
  ItemT* wkey;
  uint32_t* wpos;
  uint32_t* rankpos;
  uint32_t* Vidx;
  uint32_t* wsum;   // 2 * (BS/32 + 1)
  uint16_t* cellof;
  uint16_t* hash;
  uint16_t* list;
  uint16_t* logq;
  uint16_t* vrank;
  uint16_t* spay;
  uint16_t* wslot;
  uint16_t* V;
};

__host__ __device__ inline uint32_t ilog2(uint32_t x) {
  uint32_t r = 0;
  while ((1u << r) < x) ++r;
  return r;
}

template <typename ItemT, int BS>
__host__ __device__ inline size_t ss_carve(uint32_t k, unsigned char* base, SSSmem<ItemT, BS>* s) {
  SSSmem<ItemT, BS> L;
  L.C = next_pow2(2 * k < 64 ? 64 : 2 * k);
  L.cshift = 32 - ilog2(L.C);
  L.WT = 2 * BS;
  L.wshift = 32 - ilog2(L.WT);
  L.LOGCAP = 2 * k;
  L.SORTN = next_pow2(k);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = (off + bytes + 15) & ~(size_t)15;
    return base + o;
  };
  L.skey = (u64*)take(8ull * L.SORTN);
  L.item = (ItemT*)take(sizeof(ItemT) * k);
  L.cnt = (uint32_t*)take(4ull * k);
  L.err = (uint32_t*)take(4ull * k);
  L.touch = (uint32_t*)take(4ull * k);
  L.wkey = (ItemT*)take(sizeof(ItemT) * (L.WT + 1));
  L.wpos = (uint32_t*)take(4ull * (L.WT + 1));
  L.rankpos = (uint32_t*)take(4ull * BS);
  L.Vidx = (uint32_t*)take(4ull * BS);
  L.wsum = (uint32_t*)take(4ull * 2 * (BS / 32 + 1));
  L.cellof = (uint16_t*)take(2ull * k);
  L.hash = (uint16_t*)take(2ull * L.C);
  L.list = (uint16_t*)take(2ull * k);
  L.logq = (uint16_t*)take(2ull * L.LOGCAP);
  L.vrank = (uint16_t*)take(2ull * k);
  L.spay = (uint16_t*)take(2ull * L.SORTN);
  L.wslot = (uint16_t*)take(2ull * (L.WT + 1));
  L.V = (uint16_t*)take(2ull * BS);
  if (s) *s = L;
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

template <typename ItemT, int BS>
struct SSBlock {
  SSSmem<ItemT, BS> s;
  SSState* S;
  uint32_t k;
  uint32_t sb;  // scan scratch parity

  __device__ __forceinline__ uint32_t scan(uint32_t v, uint32_t* total) {
    uint32_t* buf = s.wsum + (sb ? (BS / 32 + 1) : 0);
    sb ^= 1;
    return block_exclusive_scan<BS>(v, buf, total);
  }

  __device__ __forceinline__ int lookup(ItemT x, uint32_t& status) const {
    uint32_t c = ItemOps<ItemT>::h1(x) >> s.cshift;
    const uint32_t mask = s.C - 1;
    for (uint32_t i = 0; i < s.C; ++i) {
      uint16_t v = s.hash[c];
      if (v == CELL_EMPTY) return -1;
      if (v != CELL_TOMB && s.item[v - 1] == x) return (int)v - 1;
      c = (c + 1) & mask;
    }
    status |= ST_PROBE;
    return -1;
  }

  // Claim the first empty or tombstone cell of x's probe sequence for slot.
  __device__ __forceinline__ void insert(ItemT x, uint32_t slot, uint32_t& status) {
    uint32_t c = ItemOps<ItemT>::h1(x) >> s.cshift;
    const uint32_t mask = s.C - 1;
    for (uint32_t i = 0; i < 4 * s.C; ++i) {
      uint16_t v = s.hash[c];
      if (v == CELL_EMPTY || v == CELL_TOMB) {
        uint16_t old = atomicCAS(&s.hash[c], v, (uint16_t)(slot + 1));
        if (old == v) {
          if (v == CELL_TOMB) atomicAdd(&S->tomb_reuse, 1u);
          s.cellof[slot] = (uint16_t)c;
          return;
        }
        continue;  // lost the race for this cell: look at it again
      }
      c = (c + 1) & mask;
    }
    status |= ST_PROBE;
  }

  // Window de-duplication table: returns the cell of x, and keeps in wpos
  // the smallest position at which x missed.
  __device__ __forceinline__ uint32_t wtab_insert(ItemT x, uint32_t t) {
    uint32_t c;
    if (x == ItemOps<ItemT>::SENT) {
      c = s.WT;
    } else {
      c = ItemOps<ItemT>::h2(x) >> s.wshift;
      for (uint32_t i = 0; i < s.WT; ++i) {
        ItemT prev = atomicCAS(&s.wkey[c], ItemOps<ItemT>::SENT, x);
        if (prev == ItemOps<ItemT>::SENT || prev == x) break;
        c = (c + 1) & (s.WT - 1);
      }
    }
    atomicMin(&s.wpos[c], t);
    return c;
  }

  __device__ void rebuild_hash(uint32_t& status) {
    for (uint32_t c = threadIdx.x; c < s.C; c += BS) s.hash[c] = CELL_EMPTY;
    __syncthreads();
    const uint32_t used = S->used;
    for (uint32_t i = threadIdx.x; i < used; i += BS) insert(s.item[i], i, status);
    __syncthreads();
    if (threadIdx.x == 0) {
      S->tombs = 0;
      S->tomb_reuse = 0;
    }
    __syncthreads();
  }

  // Build the list of the minimum-count bucket in touch order.  now = the
  // position of the next item to process.
  __device__ void rebuild_list(bool full_scan, uint32_t now) {
    uint32_t mn = 0xFFFFFFFFu;
    for (uint32_t i = threadIdx.x; i < k; i += BS) mn = min(mn, s.cnt[i]);
    mn = block_min_u32<BS>(mn, s.wsum);
    const bool incremental = !full_scan && !S->log_over && mn == S->m + 1;
    const uint32_t epoch = S->epoch_start;
    // (a) counters at count mn to sort by touch
    uint32_t n1 = 0;
    for (uint32_t base = 0; base < k; base += BS) {
      const uint32_t i = base + threadIdx.x;
      bool f = false;
      if (i < k) f = s.cnt[i] == mn && (!incremental || s.touch[i] < epoch);
      uint32_t tot;
      uint32_t ex = scan(f ? 1u : 0u, &tot);
      if (f) {
        s.skey[n1 + ex] = s.touch[i];
        s.spay[n1 + ex] = (uint16_t)i;
      }
      n1 += tot;
    }
    const uint32_t n2p = next_pow2(n1 ? n1 : 1);
    for (uint32_t i = n1 + threadIdx.x; i < n2p; i += BS) {
      s.skey[i] = ~0ull;
      s.spay[i] = 0xFFFF;
    }
    __syncthreads();
    block_bitonic_sort<BS, uint16_t>(s.skey, s.spay, n2p);
    for (uint32_t i = threadIdx.x; i < n1; i += BS) s.list[i] = s.spay[i];
    // (b) the log of counters that reached count mn during the epoch
    uint32_t n = n1;
    if (incremental) {
      const uint32_t ll = S->log_len;
      for (uint32_t base = 0; base < ll; base += BS) {
        const uint32_t j = base + threadIdx.x;
        bool f = false;
        uint16_t sl = 0;
        if (j < ll) {
          sl = s.logq[j];
          f = s.cnt[sl] == mn;
        }
        uint32_t tot;
        uint32_t ex = scan(f ? 1u : 0u, &tot);
        if (f && n + ex < k) s.list[n + ex] = sl;
        n += tot;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      S->m = mn;
      S->head = 0;
      S->list_len = n < k ? n : k;
      S->log_len = 0;
      S->log_over = 0;
      S->epoch_start = now;
    }
    __syncthreads();
  }
};

template <typename ItemT, int BS>
__global__ void __launch_bounds__(BS) ss_block_kernel(const ItemT* __restrict__ items, u64 n,
                                                      uint32_t p, uint32_t r0,
                                                      SetView<ItemT> out, uint32_t node0) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SSState S_;
  SSBlock<ItemT, BS> B;
  B.k = out.k;
  B.S = &S_;
  B.sb = 0;
  ss_carve<ItemT, BS>(B.k, smem, &B.s);
  SSState& S = S_;
  const uint32_t k = B.k;
  const uint32_t tid = threadIdx.x;
  const uint32_t r = r0 + blockIdx.x;
  const uint32_t node = node0 + blockIdx.x;
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
  auto& s = B.s;
  uint32_t status = 0;

  for (uint32_t i = tid; i < s.C; i += BS) s.hash[i] = CELL_EMPTY;
  for (uint32_t i = tid; i <= s.WT; i += BS) {
    s.wkey[i] = ItemOps<ItemT>::SENT;
    s.wpos[i] = 0xFFFFFFFFu;
  }
  for (uint32_t i = tid; i < k; i += BS) s.vrank[i] = 0;
  if (tid == 0) {
    S.m = 0; S.head = 0; S.list_len = 0; S.log_len = 0; S.log_over = 0;
    S.used = 0; S.full = 0; S.tombs = 0; S.tomb_reuse = 0; S.epoch_start = 0;
    S.P = 0; S.found = 0; S.j0 = 0; S.need_rebuild = 0; S.stall = 0; S.status = 0;
  }
  __syncthreads();

  const uint32_t hash_limit = s.C / 4 * 3;
  uint32_t t0 = 0;
  while (t0 < len) {
    const uint32_t nw = min((uint32_t)BS, len - t0);
    const uint32_t t = t0 + tid;
    const bool act = tid < nw;
    const ItemT x = act ? xs[t] : (ItemT)0;
    const int slot = act ? B.lookup(x, status) : -1;
    const uint32_t full = S.full, m = S.m;
    const bool hit = slot >= 0;
    const bool miss = act && !hit;
    const uint32_t pre = hit ? s.cnt[slot] : 0u;
    const bool lfhit = full && hit && pre == m;

    if (!__syncthreads_or(miss || lfhit)) {
      // Hits only: they commute.
      if (hit) {
        atomicAdd(&s.cnt[slot], 1u);
        atomicMax(&s.touch[slot], t);
      }
      __syncthreads();
      t0 += nw;
      continue;
    }

    if (tid == 0) {
      S.P = nw;
      S.found = 0;
      S.j0 = S.head;
    }
    uint32_t wc = 0;
    if (miss) wc = B.wtab_insert(x, t);
    __syncthreads();
    const bool first = miss && s.wpos[wc] == t;
    const bool lf = lfhit || (full && first);
    uint32_t tot;
    const uint32_t ex = B.scan((first ? 1u : 0u) | (lf ? 0x10000u : 0u), &tot);
    const uint32_t rnk = ex & 0xFFFFu, lrk = ex >> 16, M = tot & 0xFFFFu;
    if (first) s.rankpos[rnk] = t;

    // Victims: the first M counters of the bucket list still at count m.
    uint32_t Lv = 0;
    if (full && M > 0) {
      for (;;) {
        const uint32_t found = S.found, j0 = S.j0, ll = S.list_len;
        if (found >= M || j0 >= ll) break;
        const uint32_t j = j0 + tid;
        uint16_t sl = 0;
        bool valid = false;
        if (j < ll) {
          sl = s.list[j];
          valid = s.cnt[sl] == m;
        }
        uint32_t vt;
        const uint32_t ve = B.scan(valid ? 1u : 0u, &vt);
        if (valid && found + ve < M) {
          s.V[found + ve] = sl;
          s.Vidx[found + ve] = j;
        }
        if (tid == 0) {
          S.found = found + vt;
          S.j0 = j0 + BS;
        }
        __syncthreads();
      }
      Lv = min(S.found, M);
      if (tid < Lv) s.vrank[s.V[tid]] = (uint16_t)(tid + 1);
    }
    __syncthreads();

    // Cut the window at the first position where the assignment stops being exact.
    if (full && hit) {
      const uint32_t vr = s.vrank[slot];
      if (vr) atomicMin(&S.P, max(t, s.rankpos[vr - 1]) - t0);
    }
    if (tid == 0) {
      if (!full) {
        const uint32_t F = k - S.used;
        if (M > F) atomicMin(&S.P, s.rankpos[F] - t0);
      } else if (Lv < M) {
        atomicMin(&S.P, s.rankpos[Lv] - t0);
      }
    }
    __syncthreads();
    const uint32_t P = S.P, lim = t0 + P;
    const bool applyF = first && t < lim;
    const bool applyL = lf && t < lim;
    const uint32_t MP = (uint32_t)__syncthreads_count(applyF);

    // Evictions: remove the victims' items from the table.
    if (applyF && full) s.hash[s.cellof[s.V[rnk]]] = CELL_TOMB;
    __syncthreads();
    if (applyF) {
      const uint32_t v = full ? (uint32_t)s.V[rnk] : S.used + rnk;
      B.insert(x, v, status);
      s.item[v] = x;
      s.cnt[v] = full ? m + 1 : 1u;
      s.err[v] = full ? m : 0u;
      s.touch[v] = t;
      s.wslot[wc] = (uint16_t)v;
    }
    if (applyL) {
      const uint32_t idx = S.log_len + lrk;
      if (idx < s.LOGCAP) s.logq[idx] = first ? s.V[rnk] : (uint16_t)slot;
    }
    const uint32_t LGP = (uint32_t)__syncthreads_count(applyL);

    if (t < lim) {
      if (hit) {
        atomicAdd(&s.cnt[slot], 1u);
        atomicMax(&s.touch[slot], t);
      } else if (miss && !first) {
        const uint32_t v = s.wslot[wc];
        atomicAdd(&s.cnt[v], 1u);
        atomicMax(&s.touch[v], t);
      }
    }
    if (full && tid < Lv) s.vrank[s.V[tid]] = 0;
    if (tid == 0) {
      if (!full) {
        S.used += MP;
      } else {
        if (MP) S.head = s.Vidx[MP - 1] + 1;
        S.tombs += MP;
      }
      uint32_t nl = S.log_len + LGP;
      if (nl > s.LOGCAP) {
        S.log_over = 1;
        nl = s.LOGCAP;
      }
      S.log_len = nl;
      S.tombs -= S.tomb_reuse;
      S.tomb_reuse = 0;
      S.need_rebuild = 0;
      if (!full && S.used == k) {
        S.full = 1;
        S.need_rebuild = 2;
      } else if (full && Lv < M && MP == Lv) {
        S.need_rebuild = 1;
      }
      S.stall = P ? 0 : S.stall + 1;
    }
    __syncthreads();
    if (first) {
      if (wc != s.WT) s.wkey[wc] = ItemOps<ItemT>::SENT;
      s.wpos[wc] = 0xFFFFFFFFu;
    }
    const uint32_t nr = S.need_rebuild;
    if (nr) B.rebuild_list(nr == 2, lim);
    if (S.used + S.tombs > hash_limit) B.rebuild_hash(status);
    if (S.stall >= 3) {
      status |= ST_NOPROGRESS;
      break;
    }
    __syncthreads();
    t0 = lim;
  }

  // ---- output: the summary sorted by item ascending
  if (status) atomicOr(&S.status, status);
  __syncthreads();
  const uint32_t used = S.used;
  uint32_t mn = 0xFFFFFFFFu;
  for (uint32_t i = tid; i < used; i += BS) mn = min(mn, s.cnt[i]);
  mn = block_min_u32<BS>(mn, s.wsum);
  const uint32_t n2p = next_pow2(used ? used : 1);
  for (uint32_t i = tid; i < n2p; i += BS) {
    if (i < used) {
      s.skey[i] = ItemOps<ItemT>::sort_key(s.item[i], i);
      s.spay[i] = (uint16_t)i;
    } else {
      s.skey[i] = ~0ull;
      s.spay[i] = 0xFFFF;
    }
  }
  __syncthreads();
  block_bitonic_sort<BS, uint16_t>(s.skey, s.spay, n2p);
  for (uint32_t i = tid; i < used; i += BS) {
    const uint32_t sl = s.spay[i];
    out.item[obase + i] = s.item[sl];
    out.count[obase + i] = s.cnt[sl];
    out.err[obase + i] = s.err[sl];
  }
  if (tid == 0) {
    out.size[node] = used;
    out.m[node] = (used == k) ? (u64)mn : 0ull;
    out.ncov[node] = len;
    if (S.status) atomicOr(out.status, S.status);
  }
}

}  // namespace

template <typename ItemT>
size_t ss_smem_bytes(uint32_t k) {
  return ss_carve<ItemT, SS_BS>(k, nullptr, nullptr);
}

template <typename ItemT>
cudaError_t launch_summarize_blocks(const ItemT* items, u64 n, uint32_t p, uint32_t r0,
                                    uint32_t count, SetView<ItemT> out, uint32_t node0,
                                    cudaStream_t stream) {
  const size_t smem = ss_smem_bytes<ItemT>(out.k);
  auto kern = ss_block_kernel<ItemT, SS_BS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (count == 0) return cudaSuccess;
  kern<<<count, SS_BS, smem, stream>>>(items, n, p, r0, out, node0);
  return cudaGetLastError();
}

template size_t ss_smem_bytes<uint32_t>(uint32_t);
template size_t ss_smem_bytes<u64>(uint32_t);
template cudaError_t launch_summarize_blocks<uint32_t>(const uint32_t*, u64, uint32_t, uint32_t,
                                                       uint32_t, SetView<uint32_t>, uint32_t,
                                                       cudaStream_t);
template cudaError_t launch_summarize_blocks<u64>(const u64*, u64, uint32_t, uint32_t, uint32_t,
                                                  SetView<u64>, uint32_t, cudaStream_t);

}  // namespace pss
