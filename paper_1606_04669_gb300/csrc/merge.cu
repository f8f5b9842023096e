// merge.cu — the combine operator of Algorithm 2, one CTA per output summary.
//
// combine(S1, S2, k): m1, m2 are the minima of S1 and S2; every item of S1
// gets its count plus (its count in S2 if present, else m2); every item of S2
// absent from S1 gets its count plus m1; errors receive the same additions;
// Prune(k) keeps the k largest by (count descending, item ascending).
//
// Both inputs are stored sorted by item, so the union is formed without any
// hashing or sorting: it is laid out in the order of the merged sequence of
// S1 and S2 (S1 first on equal items), each thread walking its own run of
// merged positions from one merge-path search; the S2 copy of an item in both
// leaves its position empty.
// Prune(k) is an exact selection: a most-significant-digit radix select finds
// the k-th largest count c*, then the entries with count > c* and the first
// (in item order) of those with count == c* are kept.  The output is again
// sorted by item, so no level of the reduction tree ever sorts.
#include "pss_internal.cuh"
#include "pss_kernels.cuh"

namespace pss {

namespace {

constexpr uint16_t NONE = 0xFFFF;
constexpr u64 EMPTY = ~0ull;  // a merged position without a union entry

template <typename ItemT>
struct MSmem {
  ItemT* ia;
  ItemT* ib;
  u64* ca;  // STAGED: S1's counts, then its errors
  u64* cb;  // STAGED: S2's counts, then its errors
  u64* uc;
  uint16_t* srcA;
  uint16_t* srcB;
  uint32_t* hist;
  uint32_t* wsum;
  u64* red;
};

// Shared-memory layout (returns its bytes).  BIG (k above what fits): the
// union's counts and source indices live in a per-CTA slice of global memory
// (gbase; bytes to *gbytes).  STAGED: both inputs' counts (later their
// errors) are copied into shared memory as well.
template <typename ItemT, int BS, bool BIG, bool STAGED = false>
__host__ __device__ inline size_t merge_carve(uint32_t k, unsigned char* base, unsigned char* gbase,
                                              MSmem<ItemT>* s, size_t* gbytes = nullptr) {
  size_t off = 0, goff = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = (off + bytes + 15) & ~(size_t)15;
    return base + o;
  };
  auto gtake = [&](size_t bytes) {
    size_t o = goff;
    goff = (goff + bytes + 15) & ~(size_t)15;
    return gbase + o;
  };
  MSmem<ItemT> L;
  L.uc = (u64*)(BIG ? gtake(8ull * 2 * k) : take(8ull * 2 * k));
  L.red = (u64*)take(8ull * (BS / 32 + 1));
  L.ia = (ItemT*)take(sizeof(ItemT) * k);
  L.ib = (ItemT*)take(sizeof(ItemT) * k);
  L.ca = STAGED ? (u64*)take(8ull * k) : nullptr;
  L.cb = STAGED ? (u64*)take(8ull * k) : nullptr;
  L.hist = (uint32_t*)take(4ull * 512);
  L.wsum = (uint32_t*)take(4ull * 2 * (BS / 32 + 1));
  L.srcA = (uint16_t*)(BIG ? gtake(2ull * 2 * k) : take(2ull * 2 * k));
  L.srcB = (uint16_t*)(BIG ? gtake(2ull * 2 * k) : take(2ull * 2 * k));
  if (s) *s = L;
  if (gbytes) *gbytes = goff;
  return off;
}

// How many of the first d elements of the merged sequence of a and b (equal
// items: a first) come from a.
template <typename ItemT>
__device__ __forceinline__ uint32_t merge_path(const ItemT* a, uint32_t sa, const ItemT* b,
                                               uint32_t sb, uint32_t d) {
  uint32_t lo = d > sb ? d - sb : 0u, hi = d < sa ? d : sa;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= b[d - mid - 1]) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Asynchronous copies into shared memory (completed by cp_wait_all).
__device__ __forceinline__ void cp_async(void* dst, const void* src, int bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The whole CTA copies n elements from global to shared memory: 16-byte
// pieces when both addresses are 16-byte aligned, the rest element by element.
template <int BS, typename E>
__device__ __forceinline__ void stage_copy(E* dst, const E* src, uint32_t n) {
  uint32_t done = 0;
  if (((reinterpret_cast<uintptr_t>(src) | (uintptr_t)__cvta_generic_to_shared(dst)) & 15u) == 0) {
    const uint32_t pieces = (uint32_t)(n * sizeof(E) / 16);
    for (uint32_t i = threadIdx.x; i < pieces; i += BS)
      cp_async(reinterpret_cast<char*>(dst) + 16 * i, reinterpret_cast<const char*>(src) + 16 * i, 16);
    done = pieces * (uint32_t)(16 / sizeof(E));
  }
  for (uint32_t i = done + threadIdx.x; i < n; i += BS) cp_async(dst + i, src + i, (int)sizeof(E));
}

template <int BS>
__device__ __forceinline__ u64 block_reduce_u64(u64 v, u64* scratch, bool is_max) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    u64 y = __shfl_xor_sync(0xffffffffu, v, o);
    v = is_max ? (v > y ? v : y) : (v < y ? v : y);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  u64 r = scratch[0];
  for (int w = 1; w < BS / 32; ++w) r = is_max ? (r > scratch[w] ? r : scratch[w])
                                               : (r < scratch[w] ? r : scratch[w]);
  __syncthreads();
  return r;
}

// out node `no` = combine(A node na, B node nb).  MG: the merge of two
// Frequent (Misra–Gries) summaries of capacity k instead: both minima are 0,
// so the union adds the counts of equal items; when more than k items remain,
// the (k+1)-th largest count c* is subtracted from every count and only the
// counts above c* stay (their minimum and errors stay 0).
//
// One merge is a short chain of dependent steps in one CTA, so its time is
// latency and instruction count: global loads are issued several at a time
// before their values are used, the union costs one merge-path search per
// thread, the keep phase exchanges per-warp totals once (one barrier), and the
// radix histogram adds each warp's equal digits with one atomic.  (Bounding
// the kernels to three CTAs per SM, as many as the shared memory of k = 2000
// allows, forces spills at 40 registers and was slower.)
template <typename ItemT, int BS, bool BIG, bool MG = false, bool STAGED = false>
__device__ void merge_nodes(const SetView<ItemT>& A, uint32_t na, const SetView<ItemT>& B,
                            uint32_t nb, const SetView<ItemT>& O, uint32_t no,
                            unsigned char* smem, unsigned char* gslice) {
  constexpr uint32_t NW = BS / 32;
  constexpr int G = 2;
  __shared__ u64 sh_prefix;
  __shared__ uint32_t sh_need, sh_found;
  __shared__ uint32_t sh_dup[NW];
  MSmem<ItemT> s;
  const uint32_t k = O.k;
  merge_carve<ItemT, BS, BIG, STAGED>(k, smem, gslice, &s);
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t sa = A.size[na], sb = B.size[nb];
  const u64 mA = A.m[na], mB = B.m[nb];
  const size_t ba = (size_t)na * k, bb = (size_t)nb * k, bo = (size_t)no * k;
  if constexpr (STAGED) {
    // One round of copies: both inputs' items and counts (all k slots of
    // each node, so that the copies need not wait for the sizes).
    stage_copy<BS>(s.ia, A.item + ba, k);
    stage_copy<BS>(s.ib, B.item + bb, k);
    stage_copy<BS>(s.ca, A.count + ba, k);
    stage_copy<BS>(s.cb, B.count + bb, k);
    cp_commit();
  } else {
  for (uint32_t base = 0; base < sa; base += G * BS) {
    ItemT v[G];
#pragma unroll
    for (int t = 0; t < G; ++t) {
      const uint32_t i = base + t * BS + tid;
      if (i < sa) v[t] = A.item[ba + i];
    }
#pragma unroll
    for (int t = 0; t < G; ++t) {
      const uint32_t i = base + t * BS + tid;
      if (i < sa) s.ia[i] = v[t];
    }
  }
  for (uint32_t base = 0; base < sb; base += G * BS) {
    ItemT v[G];
#pragma unroll
    for (int t = 0; t < G; ++t) {
      const uint32_t j = base + t * BS + tid;
      if (j < sb) v[t] = B.item[bb + j];
    }
#pragma unroll
    for (int t = 0; t < G; ++t) {
      const uint32_t j = base + t * BS + tid;
      if (j < sb) s.ib[j] = v[t];
    }
  }
  }
  if (tid < 256) s.hist[tid] = 0;  // first radix pass (BS >= 256)
  if constexpr (STAGED) cp_wait_all();
  __syncthreads();

  // The union in merged order: position d holds the entry of the d-th
  // element of the merged sequence, or EMPTY for S2's copy of an item also in
  // S1 (it follows S1's copy).  Each thread walks its own run of positions
  // (an odd length, so that lanes' 8-byte stores fall in different banks),
  // WS steps at a time with their global loads issued together.
  const uint32_t L = sa + sb;
  if constexpr (STAGED) {
    const uint32_t per = ((L + BS - 1) / BS) | 1u;
    const uint32_t d0 = min(L, tid * per), d1 = min(L, d0 + per);
    uint32_t i = merge_path(s.ia, sa, s.ib, sb, d0), j = d0 - i, ndup = 0;
    for (uint32_t d = d0; d < d1; ++d) {
      uint16_t pa = NONE, pb = NONE;
      u64 v = EMPTY;
      if (j >= sb || (i < sa && s.ia[i] <= s.ib[j])) {
        pa = (uint16_t)i;
        if (j < sb && s.ib[j] == s.ia[i]) {
          pb = (uint16_t)j;
          v = s.ca[i] + s.cb[j];
        } else {
          v = s.ca[i] + mB;
        }
        ++i;
      } else {
        if (i > 0 && s.ia[i - 1] == s.ib[j]) {
          ++ndup;
        } else {
          pb = (uint16_t)j;
          v = s.cb[j] + mA;
        }
        ++j;
      }
      s.uc[d] = v;
      s.srcA[d] = pa;
      s.srcB[d] = pb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ndup += __shfl_xor_sync(0xffffffffu, ndup, o);
    if (lane == 0) sh_dup[warp] = ndup;
  } else {
    constexpr int WS = 3;
    const uint32_t per = ((L + BS - 1) / BS) | 1u;
    const uint32_t d0 = min(L, tid * per), d1 = min(L, d0 + per);
    uint32_t i = merge_path(s.ia, sa, s.ib, sb, d0), j = d0 - i, ndup = 0;
    for (uint32_t d = d0; d < d1; d += WS) {
      uint16_t pa[WS], pb[WS];
      u64 c[WS], c2[WS];
#pragma unroll
      for (int t = 0; t < WS; ++t) {
        pa[t] = NONE;
        pb[t] = NONE;
        if (d + t < d1) {
          if (j >= sb || (i < sa && s.ia[i] <= s.ib[j])) {
            pa[t] = (uint16_t)i;
            if (j < sb && s.ib[j] == s.ia[i]) pb[t] = (uint16_t)j;
            ++i;
          } else {
            if (i > 0 && s.ia[i - 1] == s.ib[j]) ++ndup;
            else pb[t] = (uint16_t)j;
            ++j;
          }
        }
      }
#pragma unroll
      for (int t = 0; t < WS; ++t) {
        c[t] = 0;
        c2[t] = 0;
        if (pa[t] != NONE) c[t] = A.count[ba + pa[t]];
        else if (pb[t] != NONE) c[t] = B.count[bb + pb[t]];
        if (pa[t] != NONE && pb[t] != NONE) c2[t] = B.count[bb + pb[t]];
      }
#pragma unroll
      for (int t = 0; t < WS; ++t) {
        if (d + t < d1) {
          u64 v = EMPTY;
          if (pa[t] != NONE) v = c[t] + (pb[t] != NONE ? c2[t] : mB);
          else if (pb[t] != NONE) v = c[t] + mA;
          s.uc[d + t] = v;
          s.srcA[d + t] = pa[t];
          s.srcB[d + t] = pb[t];
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ndup += __shfl_xor_sync(0xffffffffu, ndup, o);
    if (lane == 0) sh_dup[warp] = ndup;
  }
  __syncthreads();
  if constexpr (STAGED) {
    // The counts are dead: the errors take their place while the select runs.
    stage_copy<BS>(s.ca, A.err + ba, k);
    stage_copy<BS>(s.cb, B.err + bb, k);
    cp_commit();
  }
  uint32_t dups = 0;
  for (uint32_t w = 0; w < NW; ++w) dups += sh_dup[w];
  const uint32_t U = L - dups;

  // Prune(k): the k-th largest count c*, and how many entries equal to c* to
  // keep (MG: the (k+1)-th largest, none kept).  c* is the (U - need + 1)-th
  // smallest count.  A first histogram of the counts' distances from the
  // union's minimum (255 and above in one bin), scanned from the bottom,
  // finds it when it lies within 254 of the minimum: the union's low end is
  // dense (every item absent from one input sits at m1 + m2 or just above),
  // and in the trees measured c* is the minimum or one above.  Otherwise a
  // most-significant-digit radix select finds it, 8 bits a pass; two
  // histogram buffers alternate, so a pass needs two barriers.
  const bool cut = U > k;
  u64 cstar = 0;
  uint32_t need = 0;
  if (cut) {
    need = MG ? k + 1 : k;
    u64 mn = EMPTY;
    for (uint32_t u = tid; u < L; u += BS) {
      const u64 c = s.uc[u];
      mn = c < mn ? c : mn;  // EMPTY is the largest value
    }
    mn = block_reduce_u64<BS>(mn, s.red, false);
    for (uint32_t base = 0; base < L; base += BS) {
      const uint32_t u = base + tid;
      const u64 c = u < L ? s.uc[u] : EMPTY;
      const bool in = c != EMPTY;
      if (__any_sync(0xffffffffu, in)) {
        const uint32_t d = in ? (uint32_t)min(c - mn, (u64)255) : 256u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (in && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&s.hist[d], (uint32_t)__popc(peers));
      }
    }
    if (tid < 256) s.hist[256 + tid] = 0;  // the radix select's first buffer
    __syncthreads();
    if (warp == 0) {
      // lane l holds bins 8l .. 8l + 7; the total over all bins is U >= r
      const uint32_t r = U - need + 1;
      uint32_t v[8], sum = 0;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        v[t] = s.hist[8 * lane + t];
        sum += v[t];
      }
      uint32_t inc = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= (uint32_t)o) inc += y;
      }
      const unsigned reach = __ballot_sync(0xffffffffu, inc >= r);
      if (lane == (uint32_t)(__ffs(reach) - 1)) {
        uint32_t acc = inc - sum, b = 255;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          acc += v[t];
          if (acc >= r) {
            b = 8 * lane + t;
            break;
          }
        }
        // acc: entries with a count <= c*, so need - (U - acc) of those equal to c* are kept
        sh_found = b < 255u;
        sh_prefix = mn + b;
        sh_need = need - (U - acc);
      }
    }
    __syncthreads();
  }
  if (cut && sh_found) {
    cstar = sh_prefix;
    need = sh_need;
  } else if (cut) {
    u64 mx = 0;
    for (uint32_t u = tid; u < L; u += BS) {
      const u64 c = s.uc[u];
      if (c != EMPTY && c > mx) mx = c;
    }
    mx = block_reduce_u64<BS>(mx, s.red, true);
    int shift = ((63 - __clzll((long long)mx)) / 8) * 8;
    u64 prefix = 0, pmask = 0;
    for (uint32_t buf = 1; shift >= 0; shift -= 8, buf ^= 1u) {
      uint32_t* h = s.hist + 256 * buf;
      for (uint32_t base = 0; base < L; base += BS) {
        const uint32_t u = base + tid;
        const u64 c = u < L ? s.uc[u] : EMPTY;
        const bool in = c != EMPTY && (c & pmask) == prefix;
        if (__any_sync(0xffffffffu, in)) {
          const uint32_t d = in ? (uint32_t)(c >> shift) & 255u : 256u + lane;
          const unsigned peers = __match_any_sync(0xffffffffu, d);
          if (in && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&h[d], (uint32_t)__popc(peers));
        }
      }
      if (tid < 256) s.hist[256 * (buf ^ 1u) + tid] = 0;  // the next pass's buffer
      __syncthreads();
      if (warp == 0) {
        // lane l holds digits 255 - 8l down to 248 - 8l; the first lane whose
        // running total (from the top digit) reaches `need` holds c*'s digit.
        // As in a walk down from 255 that stops at 0, digit 0 is taken
        // without checking its bin.
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          v[t] = h[255 - 8 * lane - t];
          sum += v[t];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= (uint32_t)o) inc += y;
        }
        const unsigned reach = __ballot_sync(0xffffffffu, inc >= need);
        const uint32_t L = reach ? (uint32_t)(__ffs(reach) - 1) : 31u;
        if (lane == L) {
          uint32_t acc = inc - sum, d = 0;
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const uint32_t dd = 255u - 8u * lane - (uint32_t)t;
            if (dd == 0 || acc + v[t] >= need) {
              d = dd;
              break;
            }
            acc += v[t];
          }
          sh_need = need - acc;
          sh_prefix = prefix | ((u64)d << shift);
        }
      }
      __syncthreads();
      need = sh_need;
      prefix = sh_prefix;
      pmask |= 255ull << shift;
    }
    cstar = prefix;
  }

  // Keep and write in item order: warp w takes its own run of merged
  // positions, counts what it keeps, and learns from the other warps' totals
  // where its output starts.  Entries above c* (all, without a cut) are kept; of those
  // equal to c*, the first `need` in item order (none for MG).
  uint32_t nkeep = 0;
  {
    const uint32_t seg = (L + NW - 1) / NW;
    const uint32_t u0 = min(L, warp * seg), u1 = min(L, u0 + seg);
    uint32_t ngt = 0, neq = 0;
    for (uint32_t ub = u0; ub < u1; ub += 32) {
      const uint32_t u = ub + lane;
      const u64 c = u < u1 ? s.uc[u] : EMPTY;
      const bool live = c != EMPTY;
      ngt += __popc(__ballot_sync(0xffffffffu, live && (!cut || c > cstar)));
      neq += __popc(__ballot_sync(0xffffffffu, live && cut && !MG && c == cstar));
    }
    if (lane == 0) {
      s.wsum[warp] = ngt;
      s.wsum[NW + 1 + warp] = neq;
    }
    if constexpr (STAGED) cp_wait_all();
    __syncthreads();
    uint32_t gbefore = 0, ebefore = 0, gtot = 0, etot = 0;
    for (uint32_t w = 0; w < NW; ++w) {
      const uint32_t g = s.wsum[w], e = s.wsum[NW + 1 + w];
      gbefore += w < warp ? g : 0u;
      ebefore += w < warp ? e : 0u;
      gtot += g;
      etot += e;
    }
    nkeep = gtot + min(etot, need);
    for (uint32_t ub = u0; ub < u1; ub += 32 * G) {
      u64 c[G], ea[G], eb[G];
      uint16_t a[G], b[G];
      uint32_t pos[G];
      bool keep[G];
#pragma unroll
      for (int t = 0; t < G; ++t) {
        const uint32_t u = ub + 32 * t + lane;
        c[t] = u < u1 ? s.uc[u] : EMPTY;
        const bool in = c[t] != EMPTY;
        const bool gt = in && (!cut || c[t] > cstar);
        const bool eq = in && cut && !MG && c[t] == cstar;
        const unsigned bg = __ballot_sync(0xffffffffu, gt), be = __ballot_sync(0xffffffffu, eq);
        const uint32_t r = ebefore + __popc(be & lt);
        keep[t] = gt || (eq && r < need);
        pos[t] = gbefore + __popc(bg & lt) + min(r, need);
        gbefore += __popc(bg);
        ebefore += __popc(be);
        a[t] = keep[t] ? s.srcA[u] : NONE;
        b[t] = keep[t] ? s.srcB[u] : NONE;
      }
#pragma unroll
      for (int t = 0; t < G; ++t) {
        if (keep[t]) {
          if constexpr (STAGED) {
            ea[t] = a[t] != NONE ? s.ca[a[t]] : mA;
            eb[t] = b[t] != NONE ? s.cb[b[t]] : mB;
          } else {
            ea[t] = a[t] != NONE ? A.err[ba + a[t]] : mA;
            eb[t] = b[t] != NONE ? B.err[bb + b[t]] : mB;
          }
        }
      }
#pragma unroll
      for (int t = 0; t < G; ++t) {
        if (keep[t]) {
          O.item[bo + pos[t]] = a[t] != NONE ? s.ia[a[t]] : s.ib[b[t]];
          O.count[bo + pos[t]] = (MG && cut) ? c[t] - cstar : c[t];
          O.err[bo + pos[t]] = ea[t] + eb[t];
        }
      }
    }
  }
  u64 mout = 0;
  if (MG) {
    mout = 0;
  } else if (cut) {
    mout = cstar;
  } else if (U == k) {
    u64 mn = ~0ull;
    for (uint32_t u = tid; u < L; u += BS) mn = s.uc[u] < mn ? s.uc[u] : mn;  // EMPTY is the largest
    mout = block_reduce_u64<BS>(mn, s.red, false);
  }
  if (tid == 0) {
    O.size[no] = nkeep;
    O.m[no] = mout;
    O.ncov[no] = A.ncov[na] + B.ncov[nb];
    const uint32_t st = *A.status | *B.status;
    if (st) atomicOr(O.status, st);
  }
}

template <typename ItemT, int BS>
__device__ void copy_node(const SetView<ItemT>& in, uint32_t ni, const SetView<ItemT>& O,
                          uint32_t no) {
  const uint32_t k = O.k, sz = in.size[ni];
  const size_t bi = (size_t)ni * k, bo = (size_t)no * k;
  for (uint32_t i = threadIdx.x; i < sz; i += BS) {
    O.item[bo + i] = in.item[bi + i];
    O.count[bo + i] = in.count[bi + i];
    O.err[bo + i] = in.err[bi + i];
  }
  if (threadIdx.x == 0) {
    O.size[no] = sz;
    O.m[no] = in.m[ni];
    O.ncov[no] = in.ncov[ni];
    if (*in.status) atomicOr(O.status, *in.status);
  }
}

template <typename ItemT, int BS, bool BIG, bool MG, bool STAGED>
__global__ void __launch_bounds__(BS) merge_level_kernel(SetView<ItemT> in, SetView<ItemT> out,
                                                         unsigned char* gscratch, size_t gslice) {
  extern __shared__ __align__(16) unsigned char smem[];
  // Launched as a programmatic dependent of the previous level: wait until
  // that grid has finished and its writes are visible, then let the next
  // level's CTAs be scheduled (they wait the same way).  Without the launch
  // attribute both instructions return at once.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const uint32_t j = blockIdx.x;
  if (2 * j + 1 >= in.nodes) {
    copy_node<ItemT, BS>(in, 2 * j, out, j);
    return;
  }
  merge_nodes<ItemT, BS, BIG, MG, STAGED>(in, 2 * j, in, 2 * j + 1, out, j, smem,
                                          BIG ? gscratch + (size_t)j * gslice : nullptr);
}

template <typename ItemT, int BS, bool BIG, bool MG, bool STAGED>
__global__ void __launch_bounds__(BS) merge_pair_kernel(SetView<ItemT> a, uint32_t ia,
                                                        SetView<ItemT> b, uint32_t ib,
                                                        SetView<ItemT> out, unsigned char* gscratch) {
  extern __shared__ __align__(16) unsigned char smem[];
  merge_nodes<ItemT, BS, BIG, MG, STAGED>(a, ia, b, ib, out, 0, smem, gscratch);
}

// Batch form: task (d, j) builds node j of the next level of descriptor d
// (MG: the Frequent merge).
template <typename ItemT, int BS, bool MG, bool STAGED>
__global__ void __launch_bounds__(BS) merge_tasks_kernel(const MergeDesc* __restrict__ descs,
                                                         const BatchTask* __restrict__ tasks) {
  extern __shared__ __align__(16) unsigned char smem[];
  const BatchTask t = tasks[blockIdx.x];
  const MergeDesc d = descs[t.stream];
  const SetView<ItemT> in = set_view_dev<ItemT>(d.in, d.in_nodes, d.k);
  const SetView<ItemT> out = set_view_dev<ItemT>(d.out, (d.in_nodes + 1) / 2, d.k);
  const uint32_t j = t.index;
  if (2 * j + 1 >= d.in_nodes) {
    copy_node<ItemT, BS>(in, 2 * j, out, j);
    return;
  }
  merge_nodes<ItemT, BS, false, MG, STAGED>(in, 2 * j, in, 2 * j + 1, out, j, smem, nullptr);
}

template <typename ItemT, int BS>
__global__ void __launch_bounds__(BS) copy_node_kernel(SetView<ItemT> in, uint32_t ni,
                                                       SetView<ItemT> out, uint32_t no) {
  copy_node<ItemT, BS>(in, ni, out, no);
}

}  // namespace

namespace {

// Shared memory a staged combine may take: below the 227 KB a CTA can opt
// into, with room for the kernel's static shared memory.
constexpr size_t MERGE_STAGED_MAX = 224 * 1024;

// Whether the combine of k-entry summaries runs staged (both inputs' items
// and counts copied into shared memory in one round).
template <typename ItemT>
bool merge_staged(uint32_t k) {
  return k <= SS_SMEM_MAX_K &&
         merge_carve<ItemT, MERGE_BS, false, true>(k, nullptr, nullptr, nullptr) <= MERGE_STAGED_MAX;
}

}  // namespace

template <typename ItemT>
size_t merge_smem_bytes(uint32_t k) {
  if (k > SS_SMEM_MAX_K) return merge_carve<ItemT, MERGE_BS, true>(k, nullptr, nullptr, nullptr);
  return merge_staged<ItemT>(k) ? merge_carve<ItemT, MERGE_BS, false, true>(k, nullptr, nullptr, nullptr)
                                : merge_carve<ItemT, MERGE_BS, false>(k, nullptr, nullptr, nullptr);
}

namespace {

// Global scratch of `ctas` large-k merges, ordered on the stream.
template <typename ItemT>
cudaError_t merge_scratch(uint32_t k, uint32_t ctas, cudaStream_t stream, void** g, size_t* gslice) {
  merge_carve<ItemT, MERGE_BS, true>(k, nullptr, nullptr, nullptr, gslice);
  return cudaMallocAsync(g, *gslice * (ctas ? ctas : 1), stream);
}

}  // namespace

template <typename ItemT>
cudaError_t launch_merge_level(SetView<ItemT> in, SetView<ItemT> out, cudaStream_t stream,
                               bool mg) {
  const size_t smem = merge_smem_bytes<ItemT>(in.k);
  if (mg && in.k > SS_SMEM_MAX_K) return cudaErrorInvalidValue;
  if (in.k <= SS_SMEM_MAX_K) {
    const bool st = merge_staged<ItemT>(in.k);
    auto kern = mg ? (st ? merge_level_kernel<ItemT, MERGE_BS, false, true, true>
                         : merge_level_kernel<ItemT, MERGE_BS, false, true, false>)
                   : (st ? merge_level_kernel<ItemT, MERGE_BS, false, false, true>
                         : merge_level_kernel<ItemT, MERGE_BS, false, false, false>);
    cudaError_t e = ensure_kernel_attrs((const void*)kern);
    if (e != cudaSuccess) return e;
    // programmatic dependent launch: the level's CTAs may be scheduled while
    // the previous kernel on the stream drains (the kernel waits for it)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(out.nodes);
    cfg.blockDim = dim3(MERGE_BS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    unsigned char* noscratch = nullptr;
    size_t noslice = 0;
    return cudaLaunchKernelEx(&cfg, kern, in, out, noscratch, noslice);
  }
  auto kern = merge_level_kernel<ItemT, MERGE_BS, true, false, false>;
  cudaError_t e = ensure_kernel_attrs((const void*)kern);
  if (e != cudaSuccess) return e;
  void* g = nullptr;
  size_t gslice = 0;
  if ((e = merge_scratch<ItemT>(in.k, out.nodes, stream, &g, &gslice)) != cudaSuccess) return e;
  kern<<<out.nodes, MERGE_BS, smem, stream>>>(in, out, (unsigned char*)g, gslice);
  e = cudaGetLastError();
  const cudaError_t f = cudaFreeAsync(g, stream);
  return e != cudaSuccess ? e : f;
}

template <typename ItemT>
cudaError_t launch_merge_pair(SetView<ItemT> a, uint32_t ia, SetView<ItemT> b, uint32_t ib,
                              SetView<ItemT> out, cudaStream_t stream, bool mg) {
  const size_t smem = merge_smem_bytes<ItemT>(out.k);
  if (mg && out.k > SS_SMEM_MAX_K) return cudaErrorInvalidValue;
  if (out.k <= SS_SMEM_MAX_K) {
    const bool st = merge_staged<ItemT>(out.k);
    auto kern = mg ? (st ? merge_pair_kernel<ItemT, MERGE_BS, false, true, true>
                         : merge_pair_kernel<ItemT, MERGE_BS, false, true, false>)
                   : (st ? merge_pair_kernel<ItemT, MERGE_BS, false, false, true>
                         : merge_pair_kernel<ItemT, MERGE_BS, false, false, false>);
    cudaError_t e = ensure_kernel_attrs((const void*)kern);
    if (e != cudaSuccess) return e;
    kern<<<1, MERGE_BS, smem, stream>>>(a, ia, b, ib, out, nullptr);
    return cudaGetLastError();
  }
  auto kern = merge_pair_kernel<ItemT, MERGE_BS, true, false, false>;
  cudaError_t e = ensure_kernel_attrs((const void*)kern);
  if (e != cudaSuccess) return e;
  void* g = nullptr;
  size_t gslice = 0;
  if ((e = merge_scratch<ItemT>(out.k, 1, stream, &g, &gslice)) != cudaSuccess) return e;
  kern<<<1, MERGE_BS, smem, stream>>>(a, ia, b, ib, out, (unsigned char*)g);
  e = cudaGetLastError();
  const cudaError_t f = cudaFreeAsync(g, stream);
  return e != cudaSuccess ? e : f;
}

template <typename ItemT>
cudaError_t launch_copy_node(SetView<ItemT> in, uint32_t node, SetView<ItemT> out,
                             uint32_t out_node, cudaStream_t stream) {
  copy_node_kernel<ItemT, MERGE_BS><<<1, MERGE_BS, 0, stream>>>(in, node, out, out_node);
  return cudaGetLastError();
}

template <typename ItemT>
cudaError_t launch_merge_tasks(const MergeDesc* descs, const BatchTask* tasks, uint32_t ntasks,
                               uint32_t k, cudaStream_t stream, bool mg) {
  if (k > SS_SMEM_MAX_K) return cudaErrorInvalidValue;  // the batch keeps k in shared memory
  const size_t smem = merge_smem_bytes<ItemT>(k);
  const bool st = merge_staged<ItemT>(k);
  auto kern = mg ? (st ? merge_tasks_kernel<ItemT, MERGE_BS, true, true>
                       : merge_tasks_kernel<ItemT, MERGE_BS, true, false>)
                 : (st ? merge_tasks_kernel<ItemT, MERGE_BS, false, true>
                       : merge_tasks_kernel<ItemT, MERGE_BS, false, false>);
  cudaError_t e = ensure_kernel_attrs((const void*)kern);
  if (e != cudaSuccess) return e;
  if (ntasks == 0) return cudaSuccess;
  kern<<<ntasks, MERGE_BS, smem, stream>>>(descs, tasks);
  return cudaGetLastError();
}

template cudaError_t launch_merge_tasks<uint32_t>(const MergeDesc*, const BatchTask*, uint32_t,
                                                  uint32_t, cudaStream_t, bool);
template cudaError_t launch_merge_tasks<u64>(const MergeDesc*, const BatchTask*, uint32_t, uint32_t,
                                             cudaStream_t, bool);
template size_t merge_smem_bytes<uint32_t>(uint32_t);
template size_t merge_smem_bytes<u64>(uint32_t);
template cudaError_t launch_merge_level<uint32_t>(SetView<uint32_t>, SetView<uint32_t>, cudaStream_t,
                                                  bool);
template cudaError_t launch_merge_level<u64>(SetView<u64>, SetView<u64>, cudaStream_t, bool);
template cudaError_t launch_merge_pair<uint32_t>(SetView<uint32_t>, uint32_t, SetView<uint32_t>,
                                                 uint32_t, SetView<uint32_t>, cudaStream_t, bool);
template cudaError_t launch_merge_pair<u64>(SetView<u64>, uint32_t, SetView<u64>, uint32_t,
                                            SetView<u64>, cudaStream_t, bool);
template cudaError_t launch_copy_node<uint32_t>(SetView<uint32_t>, uint32_t, SetView<uint32_t>,
                                                uint32_t, cudaStream_t);
template cudaError_t launch_copy_node<u64>(SetView<u64>, uint32_t, SetView<u64>, uint32_t,
                                           cudaStream_t);

}  // namespace pss
