// merge.cu — the combine operator of Algorithm 2, one CTA per output summary.
//
// combine(S1, S2, k): m1, m2 are the minima of S1 and S2; every item of S1
// gets its count plus (its count in S2 if present, else m2); every item of S2
// absent from S1 gets its count plus m1; errors receive the same additions;
// Prune(k) keeps the k largest by (count descending, item ascending).
//
// Both inputs are stored sorted by item, so the union is formed without any
// hashing or sorting: the position of an S1 entry in the item-ordered union is
// its own index plus the number of S2-only items before it, and symmetrically
// for S2-only entries (binary searches in shared memory plus one prefix sum).
// Prune(k) is an exact selection: a most-significant-digit radix select finds
// the k-th largest count c*, then the entries with count > c* and the first
// (in item order) of those with count == c* are kept.  The output is again
// sorted by item, so no level of the reduction tree ever sorts.
#include "pss_internal.cuh"
#include "pss_kernels.cuh"

namespace pss {

namespace {

constexpr uint16_t NONE = 0xFFFF;

template <typename ItemT>
struct MSmem {
  ItemT* ia;
  ItemT* ib;
  uint32_t* borank;
  u64* uc;
  uint16_t* srcA;
  uint16_t* srcB;
  uint32_t* hist;
  uint32_t* wsum;
  u64* red;
};

// Shared-memory layout (returns its bytes).  BIG (k above what fits): the
// union's counts and source indices live in a per-CTA slice of global memory
// (gbase; bytes to *gbytes).
template <typename ItemT, int BS, bool BIG>
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
  L.borank = (uint32_t*)take(4ull * (k + 1));
  L.hist = (uint32_t*)take(4ull * 256);
  L.wsum = (uint32_t*)take(4ull * 2 * (BS / 32 + 1));
  L.srcA = (uint16_t*)(BIG ? gtake(2ull * 2 * k) : take(2ull * 2 * k));
  L.srcB = (uint16_t*)(BIG ? gtake(2ull * 2 * k) : take(2ull * 2 * k));
  if (s) *s = L;
  if (gbytes) *gbytes = goff;
  return off;
}

template <typename ItemT>
__device__ __forceinline__ uint32_t lower_bound(const ItemT* a, uint32_t n, ItemT x) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
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
template <typename ItemT, int BS, bool BIG, bool MG = false>
__device__ void merge_nodes(const SetView<ItemT>& A, uint32_t na, const SetView<ItemT>& B,
                            uint32_t nb, const SetView<ItemT>& O, uint32_t no,
                            unsigned char* smem, unsigned char* gslice) {
  __shared__ u64 sh_prefix;
  __shared__ uint32_t sh_need;
  MSmem<ItemT> s;
  const uint32_t k = O.k;
  merge_carve<ItemT, BS, BIG>(k, smem, gslice, &s);
  const uint32_t tid = threadIdx.x;
  const uint32_t sa = A.size[na], sb = B.size[nb];
  const u64 mA = A.m[na], mB = B.m[nb];
  const size_t ba = (size_t)na * k, bb = (size_t)nb * k, bo = (size_t)no * k;
  for (uint32_t i = tid; i < sa; i += BS) s.ia[i] = A.item[ba + i];
  for (uint32_t j = tid; j < sb; j += BS) s.ib[j] = B.item[bb + j];
  __syncthreads();

  uint32_t par = 0;
  auto scan = [&](uint32_t v, uint32_t* tot) {
    uint32_t* buf = s.wsum + (par ? (BS / 32 + 1) : 0);
    par ^= 1;
    return block_exclusive_scan<BS>(v, buf, tot);
  };

  // Ranks of the S2-only items.
  uint32_t run = 0;
  for (uint32_t base = 0; base < sb; base += BS) {
    const uint32_t j = base + tid;
    bool only = false;
    if (j < sb) {
      const ItemT x = s.ib[j];
      const uint32_t ii = lower_bound(s.ia, sa, x);
      only = !(ii < sa && s.ia[ii] == x);
    }
    uint32_t tot;
    const uint32_t ex = scan(only ? 1u : 0u, &tot);
    if (j < sb) s.borank[j] = run + ex;
    run += tot;
  }
  if (tid == 0) s.borank[sb] = run;
  __syncthreads();
  const uint32_t U = sa + run;

  // The union in item order.
  for (uint32_t i = tid; i < sa; i += BS) {
    const ItemT x = s.ia[i];
    const uint32_t jj = lower_bound(s.ib, sb, x);
    const bool both = jj < sb && s.ib[jj] == x;
    const uint32_t pos = i + s.borank[jj];
    s.uc[pos] = A.count[ba + i] + (both ? B.count[bb + jj] : mB);
    s.srcA[pos] = (uint16_t)i;
    s.srcB[pos] = both ? (uint16_t)jj : NONE;
  }
  for (uint32_t j = tid; j < sb; j += BS) {
    if (s.borank[j + 1] != s.borank[j]) {
      const uint32_t ii = lower_bound(s.ia, sa, s.ib[j]);
      const uint32_t pos = ii + s.borank[j];
      s.uc[pos] = B.count[bb + j] + mA;
      s.srcA[pos] = NONE;
      s.srcB[pos] = (uint16_t)j;
    }
  }
  __syncthreads();

  // Prune(k): the k-th largest count c*, and how many entries equal to c* to
  // keep (MG: the (k+1)-th largest, none kept).
  const bool cut = U > k;
  u64 cstar = 0;
  uint32_t need = 0;
  if (cut) {
    u64 mx = 0;
    for (uint32_t u = tid; u < U; u += BS) mx = s.uc[u] > mx ? s.uc[u] : mx;
    mx = block_reduce_u64<BS>(mx, s.red, true);
    int shift = ((63 - __clzll((long long)mx)) / 8) * 8;
    u64 prefix = 0, pmask = 0;
    need = MG ? k + 1 : k;
    for (; shift >= 0; shift -= 8) {
      for (uint32_t i = tid; i < 256; i += BS) s.hist[i] = 0;
      __syncthreads();
      for (uint32_t u = tid; u < U; u += BS) {
        const u64 c = s.uc[u];
        if ((c & pmask) == prefix) atomicAdd(&s.hist[(c >> shift) & 255u], 1u);
      }
      __syncthreads();
      if (tid == 0) {
        uint32_t acc = 0;
        int d = 255;
        for (; d > 0; --d) {
          if (acc + s.hist[d] >= need) break;
          acc += s.hist[d];
        }
        sh_need = need - acc;
        sh_prefix = prefix | ((u64)d << shift);
      }
      __syncthreads();
      need = sh_need;
      prefix = sh_prefix;
      pmask |= 255ull << shift;
      __syncthreads();
    }
    cstar = prefix;
  }

  // Keep and write in item order.
  uint32_t run_eq = 0, run_keep = 0;
  for (uint32_t base = 0; base < U; base += BS) {
    const uint32_t u = base + tid;
    const bool in = u < U;
    const u64 c = in ? s.uc[u] : 0;
    const bool eq = in && cut && c == cstar;
    uint32_t te;
    const uint32_t ee = scan(eq ? 1u : 0u, &te);
    const bool keep = in && (!cut || c > cstar || (!MG && eq && run_eq + ee < need));
    uint32_t tk;
    const uint32_t ek = scan(keep ? 1u : 0u, &tk);
    if (keep) {
      const uint32_t o = run_keep + ek;
      const uint16_t a = s.srcA[u], b = s.srcB[u];
      O.item[bo + o] = (a != NONE) ? s.ia[a] : s.ib[b];
      O.count[bo + o] = (MG && cut) ? c - cstar : c;
      O.err[bo + o] = ((a != NONE) ? A.err[ba + a] : mA) + ((b != NONE) ? B.err[bb + b] : mB);
    }
    run_eq += te;
    run_keep += tk;
  }
  u64 mout = 0;
  if (MG) {
    mout = 0;
  } else if (cut) {
    mout = cstar;
  } else if (U == k) {
    u64 mn = ~0ull;
    for (uint32_t u = tid; u < U; u += BS) mn = s.uc[u] < mn ? s.uc[u] : mn;
    mout = block_reduce_u64<BS>(mn, s.red, false);
  }
  if (tid == 0) {
    O.size[no] = run_keep;
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

template <typename ItemT, int BS, bool BIG, bool MG>
__global__ void __launch_bounds__(BS) merge_level_kernel(SetView<ItemT> in, SetView<ItemT> out,
                                                         unsigned char* gscratch, size_t gslice) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t j = blockIdx.x;
  if (2 * j + 1 >= in.nodes) {
    copy_node<ItemT, BS>(in, 2 * j, out, j);
    return;
  }
  merge_nodes<ItemT, BS, BIG, MG>(in, 2 * j, in, 2 * j + 1, out, j, smem,
                                  BIG ? gscratch + (size_t)j * gslice : nullptr);
}

template <typename ItemT, int BS, bool BIG, bool MG>
__global__ void __launch_bounds__(BS) merge_pair_kernel(SetView<ItemT> a, uint32_t ia,
                                                        SetView<ItemT> b, uint32_t ib,
                                                        SetView<ItemT> out, unsigned char* gscratch) {
  extern __shared__ __align__(16) unsigned char smem[];
  merge_nodes<ItemT, BS, BIG, MG>(a, ia, b, ib, out, 0, smem, gscratch);
}

// Batch form: task (d, j) builds node j of the next level of descriptor d
// (MG: the Frequent merge).
template <typename ItemT, int BS, bool MG>
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
  merge_nodes<ItemT, BS, false, MG>(in, 2 * j, in, 2 * j + 1, out, j, smem, nullptr);
}

template <typename ItemT, int BS>
__global__ void __launch_bounds__(BS) copy_node_kernel(SetView<ItemT> in, uint32_t ni,
                                                       SetView<ItemT> out, uint32_t no) {
  copy_node<ItemT, BS>(in, ni, out, no);
}

}  // namespace

template <typename ItemT>
size_t merge_smem_bytes(uint32_t k) {
  return k > SS_SMEM_MAX_K ? merge_carve<ItemT, MERGE_BS, true>(k, nullptr, nullptr, nullptr)
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
  if (mg) {
    if (in.k > SS_SMEM_MAX_K) return cudaErrorInvalidValue;
    auto kern = merge_level_kernel<ItemT, MERGE_BS, false, true>;
    cudaError_t e = ensure_kernel_attrs((const void*)kern);
    if (e != cudaSuccess) return e;
    kern<<<out.nodes, MERGE_BS, smem, stream>>>(in, out, nullptr, 0);
    return cudaGetLastError();
  }
  if (in.k <= SS_SMEM_MAX_K) {
    auto kern = merge_level_kernel<ItemT, MERGE_BS, false, false>;
    cudaError_t e = ensure_kernel_attrs((const void*)kern);
    if (e != cudaSuccess) return e;
    kern<<<out.nodes, MERGE_BS, smem, stream>>>(in, out, nullptr, 0);
    return cudaGetLastError();
  }
  auto kern = merge_level_kernel<ItemT, MERGE_BS, true, false>;
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
  if (mg) {
    if (out.k > SS_SMEM_MAX_K) return cudaErrorInvalidValue;
    auto kern = merge_pair_kernel<ItemT, MERGE_BS, false, true>;
    cudaError_t e = ensure_kernel_attrs((const void*)kern);
    if (e != cudaSuccess) return e;
    kern<<<1, MERGE_BS, smem, stream>>>(a, ia, b, ib, out, nullptr);
    return cudaGetLastError();
  }
  if (out.k <= SS_SMEM_MAX_K) {
    auto kern = merge_pair_kernel<ItemT, MERGE_BS, false, false>;
    cudaError_t e = ensure_kernel_attrs((const void*)kern);
    if (e != cudaSuccess) return e;
    kern<<<1, MERGE_BS, smem, stream>>>(a, ia, b, ib, out, nullptr);
    return cudaGetLastError();
  }
  auto kern = merge_pair_kernel<ItemT, MERGE_BS, true, false>;
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
  auto kern = mg ? merge_tasks_kernel<ItemT, MERGE_BS, true> : merge_tasks_kernel<ItemT, MERGE_BS, false>;
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
