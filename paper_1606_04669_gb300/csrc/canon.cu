// canon.cu — the query (Pruned of Algorithm 1) and the canonical export.
//
// Pruned(global, n, k) keeps the entries whose count exceeds n / k, the
// k-majority threshold of Section 3 (f >= floor(n/k) + 1, i.e. count * k > n,
// evaluated exactly in 128 bits).  Results are reported in canonical order:
// count descending, then item ascending.  One CTA: the summary (at most
// PSS_MAX_K entries) is compacted and bitonic-sorted in shared memory.
#include "pss_internal.cuh"
#include "pss_kernels.cuh"

namespace pss {

namespace {

// Ascending sort of (k1, k2) pairs with a payload; all threads call it.
template <int BS>
__device__ void bitonic_sort_2key(u64* k1, u64* k2, uint16_t* pay, uint32_t n2) {
  for (uint32_t size = 2; size <= n2; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < (n2 >> 1); i += BS) {
        const uint32_t lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
        const bool asc = (lo & size) == 0;
        const u64 a1 = k1[lo], b1 = k1[hi], a2 = k2[lo], b2 = k2[hi];
        const bool greater = (a1 > b1) || (a1 == b1 && a2 > b2);
        if (greater == asc) {
          k1[lo] = b1; k1[hi] = a1;
          k2[lo] = b2; k2[hi] = a2;
          const uint16_t t = pay[lo]; pay[lo] = pay[hi]; pay[hi] = t;
        }
      }
      __syncthreads();
    }
  }
}

__host__ __device__ inline size_t canon_carve(uint32_t k, unsigned char* base, u64** k1, u64** k2,
                                              uint16_t** pay, uint32_t** wsum) {
  const uint32_t n2 = next_pow2(k);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = (off + bytes + 15) & ~(size_t)15;
    return base + o;
  };
  u64* a = (u64*)take(8ull * n2);
  u64* b = (u64*)take(8ull * n2);
  uint16_t* c = (uint16_t*)take(2ull * n2);
  uint32_t* d = (uint32_t*)take(4ull * 2 * (CANON_BS / 32 + 1));
  if (k1) { *k1 = a; *k2 = b; *pay = c; *wsum = d; }
  return off;
}

template <typename ItemT, int BS>
__device__ void canon_node(const SetView<ItemT>& in, uint32_t node, u64 n, uint32_t kq, int filter,
                           pss_entry* out, uint32_t* out_n, unsigned char* smem) {
  u64 *k1, *k2;
  uint16_t* pay;
  uint32_t* wsum;
  const uint32_t k = in.k;
  canon_carve(k, smem, &k1, &k2, &pay, &wsum);
  const uint32_t tid = threadIdx.x;
  const uint32_t size = in.size[node];
  const size_t base = (size_t)node * k;
  // Frequent summaries: delta = floor((n_covered - sum of counts) / kq)
  const bool mg = filter >= 3;
  u64 delta = 0;
  if (mg) {
    __shared__ u64 part[BS / 32];
    u64 sum = 0;
    for (uint32_t i = tid; i < size; i += BS) sum += in.count[base + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((tid & 31) == 0) part[tid >> 5] = sum;
    __syncthreads();
    sum = 0;
    for (int w = 0; w < BS / 32; ++w) sum += part[w];
    delta = (in.ncov[node] - sum) / kq;
  }
  uint32_t nk = 0, par = 0;
  for (uint32_t b0 = 0; b0 < size; b0 += BS) {
    const uint32_t i = b0 + tid;
    bool keep = false;
    u64 c = 0;
    if (i < size) {
      c = in.count[base + i];
      // filter 1: count k > n (candidates); 2: (count - err) k > n (guaranteed,
      // since count - err <= f); 3: (count + delta) k > n (Frequent
      // candidates: count <= f <= count + delta); 4: count k > n (Frequent
      // guaranteed)
      const u64 t = filter == 2 ? c - in.err[base + i] : (filter == 3 ? c + delta : c);
      keep = !filter || __umul64hi(t, (u64)kq) != 0 || t * (u64)kq > n;
    }
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan<BS>(keep ? 1u : 0u, wsum + (par ? (BS / 32 + 1) : 0), &tot);
    par ^= 1;
    if (keep) {
      k1[nk + ex] = ~c;  // ascending ~count = descending count
      k2[nk + ex] = (u64)in.item[base + i];
      pay[nk + ex] = (uint16_t)i;
    }
    nk += tot;
  }
  const uint32_t n2 = next_pow2(nk ? nk : 1);
  for (uint32_t i = nk + tid; i < n2; i += BS) {
    k1[i] = ~0ull;
    k2[i] = ~0ull;
    pay[i] = 0xFFFF;
  }
  __syncthreads();
  bitonic_sort_2key<BS>(k1, k2, pay, n2);
  for (uint32_t i = tid; i < nk; i += BS) {
    pss_entry e;
    e.item = k2[i];
    e.count = ~k1[i];
    e.err = mg ? delta : in.err[base + pay[i]];
    out[i] = e;
  }
  if (tid == 0) {
    out_n[0] = nk;
    out_n[1] = *in.status;
  }
}

template <typename ItemT, int BS>
__global__ void __launch_bounds__(BS) canon_kernel(SetView<ItemT> in, uint32_t node, u64 n,
                                                   uint32_t kq, int filter, pss_entry* out,
                                                   uint32_t* out_n) {
  extern __shared__ __align__(16) unsigned char smem[];
  canon_node<ItemT, BS>(in, node, n, kq, filter, out, out_n, smem);
}

// Batch form: CTA d answers the query of descriptor d (its root is node 0 of
// a one-node set); results at out + out_off, counts at out_n[2 d], status at
// out_n[2 d + 1].
template <typename ItemT, int BS>
__global__ void __launch_bounds__(BS) query_batch_kernel(const QueryDesc* __restrict__ descs,
                                                         pss_entry* out, uint32_t* out_n,
                                                         const uint32_t* __restrict__ ids) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t id = ids[blockIdx.x];
  const QueryDesc d = descs[id];
  const SetView<ItemT> root = set_view_dev<ItemT>(d.root, 1, d.k);
  canon_node<ItemT, BS>(root, 0, d.n, d.kq, d.filter, out + d.out_off, out_n + 2 * id, smem);
}

}  // namespace

template <typename ItemT>
cudaError_t launch_canon(SetView<ItemT> in, uint32_t node, u64 n, uint32_t kq, int filter,
                         pss_entry* out, uint32_t* out_n, cudaStream_t stream) {
  const size_t smem = canon_carve(in.k, nullptr, nullptr, nullptr, nullptr, nullptr);
  auto kern = canon_kernel<ItemT, CANON_BS>;
  cudaError_t e = ensure_kernel_attrs((const void*)kern);
  if (e != cudaSuccess) return e;
  kern<<<1, CANON_BS, smem, stream>>>(in, node, n, kq, filter, out, out_n);
  return cudaGetLastError();
}

template <typename ItemT>
cudaError_t launch_query_batch(const QueryDesc* descs, const uint32_t* ids, uint32_t count,
                               uint32_t k, pss_entry* out, uint32_t* out_n, cudaStream_t stream) {
  const size_t smem = canon_carve(k, nullptr, nullptr, nullptr, nullptr, nullptr);
  auto kern = query_batch_kernel<ItemT, CANON_BS>;
  cudaError_t e = ensure_kernel_attrs((const void*)kern);
  if (e != cudaSuccess) return e;
  if (count == 0) return cudaSuccess;
  kern<<<count, CANON_BS, smem, stream>>>(descs, out, out_n, ids);
  return cudaGetLastError();
}

template cudaError_t launch_query_batch<uint32_t>(const QueryDesc*, const uint32_t*, uint32_t,
                                                  uint32_t, pss_entry*, uint32_t*, cudaStream_t);
template cudaError_t launch_query_batch<u64>(const QueryDesc*, const uint32_t*, uint32_t, uint32_t,
                                             pss_entry*, uint32_t*, cudaStream_t);
template cudaError_t launch_canon<uint32_t>(SetView<uint32_t>, uint32_t, u64, uint32_t, int,
                                            pss_entry*, uint32_t*, cudaStream_t);
template cudaError_t launch_canon<u64>(SetView<u64>, uint32_t, u64, uint32_t, int, pss_entry*,
                                       uint32_t*, cudaStream_t);

}  // namespace pss
