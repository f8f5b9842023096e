// accuracy.cu — exact frequencies and the accuracy metrics of a summary, as
// the paper defines them for its experiments (Section 4): the relative error
// |f - f^| / f of each reported frequency, averaged over the reported items
// (ARE); precision = true k-majority items reported / items reported; recall =
// true k-majority items reported / true k-majority items.  "Reported" is the
// query's output (count k > n); "guaranteed" counts the reported entries
// whose lower bound count - err already exceeds n/k.
#include "pss_internal.cuh"
#include "pss_kernels.cuh"

namespace pss {

namespace {

constexpr int ACC_BS = 256;

// counts[x] += 1 for every item x < 2^log2u; counts[2^log2u] counts the rest.
template <typename ItemT>
__global__ void exact_counts_kernel(const ItemT* __restrict__ items, u64 n, int log2u,
                                    uint32_t* counts) {
  const u64 u = 1ull << log2u;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  // whole warps iterate together; equal items of a warp add with one atomic
  const u64 n_round = (n + 31) / 32 * 32;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
    const u64 x = i < n ? (u64)items[i] : ~0ull;
    const u64 c = i < n ? (x < u ? x : u) : ~0ull;
    const unsigned grp = __match_any_sync(0xffffffffu, c);
    if (c != ~0ull && (threadIdx.x & 31) == (unsigned)(__ffs(grp) - 1))
      atomicAdd(&counts[c], (uint32_t)__popc(grp));
  }
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  T r = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < ACC_BS / 32; ++w) r += scratch[w];
  __syncthreads();
  return r;  // valid in thread 0
}

// One CTA over the summary's entries.  mg: a Frequent summary, whose counts
// are lower bounds: reported when count + delta exceeds the threshold,
// guaranteed when count does.
template <typename ItemT>
__global__ void __launch_bounds__(ACC_BS) accuracy_entries_kernel(SetView<ItemT> in,
                                                                  const uint32_t* __restrict__ counts,
                                                                  int log2u, u64 n, uint32_t kq,
                                                                  bool mg, AccOut* out) {
  __shared__ unsigned long long su[ACC_BS / 32];
  __shared__ double sd[ACC_BS / 32];
  __shared__ u64 sdelta;
  const u64 u = 1ull << log2u;
  const u64 thr = n / kq;  // count k > n  <=>  count > floor(n / k)
  const uint32_t size = in.size[0];
  if (mg) {  // delta = floor((n_covered - sum of counts) / k)
    unsigned long long sum = 0;
    for (uint32_t i = threadIdx.x; i < size; i += ACC_BS) sum += in.count[i];
    sum = block_sum(sum, su);
    if (threadIdx.x == 0) sdelta = (in.ncov[0] - sum) / kq;
    __syncthreads();
  }
  const u64 delta = mg ? sdelta : 0;
  unsigned long long rep = 0, tp = 0, gu = 0;
  double are = 0.0;
  for (uint32_t i = threadIdx.x; i < size; i += ACC_BS) {
    const u64 c = in.count[i], e = in.err[i];
    if (c + delta <= thr) continue;
    const u64 x = (u64)in.item[i];
    const u64 f = x < u ? counts[x] : 0;
    ++rep;
    tp += f > thr ? 1 : 0;
    gu += (mg ? c : c - e) > thr ? 1 : 0;
    if (f) are += (double)(c > f ? c - f : f - c) / (double)f;
  }
  rep = block_sum(rep, su);
  tp = block_sum(tp, su);
  gu = block_sum(gu, su);
  are = block_sum(are, sd);
  if (threadIdx.x == 0) {
    out->reported = rep;
    out->true_positive = tp;
    out->guaranteed = gu;
    out->are_sum = are;
  }
}

// Items with f k > n over the whole universe, and the count outside it.
__global__ void true_frequent_kernel(const uint32_t* __restrict__ counts, u64 u, u64 thr,
                                     AccOut* out) {
  unsigned long long c = 0;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 x = (u64)blockIdx.x * blockDim.x + threadIdx.x; x < u; x += stride)
    c += counts[x] > thr ? 1 : 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&out->true_frequent, c);
  if (blockIdx.x == 0 && threadIdx.x == 0) out->outside = counts[u];
}

int grid_for(u64 work) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  u64 blocks = (work + 255) / 256;
  const u64 cap = (u64)(sms > 0 ? sms : 1) * 8;
  if (blocks > cap) blocks = cap;
  return (int)(blocks ? blocks : 1);
}

}  // namespace

cudaError_t launch_exact_counts(const void* items, u64 n, int item_bytes, int log2u,
                                uint32_t* counts, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(counts, 0, ((1ull << log2u) + 1) * sizeof(uint32_t), stream);
  if (e != cudaSuccess || n == 0) return e;
  count_launches(1);
  if (item_bytes == 4)
    exact_counts_kernel<uint32_t><<<grid_for(n), 256, 0, stream>>>((const uint32_t*)items, n, log2u, counts);
  else
    exact_counts_kernel<u64><<<grid_for(n), 256, 0, stream>>>((const u64*)items, n, log2u, counts);
  return cudaGetLastError();
}

template <typename ItemT>
cudaError_t launch_accuracy(SetView<ItemT> in, const uint32_t* counts, int log2u, u64 n,
                            uint32_t kq, AccOut* out, cudaStream_t stream, bool mg) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(AccOut), stream);
  if (e != cudaSuccess) return e;
  count_launches(2);
  accuracy_entries_kernel<ItemT><<<1, ACC_BS, 0, stream>>>(in, counts, log2u, n, kq, mg, out);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const u64 u = 1ull << log2u;
  true_frequent_kernel<<<grid_for(u), 256, 0, stream>>>(counts, u, n / kq, out);
  return cudaGetLastError();
}

template cudaError_t launch_accuracy<uint32_t>(SetView<uint32_t>, const uint32_t*, int, u64, uint32_t,
                                               AccOut*, cudaStream_t, bool);
template cudaError_t launch_accuracy<u64>(SetView<u64>, const uint32_t*, int, u64, uint32_t, AccOut*,
                                          cudaStream_t, bool);

}  // namespace pss
