// skew.cu — the batch planner's skew estimate, from the data itself.
//
// The planner picks a stream's block-summary kernel and block length by its
// Zipf skew (batch.cu, pss_plan_blocks).  Without a caller's hint, the skew
// is estimated from the stream's first S items (S = min(n, sample) <= 4096):
// the number P of pairs of equal items among them, an exact integer and so a
// pure function of the stream's bytes, gives the collision rate
// q = P / C(S, 2), an unbiased estimate of sum_i p_i^2.  For Zipf(s) over
// [0, 2^32) that rate is q(s) = H(2^32, 2s) / H(2^32, s)^2, increasing in s;
// skew_table.inc holds it for s = 0.30 .. 4.00 and the estimate is its
// inverse by linear interpolation (IEEE +, -, *, / only: the same on every
// machine, so a recorded plan can be replayed).  This is planning, not part
// of the Space Saving method: results never depend on it, only speed.
#include <algorithm>
#include <vector>

#include "pss_internal.cuh"
#include "pss_kernels.cuh"

namespace pss {
namespace {

#include "skew_table.inc"

constexpr int SKEW_BS = 256;
constexpr uint32_t SKEW_MAX_SAMPLE = 4096;

struct SkewDesc {
  const void* items;
  u64 n;
};

// One CTA per stream: the sample (widened to 64 bits, padded with the
// largest value) sorted in shared memory, then one thread counts the pairs
// of equal items run by run (a run of c equal items holds c(c-1)/2 pairs).
// Padding sorts last, so the first S sorted values are the sample's.
template <typename ItemT>
__global__ void __launch_bounds__(SKEW_BS)
    skew_pairs_kernel(const SkewDesc* __restrict__ descs, uint32_t sample, u64* __restrict__ pairs) {
  __shared__ u64 key[SKEW_MAX_SAMPLE];
  const SkewDesc d = descs[blockIdx.x];
  const uint32_t S = (uint32_t)(d.n < sample ? d.n : sample);
  const uint32_t n2 = next_pow2(S < 2 ? 2 : S);
  const ItemT* __restrict__ xs = (const ItemT*)d.items;
  for (uint32_t i = threadIdx.x; i < n2; i += SKEW_BS) key[i] = i < S ? (u64)xs[i] : ~0ull;
  __syncthreads();
  for (uint32_t size = 2; size <= n2; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < (n2 >> 1); i += SKEW_BS) {
        const uint32_t lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
        const bool asc = (lo & size) == 0;
        const u64 a = key[lo], b = key[hi];
        if ((a > b) == asc) {
          key[lo] = b;
          key[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    u64 p = 0;
    uint32_t run = 1;
    for (uint32_t i = 1; i < S; ++i) {
      if (key[i] == key[i - 1]) {
        p += run;
        ++run;
      } else {
        run = 1;
      }
    }
    pairs[blockIdx.x] = p;
  }
}

int from_cuda_skew(cudaError_t e) {
  if (e == cudaSuccess) return PSS_OK;
  if (e == cudaErrorMemoryAllocation) return PSS_ENOMEM;
  return PSS_ECUDA;
}

}  // namespace
}  // namespace pss

using namespace pss;

extern "C" double pss_skew_of_pairs(uint64_t pairs, uint64_t sample) {
  if (sample < 2) return 0.0;  // nothing to estimate from: the planner's "unknown"
  const double q = (double)pairs / ((double)sample * (double)(sample - 1) / 2.0);
  const double smax = SKEW_TABLE_S0 + SKEW_TABLE_STEP * (SKEW_TABLE_N - 1);
  if (q <= SKEW_TABLE_Q[0]) return SKEW_TABLE_S0;
  if (q >= SKEW_TABLE_Q[SKEW_TABLE_N - 1]) return smax;
  int lo = 0, hi = SKEW_TABLE_N - 1;  // SKEW_TABLE_Q[lo] < q <= SKEW_TABLE_Q[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (SKEW_TABLE_Q[mid] < q) lo = mid;
    else hi = mid;
  }
  const double f = (q - SKEW_TABLE_Q[lo]) / (SKEW_TABLE_Q[hi] - SKEW_TABLE_Q[lo]);
  return SKEW_TABLE_S0 + SKEW_TABLE_STEP * ((double)lo + f);
}

extern "C" int pss_estimate_skew(const void* const* d_items, const uint64_t* n, uint32_t nstreams,
                                 int item_bytes, uint32_t sample, void* stream, double* skew_out,
                                 uint64_t* pairs_out) {
  if (!d_items || !n || !skew_out || nstreams == 0 || (item_bytes != 4 && item_bytes != 8) ||
      sample < 2 || sample > SKEW_MAX_SAMPLE)
    return PSS_EINVAL;
  for (uint32_t i = 0; i < nstreams; ++i)
    if (n[i] > 0 && !d_items[i]) return PSS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<SkewDesc> descs(nstreams);
  for (uint32_t i = 0; i < nstreams; ++i) descs[i] = SkewDesc{d_items[i], n[i]};
  std::vector<u64> pairs(nstreams);
  void* dmem = nullptr;
  const size_t dbytes = align_up(sizeof(SkewDesc) * nstreams, 256) + sizeof(u64) * nstreams;
  cudaError_t e = cudaMallocAsync(&dmem, dbytes, s);
  if (e != cudaSuccess) return from_cuda_skew(e);
  SkewDesc* ddesc = (SkewDesc*)dmem;
  u64* dpairs = (u64*)((char*)dmem + align_up(sizeof(SkewDesc) * nstreams, 256));
  e = cudaMemcpyAsync(ddesc, descs.data(), sizeof(SkewDesc) * nstreams, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    count_launches(1);
    if (item_bytes == 4)
      skew_pairs_kernel<uint32_t><<<nstreams, SKEW_BS, 0, s>>>(ddesc, sample, dpairs);
    else
      skew_pairs_kernel<u64><<<nstreams, SKEW_BS, 0, s>>>(ddesc, sample, dpairs);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pairs.data(), dpairs, sizeof(u64) * nstreams, cudaMemcpyDeviceToHost, s);
  const cudaError_t f = cudaFreeAsync(dmem, s);
  if (e == cudaSuccess) e = f;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda_skew(e);
  for (uint32_t i = 0; i < nstreams; ++i) {
    const uint64_t S = n[i] < sample ? n[i] : sample;
    skew_out[i] = pss_skew_of_pairs(pairs[i], S);
    if (pairs_out) pairs_out[i] = pairs[i];
  }
  return PSS_OK;
}
