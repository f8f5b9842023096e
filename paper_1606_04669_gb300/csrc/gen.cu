// gen.cu — device side of the seeded synthetic input generator.
//
// The stream definition lives in ../gen/pss_zipf.h (shared, bit for bit, with
// the host side); this file only runs it over a grid.  The paper's inputs are
// Zipf streams of skew 1.1 and 1.8 (Section 4.1).
#include "../gen/pss_zipf.h"
#include "pss_internal.cuh"
#include "pss_kernels.cuh"

namespace pss {

namespace {

// The tables and the sampler's constants are built once per CTA (the same
// functions build them on the host).
__global__ void __launch_bounds__(256) gen_zipf_kernel(void* out, u64 count, int item_bytes,
                                                       u64 seed, uint32_t sid, u64 start,
                                                       double s, int log2u) {
  __shared__ pssg_tables tb;
  __shared__ pssg_zipf zs;
  for (int i = threadIdx.x; i < PSSG_LOG_TAB; i += blockDim.x) pssg_tables_entry(&tb, i);
  __syncthreads();
  if (threadIdx.x == 0) pssg_zipf_init(&zs, &tb, s, (log2u >= 64) ? ~0ull : (1ull << log2u));
  __syncthreads();
  const pssg_zipf z = zs;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const u64 x = pssg_zipf_item(&z, &tb, log2u, seed, sid, start + i);
    if (item_bytes == 4)
      ((uint32_t*)out)[i] = (uint32_t)x;
    else
      ((u64*)out)[i] = x;
  }
}

}  // namespace

cudaError_t launch_gen_zipf(void* out, u64 count, int item_bytes, u64 seed, uint32_t stream_id,
                            u64 start, double s, int log2u, cudaStream_t stream) {
  if (count == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  u64 blocks = (count + 255) / 256;
  const u64 cap = (u64)(sms > 0 ? sms : 1) * 8;
  if (blocks > cap) blocks = cap;
  gen_zipf_kernel<<<(unsigned)blocks, 256, 0, stream>>>(out, count, item_bytes, seed, stream_id,
                                                        start, s, log2u);
  return cudaGetLastError();
}

}  // namespace pss
