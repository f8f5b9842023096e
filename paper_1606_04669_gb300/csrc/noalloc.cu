// noalloc.cu — pss_summarize for callers that cannot allocate device memory.
//
// Some callers own every byte of device memory through their own allocator,
// or run under a fixed memory budget and must not allocate once they have
// started (a serving process, for instance); for them a call that takes
// memory from CUDA's allocator behind their back is not usable.  This entry
// point runs the same kernels as pss_summarize, but keeps the block summaries
// and the reduction tree in a fixed array compiled into the library, and
// writes the root summary into buffers the caller passes in.  It calls no
// cudaMalloc, cudaFree or stream-ordered allocation.
//
// The array lives in the library's device image: every GPU that loads the
// library holds it until the process exits.  Every call uses the same array,
// so calls whose work overlaps on the GPU race; the caller serializes them.
#include <mutex>
#include <utility>
#include <vector>

#include "pss_internal.cuh"
#include "pss_kernels.cuh"

// The scratch array (file scope; its size is the public PSS_NOALLOC_SCRATCH_BYTES).
static __device__ __align__(256) unsigned char g_noalloc_scratch[PSS_NOALLOC_SCRATCH_BYTES];

namespace pss {

namespace {

std::mutex g_addr_mu;
std::vector<std::pair<int, void*>> g_addr;  // device -> address of the array

// The array's device address on the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device, with that device current.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_addr_mu);
  for (auto& da : g_addr)
    if (da.first == dev) {
      *out = da.second;
      return cudaSuccess;
    }
  void* ptr = nullptr;
  e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  g_addr.push_back({dev, ptr});
  *out = ptr;
  return cudaSuccess;
}

// Copy the root (node 0 of `root`) into the caller's arrays.
template <typename ItemT>
__global__ void root_out_kernel(SetView<ItemT> root, ItemT* items, u64* counts, u64* errs,
                                u64* header) {
  const uint32_t sz = root.size[0];
  for (uint32_t i = threadIdx.x; i < sz; i += blockDim.x) {
    items[i] = root.item[i];
    counts[i] = root.count[i];
    errs[i] = root.err[i];
  }
  if (threadIdx.x == 0) {
    header[0] = sz;
    header[1] = root.m[0];
    header[2] = root.ncov[0];
    header[3] = *root.status;
  }
}

template <typename ItemT>
int run(const void* d_items, uint64_t n, uint32_t k, uint32_t p, void* out_items,
        uint64_t* out_counts, uint64_t* out_errs, uint64_t* out_header, cudaStream_t s) {
  const int w = (int)sizeof(ItemT);
  const uint32_t p2 = (p + 1) / 2;
  const SetLayout la = set_layout(p, k, w);
  const size_t b_off = align_up(la.total, 256);
  if (b_off + set_layout(p2 > 0 ? p2 : 1, k, w).total > (size_t)PSS_NOALLOC_SCRATCH_BYTES)
    return PSS_ERANGE;
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return PSS_ECUDA;
  char* region[2] = {(char*)base, (char*)base + b_off};
  // The array keeps the previous call's contents: clear the status words.
  uint32_t nodes = p;
  int cur = 0;
  e = cudaMemsetAsync(region[0] + set_layout(nodes, k, w).status, 0, 4, s);
  if (e == cudaSuccess) {
    count_launches(1);
    e = launch_summarize_blocks<ItemT>((const ItemT*)d_items, n, p, 0, p,
                                       set_view<ItemT>(region[0], nodes, k), 0, s, false);
  }
  while (e == cudaSuccess && nodes > 1) {
    const uint32_t nxt = (nodes + 1) / 2;
    e = cudaMemsetAsync(region[cur ^ 1] + set_layout(nxt, k, w).status, 0, 4, s);
    if (e != cudaSuccess) break;
    count_launches(1);
    e = launch_merge_level<ItemT>(set_view<ItemT>(region[cur], nodes, k),
                                  set_view<ItemT>(region[cur ^ 1], nxt, k), s);
    cur ^= 1;
    nodes = nxt;
  }
  if (e == cudaSuccess) {
    count_launches(1);
    root_out_kernel<ItemT><<<1, 256, 0, s>>>(set_view<ItemT>(region[cur], 1, k), (ItemT*)out_items,
                                             (u64*)out_counts, (u64*)out_errs, (u64*)out_header);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? PSS_OK : PSS_ECUDA;
}

}  // namespace

}  // namespace pss

extern "C" int pss_summarize_noalloc(const void* d_items, uint64_t n, int item_bytes, uint32_t k,
                                     uint32_t p, void* d_out_items, uint64_t* d_out_counts,
                                     uint64_t* d_out_errs, uint64_t* d_out_header, void* stream) {
  using namespace pss;
  if (item_bytes != 4 && item_bytes != 8) return PSS_EINVAL;
  if (k < 2 || k > PSS_MAX_K_RESIDENT || p == 0) return PSS_EINVAL;
  if (n > 0 && !d_items) return PSS_EINVAL;
  if (!d_out_items || !d_out_counts || !d_out_errs || !d_out_header) return PSS_EINVAL;
  if ((n + p - 1) / p >= (1ull << 32)) return PSS_EINVAL;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return PSS_ECUDA;
  const size_t need = item_bytes == 4 ? ss_smem_bytes<uint32_t>(k) : ss_smem_bytes<u64>(k);
  const size_t need_m = item_bytes == 4 ? merge_smem_bytes<uint32_t>(k) : merge_smem_bytes<u64>(k);
  if (need > (size_t)optin || need_m > (size_t)optin) return PSS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  return item_bytes == 4
             ? run<uint32_t>(d_items, n, k, p, d_out_items, d_out_counts, d_out_errs, d_out_header, s)
             : run<u64>(d_items, n, k, p, d_out_items, d_out_counts, d_out_errs, d_out_header, s);
}
