// pss_kernels.cuh — launch entry points of the device kernels (host side).
#pragma once

#include <mutex>
#include <utility>
#include <vector>

#include "pss_internal.cuh"

namespace pss {

// Allow a kernel the device's largest opt-in shared memory and prefer shared
// memory over L1, once per kernel (keyed by its address; instantiations with
// the same signature are different kernels), so that later launches, and
// stream captures, do not set attributes.
inline cudaError_t ensure_kernel_attrs(const void* kern) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, cudaError_t>> done;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& kd : done)
    if (kd.first == kern) return kd.second;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
  // dynamic + static shared memory may not exceed the opt-in limit
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  done.push_back({kern, e});
  return e;
}

constexpr uint32_t SS_SMEM_MAX_K = 4096;  // larger k keep part of the summarize and merge state in HBM
constexpr int SS_BS = 512;     // threads per CTA of the summarize kernel (wide shape)
constexpr int SS_IPT = 2;      // items per thread per window (window = SS_BS * SS_IPT)
// Narrow shape: the same 1024-item window on half the threads, for k whose
// state is small enough that twice as many CTAs (independent blocks) fit on
// an SM.  The result does not depend on the shape.
constexpr int SS_BS_NARROW = 256;
constexpr int SS_IPT_NARROW = 4;
static_assert(SS_BS * SS_IPT == SS_BS_NARROW * SS_IPT_NARROW, "both shapes use one window size");
// Small shape: a 512-item window on 256 threads, whose smaller state lets four
// CTAs share an SM at k where the narrow shape fits only three.
constexpr int SS_BS_SMALL = 256;
constexpr int SS_IPT_SMALL = 2;
enum SSShape { SS_SHAPE_WIDE = 0, SS_SHAPE_NARROW = 1, SS_SHAPE_SMALL = 2 };
constexpr int MERGE_BS = 512;  // threads per CTA of the combine kernel
constexpr int CANON_BS = 1024; // threads per CTA of the query/export kernel

// Shared memory of one summarize CTA for k counters (the wide shape, the
// larger of the two).
template <typename ItemT>
size_t ss_smem_bytes(uint32_t k);

// Shape of the summarize kernel for k counters (`batch`: the persistent
// batch kernel): the shape that keeps the most threads resident per SM; on a
// tie the narrow shape, then the small one, then the wide one (measured:
// the 1024-item window wins where four CTAs of it fit, the 512-item window
// where only it fits four).  Decided once per (item type, k, kernel) by the
// occupancy calculator.
template <typename ItemT>
int ss_shape(uint32_t k, bool batch);

// Blocks r0 .. r0+count-1 of p (Algorithm 1 bounds over n items) into nodes
// node0 .. node0+count-1 of `out`.
template <typename ItemT>
// may_allocate = false: k <= SS_SMEM_MAX_K keeps the whole state in shared
// memory (no stream-ordered scratch is taken).
cudaError_t launch_summarize_blocks(const ItemT* items, u64 n, uint32_t p, uint32_t r0,
                                    uint32_t count, SetView<ItemT> out, uint32_t node0,
                                    cudaStream_t stream, bool may_allocate = true);

template <typename ItemT>
size_t merge_smem_bytes(uint32_t k);

// One level of the reduction tree: out node j = combine(in node 2j, in node
// 2j+1), or a copy of in node 2j when it has no partner.  mg: the merge of
// Frequent (Misra–Gries) summaries of capacity in.k instead.
template <typename ItemT>
cudaError_t launch_merge_level(SetView<ItemT> in, SetView<ItemT> out, cudaStream_t stream,
                               bool mg = false);

// Merge of two single summaries (node ia of a, node ib of b) into node 0 of out.
template <typename ItemT>
cudaError_t launch_merge_pair(SetView<ItemT> a, uint32_t ia, SetView<ItemT> b, uint32_t ib,
                              SetView<ItemT> out, cudaStream_t stream, bool mg = false);

// Frequent (Misra–Gries) summaries with out.k counters (frequent.cu): blocks
// r0 .. r0+count-1 of p into nodes node0 .. node0+count-1, one warp each.
template <typename ItemT>
cudaError_t launch_frequent_blocks(const ItemT* items, u64 n, uint32_t p, uint32_t r0,
                                   uint32_t count, SetView<ItemT> out, uint32_t node0,
                                   cudaStream_t stream);

// Shared memory of one Frequent warp with kc counters.
size_t frequent_warp_bytes(uint32_t kc, int item_bytes);

// Space Saving block summaries by one warp per block in rounds of 32 items
// (summarize_round.cu); k <= PSS_MAX_K_RESIDENT.  round_kmax(): the largest k
// the plain path sends there (0: none).
template <typename ItemT>
cudaError_t launch_summarize_round_blocks(const ItemT* items, u64 n, uint32_t p, uint32_t r0,
                                          uint32_t count, SetView<ItemT> out, uint32_t node0,
                                          cudaStream_t stream);
template <typename ItemT>
cudaError_t launch_summarize_round_batch(const BatchStream* streams, const BatchTask* tasks,
                                         uint32_t ntasks, uint32_t* counter, uint32_t k,
                                         uint32_t grid, cudaStream_t stream);
template <typename ItemT>
uint32_t round_batch_grid(uint32_t k, uint32_t ntasks, int sms);
size_t round_warp_bytes(uint32_t k, int item_bytes);
uint32_t round_kmax();
// Warps of the round kernel resident per SM at k (0 if it cannot run).
template <typename ItemT>
uint32_t round_resident_warps(uint32_t k);

// Canonical export of node `node`: every entry (filter 0), entries with
// count * kq > n (filter 1) or (count - err) * kq > n (filter 2), sorted by
// (count desc, item asc), written to out[0..*out_n).  Frequent summaries:
// with delta = floor((n_covered - sum of counts) / kq), entries with
// (count + delta) * kq > n (filter 3) or count * kq > n (filter 4), each with
// err = delta.
template <typename ItemT>
cudaError_t launch_canon(SetView<ItemT> in, uint32_t node, u64 n, uint32_t kq, int filter,
                         pss_entry* out, uint32_t* out_n, cudaStream_t stream);

template <typename ItemT>
cudaError_t launch_copy_node(SetView<ItemT> in, uint32_t node, SetView<ItemT> out,
                             uint32_t out_node, cudaStream_t stream);

// Batch forms (batch.cu).  Persistent block summaries over a task list (the
// window-parallel CTA kernel; the warp kernel has its own entry point).
template <typename ItemT>
cudaError_t launch_summarize_batch(const BatchStream* streams, const BatchTask* tasks,
                                   uint32_t ntasks, uint32_t* counter, uint32_t k, uint32_t grid,
                                   cudaStream_t stream);

// Exact frequencies and the accuracy metrics of a summary (accuracy.cu).
struct AccOut {
  unsigned long long reported, true_frequent, true_positive, guaranteed, outside;
  double are_sum;
};

cudaError_t launch_exact_counts(const void* items, u64 n, int item_bytes, int log2u,
                                uint32_t* counts, cudaStream_t stream);

template <typename ItemT>
cudaError_t launch_accuracy(SetView<ItemT> in, const uint32_t* counts, int log2u, u64 n,
                            uint32_t kq, AccOut* out, cudaStream_t stream, bool mg = false);

// Warp-per-block summaries for k <= WARP_SS_MAX_K (summarize_warp.cu).  The
// plain path (launch_summarize_blocks) uses them for k <= warp_kmax()
// (default WARP_SS_DEFAULT_K); the batch picks per stream (batch.cu).
constexpr uint32_t WARP_SS_MAX_K = 256;
constexpr uint32_t WARP_SS_DEFAULT_K = 64;
constexpr uint32_t ROUND_SS_DEFAULT_K = 256;  // plain path: the round kernel up to this k
uint32_t warp_kmax();

template <typename ItemT>
cudaError_t launch_summarize_warp_blocks(const ItemT* items, u64 n, uint32_t p, uint32_t r0,
                                         uint32_t count, SetView<ItemT> out, uint32_t node0,
                                         cudaStream_t stream);

template <typename ItemT>
cudaError_t launch_summarize_warp_batch(const BatchStream* streams, const BatchTask* tasks,
                                        uint32_t ntasks, uint32_t* counter, uint32_t k,
                                        uint32_t grid, cudaStream_t stream);

template <typename ItemT>
int summarize_warp_ctas_per_sm(uint32_t k);

// Resident CTAs per SM of the persistent CTA kernel for k counters and
// ntasks blocks, in the shape the launch picks (0 if it cannot run).
template <typename ItemT>
int summarize_ctas_per_sm(uint32_t k, uint64_t ntasks);

// One CTA per task: node task.index of the next level of descriptor task.stream
// (mg: the Frequent merge).
template <typename ItemT>
cudaError_t launch_merge_tasks(const MergeDesc* descs, const BatchTask* tasks, uint32_t ntasks,
                               uint32_t k, cudaStream_t stream, bool mg = false);

// Persistent Frequent block summaries over a task list (frequent.cu): each
// warp takes (stream, block) tasks from *counter; streams[i].k is the
// capacity k - 1.  frequent_batch_grid gives the CTAs for ntasks tasks (0 if
// it cannot run).
template <typename ItemT>
cudaError_t launch_frequent_batch(const BatchStream* streams, const BatchTask* tasks,
                                  uint32_t ntasks, uint32_t* counter, uint32_t kc, uint32_t grid,
                                  cudaStream_t stream);
template <typename ItemT>
uint32_t frequent_batch_grid(uint32_t kc, uint32_t ntasks, int sms);

// One CTA per id: the query of descs[ids[i]].
template <typename ItemT>
cudaError_t launch_query_batch(const QueryDesc* descs, const uint32_t* ids, uint32_t count,
                               uint32_t k, pss_entry* out, uint32_t* out_n, cudaStream_t stream);

// Host-side: the root set of the whole path (api.cu), stream-ordered on s.
int summarize_to_set(const void* d_items, uint64_t n, int w, uint32_t k, uint32_t p,
                     cudaStream_t s, void** root);

// Host-side accessors of a batch (batch.cu): stream i's root set (one node),
// and its query result (entries, then {count, status}) on the device.
void* batch_root(pss_batch* b, uint32_t i);
void batch_query_device(pss_batch* b, uint32_t i, pss_entry** entries, uint32_t** counts);

// Kernel-group timing (profile.cu): categories of ProfScope.
enum ProfCat : int { PROF_SUMMARIZE = 0, PROF_MERGE = 1, PROF_QUERY = 2 };

// Records CUDA events on `s` around its lifetime when profiling is enabled;
// `units` is what the group counts as launches of its category.
class ProfScope {
 public:
  ProfScope(int cat, cudaStream_t s, uint64_t units);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  int cat_;
  cudaStream_t s_;
  uint64_t units_;
  cudaEvent_t start_ = nullptr, end_ = nullptr;
  bool active_ = false;
};

// Host image of a one-node set holding canonical entries (api.cu).
int summary_image(const pss_entry* entries, uint32_t size, uint64_t m, uint64_t n_covered,
                  uint32_t k, int w, std::vector<char>& image);

// Adds n (modulo 2^64) to the library's launch counter; launch_count reads it.
void count_launches(uint64_t n);
uint64_t launch_count();

cudaError_t launch_gen_zipf(void* out, u64 count, int item_bytes, u64 seed, uint32_t stream_id,
                            u64 start, double s, int log2u, cudaStream_t stream);

}  // namespace pss
