// batch.cu — many independent streams, each summarized with its own k and p,
// in one launch graph: for every distinct k a persistent summarize kernel
// takes (stream, block) tasks from a work list (longest blocks first), then
// one combine launch per tree level covers that level of every stream, then
// one launch answers every stream's query.  The k classes run on forked
// streams; the whole sequence can be captured once as a CUDA graph and
// replayed.  Each stream's result is exactly pss_summarize + pss_query with
// the same k and p (the tree of Algorithm 1 and the combine of Algorithm 2 are
// per stream; batching only changes the launch structure).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "pss_internal.cuh"
#include "pss_kernels.cuh"

using namespace pss;

namespace {

struct StreamPlan {
  const void* items;
  uint64_t n;
  uint32_t k, p;
  uint32_t cap;                      // entries per node: k, or k - 1 (Frequent)
  std::vector<size_t> level_off;     // arena offset of each level's set
  std::vector<uint32_t> level_nodes;
  uint32_t out_off;                  // first result entry of this stream
  int kernel;                        // block summaries: KERN_CTA, KERN_WARP or KERN_ROUND
};

enum { KERN_CTA = 0, KERN_WARP = 1, KERN_ROUND = 2 };

// Kernel for a stream's block summaries.  The three kernels compute the same
// summaries; the warp kernel (counters in registers, one item at a time)
// wins where misses dominate, the window-parallel CTA kernel where hits do,
// and its cost rises with k.  The skew band [lo, hi) in which the warp
// kernel is faster, per k class, measured on a GB300 at full occupancy (u64
// items, 2^28 items in blocks of 2^15; warp / CTA items/s): k = 32: 11.9 at
// s = 0.5, 1.27 at 1.9; k = 64: 1.04 at 1.7, 0.80 at 1.8; k = 96: 1.28 at
// 1.4, 0.85 at 1.5; k = 128: 1.38 at 1.3, 0.88 at 1.4; k = 160: 1.03 at
// 1.2, 0.71 at 1.3; k = 192: 0.88 at 0.7, 1.13 at 0.9 and 1.1, 0.84 at 1.2;
// k = 224: <= 1.08 (at 1.0 only); k = 256: <= 0.93.  An unknown skew (hint
// <= 0) counts as weak.
struct WarpBand {
  uint32_t kmax;
  double lo, hi;
};
constexpr WarpBand WARP_BANDS[] = {{32, 0.0, 1.95},  {64, 0.0, 1.75},  {96, 0.0, 1.45},
                                   {128, 0.0, 1.35}, {160, 0.0, 1.25}, {192, 0.85, 1.15}};

bool use_warp_kernel(uint32_t k, double skew) {
  if (warp_kmax() == 0 || k > WARP_SS_MAX_K) return false;
  if (skew <= 0.0) return k <= 64;
  for (const WarpBand& b : WARP_BANDS)
    if (k <= b.kmax) return skew >= b.lo && skew < b.hi;
  return false;
}

// The round kernel (one warp per block in rounds of 32 items) against the
// best of the other two, measured on a GB300 with the batch's block length
// (autotune.sweep_kernels: 2^28 u64 items in blocks of 2^15; round / best
// other items/s): k = 32: 0.61..0.88 at s <= 1.3, 1.03..2.34 at s >= 1.4;
// k = 48..64: 1.11..1.17 at s <= 0.7, 0.77..0.98 at 0.9..1.2, 1.17..1.94 at
// s >= 1.4; k = 96..256: 1.08..4.05 at every skew; k = 320..384: 1.02..1.79
// at s <= 1.3, 0.81..0.92 above; k = 448: 1.06..1.14 at s <= 1.1, 0.77..0.97
// above.  It is off when pss_set_round_kmax(0).
bool use_round_kernel(uint32_t k, double skew) {
  if (round_kmax() == 0 || k > 448) return false;
  if (skew <= 0.0) return k > 64 && k <= 256;
  if (k <= 32) return skew >= 1.4;
  if (k <= 64) return skew >= 1.4 || skew < 0.8;
  if (k <= 256) return true;
  if (k <= 384) return skew < 1.3;
  return skew < 1.1;
}

int choose_kernel(uint32_t k, double skew) {
  if (use_round_kernel(k, skew)) return KERN_ROUND;
  return use_warp_kernel(k, skew) ? KERN_WARP : KERN_CTA;
}

struct LevelLaunch {
  size_t descs_off, tasks_off;
  uint32_t ntasks;
};

struct KClass {
  uint32_t k = 0;
  std::vector<uint32_t> sids;
  size_t tasks_off = 0, counter_off = 0, qids_off = 0;
  uint32_t ntasks = 0, grid = 0;
  size_t wtasks_off = 0, wcounter_off = 0;  // the class's streams on the warp kernel
  uint32_t wntasks = 0, wgrid = 0;
  size_t rtasks_off = 0, rcounter_off = 0;  // ... and on the round kernel
  uint32_t rntasks = 0, rgrid = 0;
  std::vector<LevelLaunch> levels;
  cudaStream_t side = nullptr;
  cudaEvent_t join = nullptr;
};

int from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return PSS_OK;
  if (e == cudaErrorMemoryAllocation) return PSS_ENOMEM;
  return PSS_ECUDA;
}

__global__ void zero_words_kernel(char* arena, const size_t* offs, uint32_t count) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    *(uint32_t*)(arena + offs[i]) = 0u;
}

}  // namespace

struct pss_batch {
  uint32_t nstreams = 0;
  int w = 4;
  int kind = PSS_KIND_SPACE_SAVING;
  std::vector<StreamPlan> s;
  std::vector<KClass> kc;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  size_t streams_off = 0, qdesc_off = 0, results_off = 0, nout_off = 0, status_offs_off = 0;
  uint32_t nstatus = 0;
  uint64_t total_k = 0;
  uint64_t total_items = 0;
  cudaStream_t owner = nullptr;
  cudaStream_t capture = nullptr;  // the graph is captured here, launched on the caller's stream
  uint64_t graph_launches = 0;     // kernels per graph launch
  cudaEvent_t fork = nullptr;
  cudaEvent_t ready = nullptr;            // the descriptors have landed (on the creating stream)
  std::vector<std::vector<char>> staged;  // host images of the descriptors, kept until destroy
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

// Blocks for n items with block length 2^len_log2[k class][skew class]; an
// unknown skew (hint <= 0) takes the middle class.
uint32_t plan_from(const uint32_t (*len_log2)[3], uint64_t n, uint32_t k, double skew_hint) {
  const double sk = skew_hint > 0.0 ? skew_hint : 1.4;
  static const double classes[3] = {0.8, 1.4, 2.0};
  int sc = 0;  // the nearest class, ties to the lower one
  for (int c = 1; c < 3; ++c)
    if (std::fabs(sk - classes[c]) < std::fabs(sk - classes[sc])) sc = c;
  const int kc = k <= 64 ? 0 : (k <= 256 ? 1 : (k <= 1024 ? 2 : 3));
  const uint64_t len = 1ull << len_log2[kc][sc];
  uint64_t p = (n + len - 1) / len;
  if (p == 0) p = 1;
  while ((n + p - 1) / p >= (1ull << 32)) ++p;
  if (p > 0x7FFFFFFFull) p = 0x7FFFFFFFull;
  return (uint32_t)p;
}

}  // namespace

extern "C" uint32_t pss_plan_blocks(uint64_t n, uint32_t k, int item_bytes, double skew_hint) {
  (void)item_bytes;
  // Block length per (k class, skew class), measured on a GB300 by the
  // project's autotuner (one 2^27-item stream per class through the batch
  // path; paper_1606_04669_gb300/autotune.py holds the same table): short
  // blocks for small k (more blocks in flight), 2^17 at k = 4096.
  static const uint32_t len_log2[4][3] = {{15, 15, 15}, {15, 15, 15}, {15, 16, 16}, {17, 17, 17}};
  return plan_from(len_log2, n, k, skew_hint);
}

extern "C" uint32_t pss_frequent_plan_blocks(uint64_t n, uint32_t k, int item_bytes,
                                             double skew_hint) {
  (void)item_bytes;
  // The same measurement for the Frequent batch (autotune.FREQUENT_TABLE):
  // one warp per block favours shorter blocks than the CTA kernel, 2^14 at
  // k = 1024 and 2^16 at k = 4096.
  static const uint32_t len_log2[4][3] = {{15, 15, 15}, {15, 15, 15}, {14, 14, 15}, {16, 16, 16}};
  return plan_from(len_log2, n, k, skew_hint);
}

namespace {

template <typename ItemT>
int enqueue(pss_batch* b, cudaStream_t s) {
  cudaError_t e = cudaEventRecord(b->fork, s);
  if (e != cudaSuccess) return from_cuda(e);
  // status words of every set start clear (a set's status collects kernel errors)
  e = cudaStreamWaitEvent(b->kc[0].side, b->fork, 0);
  if (e != cudaSuccess) return from_cuda(e);
  count_launches(1);
  zero_words_kernel<<<64, 256, 0, b->kc[0].side>>>(
      b->arena, (const size_t*)(b->arena + b->status_offs_off), b->nstatus);
  if ((e = cudaGetLastError()) != cudaSuccess) return from_cuda(e);
  e = cudaEventRecord(b->kc[0].join, b->kc[0].side);
  if (e != cudaSuccess) return from_cuda(e);
  const bool mg = b->kind == PSS_KIND_FREQUENT;
  for (KClass& c : b->kc) {
    const uint32_t cap = mg ? c.k - 1 : c.k;
    e = cudaStreamWaitEvent(c.side, b->kc[0].join, 0);
    if (e != cudaSuccess) return from_cuda(e);
    e = cudaMemsetAsync(b->arena + c.counter_off, 0, 4, c.side);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->arena + c.wcounter_off, 0, 4, c.side);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->arena + c.rcounter_off, 0, 4, c.side);
    if (e != cudaSuccess) return from_cuda(e);
    {
      ProfScope prof(PROF_SUMMARIZE, c.side,
                     (c.ntasks ? 1 : 0) + (c.wntasks ? 1 : 0) + (c.rntasks ? 1 : 0));
      if (c.rntasks) {
        count_launches(1);
        e = launch_summarize_round_batch<ItemT>((const BatchStream*)(b->arena + b->streams_off),
                                                (const BatchTask*)(b->arena + c.rtasks_off),
                                                c.rntasks, (uint32_t*)(b->arena + c.rcounter_off),
                                                c.k, c.rgrid, c.side);
        if (e != cudaSuccess) return from_cuda(e);
      }
      if (c.wntasks) {
        count_launches(1);
        e = launch_summarize_warp_batch<ItemT>((const BatchStream*)(b->arena + b->streams_off),
                                               (const BatchTask*)(b->arena + c.wtasks_off),
                                               c.wntasks, (uint32_t*)(b->arena + c.wcounter_off),
                                               c.k, c.wgrid, c.side);
        if (e != cudaSuccess) return from_cuda(e);
      }
      if (c.ntasks) {
        count_launches(1);
        if (mg)
          e = launch_frequent_batch<ItemT>((const BatchStream*)(b->arena + b->streams_off),
                                           (const BatchTask*)(b->arena + c.tasks_off), c.ntasks,
                                           (uint32_t*)(b->arena + c.counter_off), cap, c.grid,
                                           c.side);
        else
          e = launch_summarize_batch<ItemT>((const BatchStream*)(b->arena + b->streams_off),
                                            (const BatchTask*)(b->arena + c.tasks_off), c.ntasks,
                                            (uint32_t*)(b->arena + c.counter_off), c.k, c.grid,
                                            c.side);
      }
    }
    if (e != cudaSuccess) return from_cuda(e);
    {
      ProfScope prof(PROF_MERGE, c.side, c.levels.size());
      for (const LevelLaunch& L : c.levels) {
        count_launches(1);
        e = launch_merge_tasks<ItemT>((const MergeDesc*)(b->arena + L.descs_off),
                                      (const BatchTask*)(b->arena + L.tasks_off), L.ntasks, cap,
                                      c.side, mg);
        if (e != cudaSuccess) return from_cuda(e);
      }
    }
    {
      ProfScope prof(PROF_QUERY, c.side, 1);
      count_launches(1);
      e = launch_query_batch<ItemT>((const QueryDesc*)(b->arena + b->qdesc_off),
                                    (const uint32_t*)(b->arena + c.qids_off),
                                    (uint32_t)c.sids.size(), cap,
                                    (pss_entry*)(b->arena + b->results_off),
                                    (uint32_t*)(b->arena + b->nout_off), c.side);
    }
    if (e != cudaSuccess) return from_cuda(e);
    e = cudaEventRecord(c.join, c.side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c.join, 0);
    if (e != cudaSuccess) return from_cuda(e);
  }
  return PSS_OK;
}

void destroy(pss_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->arena) cudaFreeAsync(b->arena, b->owner);
  for (KClass& c : b->kc) {
    if (c.side) {
      cudaStreamSynchronize(c.side);
      cudaStreamDestroy(c.side);
    }
    if (c.join) cudaEventDestroy(c.join);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->ready) {
    cudaEventSynchronize(b->ready);  // the staged host images may still be read
    cudaEventDestroy(b->ready);
  }
  if (b->capture) {
    cudaStreamSynchronize(b->capture);
    cudaStreamDestroy(b->capture);
  }
  delete b;
}

}  // namespace

namespace {

int batch_create(const pss_batch_desc* desc, void* stream, pss_batch** out, int kind) {
  if (!desc || !out) return PSS_EINVAL;
  *out = nullptr;
  const uint32_t ns = desc->nstreams;
  const int w = desc->item_bytes;
  if (ns == 0 || (w != 4 && w != 8) || !desc->d_items || !desc->n || !desc->k) return PSS_EINVAL;
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return PSS_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  pss_batch* b = new (std::nothrow) pss_batch;
  if (!b) return PSS_ENOMEM;
  b->nstreams = ns;
  b->w = w;
  b->kind = kind;
  b->owner = s;
  const bool mg = kind == PSS_KIND_FREQUENT;
  b->s.resize(ns);
  // ---- plan every stream and lay out its tree levels
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = align_up(off, 256);
    off = o + bytes;
    return o;
  };
  std::vector<uint32_t> kvals;
  for (uint32_t i = 0; i < ns; ++i) {
    StreamPlan& sp = b->s[i];
    sp.items = desc->d_items[i];
    sp.n = desc->n[i];
    sp.k = desc->k[i];
    const double skew = desc->skew_hint ? desc->skew_hint[i] : 0.0;
    sp.p = (desc->p && desc->p[i]) ? desc->p[i]
                                   : (mg ? pss_frequent_plan_blocks(sp.n, sp.k, w, skew)
                                         : pss_plan_blocks(sp.n, sp.k, w, skew));
    sp.kernel = mg ? KERN_CTA : choose_kernel(sp.k, skew);
    if (sp.k < 2 || sp.k > PSS_MAX_K_RESIDENT || sp.p == 0 || (sp.n > 0 && !sp.items) ||
        (sp.n + sp.p - 1) / sp.p >= (1ull << 32)) {
      destroy(b);
      return PSS_EINVAL;
    }
    sp.cap = mg ? sp.k - 1 : sp.k;
    const size_t need = mg ? frequent_warp_bytes(sp.cap, w)
                           : (w == 4 ? ss_smem_bytes<uint32_t>(sp.k) : ss_smem_bytes<u64>(sp.k));
    const size_t need_m =
        w == 4 ? merge_smem_bytes<uint32_t>(sp.cap) : merge_smem_bytes<u64>(sp.cap);
    if (need > (size_t)optin || need_m > (size_t)optin) {
      destroy(b);
      return PSS_EINVAL;
    }
    for (uint32_t nodes = sp.p;; nodes = (nodes + 1) / 2) {
      sp.level_nodes.push_back(nodes);
      sp.level_off.push_back(take(set_layout(nodes, sp.cap, w).total));
      if (nodes == 1) break;
    }
    sp.out_off = (uint32_t)b->total_k;
    b->total_k += sp.k;
    b->total_items += sp.n;
    if (std::find(kvals.begin(), kvals.end(), sp.k) == kvals.end()) kvals.push_back(sp.k);
  }
  std::sort(kvals.begin(), kvals.end());
  b->streams_off = take(sizeof(BatchStream) * ns);
  b->qdesc_off = take(sizeof(QueryDesc) * ns);
  b->results_off = take(sizeof(pss_entry) * b->total_k);
  b->nout_off = take(sizeof(uint32_t) * 2 * ns);
  // ---- per k class: tasks (longest blocks first), merge levels, query ids
  std::vector<char> host;  // image of the descriptor part of the arena, filled below
  struct Pending {
    size_t off;
    std::vector<char> bytes;
  };
  std::vector<Pending> uploads;
  auto upload = [&](size_t o, const void* src, size_t bytes) {
    Pending pd;
    pd.off = o;
    pd.bytes.assign((const char*)src, (const char*)src + bytes);
    uploads.push_back(std::move(pd));
  };
  b->kc.resize(kvals.size());
  for (size_t ci = 0; ci < kvals.size(); ++ci) {
    KClass& c = b->kc[ci];
    c.k = kvals[ci];
    for (uint32_t i = 0; i < ns; ++i)
      if (b->s[i].k == c.k) c.sids.push_back(i);
    // tasks of each kernel, longest blocks first so that the last wave is short
    auto plan_tasks = [&](int kernel, size_t* off, size_t* counter, uint32_t* count) {
      std::vector<BatchTask> tasks;
      for (uint32_t i : c.sids)
        if (b->s[i].kernel == kernel)
          for (uint32_t r = 0; r < b->s[i].p; ++r) tasks.push_back(BatchTask{i, r});
      std::vector<uint64_t> key(tasks.size());
      for (size_t t = 0; t < tasks.size(); ++t) {
        const StreamPlan& sp = b->s[tasks[t].stream];
        key[t] = block_bound(tasks[t].index + 1ull, sp.n, sp.p) -
                 block_bound(tasks[t].index, sp.n, sp.p);
      }
      std::vector<size_t> order(tasks.size());
      for (size_t t = 0; t < order.size(); ++t) order[t] = t;
      std::stable_sort(order.begin(), order.end(),
                       [&](size_t a, size_t bb) { return key[a] > key[bb]; });
      std::vector<BatchTask> sorted(tasks.size());
      for (size_t t = 0; t < order.size(); ++t) sorted[t] = tasks[order[t]];
      *count = (uint32_t)sorted.size();
      *off = take(sizeof(BatchTask) * (sorted.size() ? sorted.size() : 1));
      upload(*off, sorted.data(), sizeof(BatchTask) * sorted.size());
      *counter = take(4);
    };
    plan_tasks(KERN_CTA, &c.tasks_off, &c.counter_off, &c.ntasks);
    plan_tasks(KERN_WARP, &c.wtasks_off, &c.wcounter_off, &c.wntasks);
    plan_tasks(KERN_ROUND, &c.rtasks_off, &c.rcounter_off, &c.rntasks);
    if (c.rntasks) {
      c.rgrid = w == 4 ? round_batch_grid<uint32_t>(c.k, c.rntasks, sms)
                       : round_batch_grid<u64>(c.k, c.rntasks, sms);
      if (c.rgrid == 0) {
        destroy(b);
        return PSS_EINVAL;
      }
    }
    if (c.ntasks && mg) {
      c.grid = w == 4 ? frequent_batch_grid<uint32_t>(c.k - 1, c.ntasks, sms)
                      : frequent_batch_grid<u64>(c.k - 1, c.ntasks, sms);
      if (c.grid == 0) {
        destroy(b);
        return PSS_EINVAL;
      }
    } else if (c.ntasks) {
      const int per_sm = w == 4 ? summarize_ctas_per_sm<uint32_t>(c.k, c.ntasks)
                                : summarize_ctas_per_sm<u64>(c.k, c.ntasks);
      if (per_sm <= 0) {
        destroy(b);
        return PSS_EINVAL;
      }
      c.grid = (uint32_t)std::min<uint64_t>((uint64_t)sms * per_sm, c.ntasks);
    }
    if (c.wntasks) {
      const int per_sm = w == 4 ? summarize_warp_ctas_per_sm<uint32_t>(c.k)
                                : summarize_warp_ctas_per_sm<u64>(c.k);
      if (per_sm <= 0) {
        destroy(b);
        return PSS_EINVAL;
      }
      // WS_WPB blocks per CTA
      c.wgrid = (uint32_t)std::min<uint64_t>((uint64_t)sms * per_sm, (c.wntasks + 3) / 4);
    }
    // merge levels: level l -> l + 1 for every stream of the class that has it
    for (uint32_t l = 0;; ++l) {
      std::vector<MergeDesc> descs;
      std::vector<BatchTask> mt;
      for (uint32_t i : c.sids) {
        const StreamPlan& sp = b->s[i];
        if (l + 1 >= sp.level_nodes.size()) continue;
        const uint32_t d = (uint32_t)descs.size();
        descs.push_back(MergeDesc{nullptr, nullptr, sp.level_nodes[l], sp.cap});
        // pointers are fixed once the arena exists; record offsets for now
        descs.back().in = (void*)(uintptr_t)sp.level_off[l];
        descs.back().out = (void*)(uintptr_t)sp.level_off[l + 1];
        for (uint32_t j = 0; j < sp.level_nodes[l + 1]; ++j) mt.push_back(BatchTask{d, j});
      }
      if (descs.empty()) break;
      LevelLaunch L;
      L.descs_off = take(sizeof(MergeDesc) * descs.size());
      L.tasks_off = take(sizeof(BatchTask) * mt.size());
      L.ntasks = (uint32_t)mt.size();
      upload(L.descs_off, descs.data(), sizeof(MergeDesc) * descs.size());
      upload(L.tasks_off, mt.data(), sizeof(BatchTask) * mt.size());
      c.levels.push_back(L);
    }
    c.qids_off = take(sizeof(uint32_t) * c.sids.size());
    upload(c.qids_off, c.sids.data(), sizeof(uint32_t) * c.sids.size());
  }
  // status words of every set
  std::vector<size_t> status_offs;
  for (const StreamPlan& sp : b->s)
    for (size_t l = 0; l < sp.level_off.size(); ++l)
      status_offs.push_back(sp.level_off[l] + set_layout(sp.level_nodes[l], sp.cap, w).status);
  b->nstatus = (uint32_t)status_offs.size();
  b->status_offs_off = take(sizeof(size_t) * status_offs.size());
  b->arena_bytes = align_up(off, 256);
  // ---- device memory and descriptors
  cudaError_t e = cudaMallocAsync((void**)&b->arena, b->arena_bytes, s);
  if (e != cudaSuccess) {
    b->arena = nullptr;
    destroy(b);
    return from_cuda(e);
  }
  std::vector<BatchStream> bs(ns);
  std::vector<QueryDesc> qd(ns);
  for (uint32_t i = 0; i < ns && e == cudaSuccess; ++i) {
    const StreamPlan& sp = b->s[i];
    bs[i] = BatchStream{sp.items, sp.n, sp.p, sp.cap, b->arena + sp.level_off[0]};
    qd[i] = QueryDesc{b->arena + sp.level_off.back(), sp.n, sp.cap, sp.out_off, sp.k, mg ? 3 : 1};
  }
  for (Pending& pd : uploads) {  // merge descriptors: offsets -> pointers
    for (KClass& c : b->kc)
      for (LevelLaunch& L : c.levels)
        if (pd.off == L.descs_off) {
          MergeDesc* md = (MergeDesc*)pd.bytes.data();
          const size_t cnt = pd.bytes.size() / sizeof(MergeDesc);
          for (size_t t = 0; t < cnt; ++t) {
            md[t].in = b->arena + (uintptr_t)md[t].in;
            md[t].out = b->arena + (uintptr_t)md[t].out;
          }
        }
  }
  // The descriptors go up in stream order after the arena's allocation; the
  // host does not wait for them (a batch per serving tick would otherwise
  // wait for the copy engine at every tick).  b->ready marks their arrival.
  auto stage = [&](size_t o, const void* src, size_t bytes) {
    if (e != cudaSuccess || bytes == 0) return;
    b->staged.emplace_back((const char*)src, (const char*)src + bytes);
    e = cudaMemcpyAsync(b->arena + o, b->staged.back().data(), bytes, cudaMemcpyHostToDevice, s);
  };
  stage(b->streams_off, bs.data(), sizeof(BatchStream) * ns);
  stage(b->qdesc_off, qd.data(), sizeof(QueryDesc) * ns);
  stage(b->status_offs_off, status_offs.data(), sizeof(size_t) * status_offs.size());
  for (Pending& pd : uploads) stage(pd.off, pd.bytes.data(), pd.bytes.size());
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(b->ready, s);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  for (KClass& c : b->kc) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.join, cudaEventDisableTiming);
    // set kernel attributes outside any capture
    const uint32_t cap = mg ? c.k - 1 : c.k;
    if (e == cudaSuccess)
      e = w == 4 ? launch_merge_tasks<uint32_t>(nullptr, nullptr, 0, cap, c.side, mg)
                 : launch_merge_tasks<u64>(nullptr, nullptr, 0, cap, c.side, mg);
    if (e == cudaSuccess)
      e = w == 4 ? launch_query_batch<uint32_t>(nullptr, nullptr, 0, cap, nullptr, nullptr, c.side)
                 : launch_query_batch<u64>(nullptr, nullptr, 0, cap, nullptr, nullptr, c.side);
  }
  if (e != cudaSuccess) {
    destroy(b);
    return from_cuda(e);
  }
  *out = b;
  return PSS_OK;
}

}  // namespace

extern "C" int pss_batch_create(const pss_batch_desc* desc, void* stream, pss_batch** out) {
  return batch_create(desc, stream, out, PSS_KIND_SPACE_SAVING);
}

extern "C" int pss_frequent_batch_create(const pss_batch_desc* desc, void* stream,
                                         pss_batch** out) {
  return batch_create(desc, stream, out, PSS_KIND_FREQUENT);
}

extern "C" int pss_batch_plan(const pss_batch* b, uint32_t* p) {
  if (!b || !p) return PSS_EINVAL;
  for (uint32_t i = 0; i < b->nstreams; ++i) p[i] = b->s[i].p;
  return PSS_OK;
}

extern "C" int pss_batch_run(pss_batch* b, int use_graph, void* stream) {
  if (!b) return PSS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!use_graph) {
    const cudaError_t e = cudaStreamWaitEvent(s, b->ready, 0);
    if (e != cudaSuccess) return from_cuda(e);
    return b->w == 4 ? enqueue<uint32_t>(b, s) : enqueue<u64>(b, s);
  }
  if (!b->exec) {
    // the capture cannot wait on an event recorded outside it: the host waits
    // once for the descriptors instead
    cudaError_t e0 = cudaEventSynchronize(b->ready);
    if (e0 != cudaSuccess) return from_cuda(e0);
    // Capture on the batch's own stream (the caller's may be the legacy
    // default stream, which cannot be captured); launches are counted per
    // replay, not at capture.
    cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return from_cuda(e);
    const uint64_t before = launch_count();
    const int rc = b->w == 4 ? enqueue<uint32_t>(b, b->capture) : enqueue<u64>(b, b->capture);
    b->graph_launches = launch_count() - before;
    count_launches(0 - b->graph_launches);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->capture, &g);
    if (rc != PSS_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return from_cuda(e);
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      return from_cuda(e);
    }
  }
  count_launches(b->graph_launches);
  return from_cuda(cudaGraphLaunch(b->exec, s));
}

extern "C" int pss_batch_results(pss_batch* b, pss_entry* host_out, uint32_t* host_counts,
                                 void* stream) {
  if (!b || !host_out || !host_counts) return PSS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<uint32_t> nout(2 * (size_t)b->nstreams);
  std::vector<pss_entry> all(b->total_k);
  cudaError_t e = cudaMemcpyAsync(all.data(), b->arena + b->results_off, sizeof(pss_entry) * b->total_k,
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(nout.data(), b->arena + b->nout_off, sizeof(uint32_t) * nout.size(),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  int rc = PSS_OK;
  for (uint32_t i = 0; i < b->nstreams; ++i) {
    const StreamPlan& sp = b->s[i];
    host_counts[i] = nout[2 * i];
    if (nout[2 * i + 1]) rc = PSS_EDEVICE;
    memcpy(host_out + sp.out_off, all.data() + sp.out_off, sizeof(pss_entry) * nout[2 * i]);
  }
  return rc;
}

extern "C" int pss_batch_export(pss_batch* b, uint32_t index, pss_entry* host_out, uint32_t cap,
                                uint32_t* size, uint64_t* m, uint64_t* n_covered, void* stream) {
  if (!b || index >= b->nstreams || !size) return PSS_EINVAL;
  if (cap > 0 && !host_out) return PSS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const StreamPlan& sp = b->s[index];
  void* root = b->arena + sp.level_off.back();
  const uint32_t k = sp.cap;
  void* dmem = nullptr;
  cudaError_t e = cudaMallocAsync(&dmem, sizeof(pss_entry) * k + 16, s);
  if (e != cudaSuccess) return from_cuda(e);
  pss_entry* d_out = (pss_entry*)dmem;
  uint32_t* d_n = (uint32_t*)((char*)dmem + sizeof(pss_entry) * k);
  count_launches(1);
  e = b->w == 4 ? launch_canon<uint32_t>(set_view<uint32_t>(root, 1, k), 0, 0, 1, 0, d_out, d_n, s)
                : launch_canon<u64>(set_view<u64>(root, 1, k), 0, 0, 1, 0, d_out, d_n, s);
  uint32_t hn[2] = {0, 0};
  const SetLayout L = set_layout(1, k, b->w);
  uint64_t hm = 0, hc = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(hn, d_n, sizeof(hn), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hm, (char*)root + L.m, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, (char*)root + L.ncov, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int rc = from_cuda(e);
  if (rc == PSS_OK && hn[1]) rc = PSS_EDEVICE;
  if (rc == PSS_OK && hn[0] > cap) rc = PSS_ERANGE;
  if (rc == PSS_OK && hn[0]) {
    e = cudaMemcpyAsync(host_out, d_out, sizeof(pss_entry) * hn[0], cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    rc = from_cuda(e);
  }
  cudaFreeAsync(dmem, s);
  if (rc == PSS_OK) {
    if (b->kind == PSS_KIND_FREQUENT) {  // m receives delta, as pss_export
      uint64_t total = 0;
      for (uint32_t i = 0; i < hn[0]; ++i) total += host_out[i].count;
      hm = (hc - total) / sp.k;
    }
    *size = hn[0];
    if (m) *m = hm;
    if (n_covered) *n_covered = hc;
  }
  return rc;
}

extern "C" int pss_batch_info(const pss_batch* b, uint32_t* nstreams, uint64_t* total_items,
                              uint64_t* total_k, uint32_t* k_classes) {
  if (!b) return PSS_EINVAL;
  if (nstreams) *nstreams = b->nstreams;
  if (total_items) *total_items = b->total_items;
  if (total_k) *total_k = b->total_k;
  if (k_classes) *k_classes = (uint32_t)b->kc.size();
  return PSS_OK;
}

extern "C" void pss_batch_free(pss_batch* b) { destroy(b); }

namespace pss {

void* batch_root(pss_batch* b, uint32_t i) { return b->arena + b->s[i].level_off.back(); }

void batch_query_device(pss_batch* b, uint32_t i, pss_entry** entries, uint32_t** counts) {
  *entries = (pss_entry*)(b->arena + b->results_off) + b->s[i].out_off;
  *counts = (uint32_t*)(b->arena + b->nout_off) + 2 * i;
}

}  // namespace pss
