// api.cu — the extern "C" boundary of libpss (declared in include/pss.h).
//
// Argument checks, device memory of summaries (CUDA stream-ordered
// allocator) and kernel sequencing.  Every step of the computation runs in
// the kernels of summarize.cu, merge.cu and canon.cu.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "pss_internal.cuh"
#include "pss_kernels.cuh"

using namespace pss;

struct pss_summary {
  uint32_t k;           // the k of the k-majority problem
  uint32_t cap;         // entries per node: k (Space Saving) or k - 1 (Frequent)
  int kind;             // PSS_KIND_*
  int item_bytes;
  void* mem;            // one set of one node (set_layout)
  cudaStream_t stream;  // stream of the creating call; frees are ordered on it
};

struct pss_tree {
  uint32_t k, cap, p;
  int kind;
  int item_bytes;
  cudaStream_t stream;
  std::vector<void*> mem;       // one set per level
  std::vector<uint32_t> nodes;  // summaries per level
};

namespace {

std::atomic<int> g_host_direct{1};  // pss_set_host_direct

int from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return PSS_OK;
  if (e == cudaErrorMemoryAllocation) return PSS_ENOMEM;
  return PSS_ECUDA;
}

// Keep freed stream-ordered memory in the pool (no return to the OS between
// calls), once per device.
std::mutex g_pool_mu;
std::vector<int> g_pool_done;

cudaError_t prepare_device() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  for (int d : g_pool_done)
    if (d == dev) return cudaSuccess;
  cudaMemPool_t pool;
  e = cudaDeviceGetDefaultMemPool(&pool, dev);
  if (e != cudaSuccess) return e;
  uint64_t thr = ~0ull;
  e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  if (e != cudaSuccess) return e;
  g_pool_done.push_back(dev);
  return cudaSuccess;
}

cudaError_t alloc_set(uint32_t nodes, uint32_t k, int w, cudaStream_t s, void** mem) {
  SetLayout L = set_layout(nodes, k, w);
  cudaError_t e = cudaMallocAsync(mem, L.total, s);
  if (e != cudaSuccess) {
    *mem = nullptr;
    return e;
  }
  e = cudaMemsetAsync((char*)*mem + L.status, 0, 4, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(*mem, s);
    *mem = nullptr;
  }
  return e;
}

size_t max_optin_smem() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  return (size_t)v;
}

int check_k_width(uint32_t k, int w) {
  if (w != 4 && w != 8) return PSS_EINVAL;
  if (k < 2 || k > PSS_MAX_K) return PSS_EINVAL;
  return PSS_OK;
}

// Level 0 (the block summaries, enqueued by `level0`) and the merge levels;
// k is the capacity of a node, mg selects the Frequent merge.
template <typename ItemT, typename Level0>
int run_tree(uint32_t k, uint32_t p, cudaStream_t s, bool keep, std::vector<void*>& mems,
             std::vector<uint32_t>& nodes, Level0 level0, bool mg = false) {
  const int w = (int)sizeof(ItemT);
  auto fail = [&](cudaError_t e) {
    for (void* m : mems)
      if (m) cudaFreeAsync(m, s);
    mems.clear();
    nodes.clear();
    return from_cuda(e);
  };
  void* m0 = nullptr;
  cudaError_t e = alloc_set(p, k, w, s, &m0);
  if (e != cudaSuccess) return fail(e);
  mems.push_back(m0);
  nodes.push_back(p);
  // k in shared memory: every level's set is allocated (and its status word
  // cleared) before the first kernel, so that the block summaries and the
  // merge levels follow one another on the stream with nothing in between
  // and each level can be launched as a programmatic dependent of the one
  // before (at the cost of holding every level, about twice level 0's bytes)
  const bool chained = k <= SS_SMEM_MAX_K;
  if (chained)
    for (uint32_t cur = p; cur > 1;) {
      cur = (cur + 1) / 2;
      void* mm = nullptr;
      e = alloc_set(cur, k, w, s, &mm);
      if (e != cudaSuccess) return fail(e);
      mems.push_back(mm);
      nodes.push_back(cur);
    }
  {
    ProfScope prof(PROF_SUMMARIZE, s, 1);
    e = level0(set_view<ItemT>(m0, p, k));
  }
  if (e != cudaSuccess) return fail(e);
  uint32_t levels = 0;
  for (uint32_t w2 = p; w2 > 1; w2 = (w2 + 1) / 2) ++levels;
  ProfScope prof(PROF_MERGE, s, levels);
  if (chained) {
    for (size_t L = 1; L < mems.size(); ++L) {
      e = launch_merge_level<ItemT>(set_view<ItemT>(mems[L - 1], nodes[L - 1], k),
                                    set_view<ItemT>(mems[L], nodes[L], k), s, mg);
      count_launches(1);
      if (e != cudaSuccess) return fail(e);
    }
    if (!keep)
      for (size_t i = 0; i + 1 < mems.size(); ++i) {
        cudaFreeAsync(mems[i], s);
        mems[i] = nullptr;
      }
    return PSS_OK;
  }
  while (nodes.back() > 1) {
    const uint32_t cur = nodes.back(), nxt = (cur + 1) / 2;
    void* mm = nullptr;
    e = alloc_set(nxt, k, w, s, &mm);
    if (e != cudaSuccess) return fail(e);
    e = launch_merge_level<ItemT>(set_view<ItemT>(mems.back(), cur, k), set_view<ItemT>(mm, nxt, k),
                                  s, mg);
    count_launches(1);
    if (e != cudaSuccess) {
      cudaFreeAsync(mm, s);
      return fail(e);
    }
    if (!keep) {
      cudaFreeAsync(mems.back(), s);
      mems.back() = nullptr;
    }
    mems.push_back(mm);
    nodes.push_back(nxt);
  }
  return PSS_OK;
}

template <typename ItemT>
int run_tree_device(const void* d_items, uint64_t n, uint32_t k, uint32_t p, cudaStream_t s,
                    bool keep, std::vector<void*>& mems, std::vector<uint32_t>& nodes) {
  return run_tree<ItemT>(k, p, s, keep, mems, nodes, [&](SetView<ItemT> v0) {
    count_launches(1);
    return launch_summarize_blocks<ItemT>((const ItemT*)d_items, n, p, 0, p, v0, 0, s);
  });
}

// The Frequent path: nodes of k - 1 counters, Misra–Gries block summaries and
// the Frequent merge.
template <typename ItemT>
int run_frequent_tree_device(const void* d_items, uint64_t n, uint32_t k, uint32_t p,
                             cudaStream_t s, bool keep, std::vector<void*>& mems,
                             std::vector<uint32_t>& nodes) {
  return run_tree<ItemT>(
      k - 1, p, s, keep, mems, nodes,
      [&](SetView<ItemT> v0) {
        count_launches(1);
        return launch_frequent_blocks<ItemT>((const ItemT*)d_items, n, p, 0, p, v0, 0, s);
      },
      true);
}

// One non-blocking copy stream per device for host-input calls.
std::mutex g_copy_mu;
std::vector<std::pair<int, cudaStream_t>> g_copy_streams;

cudaError_t copy_stream(cudaStream_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_copy_mu);
  for (auto& ds : g_copy_streams)
    if (ds.first == dev) {
      *out = ds.second;
      return cudaSuccess;
    }
  cudaStream_t cs;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  g_copy_streams.push_back({dev, cs});
  *out = cs;
  return cudaSuccess;
}

// Host input: the blocks are copied in `groups` slabs on the copy stream;
// the summarize kernel of slab g starts as soon as slab g has landed, so the
// copy of slab g+1 overlaps it.  k is the node capacity; mg: Frequent
// summaries (block kernel and merge).
template <typename ItemT>
int run_tree_host(const void* h_items, uint64_t n, uint32_t k, uint32_t p, cudaStream_t s,
                  std::vector<void*>& mems, std::vector<uint32_t>& nodes, bool mg = false) {
  const size_t w = sizeof(ItemT);
  cudaStream_t cs;
  cudaError_t e = copy_stream(&cs);
  if (e != cudaSuccess) return from_cuda(e);
  void* dbuf = nullptr;
  if (n) {
    e = cudaMallocAsync(&dbuf, n * w, s);
    if (e != cudaSuccess) return from_cuda(e);
  }
  const uint32_t groups = p < 16 ? p : 16;
  std::vector<cudaEvent_t> evs;
  auto make_event = [&](cudaEvent_t* ev) {
    cudaError_t r = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (r == cudaSuccess) evs.push_back(*ev);
    return r;
  };
  cudaEvent_t ready;
  e = make_event(&ready);
  if (e == cudaSuccess) e = cudaEventRecord(ready, s);        // dbuf allocated on s
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ready, 0);
  int rc = from_cuda(e);
  if (rc == PSS_OK) {
    rc = run_tree<ItemT>(k, p, s, false, mems, nodes, [&](SetView<ItemT> v0) {
      cudaError_t r = cudaSuccess;
      for (uint32_t g = 0; g < groups && r == cudaSuccess; ++g) {
        const uint32_t r0 = (uint32_t)((uint64_t)g * p / groups);
        const uint32_t r1 = (uint32_t)((uint64_t)(g + 1) * p / groups);
        const uint64_t lo = block_bound(r0, n, p), hi = block_bound(r1, n, p);
        if (hi > lo) {
          cudaEvent_t landed;
          r = make_event(&landed);
          if (r == cudaSuccess)
            r = cudaMemcpyAsync((char*)dbuf + lo * w, (const char*)h_items + lo * w, (hi - lo) * w,
                                cudaMemcpyHostToDevice, cs);
          if (r == cudaSuccess) r = cudaEventRecord(landed, cs);
          if (r == cudaSuccess) r = cudaStreamWaitEvent(s, landed, 0);
        }
        if (r == cudaSuccess && r1 > r0) {
          count_launches(1);
          r = mg ? launch_frequent_blocks<ItemT>((const ItemT*)dbuf, n, p, r0, r1 - r0, v0, r0, s)
                 : launch_summarize_blocks<ItemT>((const ItemT*)dbuf, n, p, r0, r1 - r0, v0, r0, s);
        }
      }
      return r;
    }, mg);
  }
  if (dbuf) cudaFreeAsync(dbuf, s);
  for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
  return rc;
}

int validate_summarize(const void* d_items, uint64_t n, int w, uint32_t k, uint32_t p) {
  int rc = check_k_width(k, w);
  if (rc) return rc;
  if (p == 0) return PSS_EINVAL;
  if (n > 0 && d_items == nullptr) return PSS_EINVAL;
  if ((n + p - 1) / p >= (1ull << 32)) return PSS_EINVAL;  // a block must be < 2^32 items
  const size_t need = w == 4 ? ss_smem_bytes<uint32_t>(k) : ss_smem_bytes<u64>(k);
  const size_t need_m = w == 4 ? merge_smem_bytes<uint32_t>(k) : merge_smem_bytes<u64>(k);
  const size_t have = max_optin_smem();
  if (need > have || need_m > have) return PSS_EINVAL;
  return PSS_OK;
}

int tree_common(const void* d_items, uint64_t n, int w, uint32_t k, uint32_t p, cudaStream_t s,
                bool keep, std::vector<void*>& mems, std::vector<uint32_t>& nodes) {
  cudaError_t e = prepare_device();
  if (e != cudaSuccess) return from_cuda(e);
  int rc = validate_summarize(d_items, n, w, k, p);
  if (rc) return rc;
  return w == 4 ? run_tree_device<uint32_t>(d_items, n, k, p, s, keep, mems, nodes)
                : run_tree_device<u64>(d_items, n, k, p, s, keep, mems, nodes);
}

int validate_frequent(const void* items, uint64_t n, int w, uint32_t k, uint32_t p) {
  if ((w != 4 && w != 8) || k < 2 || k > PSS_MAX_K_RESIDENT || p == 0) return PSS_EINVAL;
  if (n > 0 && items == nullptr) return PSS_EINVAL;
  if ((n + p - 1) / p >= (1ull << 32)) return PSS_EINVAL;
  const size_t have = max_optin_smem();
  const size_t need_m = w == 4 ? merge_smem_bytes<uint32_t>(k - 1) : merge_smem_bytes<u64>(k - 1);
  if (frequent_warp_bytes(k - 1, w) > have || need_m > have) return PSS_EINVAL;
  return PSS_OK;
}

int frequent_tree_common(const void* d_items, uint64_t n, int w, uint32_t k, uint32_t p,
                         cudaStream_t s, bool keep, std::vector<void*>& mems,
                         std::vector<uint32_t>& nodes) {
  cudaError_t e = prepare_device();
  if (e != cudaSuccess) return from_cuda(e);
  int rc = validate_frequent(d_items, n, w, k, p);
  if (rc) return rc;
  return w == 4 ? run_frequent_tree_device<uint32_t>(d_items, n, k, p, s, keep, mems, nodes)
                : run_frequent_tree_device<u64>(d_items, n, k, p, s, keep, mems, nodes);
}

// Pinned host memory mapped into the device's address space (a coherent
// CPU-GPU link): its device address, else nullptr (then the items are
// staged).
const void* mapped_host(const void* h_items, uint64_t n) {
  if (!n || !g_host_direct.load()) return nullptr;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, h_items) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
      attr.devicePointer)
    return attr.devicePointer;
  cudaGetLastError();  // an unregistered pointer is not an error here
  return nullptr;
}

// A summary object for one-node set `mem` (nullptr when out of host memory;
// the caller then frees mem).
pss_summary* new_summary(uint32_t k, int kind, int w, void* mem, cudaStream_t s) {
  pss_summary* sm = new (std::nothrow) pss_summary;
  if (!sm) return nullptr;
  sm->k = k;
  sm->cap = kind == PSS_KIND_FREQUENT ? k - 1 : k;
  sm->kind = kind;
  sm->item_bytes = w;
  sm->mem = mem;
  sm->stream = s;
  return sm;
}

// Canonical copy-out of one node; filter selects the query.
int canon_out(void* set_mem, uint32_t nodes, uint32_t node, uint32_t k, int w, uint64_t n,
              uint32_t kq, int filter, pss_entry* host_out, uint32_t cap, uint32_t* n_out,
              cudaStream_t s) {
  const size_t ebytes = (size_t)k * sizeof(pss_entry);
  void* dmem = nullptr;
  cudaError_t e = cudaMallocAsync(&dmem, ebytes + 16, s);
  if (e != cudaSuccess) return from_cuda(e);
  pss_entry* d_out = (pss_entry*)dmem;
  uint32_t* d_n = (uint32_t*)((char*)dmem + ebytes);
  {
  ProfScope prof(PROF_QUERY, s, 1);
  count_launches(1);
  e = (w == 4) ? launch_canon<uint32_t>(set_view<uint32_t>(set_mem, nodes, k), node, n, kq, filter,
                                        d_out, d_n, s)
               : launch_canon<u64>(set_view<u64>(set_mem, nodes, k), node, n, kq, filter, d_out,
                                   d_n, s);
  }
  uint32_t hn[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hn, d_n, sizeof(hn), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int rc = from_cuda(e);
  if (rc == PSS_OK && hn[1] != 0) rc = PSS_EDEVICE;
  if (rc == PSS_OK && hn[0] > cap) rc = PSS_ERANGE;
  if (rc == PSS_OK && hn[0] > 0) {
    e = cudaMemcpyAsync(host_out, d_out, (size_t)hn[0] * sizeof(pss_entry), cudaMemcpyDeviceToHost,
                        s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    rc = from_cuda(e);
  }
  cudaFreeAsync(dmem, s);
  if (rc == PSS_OK && n_out) *n_out = hn[0];
  return rc;
}

}  // namespace

namespace pss {

// Host image of a one-node set (set_layout(1, k, w)) holding the canonical
// entries in item order; PSS_EINVAL on duplicates, size > k, or items wider
// than w bytes.
int summary_image(const pss_entry* entries, uint32_t size, uint64_t m, uint64_t n_covered,
                  uint32_t k, int w, std::vector<char>& image) {
  if ((size && !entries) || size > k || (w != 4 && w != 8)) return PSS_EINVAL;
  std::vector<pss_entry> e(entries, entries + size);
  std::sort(e.begin(), e.end(), [](const pss_entry& a, const pss_entry& b) { return a.item < b.item; });
  for (uint32_t i = 0; i < size; ++i) {
    if (i && e[i].item == e[i - 1].item) return PSS_EINVAL;
    if (w == 4 && e[i].item > 0xFFFFFFFFull) return PSS_EINVAL;
  }
  const SetLayout L = set_layout(1, k, w);
  image.assign(L.total, 0);
  char* b = image.data();
  for (uint32_t i = 0; i < size; ++i) {
    if (w == 4) ((uint32_t*)(b + L.item))[i] = (uint32_t)e[i].item;
    else ((uint64_t*)(b + L.item))[i] = e[i].item;
    ((uint64_t*)(b + L.count))[i] = e[i].count;
    ((uint64_t*)(b + L.err))[i] = e[i].err;
  }
  *(uint32_t*)(b + L.size) = size;
  *(uint64_t*)(b + L.m) = m;
  *(uint64_t*)(b + L.ncov) = n_covered;
  return PSS_OK;
}

// The root set (one node) of the path over d_items, allocated stream-ordered
// on s (release with cudaFreeAsync); used by the serving runtime.
int summarize_to_set(const void* d_items, uint64_t n, int w, uint32_t k, uint32_t p,
                     cudaStream_t s, void** root) {
  std::vector<void*> mems;
  std::vector<uint32_t> nodes;
  *root = nullptr;
  int rc = tree_common(d_items, n, w, k, p, s, false, mems, nodes);
  if (rc) return rc;
  *root = mems.back();
  return PSS_OK;
}

}  // namespace pss

extern "C" {

const char* pss_strerror(int code) {
  switch (code) {
    case PSS_OK: return "success";
    case PSS_EINVAL: return "invalid argument";
    case PSS_EMISMATCH: return "summaries have different k or item width";
    case PSS_ENOMEM: return "device memory allocation failed";
    case PSS_ECUDA: return "CUDA runtime error";
    case PSS_ETIMEOUT: return "bounded device wait expired";
    case PSS_EDEVICE: return "a kernel recorded an error in the summary";
    case PSS_ERANGE: return "output capacity too small";
    default: return "unknown error";
  }
}

int pss_abi_version(void) { return 1; }

int pss_summarize(const void* d_items, uint64_t n, int item_bytes, uint32_t k, uint32_t p,
                  void* stream, pss_summary** out) {
  if (!out) return PSS_EINVAL;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<void*> mems;
  std::vector<uint32_t> nodes;
  int rc = tree_common(d_items, n, item_bytes, k, p, s, false, mems, nodes);
  if (rc) return rc;
  pss_summary* sm = new_summary(k, PSS_KIND_SPACE_SAVING, item_bytes, mems.back(), s);
  if (!sm) {
    cudaFreeAsync(mems.back(), s);
    return PSS_ENOMEM;
  }
  *out = sm;
  return PSS_OK;
}

int pss_frequent_summarize(const void* d_items, uint64_t n, int item_bytes, uint32_t k,
                           uint32_t p, void* stream, pss_summary** out) {
  if (!out) return PSS_EINVAL;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<void*> mems;
  std::vector<uint32_t> nodes;
  int rc = frequent_tree_common(d_items, n, item_bytes, k, p, s, false, mems, nodes);
  if (rc) return rc;
  pss_summary* sm = new_summary(k, PSS_KIND_FREQUENT, item_bytes, mems.back(), s);
  if (!sm) {
    cudaFreeAsync(mems.back(), s);
    return PSS_ENOMEM;
  }
  *out = sm;
  return PSS_OK;
}

int pss_set_host_direct(int on) { return g_host_direct.exchange(on ? 1 : 0); }

int pss_summarize_host(const void* h_items, uint64_t n, int item_bytes, uint32_t k, uint32_t p,
                       void* stream, pss_summary** out) {
  if (!out) return PSS_EINVAL;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = prepare_device();
  if (e != cudaSuccess) return from_cuda(e);
  int rc = validate_summarize(h_items, n, item_bytes, k, p);
  if (rc) return rc;
  std::vector<void*> mems;
  std::vector<uint32_t> nodes;
  // mapped pinned memory: the kernels read the items in place, each block's
  // windows copied into shared memory one window ahead as for device input
  const void* mapped = mapped_host(h_items, n);
  if (mapped)
    rc = item_bytes == 4 ? run_tree_device<uint32_t>(mapped, n, k, p, s, false, mems, nodes)
                         : run_tree_device<u64>(mapped, n, k, p, s, false, mems, nodes);
  else
    rc = item_bytes == 4 ? run_tree_host<uint32_t>(h_items, n, k, p, s, mems, nodes)
                         : run_tree_host<u64>(h_items, n, k, p, s, mems, nodes);
  if (rc) return rc;
  pss_summary* sm = new_summary(k, PSS_KIND_SPACE_SAVING, item_bytes, mems.back(), s);
  if (!sm) {
    cudaFreeAsync(mems.back(), s);
    return PSS_ENOMEM;
  }
  *out = sm;
  return PSS_OK;
}

int pss_frequent_summarize_host(const void* h_items, uint64_t n, int item_bytes, uint32_t k,
                                uint32_t p, void* stream, pss_summary** out) {
  if (!out) return PSS_EINVAL;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = prepare_device();
  if (e != cudaSuccess) return from_cuda(e);
  int rc = validate_frequent(h_items, n, item_bytes, k, p);
  if (rc) return rc;
  std::vector<void*> mems;
  std::vector<uint32_t> nodes;
  const void* mapped = mapped_host(h_items, n);
  if (mapped)
    rc = item_bytes == 4 ? run_frequent_tree_device<uint32_t>(mapped, n, k, p, s, false, mems, nodes)
                         : run_frequent_tree_device<u64>(mapped, n, k, p, s, false, mems, nodes);
  else
    rc = item_bytes == 4 ? run_tree_host<uint32_t>(h_items, n, k - 1, p, s, mems, nodes, true)
                         : run_tree_host<u64>(h_items, n, k - 1, p, s, mems, nodes, true);
  if (rc) return rc;
  pss_summary* sm = new_summary(k, PSS_KIND_FREQUENT, item_bytes, mems.back(), s);
  if (!sm) {
    cudaFreeAsync(mems.back(), s);
    return PSS_ENOMEM;
  }
  *out = sm;
  return PSS_OK;
}

int pss_summarize_tree(const void* d_items, uint64_t n, int item_bytes, uint32_t k, uint32_t p,
                       void* stream, pss_tree** out) {
  if (!out) return PSS_EINVAL;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  pss_tree* t = new (std::nothrow) pss_tree;
  if (!t) return PSS_ENOMEM;
  int rc = tree_common(d_items, n, item_bytes, k, p, s, true, t->mem, t->nodes);
  if (rc) {
    delete t;
    return rc;
  }
  t->k = k;
  t->cap = k;
  t->kind = PSS_KIND_SPACE_SAVING;
  t->p = p;
  t->item_bytes = item_bytes;
  t->stream = s;
  *out = t;
  return PSS_OK;
}

int pss_frequent_summarize_tree(const void* d_items, uint64_t n, int item_bytes, uint32_t k,
                                uint32_t p, void* stream, pss_tree** out) {
  if (!out) return PSS_EINVAL;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  pss_tree* t = new (std::nothrow) pss_tree;
  if (!t) return PSS_ENOMEM;
  int rc = frequent_tree_common(d_items, n, item_bytes, k, p, s, true, t->mem, t->nodes);
  if (rc) {
    delete t;
    return rc;
  }
  t->k = k;
  t->cap = k - 1;
  t->kind = PSS_KIND_FREQUENT;
  t->p = p;
  t->item_bytes = item_bytes;
  t->stream = s;
  *out = t;
  return PSS_OK;
}

int pss_tree_levels(const pss_tree* tree, uint32_t* levels) {
  if (!tree || !levels) return PSS_EINVAL;
  *levels = (uint32_t)tree->nodes.size();
  return PSS_OK;
}

int pss_tree_level_nodes(const pss_tree* tree, uint32_t level, uint32_t* nodes) {
  if (!tree || !nodes || level >= tree->nodes.size()) return PSS_EINVAL;
  *nodes = tree->nodes[level];
  return PSS_OK;
}

int pss_tree_read_level(const pss_tree* tree, uint32_t level, uint64_t* items, uint64_t* counts,
                        uint64_t* errs, uint32_t* sizes, uint64_t* m, uint64_t* n_covered,
                        void* stream) {
  if (!tree || level >= tree->nodes.size()) return PSS_EINVAL;
  if (!items || !counts || !errs || !sizes || !m || !n_covered) return PSS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t nodes = tree->nodes[level], k = tree->cap;
  const int w = tree->item_bytes;
  const SetLayout L = set_layout(nodes, k, w);
  const char* base = (const char*)tree->mem[level];
  const size_t e = (size_t)nodes * k;
  std::vector<uint32_t> narrow;
  uint32_t status = 0;
  cudaError_t ce;
  if (w == 4) {
    narrow.resize(e);
    ce = cudaMemcpyAsync(narrow.data(), base + L.item, e * 4, cudaMemcpyDeviceToHost, s);
  } else {
    ce = cudaMemcpyAsync(items, base + L.item, e * 8, cudaMemcpyDeviceToHost, s);
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(counts, base + L.count, e * 8, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(errs, base + L.err, e * 8, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(sizes, base + L.size, (size_t)nodes * 4, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(m, base + L.m, (size_t)nodes * 8, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(n_covered, base + L.ncov, (size_t)nodes * 8, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&status, base + L.status, 4, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return from_cuda(ce);
  if (w == 4)
    for (size_t i = 0; i < e; ++i) items[i] = narrow[i];
  return status ? PSS_EDEVICE : PSS_OK;
}

int pss_tree_root(const pss_tree* tree, void* stream, pss_summary** out) {
  if (!tree || !out) return PSS_EINVAL;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  const int w = tree->item_bytes;
  const SetLayout L = set_layout(1, tree->cap, w);
  void* mem = nullptr;
  cudaError_t e = cudaMallocAsync(&mem, L.total, s);
  if (e != cudaSuccess) return from_cuda(e);
  e = cudaMemcpyAsync(mem, tree->mem.back(), L.total, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(mem, s);
    return from_cuda(e);
  }
  pss_summary* sm = new_summary(tree->k, tree->kind, w, mem, s);
  if (!sm) {
    cudaFreeAsync(mem, s);
    return PSS_ENOMEM;
  }
  *out = sm;
  return PSS_OK;
}

int pss_tree_kind(const pss_tree* tree, int* kind) {
  if (!tree || !kind) return PSS_EINVAL;
  *kind = tree->kind;
  return PSS_OK;
}

void pss_tree_free(pss_tree* tree) {
  if (!tree) return;
  for (void* m : tree->mem)
    if (m) cudaFreeAsync(m, tree->stream);
  delete tree;
}

int pss_merge(const pss_summary* a, const pss_summary* b, void* stream, pss_summary** out) {
  if (!a || !b || !out) return PSS_EINVAL;
  *out = nullptr;
  if (a->k != b->k || a->item_bytes != b->item_bytes || a->kind != b->kind) return PSS_EMISMATCH;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = prepare_device();
  if (e != cudaSuccess) return from_cuda(e);
  const uint32_t k = a->cap;
  const bool mg = a->kind == PSS_KIND_FREQUENT;
  const int w = a->item_bytes;
  void* mem = nullptr;
  e = alloc_set(1, k, w, s, &mem);
  if (e != cudaSuccess) return from_cuda(e);
  ProfScope prof(PROF_MERGE, s, 1);
  count_launches(1);
  if (w == 4)
    e = launch_merge_pair<uint32_t>(set_view<uint32_t>(a->mem, 1, k), 0,
                                    set_view<uint32_t>(b->mem, 1, k), 0,
                                    set_view<uint32_t>(mem, 1, k), s, mg);
  else
    e = launch_merge_pair<u64>(set_view<u64>(a->mem, 1, k), 0, set_view<u64>(b->mem, 1, k), 0,
                               set_view<u64>(mem, 1, k), s, mg);
  if (e != cudaSuccess) {
    cudaFreeAsync(mem, s);
    return from_cuda(e);
  }
  pss_summary* sm = new_summary(a->k, a->kind, w, mem, s);
  if (!sm) {
    cudaFreeAsync(mem, s);
    return PSS_ENOMEM;
  }
  *out = sm;
  return PSS_OK;
}

int pss_query(const pss_summary* summary, uint64_t n, uint32_t k, pss_entry* host_out, uint32_t cap,
              uint32_t* n_out, void* stream) {
  if (!summary || !n_out || k < 2) return PSS_EINVAL;
  if (cap > 0 && !host_out) return PSS_EINVAL;
  const int filter = summary->kind == PSS_KIND_FREQUENT ? 3 : 1;
  return canon_out(summary->mem, 1, 0, summary->cap, summary->item_bytes, n, k, filter, host_out,
                   cap, n_out, (cudaStream_t)stream);
}

namespace {

int import_kind(const pss_entry* entries, uint32_t size, uint64_t m, uint64_t n_covered,
                uint32_t k, int item_bytes, void* stream, pss_summary** out, int kind) {
  if (!out) return PSS_EINVAL;
  *out = nullptr;
  int rc = check_k_width(k, item_bytes);
  if (rc) return rc;
  const bool mg = kind == PSS_KIND_FREQUENT;
  if (mg && k > PSS_MAX_K_RESIDENT) return PSS_EINVAL;
  std::vector<char> image;
  // a Frequent summary stores minimum 0 (its export reports delta in m)
  if ((rc = pss::summary_image(entries, size, mg ? 0 : m, n_covered, mg ? k - 1 : k, item_bytes,
                               image)))
    return rc;
  cudaError_t e = prepare_device();
  if (e != cudaSuccess) return from_cuda(e);
  cudaStream_t s = (cudaStream_t)stream;
  void* mem = nullptr;
  e = cudaMallocAsync(&mem, image.size(), s);
  if (e != cudaSuccess) return from_cuda(e);
  // pageable source: the call returns once the bytes are staged
  e = cudaMemcpyAsync(mem, image.data(), image.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFreeAsync(mem, s);
    return from_cuda(e);
  }
  pss_summary* sm = new_summary(k, kind, item_bytes, mem, s);
  if (!sm) {
    cudaFreeAsync(mem, s);
    return PSS_ENOMEM;
  }
  *out = sm;
  return PSS_OK;
}

}  // namespace

int pss_import(const pss_entry* entries, uint32_t size, uint64_t m, uint64_t n_covered, uint32_t k,
               int item_bytes, void* stream, pss_summary** out) {
  return import_kind(entries, size, m, n_covered, k, item_bytes, stream, out,
                     PSS_KIND_SPACE_SAVING);
}

int pss_frequent_import(const pss_entry* entries, uint32_t size, uint64_t n_covered, uint32_t k,
                        int item_bytes, void* stream, pss_summary** out) {
  return import_kind(entries, size, 0, n_covered, k, item_bytes, stream, out, PSS_KIND_FREQUENT);
}

int pss_query_mode(const pss_summary* summary, uint64_t n, uint32_t k, int mode, pss_entry* host_out,
                   uint32_t cap, uint32_t* n_out, void* stream) {
  if (mode != PSS_QUERY_CANDIDATES && mode != PSS_QUERY_GUARANTEED) return PSS_EINVAL;
  if (!summary || !n_out || k < 2) return PSS_EINVAL;
  if (cap > 0 && !host_out) return PSS_EINVAL;
  const bool g = mode == PSS_QUERY_GUARANTEED;
  const int filter = summary->kind == PSS_KIND_FREQUENT ? (g ? 4 : 3) : (g ? 2 : 1);
  return canon_out(summary->mem, 1, 0, summary->cap, summary->item_bytes, n, k, filter, host_out,
                   cap, n_out, (cudaStream_t)stream);
}

int pss_exact_counts(const void* d_items, uint64_t n, int item_bytes, int log2u, uint32_t* d_counts,
                     void* stream) {
  if ((item_bytes != 4 && item_bytes != 8) || log2u < 1 || log2u > 32 || !d_counts) return PSS_EINVAL;
  if (n > 0 && !d_items) return PSS_EINVAL;
  cudaError_t e = prepare_device();
  if (e != cudaSuccess) return from_cuda(e);
  return from_cuda(pss::launch_exact_counts(d_items, n, item_bytes, log2u, d_counts,
                                            (cudaStream_t)stream));
}

int pss_accuracy_of(const pss_summary* summary, const uint32_t* d_counts, int log2u, uint64_t n,
                    uint32_t k, pss_accuracy* out, void* stream) {
  if (!summary || !d_counts || !out || k < 2 || log2u < 1 || log2u > 32) return PSS_EINVAL;
  const bool mg = summary->kind == PSS_KIND_FREQUENT;
  cudaStream_t s = (cudaStream_t)stream;
  void* dmem = nullptr;
  cudaError_t e = cudaMallocAsync(&dmem, sizeof(pss::AccOut), s);
  if (e != cudaSuccess) return from_cuda(e);
  pss::AccOut* d = (pss::AccOut*)dmem;
  e = summary->item_bytes == 4
          ? pss::launch_accuracy<uint32_t>(set_view<uint32_t>(summary->mem, 1, summary->cap), d_counts,
                                           log2u, n, k, d, s, mg)
          : pss::launch_accuracy<u64>(set_view<u64>(summary->mem, 1, summary->cap), d_counts, log2u, n,
                                      k, d, s, mg);
  pss::AccOut h{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(dmem, s);
  if (e != cudaSuccess) return from_cuda(e);
  out->reported = h.reported;
  out->true_frequent = h.true_frequent;
  out->true_positive = h.true_positive;
  out->guaranteed = h.guaranteed;
  out->outside = h.outside;
  out->are = h.reported ? h.are_sum / (double)h.reported : 0.0;
  out->precision = h.reported ? (double)h.true_positive / (double)h.reported : 1.0;
  out->recall = h.true_frequent ? (double)h.true_positive / (double)h.true_frequent : 1.0;
  return PSS_OK;
}

int pss_export(const pss_summary* summary, pss_entry* host_out, uint32_t cap, uint32_t* size,
               uint64_t* m, uint64_t* n_covered, void* stream) {
  if (!summary || !size) return PSS_EINVAL;
  if (cap > 0 && !host_out) return PSS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = canon_out(summary->mem, 1, 0, summary->cap, summary->item_bytes, 0, 1, 0, host_out, cap,
                     size, s);
  if (rc) return rc;
  const SetLayout L = set_layout(1, summary->cap, summary->item_bytes);
  uint64_t hm = 0, hc = 0;
  cudaError_t e = cudaMemcpyAsync(&hm, (char*)summary->mem + L.m, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, (char*)summary->mem + L.ncov, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  if (summary->kind == PSS_KIND_FREQUENT) {
    // delta = floor((n_covered - sum of counts) / k): the bound on every count
    uint64_t total = 0;
    for (uint32_t i = 0; i < *size; ++i) total += host_out[i].count;
    hm = (hc - total) / summary->k;
  }
  if (m) *m = hm;
  if (n_covered) *n_covered = hc;
  return PSS_OK;
}

int pss_summary_info(const pss_summary* summary, uint32_t* k, int* item_bytes) {
  if (!summary) return PSS_EINVAL;
  if (k) *k = summary->k;
  if (item_bytes) *item_bytes = summary->item_bytes;
  return PSS_OK;
}

int pss_summary_kind(const pss_summary* summary, int* kind) {
  if (!summary || !kind) return PSS_EINVAL;
  *kind = summary->kind;
  return PSS_OK;
}

void pss_free(pss_summary* summary) {
  if (!summary) return;
  if (summary->mem) cudaFreeAsync(summary->mem, summary->stream);
  delete summary;
}

int pss_gen_zipf(void* d_out, uint64_t count, int item_bytes, uint64_t seed, uint32_t stream_id,
                 uint64_t start, double s, int log2u, void* stream) {
  if (item_bytes != 4 && item_bytes != 8) return PSS_EINVAL;
  if (count > 0 && !d_out) return PSS_EINVAL;
  if (log2u < 1 || log2u > 63 || (item_bytes == 4 && log2u > 32)) return PSS_EINVAL;
  if (!(s > 0.0) || s > 64.0) return PSS_EINVAL;
  if (count > 0) count_launches(1);
  return from_cuda(launch_gen_zipf(d_out, count, item_bytes, seed, stream_id, start, s, log2u,
                                   (cudaStream_t)stream));
}

}  // extern "C"
