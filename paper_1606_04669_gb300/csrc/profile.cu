// profile.cu — launch counter and CUDA-event timing of the kernel groups
// (summarize, merge tree, query/export).  The paper's scalability analysis
// separates computation from the reduction overhead (Section 4.1, fractional
// overhead); these timers give the same split on the device.
#include <atomic>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pss_internal.cuh"
#include "pss_kernels.cuh"

namespace pss {

namespace {

struct Pending {
  int cat;
  cudaEvent_t start, end;
};

std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_enabled{0};
std::mutex g_mu;
std::vector<cudaEvent_t> g_pool;
std::vector<Pending> g_pending;
double g_ms[3] = {0, 0, 0};
uint64_t g_calls[3] = {0, 0, 0};

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

}  // namespace

void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

ProfScope::ProfScope(int cat, cudaStream_t s, uint64_t units) : cat_(cat), s_(s), units_(units) {
  // a host range per kernel group for timeline tools (no cost without one)
  static const char* const names[3] = {"pss summarize", "pss merge tree", "pss query"};
  nvtxRangePushA(names[cat_ >= 0 && cat_ < 3 ? cat_ : 0]);
  if (!g_enabled.load(std::memory_order_relaxed)) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  std::lock_guard<std::mutex> lock(g_mu);
  start_ = get_event();
  end_ = get_event();
  if (start_ && end_) {
    cudaEventRecord(start_, s_);
    active_ = true;
  }
}

ProfScope::~ProfScope() {
  nvtxRangePop();
  if (!active_) return;
  std::lock_guard<std::mutex> lock(g_mu);
  cudaEventRecord(end_, s_);
  g_pending.push_back(Pending{cat_, start_, end_});
  g_calls[cat_] += units_;
}

}  // namespace pss

extern "C" int pss_profile_enable(int on) {
  pss::g_enabled.store(on ? 1 : 0);
  return PSS_OK;
}

extern "C" int pss_profile_read(pss_profile* out, int reset) {
  using namespace pss;
  std::lock_guard<std::mutex> lock(g_mu);
  int rc = PSS_OK;
  for (const Pending& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.end) != cudaSuccess ||
        cudaEventElapsedTime(&ms, p.start, p.end) != cudaSuccess) {
      rc = PSS_ECUDA;
    } else {
      g_ms[p.cat] += ms;
    }
    g_pool.push_back(p.start);
    g_pool.push_back(p.end);
  }
  g_pending.clear();
  if (out) {
    out->launches = g_launches.load();
    out->summarize_calls = g_calls[0];
    out->merge_levels = g_calls[1];
    out->query_calls = g_calls[2];
    out->summarize_ms = g_ms[0];
    out->merge_ms = g_ms[1];
    out->query_ms = g_ms[2];
  }
  if (reset) {
    g_launches.store(0);
    for (int i = 0; i < 3; ++i) {
      g_ms[i] = 0;
      g_calls[i] = 0;
    }
  }
  return rc;
}
