// serve.cu — request loop with continuous batching over resident tenant
// summaries.  Each request is a segment of one tenant's stream: its summary is
// built (Section 3 per block, Algorithm 2 tree), merged into the tenant's
// resident summary with combine (Algorithm 2) in arrival order, and both the
// segment and the tenant are queried (Algorithm 1, Pruned).
//
// Threads and streams:
//   * the caller submits requests with scheduled arrival times; a scheduler
//     thread releases each at its time (open loop), admits released requests
//     while the device-memory budget, the result slots and the per-tick limit
//     allow, and enqueues one tick per admission round;
//   * a tick's segment generation and summaries go to one of NSEG segment
//     streams (in turn), so consecutive ticks overlap on the device; the
//     tenant merges and queries go, in arrival order, to the tenant's own
//     stream (tenant t on tenant stream t mod NTEN), which waits for the
//     tick's segments -- so every tenant sees its segments in arrival order
//     whatever the mix, and a long segment of one tenant holds up only the
//     tenants that share its tick or its tenant stream;
//   * results land in pinned host slots; the scheduler completes a tick when
//     the events of every stream it used have passed, in whatever order the
//     ticks finish.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "pss_internal.cuh"
#include "pss_kernels.cuh"

using namespace pss;

namespace {

int from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return PSS_OK;
  if (e == cudaErrorMemoryAllocation) return PSS_ENOMEM;
  return PSS_ECUDA;
}

struct Admitted {
  pss_request r;
  double admitted = 0;
  uint32_t p = 0;
  uint32_t slot = 0;
  uint64_t bytes = 0;
  uint64_t tenant_items = 0;
  void* gen = nullptr;   // generated segment items
  void* root = nullptr;  // segment summary
  int status = PSS_OK;
};

struct Tick {
  std::vector<Admitted> reqs;
  pss_batch* batch = nullptr;     // the tick's segment summaries
  std::vector<cudaEvent_t> done;  // one per stream the tick used
};

constexpr int NSEG = 4;   // segment streams, taken in turn by the ticks
constexpr int NTEN = 8;   // tenant streams (tenant t on t mod NTEN)

struct Result {
  std::vector<pss_entry> seg, ten;
};

}  // namespace

struct pss_server {
  pss_server_config cfg{};
  int kind = PSS_KIND_SPACE_SAVING;  // of every summary the server keeps
  uint32_t cap = 0;                  // entries per summary: k, or k - 1 (Frequent)
  int dev = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::vector<pss_request> pending;  // submitted, not yet released (sorted by arrival)
  size_t pending_head = 0;
  bool pending_sorted = true;
  std::deque<pss_request> ready;     // released, not yet admitted
  std::deque<Tick> inflight;
  std::vector<pss_completion> completions;
  std::unordered_map<uint64_t, Result> results;
  std::unordered_set<uint64_t> live;     // ids submitted and not yet read (or failed)
  std::atomic<uint32_t> fail_allocs{0};  // injected segment allocation failures to come
  uint64_t submitted = 0, completed = 0;
  // device state
  std::vector<void*> tenant_mem[2];
  std::vector<int> tenant_cur;
  std::vector<uint64_t> tenant_items;
  cudaStream_t seg_stream[NSEG] = {};
  cudaStream_t tenant_stream[NTEN] = {};
  cudaStream_t plan_stream = nullptr;  // batch set-up, independent of segment work
  pss_entry* d_q = nullptr;    // per slot: 2 k entries
  uint32_t* d_qn = nullptr;    // per slot: 4 words
  pss_entry* h_q = nullptr;    // pinned mirror
  uint32_t* h_qn = nullptr;
  std::vector<uint32_t> free_slots;
  uint64_t inflight_bytes = 0;
  uint64_t ticks = 0;
  std::thread th;
  std::atomic<bool> stop{false};
  bool started = false;
  std::chrono::steady_clock::time_point t0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

uint64_t request_bytes(const pss_request& r, uint32_t cap, uint32_t p) {
  const uint64_t items = r.d_items ? 0 : r.n * 4;
  // block summaries and one tree level, plus the root (set_layout sizes)
  return items + set_layout(p, cap, 4).total + set_layout((p + 1) / 2, cap, 4).total +
         set_layout(1, cap, 4).total;
}

// Enqueue one tick (called by the scheduler thread without the lock held):
// generate the segments, summarize all of them as one batch (one persistent
// launch over every block of the tick), then, in arrival order on the tenant
// stream, merge each into its tenant and query the tenant.
void launch_tick(pss_server* sv, Tick& t) {
  const uint32_t k = sv->cfg.k, cap = sv->cap;
  const bool mg = sv->kind == PSS_KIND_FREQUENT;
  cudaStream_t seg = sv->seg_stream[sv->ticks % NSEG];
  ++sv->ticks;
  const uint32_t nr = (uint32_t)t.reqs.size();
  std::vector<const void*> items(nr);
  std::vector<uint64_t> ns(nr);
  std::vector<uint32_t> ks(nr, k), ps(nr);
  std::vector<uint32_t> bidx(nr, ~0u);  // request -> its stream in the tick's batch
  uint32_t nb = 0;
  for (uint32_t i = 0; i < nr; ++i) {
    Admitted& a = t.reqs[i];
    const void* src = a.r.d_items;
    if (!src && a.r.n) {
      cudaError_t e = cudaSuccess;
      uint32_t f = sv->fail_allocs.load();
      while (f && !sv->fail_allocs.compare_exchange_weak(f, f - 1)) {
      }
      if (f) e = cudaErrorMemoryAllocation;  // injected fault
      if (e == cudaSuccess) e = cudaMallocAsync(&a.gen, a.r.n * 4, seg);
      if (e == cudaSuccess)
        e = launch_gen_zipf(a.gen, a.r.n, 4, a.r.seed, a.r.stream_id, 0, a.r.s, a.r.log2u, seg);
      if (e == cudaSuccess) count_launches(1);
      if (e != cudaSuccess) a.status = from_cuda(e);
      src = a.gen;
    }
    if (a.status != PSS_OK) continue;  // a failed request leaves its tenant untouched
    bidx[i] = nb++;
    items[bidx[i]] = src;
    ns[bidx[i]] = a.r.n;
    ps[bidx[i]] = a.p;
  }
  int rc = PSS_OK;
  if (nb) {
    pss_batch_desc desc{nb, 4, items.data(), ns.data(), ks.data(), ps.data(), nullptr};
    rc = mg ? pss_frequent_batch_create(&desc, sv->plan_stream, &t.batch)
            : pss_batch_create(&desc, sv->plan_stream, &t.batch);
    if (rc == PSS_OK) rc = pss_batch_run(t.batch, 0, seg);
  }
  if (rc != PSS_OK) {
    for (Admitted& a : t.reqs)
      if (a.status == PSS_OK) a.status = rc;
  }
  // the generated items are read by the batch only (on seg)
  for (Admitted& a : t.reqs)
    if (a.gen) cudaFreeAsync(a.gen, seg);
  cudaEvent_t segs_done;
  cudaEventCreateWithFlags(&segs_done, cudaEventDisableTiming);
  cudaEventRecord(segs_done, seg);
  bool used[NTEN] = {};
  for (uint32_t i = 0; i < nr; ++i) {
    Admitted& a = t.reqs[i];
    if (a.status != PSS_OK) continue;
    const uint32_t T = a.r.tenant;
    cudaStream_t ts = sv->tenant_stream[T % NTEN];
    if (!used[T % NTEN]) {
      cudaStreamWaitEvent(ts, segs_done, 0);
      used[T % NTEN] = true;
    }
    const int cur = sv->tenant_cur[T];
    void* in = sv->tenant_mem[cur][T];
    void* out = sv->tenant_mem[cur ^ 1][T];
    void* root = batch_root(t.batch, bidx[i]);
    cudaError_t e = launch_merge_pair<uint32_t>(set_view<uint32_t>(in, 1, cap), 0,
                                                set_view<uint32_t>(root, 1, cap), 0,
                                                set_view<uint32_t>(out, 1, cap), ts, mg);
    count_launches(1);
    sv->tenant_cur[T] = cur ^ 1;
    sv->tenant_items[T] += a.r.n;
    a.tenant_items = sv->tenant_items[T];
    pss_entry* q = sv->d_q + (size_t)a.slot * 2 * k;
    uint32_t* qn = sv->d_qn + (size_t)a.slot * 4;
    if (e == cudaSuccess)
      e = launch_canon<uint32_t>(set_view<uint32_t>(out, 1, cap), 0, a.tenant_items, k,
                                 mg ? 3 : 1, q + k, qn + 2, ts);
    count_launches(1);
    pss_entry* sq;
    uint32_t* sqn;
    batch_query_device(t.batch, bidx[i], &sq, &sqn);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sv->h_q + (size_t)a.slot * 2 * k, sq, sizeof(pss_entry) * k,
                          cudaMemcpyDeviceToHost, ts);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sv->h_qn + (size_t)a.slot * 4, sqn, sizeof(uint32_t) * 2,
                          cudaMemcpyDeviceToHost, ts);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sv->h_q + (size_t)a.slot * 2 * k + k, q + k, sizeof(pss_entry) * k,
                          cudaMemcpyDeviceToHost, ts);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sv->h_qn + (size_t)a.slot * 4 + 2, qn + 2, sizeof(uint32_t) * 2,
                          cudaMemcpyDeviceToHost, ts);
    if (e != cudaSuccess) a.status = from_cuda(e);
  }
  cudaEventDestroy(segs_done);
  auto mark = [&](cudaStream_t st) {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return;
    cudaEventRecord(ev, st);
    t.done.push_back(ev);
  };
  mark(seg);
  for (int j = 0; j < NTEN; ++j)
    if (used[j]) mark(sv->tenant_stream[j]);
}

// Complete the ticks whose work has finished, in any order (lock held by
// the caller).
void reap(pss_server* sv) {
  const uint32_t k = sv->cfg.k;
  for (size_t ti = 0; ti < sv->inflight.size();) {
    Tick& t = sv->inflight[ti];
    bool finished = true;
    for (cudaEvent_t ev : t.done)
      if (cudaEventQuery(ev) == cudaErrorNotReady) {
        finished = false;
        break;
      }
    if (!finished) {
      ++ti;
      continue;
    }
    const double done = sv->now();
    for (Admitted& a : t.reqs) {
      pss_completion c{};
      c.id = a.r.id;
      c.tenant = a.r.tenant;
      c.p = a.p;
      c.arrival = a.r.arrival;
      c.admitted = a.admitted;
      c.completed = done;
      c.tenant_items = a.tenant_items;
      c.status = a.status;
      if (a.status == PSS_OK) {
        const uint32_t* qn = sv->h_qn + (size_t)a.slot * 4;
        const pss_entry* q = sv->h_q + (size_t)a.slot * 2 * k;
        c.n_segment = qn[0];
        c.n_tenant = qn[2];
        if (qn[1] || qn[3]) c.status = PSS_EDEVICE;
        Result res;
        res.seg.assign(q, q + std::min(qn[0], k));
        res.ten.assign(q + k, q + k + std::min(qn[2], k));
        sv->results[a.r.id] = std::move(res);
      } else {
        sv->live.erase(a.r.id);  // nothing to read
      }
      sv->completions.push_back(c);
      sv->free_slots.push_back(a.slot);
      sv->inflight_bytes -= a.bytes;
      ++sv->completed;
    }
    for (cudaEvent_t ev : t.done) cudaEventDestroy(ev);
    if (t.batch) pss_batch_free(t.batch);  // its work has completed
    sv->inflight.erase(sv->inflight.begin() + (std::ptrdiff_t)ti);
    sv->cv.notify_all();
  }
}

void scheduler(pss_server* sv) {
  cudaSetDevice(sv->dev);
  const uint32_t k = sv->cfg.k;
  while (!sv->stop.load()) {
    Tick tick;
    {
      std::unique_lock<std::mutex> lock(sv->mu);
      const double now = sv->now();
      if (!sv->pending_sorted) {
        std::stable_sort(sv->pending.begin() + sv->pending_head, sv->pending.end(),
                         [](const pss_request& a, const pss_request& b) { return a.arrival < b.arrival; });
        sv->pending_sorted = true;
      }
      while (sv->pending_head < sv->pending.size() && sv->pending[sv->pending_head].arrival <= now)
        sv->ready.push_back(sv->pending[sv->pending_head++]);
      reap(sv);
      while (!sv->ready.empty() && tick.reqs.size() < sv->cfg.max_batch && !sv->free_slots.empty()) {
        const pss_request& r = sv->ready.front();
        const uint32_t p = r.p ? r.p
                               : (sv->kind == PSS_KIND_FREQUENT ? pss_frequent_plan_blocks(r.n, k, 4, r.s)
                                                                : pss_plan_blocks(r.n, k, 4, r.s));
        const uint64_t bytes = request_bytes(r, sv->cap, p);
        // admit while the budget allows; a request larger than the whole
        // budget runs alone
        if (sv->inflight_bytes + bytes > sv->cfg.budget_bytes &&
            !(sv->inflight_bytes == 0 && tick.reqs.empty()))
          break;
        Admitted a;
        a.r = r;
        a.p = p;
        a.bytes = bytes;
        a.admitted = now;
        a.slot = sv->free_slots.back();
        sv->free_slots.pop_back();
        sv->inflight_bytes += bytes;
        tick.reqs.push_back(a);
        sv->ready.pop_front();
      }
      if (tick.reqs.empty()) {
        // nothing to admit: wait for an arrival, a completion or a stop
        double wait = 5e-5;
        if (sv->pending_head < sv->pending.size() && sv->inflight.empty())
          wait = std::min(wait, std::max(0.0, sv->pending[sv->pending_head].arrival - now));
        if (sv->inflight.empty() && sv->ready.empty() && sv->pending_head >= sv->pending.size()) {
          sv->cv.notify_all();
          sv->cv.wait_for(lock, std::chrono::milliseconds(1));
        } else if (wait > 0) {
          lock.unlock();
          std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 5e-5)));
        }
        continue;
      }
    }
    launch_tick(sv, tick);
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      sv->inflight.push_back(std::move(tick));
    }
  }
}

void destroy(pss_server* sv) {
  if (!sv) return;
  if (sv->th.joinable()) {
    sv->stop.store(true);
    sv->cv.notify_all();
    sv->th.join();
  }
  cudaSetDevice(sv->dev);
  for (auto st : sv->tenant_stream)
    if (st) cudaStreamSynchronize(st);
  for (auto st : sv->seg_stream)
    if (st) cudaStreamSynchronize(st);
  for (auto& t : sv->inflight)
    for (cudaEvent_t ev : t.done) cudaEventDestroy(ev);
  for (int b = 0; b < 2; ++b)
    for (void* m : sv->tenant_mem[b])
      if (m) cudaFree(m);
  if (sv->d_q) cudaFree(sv->d_q);
  if (sv->d_qn) cudaFree(sv->d_qn);
  if (sv->h_q) cudaFreeHost(sv->h_q);
  if (sv->h_qn) cudaFreeHost(sv->h_qn);
  for (auto& t : sv->inflight)
    if (t.batch) pss_batch_free(t.batch);
  for (auto st : sv->tenant_stream)
    if (st) cudaStreamDestroy(st);
  if (sv->plan_stream) {
    cudaStreamSynchronize(sv->plan_stream);
    cudaStreamDestroy(sv->plan_stream);
  }
  for (auto st : sv->seg_stream)
    if (st) cudaStreamDestroy(st);
  delete sv;
}

}  // namespace

namespace {

int server_create(const pss_server_config* cfg, pss_server** out, int kind) {
  if (!cfg || !out) return PSS_EINVAL;
  *out = nullptr;
  if (cfg->tenants == 0 || cfg->k < 2 || cfg->k > PSS_MAX_K_RESIDENT || cfg->max_batch == 0 ||
      cfg->max_inflight == 0)
    return PSS_EINVAL;
  pss_server* sv = new (std::nothrow) pss_server;
  if (!sv) return PSS_ENOMEM;
  sv->cfg = *cfg;
  sv->kind = kind;
  sv->cap = kind == PSS_KIND_FREQUENT ? cfg->k - 1 : cfg->k;
  cudaError_t e = cudaGetDevice(&sv->dev);
  const uint32_t k = cfg->k, T = cfg->tenants;
  const SetLayout L = set_layout(1, sv->cap, 4);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    sv->tenant_mem[b].assign(T, nullptr);
    for (uint32_t t = 0; t < T && e == cudaSuccess; ++t) {
      e = cudaMalloc(&sv->tenant_mem[b][t], L.total);
      if (e == cudaSuccess) e = cudaMemset(sv->tenant_mem[b][t], 0, L.total);  // empty summary
    }
  }
  sv->tenant_cur.assign(T, 0);
  sv->tenant_items.assign(T, 0);
  const size_t slots = cfg->max_inflight;
  if (e == cudaSuccess) e = cudaMalloc(&sv->d_q, sizeof(pss_entry) * 2 * k * slots);
  if (e == cudaSuccess) e = cudaMalloc(&sv->d_qn, sizeof(uint32_t) * 4 * slots);
  if (e == cudaSuccess) e = cudaHostAlloc(&sv->h_q, sizeof(pss_entry) * 2 * k * slots, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc(&sv->h_qn, sizeof(uint32_t) * 4 * slots, cudaHostAllocDefault);
  for (int i = 0; i < NSEG && e == cudaSuccess; ++i)
    e = cudaStreamCreateWithFlags(&sv->seg_stream[i], cudaStreamNonBlocking);
  for (int i = 0; i < NTEN && e == cudaSuccess; ++i)
    e = cudaStreamCreateWithFlags(&sv->tenant_stream[i], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->plan_stream, cudaStreamNonBlocking);
  for (uint32_t i = 0; i < slots; ++i) sv->free_slots.push_back((uint32_t)(slots - 1 - i));
  if (e != cudaSuccess) {
    destroy(sv);
    return from_cuda(e);
  }
  *out = sv;
  return PSS_OK;
}

}  // namespace

extern "C" int pss_server_create(const pss_server_config* cfg, pss_server** out) {
  return server_create(cfg, out, PSS_KIND_SPACE_SAVING);
}

extern "C" int pss_frequent_server_create(const pss_server_config* cfg, pss_server** out) {
  return server_create(cfg, out, PSS_KIND_FREQUENT);
}

extern "C" int pss_server_submit(pss_server* sv, const pss_request* reqs, uint32_t count) {
  if (!sv || (count && !reqs)) return PSS_EINVAL;
  for (uint32_t i = 0; i < count; ++i) {
    const pss_request& r = reqs[i];
    if (r.tenant >= sv->cfg.tenants) return PSS_EINVAL;
    if (!r.d_items && r.n && (r.log2u < 1 || r.log2u > 32 || !(r.s > 0.0))) return PSS_EINVAL;
    if (r.p && (r.n + r.p - 1) / r.p >= (1ull << 32)) return PSS_EINVAL;
  }
  std::lock_guard<std::mutex> lock(sv->mu);
  // ids must be unique among the requests not yet read back
  std::unordered_set<uint64_t> mine;
  for (uint32_t i = 0; i < count; ++i)
    if (sv->live.count(reqs[i].id) || !mine.insert(reqs[i].id).second) return PSS_EINVAL;
  for (uint32_t i = 0; i < count; ++i) {
    sv->pending.push_back(reqs[i]);
    sv->live.insert(reqs[i].id);
  }
  sv->pending_sorted = false;
  sv->submitted += count;
  sv->cv.notify_all();
  return PSS_OK;
}

extern "C" int pss_server_start(pss_server* sv) {
  if (!sv) return PSS_EINVAL;
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->started) return PSS_OK;
  sv->t0 = std::chrono::steady_clock::now();
  sv->started = true;
  sv->th = std::thread(scheduler, sv);
  return PSS_OK;
}

extern "C" int pss_server_wait(pss_server* sv, double timeout_s) {
  if (!sv) return PSS_EINVAL;
  std::unique_lock<std::mutex> lock(sv->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (sv->completed < sv->submitted) {
    if (sv->cv.wait_until(lock, deadline) == std::cv_status::timeout &&
        sv->completed < sv->submitted)
      return PSS_ETIMEOUT;
  }
  return PSS_OK;
}

extern "C" int pss_server_poll(pss_server* sv, pss_completion* out, uint32_t cap, uint32_t* n_out) {
  if (!sv || !n_out || (cap && !out)) return PSS_EINVAL;
  std::lock_guard<std::mutex> lock(sv->mu);
  const uint32_t n = (uint32_t)std::min<size_t>(cap, sv->completions.size());
  std::copy(sv->completions.begin(), sv->completions.begin() + n, out);
  sv->completions.erase(sv->completions.begin(), sv->completions.begin() + n);
  *n_out = n;
  return PSS_OK;
}

extern "C" int pss_server_result(pss_server* sv, uint64_t id, pss_entry* seg_out, uint32_t* n_seg,
                                 pss_entry* ten_out, uint32_t* n_ten) {
  if (!sv || !seg_out || !n_seg || !ten_out || !n_ten) return PSS_EINVAL;
  std::lock_guard<std::mutex> lock(sv->mu);
  auto it = sv->results.find(id);
  if (it == sv->results.end()) return PSS_EINVAL;
  std::copy(it->second.seg.begin(), it->second.seg.end(), seg_out);
  std::copy(it->second.ten.begin(), it->second.ten.end(), ten_out);
  *n_seg = (uint32_t)it->second.seg.size();
  *n_ten = (uint32_t)it->second.ten.size();
  sv->results.erase(it);
  sv->live.erase(id);
  return PSS_OK;
}

extern "C" int pss_server_inject_alloc_failures(pss_server* sv, uint32_t count) {
  if (!sv) return PSS_EINVAL;
  sv->fail_allocs.store(count);
  return PSS_OK;
}

extern "C" int pss_server_tenant_import(pss_server* sv, uint32_t tenant, const pss_entry* entries,
                                        uint32_t size, uint64_t m, uint64_t n_covered) {
  if (!sv || tenant >= sv->cfg.tenants) return PSS_EINVAL;
  std::vector<char> image;
  // a Frequent summary stores minimum 0 (export reports delta in m instead)
  const bool mg = sv->kind == PSS_KIND_FREQUENT;
  int rc = summary_image(entries, size, mg ? 0 : m, n_covered, sv->cap, 4, image);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->started) return PSS_EINVAL;
  cudaError_t e = cudaMemcpy(sv->tenant_mem[sv->tenant_cur[tenant]][tenant], image.data(),
                             image.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return from_cuda(e);
  sv->tenant_items[tenant] = n_covered;
  return PSS_OK;
}

extern "C" int pss_server_tenant_export(pss_server* sv, uint32_t tenant, pss_entry* host_out,
                                        uint32_t cap, uint32_t* size, uint64_t* m,
                                        uint64_t* n_covered) {
  if (!sv || tenant >= sv->cfg.tenants || !size) return PSS_EINVAL;
  void* mem;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    mem = sv->tenant_mem[sv->tenant_cur[tenant]][tenant];
  }
  const uint32_t k = sv->cap;
  pss_entry* d_out = nullptr;
  cudaError_t e = cudaMalloc(&d_out, sizeof(pss_entry) * k + 16);
  if (e != cudaSuccess) return from_cuda(e);
  uint32_t* d_n = (uint32_t*)((char*)d_out + sizeof(pss_entry) * k);
  cudaStream_t ts = sv->tenant_stream[tenant % NTEN];
  const SetLayout L = set_layout(1, k, 4);
  uint32_t hn[2] = {0, 0};
  uint64_t hm = 0, hc = 0;
  e = launch_canon<uint32_t>(set_view<uint32_t>(mem, 1, k), 0, 0, 1, 0, d_out, d_n, ts);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hn, d_n, sizeof(hn), cudaMemcpyDeviceToHost, ts);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hm, (char*)mem + L.m, 8, cudaMemcpyDeviceToHost, ts);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, (char*)mem + L.ncov, 8, cudaMemcpyDeviceToHost, ts);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ts);
  int rc = from_cuda(e);
  if (rc == PSS_OK && hn[1]) rc = PSS_EDEVICE;
  if (rc == PSS_OK && hn[0] > cap) rc = PSS_ERANGE;
  std::vector<pss_entry> ents(hn[0]);
  if (rc == PSS_OK && hn[0])
    rc = from_cuda(cudaMemcpy(ents.data(), d_out, sizeof(pss_entry) * hn[0], cudaMemcpyDeviceToHost));
  if (rc == PSS_OK && hn[0] && host_out) memcpy(host_out, ents.data(), sizeof(pss_entry) * hn[0]);
  cudaFree(d_out);
  if (rc == PSS_OK && sv->kind == PSS_KIND_FREQUENT) {  // m receives delta, as pss_export
    uint64_t total = 0;
    for (const pss_entry& en : ents) total += en.count;
    hm = (hc - total) / sv->cfg.k;
  }
  if (rc == PSS_OK) {
    *size = hn[0];
    if (m) *m = hm;
    if (n_covered) *n_covered = hc;
  }
  return rc;
}

extern "C" void pss_server_destroy(pss_server* sv) { destroy(sv); }
