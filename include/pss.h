/*
 * pss.h — C ABI of libpss: Parallel Space Saving on one GB300 (sm_103a).
 *
 * The method is M. Cafaro, M. Pulimeno, I. Epicoco, G. Aloisio, "Parallel
 * Space Saving on Multi and Many-Core Processors" (arXiv:1606.04669):
 *   - the input of n items is split into p blocks with the bounds of
 *     Algorithm 1 (block r is [floor(r n / p), floor((r+1) n / p)));
 *   - each block is reduced to a k-counter Space Saving summary (Section 3);
 *   - the p summaries are merged by the combine operator of Algorithm 2
 *     (union, count addition, the other summary's minimum added for absent
 *     items, Prune(k)) in a binary reduction tree (Algorithm 1,
 *     ParallelReduction);
 *   - the query reports the k-majority candidates: entries whose count
 *     exceeds n / k (Algorithm 1, Pruned; threshold of Section 3).
 *
 * Conventions shared by every call:
 *   - Items are unsigned integers of item_bytes = 4 or 8 bytes.
 *   - Counts and errors are exact unsigned 64-bit integers.  Every entry
 *     satisfies count - err <= f <= count, f the item's true frequency.
 *   - A summary keeps at most k entries; its minimum m is the smallest count
 *     when k entries are in use and 0 otherwise.  Ties are broken
 *     deterministically: the evicted counter is the least recently updated
 *     among those with the minimum count; Prune(k) keeps the k largest by
 *     (count descending, item ascending).
 *   - Device pointers are plain CUDA device addresses; host pointers are
 *     ordinary (pageable or pinned) host memory.  `stream` is a cudaStream_t
 *     passed as void* (NULL = the legacy default stream).
 *   - Calls that only enqueue GPU work are asynchronous on `stream`; calls
 *     that return data to the host synchronize `stream`.
 *   - Every function returns PSS_OK (0) or a negative PSS_E* code; on error
 *     no output handle is created and nothing is enqueued.
 *   - Summaries and trees are device-resident and owned by the library;
 *     release them with pss_free / pss_tree_free.  Their memory comes from
 *     CUDA's stream-ordered allocator on the stream of the creating call.
 *     An input buffer is borrowed: it must stay valid until the work enqueued
 *     on `stream` has passed it.
 *   - Errors raised inside a kernel (a bounded device loop that ran out)
 *     are recorded in the produced summary and reported as PSS_EDEVICE by
 *     the next call that reads it back (pss_export, pss_query,
 *     pss_tree_read_level).
 */
#ifndef PSS_H_
#define PSS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PSS_OK 0
#define PSS_EINVAL (-1)    /* bad argument: null pointer, k < 2, k > PSS_MAX_K, width not 4/8 ... */
#define PSS_EMISMATCH (-2) /* merging summaries of different k, item width or kind */
#define PSS_ENOMEM (-3)    /* device allocation failed */
#define PSS_ECUDA (-4)     /* a CUDA runtime call failed (launch, copy, sync) */
#define PSS_ETIMEOUT (-5)  /* a bounded device wait expired */
#define PSS_EDEVICE (-6)   /* a kernel recorded an error in the summary */
#define PSS_ERANGE (-7)    /* output capacity too small */

/* Largest k the shared-memory resident summarize kernel supports. */
#define PSS_MAX_K 8192u          /* pss_summarize*, pss_merge, pss_query*, pss_export */
#define PSS_MAX_K_RESIDENT 4096u /* the batch, server and allocation-free forms */

typedef struct pss_summary pss_summary; /* one summary (opaque, device-resident) */
typedef struct pss_tree pss_tree;       /* every level of one reduction tree */

typedef struct {
  uint64_t item;  /* the monitored item */
  uint64_t count; /* estimated frequency f^ (an upper bound on f) */
  uint64_t err;   /* maximum over-estimation: count - err <= f */
} pss_entry;

/* Text of a PSS_E* code (static storage). */
const char* pss_strerror(int code);

/* ABI version of this header (incremented on incompatible changes). */
int pss_abi_version(void);

/*
 * pss_summarize — ParallelSpaceSaving(N, n, p, k) of Algorithm 1 up to the
 * reduction: p block summaries (Section 3 update rule) merged by Algorithm 2
 * in a binary tree over adjacent pairs (an odd last summary is carried up).
 *   d_items     device array of n items of item_bytes each (4 or 8);
 *               may be NULL only when n == 0.
 *   k           counters per summary, 2 <= k <= PSS_MAX_K (the paper's k
 *               sweep reaches 8000); above 4096 part of each block's state
 *               and of each combine's union lives in HBM scratch taken on
 *               the stream for the call.
 *   p           number of blocks, p >= 1; blocks may be empty when n < p;
 *               a block must hold fewer than 2^32 items.
 *   out         receives a new summary (release with pss_free).
 * Asynchronous on stream.
 */
int pss_summarize(const void* d_items, uint64_t n, int item_bytes, uint32_t k, uint32_t p,
                  void* stream, pss_summary** out);

/*
 * pss_summarize_host — pss_summarize for items in HOST memory.  Pinned memory
 * that the device can address (cudaHostAlloc / cudaHostRegister memory is
 * mapped into the unified address space; on a coherent CPU-GPU link such as
 * NVLink-C2C the kernels read it at link bandwidth) is read in place by the
 * summarize kernel.  Other host memory, or every call after
 * pss_set_host_direct(0), is copied to the device in up to 16 slabs on a
 * library-owned copy stream, each slab's block summaries starting as soon as
 * it has landed.  h_items must stay valid until the work enqueued on stream
 * has completed.  Asynchronous on stream.
 */
/* Whether pss_summarize_host reads mapped pinned host memory in place (1,
 * the default) or always stages copies (0).  Results are the same either way.
 * Process-wide; returns the previous value. */
int pss_set_host_direct(int on);

int pss_summarize_host(const void* h_items, uint64_t n, int item_bytes, uint32_t k, uint32_t p,
                       void* stream, pss_summary** out);

/* Size of the fixed device array pss_summarize_noalloc works in (32 MiB). */
#define PSS_NOALLOC_SCRATCH_BYTES (32ull << 20)

/*
 * pss_summarize_noalloc — the computation of pss_summarize for callers that
 * cannot allocate device memory: processes that own all device memory
 * through their own allocator, or that run under a fixed budget and must not
 * allocate once started (a serving process, for instance).  The paper has no
 * counterpart; this is a deployment variant of the same kernels.
 *   - It calls no cudaMalloc, cudaFree or stream-ordered allocation.  The
 *     block summaries and the reduction tree live in one fixed array of
 *     PSS_NOALLOC_SCRATCH_BYTES compiled into the library; every GPU that
 *     loads the library holds that array until the process exits.
 *   - k <= PSS_MAX_K_RESIDENT (larger k need stream-ordered scratch).
 *   - Limit: the p block summaries plus ceil(p/2) merged summaries must fit
 *     in the array (about 1.5 p k (item_bytes + 16) bytes; e.g. p = 8,
 *     k = 2000 fits, p = 4096, k = 2000 does not); otherwise PSS_ERANGE and
 *     nothing is enqueued.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call uses the same array and leaves its contents there: calls
 *     whose work overlaps on the GPU (other streams, other host threads) race
 *     and must be serialized by the caller.
 *   - Outputs, in caller-owned device memory: d_out_items (k items of
 *     item_bytes), d_out_counts and d_out_errs (k values) receive the root
 *     summary sorted by item ascending; d_out_header[4] = {size, m,
 *     n_covered, status}, status != 0 meaning a kernel recorded an error.
 * Arguments otherwise as pss_summarize.  Asynchronous on stream.
 */
int pss_summarize_noalloc(const void* d_items, uint64_t n, int item_bytes, uint32_t k, uint32_t p,
                          void* d_out_items, uint64_t* d_out_counts, uint64_t* d_out_errs,
                          uint64_t* d_out_header, void* stream);

/*
 * pss_summarize_tree — the same computation as pss_summarize, keeping every
 * level of the reduction tree (level 0 = the p block summaries, last level =
 * the root) for inspection with pss_tree_read_level.  Asynchronous.
 */
int pss_summarize_tree(const void* d_items, uint64_t n, int item_bytes, uint32_t k, uint32_t p,
                       void* stream, pss_tree** out);

/* Number of levels of a tree (1 + ceil(log2 p)). */
int pss_tree_levels(const pss_tree* tree, uint32_t* levels);

/* Number of summaries at `level` of a tree. */
int pss_tree_level_nodes(const pss_tree* tree, uint32_t level, uint32_t* nodes);

/*
 * pss_tree_read_level — copy every summary of one tree level to the host,
 * in the device layout: node j's entries are at [j*c, j*c + sizes[j]) of
 * items/counts/errs, sorted by item ascending (items widened to 64 bits);
 * c = k for a Space Saving tree, k - 1 for a Frequent one.  Arrays items,
 * counts, errs hold nodes*c values; sizes, m, n_covered hold nodes values.  Synchronizes stream.  PSS_EDEVICE if a kernel recorded an
 * error in that level.
 */
int pss_tree_read_level(const pss_tree* tree, uint32_t level, uint64_t* items, uint64_t* counts,
                        uint64_t* errs, uint32_t* sizes, uint64_t* m, uint64_t* n_covered,
                        void* stream);

/* A new summary holding a copy of the tree's root (release with pss_free). */
int pss_tree_root(const pss_tree* tree, void* stream, pss_summary** out);

/* Release a tree (stream-ordered on the stream that created it). */
void pss_tree_free(pss_tree* tree);

/*
 * Frequent (Misra–Gries) summaries: the second counter-based summary the
 * paper discusses (Section 2, related work: Misra and Gries; Frequent of
 * Demaine et al.; the parallel merge of Frequent summaries), on the same
 * blocks and reduction tree as Space Saving.  The paper names the algorithm
 * and its merge but does not define them; the library follows the published
 * definitions:
 *   - block summary (Misra and Gries, 1982) with k - 1 counters: an item
 *     already counted adds 1; an item not counted takes a free counter with
 *     count 1; when no counter is free every counter loses 1, counters that
 *     reach 0 are freed and the item is not stored;
 *   - merge (Agarwal et al., "Mergeable summaries", 2012): counts of equal
 *     items add (absent = 0); when more than k - 1 items remain, the k-th
 *     largest count is subtracted from every count and only positive counts
 *     stay.
 * A Frequent summary holds at most k - 1 entries with err = 0 and minimum 0.
 * Its counts are lower bounds: with delta = floor((n_covered - sum of
 * counts) / k), every stored item satisfies count <= f <= count + delta and
 * every other item f <= delta, so every item with f * k > n is stored.
 * The same calls read and combine both kinds of summary: pss_merge (both
 * arguments of one kind, else PSS_EMISMATCH), pss_query / pss_query_mode,
 * pss_export, pss_free, and pss_tree_levels / _level_nodes / _read_level /
 * _root / _free for trees.  Not available for Frequent summaries:
 * the allocation-free form (pss_import makes a Space Saving summary,
 * pss_frequent_import a Frequent one; pss_frequent_summarize_host takes host
 * input; pss_accuracy_of uses the Frequent bounds).  The batched form is
 * pss_frequent_batch_create, the served form pss_frequent_server_create.
 *
 * pss_frequent_summarize — p Misra–Gries block summaries (Algorithm 1
 * bounds) merged in the binary tree over adjacent pairs (an odd last summary
 * carried up).  2 <= k <= PSS_MAX_K_RESIDENT; otherwise as pss_summarize.
 * Asynchronous on stream.
 */
#define PSS_KIND_SPACE_SAVING 0
#define PSS_KIND_FREQUENT 1
int pss_frequent_summarize(const void* d_items, uint64_t n, int item_bytes, uint32_t k,
                           uint32_t p, void* stream, pss_summary** out);

/* pss_frequent_summarize for items in HOST memory, read in place when
 * mapped pinned, else copied in slabs overlapped with the block summaries
 * (as pss_summarize_host).  Asynchronous on stream. */
int pss_frequent_summarize_host(const void* h_items, uint64_t n, int item_bytes, uint32_t k,
                                uint32_t p, void* stream, pss_summary** out);

/* pss_frequent_summarize keeping every level of the tree (nodes hold k - 1
 * entries: pss_tree_read_level's stride is k - 1).  Asynchronous. */
int pss_frequent_summarize_tree(const void* d_items, uint64_t n, int item_bytes, uint32_t k,
                                uint32_t p, void* stream, pss_tree** out);

/* PSS_KIND_SPACE_SAVING or PSS_KIND_FREQUENT. */
int pss_summary_kind(const pss_summary* summary, int* kind);
int pss_tree_kind(const pss_tree* tree, int* kind);

/*
 * Batched form: many independent streams, each with its own k and p, in one
 * launch graph.  For every distinct k one persistent summarize kernel takes
 * (stream, block) tasks from a work list, longest blocks first; one combine
 * launch per tree level covers that level of every stream; one launch
 * answers every stream's query.  Each stream's result is exactly that of
 * pss_summarize + pss_query with the same k and p (Algorithm 1 and 2 are
 * applied per stream; batching changes only the launch structure).
 */
typedef struct pss_batch pss_batch;

typedef struct {
  uint32_t nstreams;
  int item_bytes;                /* 4 or 8, the same for every stream */
  const void* const* d_items;    /* nstreams device pointers */
  const uint64_t* n;             /* nstreams lengths */
  const uint32_t* k;             /* nstreams counter counts, 2 <= k <= PSS_MAX_K_RESIDENT */
  const uint32_t* p;             /* nstreams block counts; NULL or 0 entries: pss_plan_blocks */
  const double* skew_hint;       /* optional per-stream skew for the planner (NULL: unknown) */
} pss_batch_desc;

/* The planner's block count for a stream of n items with k counters: a pure
 * function of its arguments (never of load), so a result can be replayed.
 * Block lengths come from the autotuner's measured table per (k class:
 * <= 64, <= 256, <= 1024, larger; skew class: nearest of 0.8, 1.4, 2.0;
 * skew_hint <= 0 means unknown and takes 1.4). */
uint32_t pss_plan_blocks(uint64_t n, uint32_t k, int item_bytes, double skew_hint);

/* The planner of the Frequent batch and server (same classes; its own
 * measured block lengths: 2^15 for k <= 256, 2^14 at k <= 1024 (2^15 at skew
 * class 2.0), 2^16 above). */
uint32_t pss_frequent_plan_blocks(uint64_t n, uint32_t k, int item_bytes, double skew_hint);

/* The planner's skew estimate for streams the caller knows nothing about (no
 * counterpart in the paper: it only steers the kernel choice and block
 * length, never a result).  For each stream, P = the number of pairs of
 * equal items among its first S = min(n[i], sample) items, counted exactly
 * on the device; skew_out[i] = pss_skew_of_pairs(P, S) and, if pairs_out is
 * not NULL, pairs_out[i] = P.  Both are pure functions of the stream's bytes,
 * so a plan built from them can be replayed.
 *   d_items: nstreams device pointers (NULL allowed where n[i] == 0);
 *   item_bytes 4 or 8; 2 <= sample <= 4096.
 * Allocates a small stream-ordered buffer; synchronizes stream.  PSS_EINVAL
 * on bad arguments. */
int pss_estimate_skew(const void* const* d_items, const uint64_t* n, uint32_t nstreams,
                      int item_bytes, uint32_t sample, void* stream, double* skew_out,
                      uint64_t* pairs_out);

/* Host only: the Zipf exponent s whose collision rate over [0, 2^32),
 * H(2^32, 2s) / H(2^32, s)^2 (H(U, s) = sum of r^-s for r = 1..U), equals
 * pairs / C(sample, 2), by interpolation in a table for s = 0.30 .. 4.00
 * (clamped to that range; 0.0 = unknown when sample < 2). */
double pss_skew_of_pairs(uint64_t pairs, uint64_t sample);

/* Plan and allocate a batch (device memory for every stream's tree, task
 * lists, results).  The streams' item buffers are borrowed for the batch's
 * lifetime.  Synchronizes stream. */
int pss_batch_create(const pss_batch_desc* desc, void* stream, pss_batch** out);

/* The batched form of the Frequent (Misra–Gries) summary: every stream of
 * desc is summarized with pss_frequent_summarize's blocks, merges and query
 * (k - 1 counters; each stream's result equals pss_frequent_summarize +
 * pss_query with the same k and p).  The block count comes from the same
 * planner.  pss_batch_run, _results, _export (m receives delta), _plan,
 * _info and _free apply unchanged. */
int pss_frequent_batch_create(const pss_batch_desc* desc, void* stream, pss_batch** out);

/* The block count used for each stream (nstreams values). */
int pss_batch_plan(const pss_batch* batch, uint32_t* p);

/* Counts of a batch (any pointer may be NULL). */
int pss_batch_info(const pss_batch* batch, uint32_t* nstreams, uint64_t* total_items,
                   uint64_t* total_k, uint32_t* k_classes);

/* Enqueue the whole batch on stream.  use_graph != 0: captured as a CUDA
 * graph on the first call (stream must not be capturing) and replayed
 * afterwards.  Asynchronous. */
int pss_batch_run(pss_batch* batch, int use_graph, void* stream);

/* Every stream's query result: stream i's entries are at host_out + (sum of
 * k over streams before i), host_counts[i] of them.  Synchronizes stream;
 * PSS_EDEVICE if a kernel recorded an error in any stream. */
int pss_batch_results(pss_batch* batch, pss_entry* host_out, uint32_t* host_counts, void* stream);

/* Canonical export of stream `index`'s root summary (as pss_export). */
int pss_batch_export(pss_batch* batch, uint32_t index, pss_entry* host_out, uint32_t cap,
                     uint32_t* size, uint64_t* m, uint64_t* n_covered, void* stream);

/* Release a batch (stream-ordered on the stream that created it). */
void pss_batch_free(pss_batch* batch);

/*
 * pss_merge — combine(S1, S2, k) of Algorithm 2: union of the items; an item
 * in both gets count1 + count2 (err1 + err2); an item in one only gets the
 * other summary's minimum added to its count and to its err; Prune(k) keeps
 * the k largest by (count descending, item ascending).  Both summaries must
 * have the same k, item width and kind (else PSS_EMISMATCH).  Two Frequent
 * summaries are merged by the Frequent merge instead.  Asynchronous.
 */
int pss_merge(const pss_summary* a, const pss_summary* b, void* stream, pss_summary** out);

/*
 * pss_query — Pruned(global, n, k) of Algorithm 1: the entries whose count
 * exceeds n / k (count * k > n, i.e. count >= floor(n/k) + 1, the k-majority
 * threshold of Section 3), in order of count descending then item
 * ascending.  n is the length of the stream the summary describes.
 *   host_out    array of cap entries; *n_out receives the number reported.
 * PSS_ERANGE if more than cap entries qualify (nothing is written).
 * A Frequent summary reports the entries whose upper bound exceeds n / k,
 * (count + delta) * k > n (no k-majority item is missed), each with
 * err = delta (count <= f <= count + err).
 * Synchronizes stream.
 */
int pss_query(const pss_summary* summary, uint64_t n, uint32_t k, pss_entry* host_out, uint32_t cap,
              uint32_t* n_out, void* stream);

/*
 * pss_query_mode — pss_query with a choice of bound.  PSS_QUERY_CANDIDATES is
 * pss_query (count * k > n: every true k-majority item is among them, the
 * 100% recall of Section 4).  PSS_QUERY_GUARANTEED keeps the entries whose
 * lower bound already exceeds the threshold, (count - err) * k > n: since
 * count - err <= f, each of them is a true k-majority item (no false
 * positive).  The paper reports only the first; the second is its
 * counterpart from the same error bound.  For a Frequent summary the
 * guaranteed entries are count * k > n (count <= f), each with err = delta.
 * Same order, arguments and errors as pss_query; any other mode is PSS_EINVAL.
 */
#define PSS_QUERY_CANDIDATES 0
#define PSS_QUERY_GUARANTEED 1
int pss_query_mode(const pss_summary* summary, uint64_t n, uint32_t k, int mode, pss_entry* host_out,
                   uint32_t cap, uint32_t* n_out, void* stream);

/*
 * Exact frequencies, the reference of the paper's accuracy metrics
 * (Section 4).  pss_exact_counts overwrites d_counts[0 .. 2^log2u] (caller
 * memory, 2^log2u + 1 u32 words, 1 <= log2u <= 32): word x is the number of
 * occurrences of item x among the n items at d_items (item_bytes 4 or 8), the
 * last word the number of items outside [0, 2^log2u).  Counts wrap past
 * 2^32 - 1 occurrences of one item.  Asynchronous.
 */
int pss_exact_counts(const void* d_items, uint64_t n, int item_bytes, int log2u, uint32_t* d_counts,
                     void* stream);

/*
 * pss_accuracy_of — the accuracy of a summary's answer against exact counts
 * (from pss_exact_counts over the same n items), as Section 4 defines it:
 * the relative error |f - count| / f of every reported item averaged over
 * the reported items (ARE), precision = reported true k-majority items /
 * reported items, recall = reported true k-majority items / true k-majority
 * items.  "Reported" means pss_query's answer (count * k > n), "true
 * k-majority" f * k > n.  Empty denominators give ARE 0, precision 1,
 * recall 1.  For a Frequent summary "reported" is its query's answer,
 * (count + delta) * k > n, and "guaranteed" count * k > n.  Synchronizes
 * stream.
 */
typedef struct {
  uint64_t reported;      /* entries with count * k > n */
  uint64_t true_frequent; /* items with f * k > n */
  uint64_t true_positive; /* reported items that are truly frequent */
  uint64_t guaranteed;    /* reported entries with (count - err) * k > n */
  uint64_t outside;       /* items of the stream outside [0, 2^log2u) */
  double are;
  double precision;
  double recall;
} pss_accuracy;
int pss_accuracy_of(const pss_summary* summary, const uint32_t* d_counts, int log2u, uint64_t n,
                    uint32_t k, pss_accuracy* out, void* stream);

/*
 * pss_export — copy a whole summary to the host in canonical order (count
 * descending, item ascending) with its minimum m and the number of stream
 * items it describes.  host_out holds cap >= k entries (PSS_ERANGE if the
 * summary holds more than cap).  For a Frequent summary *m receives delta =
 * floor((n_covered - sum of counts) / k) (every stored item has count <= f
 * <= count + delta, every other item f <= delta) and every err is 0.
 * Synchronizes stream.
 */
int pss_export(const pss_summary* summary, pss_entry* host_out, uint32_t cap, uint32_t* size,
               uint64_t* m, uint64_t* n_covered, void* stream);

/* k and item width of a summary. */
int pss_summary_info(const pss_summary* summary, uint32_t* k, int* item_bytes);

/*
 * pss_import — a device summary from canonical host entries, the output of
 * pss_export: entries[0 .. size) with distinct items, the summary's minimum
 * m and the stream length n_covered it describes.  Summaries are mergeable
 * (Algorithm 2), so an exported summary with its n_covered is a complete
 * checkpoint: importing it and merging on (pss_merge) continues a
 * computation exactly.  size <= k <= PSS_MAX_K; item_bytes 4 (items must fit
 * in 32 bits) or 8; duplicate items or size > k are PSS_EINVAL.  The entries
 * are read before the call returns; the summary is ready in stream order.
 */
int pss_import(const pss_entry* entries, uint32_t size, uint64_t m, uint64_t n_covered, uint32_t k,
               int item_bytes, void* stream, pss_summary** out);

/* pss_import for a Frequent summary: entries[0 .. size) (the counts of
 * pss_export's output; err is ignored), size <= k - 1, 2 <= k <=
 * PSS_MAX_K_RESIDENT.  Its delta follows from n_covered and the counts. */
int pss_frequent_import(const pss_entry* entries, uint32_t size, uint64_t n_covered, uint32_t k,
                        int item_bytes, void* stream, pss_summary** out);

/* Release a summary (stream-ordered on the stream that created it). */
void pss_free(pss_summary* summary);

/*
 * Served form: a request loop with continuous batching.  Each request is a
 * segment of one tenant's stream; the server keeps every tenant's summary
 * resident on the device and merges each new segment into it with combine
 * (Algorithm 2), strictly in arrival order per tenant, then answers two
 * queries (Algorithm 1, Pruned): the segment's own and the tenant's running
 * one.  Requests are released at their scheduled arrival times (open loop);
 * a scheduler thread admits them while the device-memory budget and the
 * per-tick limit allow, so requests that arrive while others are on the GPU
 * join the next tick, and ticks overlap on the device (segment work on
 * streams taken in turn, each tenant's merges in order on the tenant's own
 * stream; ticks complete in the order they finish).  Results are
 * independent of the mix: a request's results equal those of running its
 * tenant's requests alone, in order.
 */
typedef struct pss_server pss_server;

typedef struct {
  uint32_t tenants;        /* tenant summaries kept resident */
  uint32_t k;              /* counters of every segment and tenant summary (<= PSS_MAX_K_RESIDENT) */
  uint64_t budget_bytes;   /* device memory admitted requests may hold at once */
  uint32_t max_batch;      /* requests admitted per scheduling tick */
  uint32_t max_inflight;   /* admitted, not yet completed requests (host result slots) */
} pss_server_config;

typedef struct {
  uint64_t id;             /* caller's request id (unique) */
  double arrival;          /* scheduled arrival, seconds after pss_server_start */
  uint32_t tenant;         /* < tenants */
  uint64_t n;              /* segment length (items) */
  const void* d_items;     /* segment items (uint32, device); NULL: generate them */
  double s;                /* generated segments: Zipf skew, universe 2^log2u */
  int log2u;
  uint64_t seed;           /* generated segments: seed and stream id */
  uint32_t stream_id;
  uint32_t p;              /* blocks for the segment; 0 = pss_plan_blocks */
} pss_request;

typedef struct {
  uint64_t id;
  uint32_t tenant;
  uint32_t p;              /* blocks used for the segment */
  double arrival, admitted, completed;  /* seconds after start */
  uint32_t n_segment;      /* entries of the segment query */
  uint32_t n_tenant;       /* entries of the tenant query */
  uint64_t tenant_items;   /* items merged into the tenant, this segment included */
  int status;              /* PSS_OK or an error code */
} pss_completion;

int pss_server_create(const pss_server_config* config, pss_server** out);

/* The served form with Frequent (Misra–Gries) summaries: segments are
 * summarized by the Frequent batch, merged into their tenant with the
 * Frequent merge and both are queried with the Frequent query (err = delta).
 * Tenant summaries hold k - 1 entries; pss_server_tenant_export reports delta
 * in m and pss_server_tenant_import ignores m.  Everything else as
 * pss_server_create. */
int pss_frequent_server_create(const pss_server_config* config, pss_server** out);

/* Queue requests (any order; each is released at its arrival time).  May be
 * called before or after pss_server_start.  Request ids must be unique among
 * the requests whose results have not been read (or that have not failed):
 * a repeated id rejects the whole call with PSS_EINVAL. */
int pss_server_submit(pss_server* server, const pss_request* requests, uint32_t count);

/* Start the clock and the scheduler thread. */
int pss_server_start(pss_server* server);

/* Wait until every submitted request has completed (timeout in seconds;
 * PSS_ETIMEOUT if it expires). */
int pss_server_wait(pss_server* server, double timeout_s);

/* Drain up to cap completions (in completion order). */
int pss_server_poll(pss_server* server, pss_completion* out, uint32_t cap, uint32_t* n_out);

/* The two query results of a completed request (count desc, item asc);
 * each array holds k entries.  The result is released once read. */
int pss_server_result(pss_server* server, uint64_t id, pss_entry* segment_out, uint32_t* n_segment,
                      pss_entry* tenant_out, uint32_t* n_tenant);

/* Canonical export of a tenant's resident summary (waits for the server's
 * tenant work enqueued so far). */
int pss_server_tenant_export(pss_server* server, uint32_t tenant, pss_entry* host_out, uint32_t cap,
                             uint32_t* size, uint64_t* m, uint64_t* n_covered);

/* Fault injection for tests of the serving layer: the next `count` segment
 * allocations fail as if the device were out of memory.  Each such request
 * completes with status PSS_ENOMEM and leaves its tenant untouched; the
 * other requests of its tick, and every later one, proceed. */
int pss_server_inject_alloc_failures(pss_server* server, uint32_t count);

/* Restore a tenant's resident summary from a checkpoint (pss_server_tenant_export
 * of an earlier server with the same k): entries, m and n_covered as pss_import
 * takes them.  Only before pss_server_start (else PSS_EINVAL); the tenant's
 * later segments merge into it as if the earlier server had continued. */
int pss_server_tenant_import(pss_server* server, uint32_t tenant, const pss_entry* entries,
                             uint32_t size, uint64_t m, uint64_t n_covered);

/* Stop the scheduler (after the current tick) and release everything. */
void pss_server_destroy(pss_server* server);

/*
 * Kernel choice for the block summaries of pss_summarize*.  Blocks with
 * k <= kmax counters are summarized by one warp each, the counters in the
 * warp's registers (kmax is clamped to 256); larger k, or kmax = 0, use the
 * window-parallel CTA kernel.  Both apply the same sequential rule, so the
 * summaries are the same either way; the warp kernel is the faster one where
 * misses dominate (small k, weak skew).  The default is 64.  The batch API
 * chooses per stream from k <= 256 and its skew hint, unless kmax is 0.
 * Process-wide; returns the previous value.  Launches already enqueued (or
 * captured) keep their kernel.
 */
uint32_t pss_set_warp_kmax(uint32_t kmax);

/*
 * Largest k whose block summaries the plain path computes with the round
 * kernel: one warp per block, counters and table in shared memory, 32 items
 * per round, the evictions in (count, touch) order from a queue of the
 * minimum count.  Blocks with k above the warp kernel's limit and at most
 * kmax (clamped to PSS_MAX_K_RESIDENT) use it when the launch has enough
 * blocks to fill half the warps it keeps resident; the result is the same as
 * with the other kernels.  The default is 256.  Process-wide; returns the
 * previous value.
 */
uint32_t pss_set_round_kmax(uint32_t kmax);

/* The block-summary kernel the plain path uses for `count` blocks with k
 * counters (item_bytes 4 or 8): PSS_KERNEL_CTA (window-parallel, one CTA per
 * block; k above 4096 keeps part of its state in HBM), PSS_KERNEL_WARP
 * (counters in a warp's registers) or PSS_KERNEL_ROUND (one warp per block in
 * rounds); -1 for invalid arguments.  Queries the device's occupancy once per
 * k. */
#define PSS_KERNEL_CTA 0
#define PSS_KERNEL_WARP 1
#define PSS_KERNEL_ROUND 2
int pss_plan_kernel(uint32_t k, uint32_t count, int item_bytes);

/* The CTA shape of the window-parallel block-summary kernel for k counters
 * (item_bytes 4 or 8; `batch` != 0: the persistent kernel of the batch API):
 * *threads per CTA and *items_per_thread of one window.  Three shapes exist
 * (512 x 2, 256 x 4, 256 x 2); the one that keeps the most threads resident
 * per SM at this k is used (on a tie 256 x 4, then 256 x 2, then 512 x 2) by
 * launches of more blocks than the SMs hold at once in the 512 x 2 shape;
 * smaller launches run 256 x 2 as 512 x 2 (a launch that waits for no slot
 * takes as long as one block).  The summaries do not depend on the shape.
 * Queries the device's occupancy once per k.  PSS_EINVAL for invalid
 * arguments or null outputs; k above 4096 always reports 512 x 2.  This is
 * the shape of the kernel that keeps the whole state in shared memory: for
 * 2048 < k <= 3072 the plain path (batch == 0) runs the 512 x 2 form with
 * part of the state in stream-ordered HBM scratch instead, where that keeps
 * more CTAs resident (pss_summarize_noalloc never does). */
int pss_plan_cta_shape(uint32_t k, int item_bytes, int batch, int* threads,
                       int* items_per_thread);

/*
 * Profiling.  The paper reports run time and the "fractional overhead" of
 * the reduction relative to the computation (Section 4.1); the library can
 * time its own kernel groups with CUDA events on the launching stream.
 */
typedef struct {
  uint64_t launches;        /* kernels launched by the library since the last reset (always counted) */
  uint64_t summarize_calls; /* timed summarize-kernel launches */
  uint64_t merge_levels;    /* timed merge-level launches */
  uint64_t query_calls;     /* timed query/export launches */
  double summarize_ms;      /* device time of the summarize kernels */
  double merge_ms;          /* device time of the merge tree */
  double query_ms;          /* device time of the query/export kernels */
} pss_profile;

/* on != 0: record CUDA events around every kernel group from now on. */
int pss_profile_enable(int on);

/* Accumulated counters (waits for the recorded events); reset != 0 zeroes them. */
int pss_profile_read(pss_profile* out, int reset);

/*
 * pss_gen_zipf — fill d_out with items [start, start + count) of the seeded
 * synthetic stream (seed, stream_id): Zipf(s) ranks over [1, 2^log2u] mapped
 * by a fixed bijection onto [0, 2^log2u) (the paper's inputs are Zipf
 * streams of skew 1.1 and 1.8, Section 4.1).  item_bytes 4 requires
 * log2u <= 32; log2u <= 63.  Asynchronous.
 */
int pss_gen_zipf(void* d_out, uint64_t count, int item_bytes, uint64_t seed, uint32_t stream_id,
                 uint64_t start, double s, int log2u, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PSS_H_ */
