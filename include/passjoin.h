/*
 * passjoin.h -- C ABI of the GB300 Pass-Join edit-distance similarity join.
 *
 * Problem (Def. 1, Sec. 2 of the Pass-Join paper): given string sets R and S
 * and an edit-distance threshold tau, find every pair <r, s> in R x S with
 * ED(r, s) <= tau, where ED counts single-character insertions, deletions
 * and substitutions.  R = S is the self join (Sec. 2); R != S is the join of
 * Sec. 3.2.  Every call returns the exact pair set of that definition with
 * the exact ED of each pair.
 *
 * Method (all of it runs in this library's CUDA kernels on one GPU):
 *   - strings are grouped by length and each string of length >= tau + 1 is
 *     cut into tau + 1 even segments (Sec. 3.1), kept in a segment index keyed
 *     by (string length l, segment number i, segment content) (Sec. 3.2);
 *   - every probing string selects its multi-match-aware substrings for each
 *     admissible length l (Sec. 4.2, Alg. 2, Lemma 2) and looks them up;
 *   - every hit is checked by extension-based verification (Sec. 5.2, Alg. 3)
 *     built on length-aware banded DP with expected-edit-distance early
 *     termination (Sec. 5.1, Lemma 4).
 *
 * Conventions shared by every entry point:
 *   - Return value: PJ_OK (0) or a negative PJ_E* code.  pj_strerror() names a
 *     code; pj_last_error() gives the calling thread's last detailed message.
 *   - Strings are byte strings of length 0..65535.  A string set is the
 *     concatenation of its strings (bytes) plus n + 1 non-decreasing offsets;
 *     string k is bytes[offsets[k] .. offsets[k+1]).  offsets[0] need not be 0.
 *   - pj_strings.on_device = 0: bytes and offsets are host pointers;
 *     on_device = 1: device pointers on the library's device.  The caller owns
 *     them; they are read during the call only and may be freed afterwards.
 *   - 0 <= tau <= PJ_TAU_LIMIT.  Ids are 0-based input positions.
 *   - Results are library-allocated (host memory unless
 *     pj_options.results_on_device = 1), sorted by (a, b), released with
 *     pj_result_free().
 *   - All device work of a call is ordered on pj_options.stream; a call
 *     returns after its results are complete.
 */
#ifndef PASSJOIN_H
#define PASSJOIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PJ_TAU_LIMIT 32     /* largest threshold the kernels accept */
#define PJ_MAX_STRING_LEN 65535

enum {
  PJ_OK = 0,
  PJ_EINVAL = -1,     /* bad argument: NULL, tau out of range, offsets decreasing, string too long */
  PJ_ENOMEM = -2,     /* a device or host allocation failed */
  PJ_ECUDA = -3,      /* a CUDA runtime call or kernel failed (see pj_last_error) */
  PJ_ETIMEDOUT = -4,  /* a bounded wait expired (serving) */
  PJ_ECANCELED = -5   /* the request was cancelled (serving) */
};

/* verify_mode values (pj_options.verify_mode) */
enum {
  PJ_VERIFY_AUTO = 0,       /* library's choice: the autotuner's when autotune is set, else
                               PJ_VERIFY_PAIRS for strings longer than 256 bytes on average
                               and PJ_VERIFY_EXTENSION otherwise */
  PJ_VERIFY_EXTENSION = 1,  /* extension-based verification of every candidate match
                               (Sec. 5.2, Alg. 3) */
  PJ_VERIFY_PAIRS = 2       /* materialised: the candidate pairs are made distinct by a sort and
                               each distinct pair is verified once over the whole strings with
                               the length-aware method (Sec. 5.1); same results */
};

/* partition values (pj_options.partition): where the longer segments go when
 * a string's length is not a multiple of tau + 1.  Every segment has
 * floor(|s| / (tau + 1)) or that plus one characters in both. */
enum {
  PJ_PARTITION_EVEN = 0,    /* the last segments are the longer ones (Sec. 3.1, even partition) */
  PJ_PARTITION_CENTER = 1   /* the segments nearest the middle are the longer ones, where the
                               multi-match windows (Sec. 4.2) are widest; same results, fewer
                               candidates on short strings (a scheme of this library; the paper
                               leaves other partition schemes to future work, Sec. 3.1) */
};

/* A set of n strings; see the conventions above. */
typedef struct {
  const uint8_t* bytes;
  const uint64_t* offsets; /* n + 1 entries */
  uint32_t n;
  int on_device;
} pj_strings;

/* One similar pair.  Self join: a < b are input ids of the one set.
 * pj_join: a indexes R, b indexes S.  pj_query: a indexes the query batch,
 * b indexes the indexed set.  ed = ED(a, b) exactly, 0 <= ed <= tau. */
typedef struct {
  uint32_t a;
  uint32_t b;
  uint32_t ed;
} pj_pair;

/* Work counters of one call (all exact counts) and its device times. */
typedef struct {
  uint64_t lookups;     /* selected substrings looked up in the segment index */
  uint64_t candidates;  /* (probe, indexed string, segment, position) matches verified */
  uint64_t accepted;    /* matches accepted by extension verification */
  uint64_t dp_cells;    /* DP cells evaluated by the verification kernels */
  uint64_t fallback_pairs; /* pairs verified directly because a string has length <= tau */
  uint64_t hits;        /* lookups whose posting run was non-empty */
  float probe_ms;       /* device time of selection + lookup (CUDA events on the call's stream) */
  float verify_ms;      /* device time of extension verification */
  float fallback_ms;    /* device time of the short-string verification */
  float dedupe_ms;      /* device time of sort, min-reduce and compaction */
  float partition_ms;   /* device time spent building a lazily built threshold index, else 0 */
  int32_t verify_block; /* block size of the thread-per-candidate verification */
  int32_t warp_min_len; /* self join: probes at least this long were verified one warp per candidate */
  float tune_ms;        /* time spent autotuning during this call (0 when the decision was cached) */
  int32_t verify_mode;  /* PJ_VERIFY_EXTENSION or PJ_VERIFY_PAIRS, as run */
  int32_t pair_warp;    /* PJ_VERIFY_PAIRS: 1 when one warp verified each pair */
  uint64_t filtered;    /* candidates rejected before any DP by the character-count bound
                           ED(x, y) >= max over the two directions of the summed surplus of
                           one string's character counts over the other's (characters in
                           24 buckets, counts capped at 4); not part of Pass-Join, exact */
  uint64_t distinct_pairs; /* PJ_VERIFY_PAIRS: distinct candidate pairs verified */
  int32_t graph_replay; /* 1: the self join ran as a replay of its recorded CUDA graph
                           (pj_options.graph_joins); the phase times are then 0 */
  float graph_ms;       /* device time of that replay */
  uint64_t device_peak; /* with pj_options.device_budget set: the most device bytes held at once
                           through the budgeted allocator (over the index's life so far, or over
                           the call for pj_join and pj_self_join_stream); 0 without a budget */
  uint32_t windows;     /* pj_self_join_stream: length windows joined; 0 for other calls */
  int32_t fused;        /* self join in PJ_VERIFY_PAIRS: 1 when one persistent kernel ran selection,
                           lookup, distinct-pair formation and verification together; pairs
                           beyond its shared-memory lists went through the materialised path */
} pj_stats;

typedef struct {
  pj_pair* pairs;   /* count entries; host memory, or device memory if on_device */
  uint64_t count;
  int on_device;
  pj_stats stats;
  void* priv;       /* library-owned; do not touch */
} pj_result;

/* Device memory provider.  alloc returns device memory of at least `bytes`
 * bytes usable on `stream` (NULL on failure); free releases it. */
typedef void* (*pj_alloc_fn)(void* ctx, size_t bytes, void* stream);
typedef void (*pj_free_fn)(void* ctx, void* ptr, void* stream);

typedef struct {
  void* stream;           /* cudaStream_t for all device work; NULL = default stream */
  pj_alloc_fn alloc;      /* NULL = cudaMallocAsync on the stream */
  pj_free_fn free;        /* must be set iff alloc is set */
  void* alloc_ctx;
  int verify_mode;        /* PJ_VERIFY_* */
  int results_on_device;  /* 1: pj_result.pairs stays in device memory */
  int lazy_partitions;    /* 1: pj_build_index builds only the store; each threshold's
                             segment index is built by the first call that needs it */
  int autotune;           /* 1: the first self join of a threshold times, on a prefix of its
                             candidates (probes in length order), every verification
                             configuration -- extension verification with the thread- /
                             warp-per-candidate cut-over at each length-bucket edge and block
                             sizes 128/256/512, and PJ_VERIFY_PAIRS with a thread or a warp
                             per pair -- and keeps the fastest (cached per workload signature
                             for the process, and in the file autotune_cache names) */
  int graph_joins;        /* 1: after the first self join of a threshold, its whole pipeline is
                             recorded into a CUDA graph sized from that join's counts, and
                             later self joins of the threshold replay it (one graph launch;
                             same results; a count above a recorded capacity, which an
                             unchanged index cannot produce, falls back to the eager path).
                             Not recorded: joins with a warp-per-candidate range, or with more
                             probe groups than PJ_GRAPH_MAX_GROUPS (environment, default
                             2^28; the graph probes all groups in one pass).  A recorded join
                             keeps its device buffers (about the eager join's peak scratch;
                             ~10 GB for 1M short strings at tau = 4) until pj_index_free. */
  uint64_t device_budget; /* 0 = no limit.  Most device memory held at once through this
                             index's allocator (pj_build_index: its store, every threshold's
                             segment index, the scratch of every join, device results) or
                             through one pj_join / pj_self_join_stream call's.  An allocation
                             that would pass it fails the call with PJ_ENOMEM (nothing is
                             allocated); pj_self_join_stream instead narrows its length windows
                             until each window fits. */
  const char* autotune_cache; /* file that keeps autotuning decisions across processes (read,
                                 then appended; copied at pj_build_index).  NULL = the file
                                 named by the environment variable PJ_AUTOTUNE_CACHE, if any */
  int partition;          /* PJ_PARTITION_*: partition scheme of the segment indexes
                             (pj_build_index, pj_join, pj_self_join_stream); default EVEN */
} pj_options;

typedef struct pj_index pj_index; /* opaque, library-owned */

/* Fill *opt with defaults (default stream, cudaMallocAsync, auto verify,
 * host results). */
void pj_options_init(pj_options* opt);

/*
 * pj_build_index -- build the resident segment index of S for every
 * threshold 0..tau_max (Sec. 3.1 even partition, Sec. 3.2 index
 * L_l^i keyed by length, segment number and segment content).
 *   S       : the strings to index (host or device; see conventions).
 *   tau_max : 0..PJ_TAU_LIMIT.
 *   opt     : stream and allocator used for the index's whole life (copied).
 *             NULL = defaults.
 *   out     : receives the index; release with pj_index_free().
 * Errors: PJ_EINVAL (NULL S/out, tau_max out of range, decreasing offsets,
 * a string longer than PJ_MAX_STRING_LEN), PJ_ENOMEM, PJ_ECUDA.  On error
 * *out is NULL.
 */
int pj_build_index(const pj_strings* S, int tau_max, const pj_options* opt, pj_index** out);

/*
 * pj_self_join -- Def. 1 with R = S over the indexed set (Alg. 1): every
 * unordered pair of distinct ids a < b with ED <= tau.  Equal strings with
 * different ids are reported with ed = 0.
 *   idx : from pj_build_index; tau : 0..tau_max of idx.
 *   out : receives the result (stream, allocator and results_on_device of
 *         the index's options).
 * Errors: PJ_EINVAL (NULL, tau out of range), PJ_ENOMEM, PJ_ECUDA.
 */
int pj_self_join(pj_index* idx, int tau, pj_result* out);

/*
 * pj_self_join_shard -- one of n_shards disjoint parts of pj_self_join: the
 * pairs whose later string, in the visiting order of Alg. 1 (by length, then
 * id), is among the shard's probing strings -- the partitioned strings
 * (length >= tau + 1) split into n_shards equal consecutive ranges of that
 * order.  Shard 0 also holds every pair with a string too short to partition
 * (length <= tau).  Each pair is found by exactly one probe (the later
 * string probes the earlier, Alg. 1), so the shards' results are disjoint
 * and their union is exactly pj_self_join's result; each shard's pairs are
 * sorted by (a, b).  Shards of one index can run one after another or on
 * several GPUs, each with its own copy of the index.
 *   shard : 0..n_shards-1.  Other arguments and errors as pj_self_join
 *   (PJ_EINVAL also for n_shards = 0 or shard >= n_shards).
 */
int pj_self_join_shard(pj_index* idx, int tau, uint32_t shard, uint32_t n_shards, pj_result* out);

/*
 * pj_self_join_stream -- Def. 1 with R = S for a set that is never held on
 * the device as a whole.  When strings are visited by length (Alg. 1), a
 * string of length |s| probes only the inverted lists of lengths |s| - tau
 * .. |s| (Sec. 3.2).  So the strings, ordered on the host as the store orders
 * them (by length, then first eight bytes, then id),
 * are cut into windows of consecutive probing strings; a window's device set
 * is its probing strings plus the strings before them whose length is at
 * least its first probe's length - tau.  Each window builds a temporary store
 * and segment index of its device set and self-joins it with only its own
 * strings probing; the host maps the pairs back to input ids and merges the
 * windows' results.  The result equals pj_self_join's exactly.
 *   S   : HOST strings (on_device = 0).  tau : 0..PJ_TAU_LIMIT.
 *   opt : stream, allocator, verify_mode, autotune; device_budget bounds the
 *         device memory of the call (0 = three quarters of the free device
 *         memory): windows are sized from an estimate of their bytes and a
 *         window that still exceeds the budget is split in two and retried.
 *         Results are always in host memory (results_on_device is ignored).
 *   out : pairs a < b sorted by (a, b); stats summed over the windows, with
 *         stats.windows and stats.device_peak.
 * Errors: PJ_EINVAL (NULL, device strings, tau out of range, bad offsets),
 * PJ_ENOMEM (a window of one probing string does not fit the budget, or a
 * host allocation failed), PJ_ECUDA.
 */
int pj_self_join_stream(const pj_strings* S, int tau, const pj_options* opt, pj_result* out);

/*
 * pj_join -- Def. 1 for two sets (Sec. 3.2: index S, probe every r of R over
 * the lengths [|r| - tau, |r| + tau]).  Builds a temporary index of S for
 * this tau only.
 *   R, S : string sets (host or device); tau : 0..PJ_TAU_LIMIT;
 *   opt  : NULL = defaults.  out: pairs (a in R, b in S).
 * Errors as pj_build_index / pj_self_join.
 */
int pj_join(const pj_strings* R, const pj_strings* S, int tau, const pj_options* opt,
            pj_result* out);

/*
 * pj_query -- probe a batch of query strings against a resident index
 * (Sec. 3.2 join with R = the batch): pairs (a = query position, b = indexed
 * id) with ED <= tau.  Uses the index's stream and allocator; concurrent
 * calls on one index from several host threads are serialised by the
 * library.
 *   idx : from pj_build_index; batch : query strings (host or device);
 *   tau : 0..tau_max of idx.
 * Errors: PJ_EINVAL, PJ_ENOMEM, PJ_ECUDA.
 */
int pj_query(pj_index* idx, const pj_strings* batch, int tau, pj_result* out);

/*
 * pj_query_multi -- one batched probe of many queries that carry their own
 * thresholds (Sec. 3.2 join with R = the batch; each query q uses
 * threshold taus[q] and that threshold's segment index): all queries go
 * through one sequence of probe and verification launches.  Pairs are
 * (a = query position in the batch, b = indexed id, ed) sorted by (a, b);
 * for every query they equal pj_query of that query alone at its threshold.
 *   taus : host array of batch->n thresholds, each 0..tau_max of idx.
 * Errors as pj_query.
 */
int pj_query_multi(pj_index* idx, const pj_strings* batch, const uint8_t* taus, pj_result* out);

/* ----------------------------------------------------------- query plans --
 * A query plan is pj_query_multi recorded once into a CUDA graph, for
 * batches of bounded size that arrive again and again (serving).  The eager
 * path reads sizes back to the host between its launches (hits, candidates,
 * accepted matches, pairs) and allocates per call; a plan keeps every size
 * on the device, preallocates all buffers for its capacities, and runs a
 * whole batch -- threshold groups, probe (Sec. 4.2, Alg. 2), extension
 * verification (Sec. 5.2, Alg. 3), the short-string fallback, dedupe and
 * compaction -- as ONE graph launch after the batch's host-to-device copies,
 * with one stream synchronisation at the end.  Results are written by the
 * last kernels straight into mapped pinned host memory.  When a batch needs
 * more room than the capacities (hits, accepted matches or pairs), the plan
 * enlarges that buffer, records the graph again and reruns the batch, so
 * results never depend on the capacities.  A plan reads the index only; it
 * builds every threshold 0..tau_max of a lazy index when it is created.
 * The index must outlive the plan.  A plan is used by one thread at a time
 * (calls on one plan are serialised); use one plan per concurrent caller. */
typedef struct pj_plan pj_plan;

typedef struct {
  uint32_t max_queries;      /* strings per batch (default 4096, at most 2^24) */
  uint64_t max_bytes;        /* query bytes per batch (default 1 MiB) */
  uint64_t hits_capacity;    /* initial capacities (0 = derived from the above); */
  uint64_t accepted_capacity;/* they grow when a batch needs more */
  uint64_t pairs_capacity;
} pj_plan_options;

typedef struct {
  uint64_t runs;             /* batches run */
  uint64_t recaptures;       /* graph recordings after the first (capacity growth) */
  uint32_t graph_nodes;      /* nodes of the current graph */
  uint32_t graph_kernels;    /* kernel nodes of the current graph (launches per run) */
  uint64_t hits_capacity, accepted_capacity, pairs_capacity;
  uint64_t device_bytes;     /* device memory held by the plan */
  uint64_t host_bytes;       /* pinned host memory held by the plan */
} pj_plan_info;

void pj_plan_options_init(pj_plan_options* opt);
/* Create a plan over idx (opt NULL = defaults) on its own CUDA stream.
 * Errors: PJ_EINVAL (NULL, capacities out of range), PJ_ENOMEM, PJ_ECUDA. */
int pj_plan_create(pj_index* idx, const pj_plan_options* opt, pj_plan** out);
/* Run one batch: HOST strings (batch->on_device = 0), at most max_queries of
 * them and max_bytes bytes, query q with threshold taus[q] (0..tau_max).
 * *out receives host pairs (a = query position, b = indexed id, ed) sorted
 * by (a, b) -- exactly what pj_query_multi returns -- and the counters of
 * pj_stats (the millisecond fields are 0).  Release with pj_result_free.
 * Errors: PJ_EINVAL (NULL, device batch, batch above the plan's limits, tau
 * out of range, bad offsets, a string longer than 65535 bytes), PJ_ENOMEM,
 * PJ_ECUDA (including a failed segment index consistency check). */
int pj_plan_query(pj_plan* plan, const pj_strings* batch, const uint8_t* taus, pj_result* out);
int pj_plan_get_info(const pj_plan* plan, pj_plan_info* out);
/* Release a plan (NULL is ignored). */
void pj_plan_free(pj_plan* plan);

/* ---------------------------------------------------------------- serving --
 * A continuous-batching query server over a resident index (the R != S join
 * of Sec. 3.2 per request).  Requests are queued by pj_server_submit; each
 * of `slots` worker threads owns a CUDA stream, and whenever a slot is free
 * it admits every pending request that fits its caps -- max_batch_queries,
 * max_batch_bytes, and (free device memory - device_reserve) /
 * bytes_per_query queries -- and runs them together as one pj_query_multi
 * batch.  Requests arriving while other batches run are taken by the next
 * free slot, so batches overlap on the device.  Each request's result is
 * exactly what pj_query returns for it alone.  The index must outlive the
 * server; the server builds every threshold's segment index at start and
 * then only reads the index. */
typedef struct pj_server pj_server;

typedef struct {
  int slots;                   /* concurrent batches (1..16, default 3) */
  uint32_t max_batch_queries;  /* queries per batch (default 65536) */
  uint64_t max_batch_bytes;    /* query bytes per batch (default 16 MiB) */
  uint64_t bytes_per_query;    /* device-memory estimate per query for admission (default 64 KiB) */
  uint64_t device_reserve;     /* device memory kept free (default 2 GiB) */
  int use_plans;               /* 1: each slot runs its batches through its own query plan
                                  (one CUDA graph launch per batch); 0 (default): pj_query_multi */
} pj_server_options;

/* Time a request spent queued and being served (host clock), and how many
 * requests shared its batch. */
typedef struct {
  float queue_ms;
  float service_ms;
  uint32_t batch_requests;
} pj_request_times;

typedef struct {
  uint64_t requests, batches, queries, max_batch_requests;
  uint32_t max_in_flight;
  uint64_t pending;
} pj_server_counters;

void pj_server_options_init(pj_server_options* opt);
/* Start the server (opt NULL = defaults).  Errors: PJ_EINVAL, PJ_ENOMEM, PJ_ECUDA. */
int pj_server_start(pj_index* idx, const pj_server_options* opt, pj_server** out);
/* Queue one request: host strings (copied before returning) and its tau in
 * 0..tau_max.  *ticket identifies it.  Errors: PJ_EINVAL, PJ_ECANCELED (stopping). */
int pj_server_submit(pj_server* srv, const pj_strings* batch, int tau, uint64_t* ticket);
/* Wait up to timeout_ms (< 0: no limit) for a request.  PJ_OK: *out holds its
 * pairs (a = position in the request's batch, b = indexed id), release with
 * pj_result_free; times (may be NULL) receives its timings.  PJ_ETIMEDOUT:
 * not finished, the ticket stays valid.  PJ_ECANCELED: cancelled.  Any other
 * error is the batch's error.  A ticket can be collected once. */
int pj_server_wait(pj_server* srv, uint64_t ticket, int timeout_ms, pj_result* out, pj_request_times* times);
/* Cancel a queued or running request (its result is dropped). */
int pj_server_cancel(pj_server* srv, uint64_t ticket);
int pj_server_stats(pj_server* srv, pj_server_counters* out);
/* Finish running batches, cancel queued requests, join the slots, free. */
void pj_server_stop(pj_server* srv);

/*
 * pj_query_noalloc -- pj_query for callers that cannot allocate memory on the
 * call path: a serving thread that must not block in cudaMalloc/cudaFree
 * (they can synchronise the device), or an embedder that reserved its GPU
 * memory up front.  It allocates nothing: no device or host allocation and
 * no allocating library call.  The paper has no counterpart; this is a
 * serving convenience of this library.
 *   idx       : from pj_build_index; the threshold's index must already be
 *               built (always true unless lazy_partitions was set).
 *   batch     : query strings in DEVICE memory (on_device = 1), at most
 *               PJ_NOALLOC_MAX_QUERIES of them.
 *   tau       : 0..tau_max of idx.
 *   out_pairs : caller-owned device buffer of out_cap pj_pair entries; on
 *               success it holds *out_count pairs sorted by (a, b), exactly
 *               what pj_query returns for the same input.
 *   out_count : host pointer; receives the number of pairs (also when the
 *               buffer is too small, so the caller can retry).
 * All temporaries live in one device array of PJ_NOALLOC_SCRATCH_BYTES bytes
 * inside the library; every GPU that loads the library holds it until the
 * process exits.  Every call looks up that array's device address on the
 * current device (cudaGetSymbolAddress, which allocates nothing); the first
 * call on a device also loads the library's kernels there, so make that
 * first call before any stream capture.  Every call shares the array and
 * leaves its contents behind;
 * calls are serialised on the host, but calls whose GPU work overlaps (other
 * processes, or work still running on another stream) race on it.
 * Errors: PJ_EINVAL (NULL, tau out of range, host batch, batch too large,
 * index for tau not built, output buffer too small), PJ_ENOMEM (more
 * accepted matches than the scratch holds), PJ_ECUDA.
 */
#define PJ_NOALLOC_SCRATCH_BYTES (64u << 20)
#define PJ_NOALLOC_MAX_QUERIES 65536
int pj_query_noalloc(pj_index* idx, const pj_strings* batch, int tau, pj_pair* out_pairs, uint64_t out_cap,
                     uint64_t* out_count);

/*
 * pj_count_selection -- the substring-selection ablation of Sec. 4 for the
 * self join of the indexed set at threshold tau (the counts the paper plots
 * for its selection methods).  For every probing string s, every length l
 * in [max(tau + 1, |s| - tau), |s|] such that some string of length l is
 * visited before s (Alg. 1's visiting order by length, then id), and every
 * segment i of the even partition of l (Sec. 3.1), it sums the number of
 * start positions p (substrings s[p, l_i] that exist in s) each method
 * selects:
 *   length_based   : every substring of length l_i (Sec. 4);
 *   shift_based    : p in [P_i - tau, P_i + tau] (Sec. 4);
 *   position_aware : p in [P_i - floor((tau - D)/2), P_i + floor((tau + D)/2)],
 *                    D = |s| - l (Sec. 4.1);
 *   multi_match    : the multi-match-aware window of Sec. 4.2 (Lemma 2),
 *                    which is what pj_self_join looks up;
 *   groups         : the (s, l, i) combinations counted.
 * Counts only: nothing is looked up.  Needs no segment index (a lazy index
 * is fine).  Errors: PJ_EINVAL (NULL, tau outside 0..tau_max), PJ_ECUDA.
 */
typedef struct {
  uint64_t length_based;
  uint64_t shift_based;
  uint64_t position_aware;
  uint64_t multi_match;
  uint64_t groups;
} pj_selection;
int pj_count_selection(pj_index* idx, int tau, pj_selection* out);

/*
 * pj_calibrate -- measures, on the current device, the ceilings that the
 * join's rooflines are reported against (the paper has no counterpart; it is
 * a measurement aid).  Kernels run 8 blocks of 256 threads per SM:
 *   dp_cells_per_s      : cells of the banded VERIFYSTRINGPAIR recurrence
 *                         (Sec. 5.1; the verification kernels' cell code, a
 *                         band of 5 diagonals, Lemma 4 test per row) with both
 *                         strings in registers;
 *   int32_ops_per_s     : 32-bit integer operations (independent xor + add
 *                         chains of register operands);
 *   l2_read_bytes_per_s : read bandwidth of a 64 MiB buffer held in the L2
 *                         with 16-byte loads;
 *   sm_mhz              : SM clock during the DP run (clock64 against the
 *                         global nanosecond timer);
 *   sm_count            : multiprocessors.
 * Each figure is the best of three launches on a stream of its own; the call
 * takes well under a second and allocates 64 MiB of device memory
 * (cudaMallocAsync) for its duration.  Errors: PJ_EINVAL (NULL), PJ_ENOMEM,
 * PJ_ECUDA.
 */
typedef struct {
  double dp_cells_per_s;
  double int32_ops_per_s;
  double l2_read_bytes_per_s;
  double sm_mhz;
  int32_t sm_count;
} pj_calibration;
int pj_calibrate(pj_calibration* out);

/* Number of strings / largest tau of an index (0 for NULL). */
uint32_t pj_index_size(const pj_index* idx);
int pj_index_tau_max(const pj_index* idx);
/* Device bytes held by the index (store + every threshold's tables). */
uint64_t pj_index_device_bytes(const pj_index* idx);

/* Device time of pj_build_index (store and eagerly built thresholds), ms. */
float pj_index_build_ms(const pj_index* idx);

/* Number of CUDA kernels this library has launched since it was loaded
 * (all threads, all calls). */
uint64_t pj_kernel_launches(void);

/* Release a result / an index.  NULL and already-released results are
 * ignored.  A result must be released before the index it came from. */
void pj_result_free(pj_result* res);
void pj_index_free(pj_index* idx);

/* Static name of an error code; message of the calling thread's last error. */
const char* pj_strerror(int code);
const char* pj_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PASSJOIN_H */
