/*
 * rmips.h -- C ABI of librmips: exact reverse k-MIPS on one NVIDIA GB300 GPU.
 *
 * Problem (Definition 2, "Reverse k-MIPS problem", of Amagata & Hara,
 * "Reverse Maximum Inner Product Search", RecSys 2021): given a query item
 * vector q, a user set Q, an item set P and k, return every user u in Q whose
 * k-MIPS result over P + {q} contains q.  Ties between q and an item are
 * resolved in q's favour:
 *
 *     u is returned  <=>  #{ p in P : u.p > u.q } < k
 *
 * with the inner products taken in exact arithmetic on the float32 inputs.
 * The returned set is exactly that set on every precision path; reduced
 * precision only changes how many users need the exact recheck.
 *
 * Method (Simpfer, Section 4): an offline index (Algorithm 1) keeps, per
 * user, bounds on its j-th largest inner product over P (j = 1..k_max) and
 * groups norm-sorted users into blocks; a query prunes whole blocks
 * (Lemma 3), decides most remaining users in O(1) (Lemmas 1 and 2), and
 * verifies the rest against P (Algorithm 2, Corollaries 1 and 2) with an
 * exact tie-breaking recheck.
 *
 * Conventions for every entry point:
 *  - Matrices are row-major float32, [rows][d], caller-owned, and may live in
 *    host or device memory (detected with cudaPointerGetAttributes).  The
 *    library never keeps a caller pointer after the call returns.
 *  - Ids are 0-based row numbers of the caller's original Q.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    that return counts or host results synchronise that stream.
 *  - Every call returns an rmips_status; on failure no output is partially
 *    written unless stated, and rmips_last_error() gives a message.
 *  - An index is immutable after build.  Concurrent queries on one index are
 *    safe from different host threads (each call takes its own workspace).
 */
#ifndef RMIPS_H
#define RMIPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rmips_index rmips_index;

typedef enum {
  RMIPS_OK = 0,
  RMIPS_ERR_ARG = 1,        /* bad pointer, size, option or segment */
  RMIPS_ERR_K_RANGE = 2,    /* k < 1 or k > k_max (the paper rebuilds the
                               index for k > k_max, Section 4.1) */
  RMIPS_ERR_NONFINITE = 3,  /* NaN or Inf in Q, P or a query; for a BF16 / FP16
                               index also a value of Q or a query whose copy in
                               that format would overflow (FP16: |x| > 65504) */
  RMIPS_ERR_OOM = 4,        /* device or pinned host allocation failed */
  RMIPS_ERR_CAPACITY = 5,   /* output buffer too small; the required size
                               is reported, nothing is written */
  RMIPS_ERR_TIMEOUT = 6,    /* a bounded device wait gave up */
  RMIPS_ERR_CUDA = 7,       /* a CUDA runtime call failed */
  RMIPS_ERR_INTERNAL = 8,   /* a device-side consistency check failed */
  RMIPS_ERR_BUSY = 9        /* serving: admission refused, too many pending */
} rmips_status;

/* Arithmetic of the online filter (the index always keeps float32 copies). */
enum { RMIPS_FP32 = 0, RMIPS_BF16 = 1, RMIPS_FP16 = 2 };

typedef struct {
  int32_t k_max;      /* largest k a query may use; 1..28 (Section 2: the
                         method's only parameter, 25 in Section 5) */
  int32_t block_size; /* users per block (Definition 4); 32, 64, 128 or 256;
                         0 selects 32 */
  int64_t p_prime;    /* |P'| of Algorithm 1: 0 (or >= |P|) builds the bounds
                         over all of P ("full-P"); otherwise over the first
                         p_prime items in descending norm, as in the paper */
  int32_t precision;  /* RMIPS_FP32, RMIPS_BF16 or RMIPS_FP16 */
  int32_t flags;      /* RMIPS_FLAG_* bits; 0 for the defaults */
  const char* tune_cache;  /* NULL, or a text file of autotuner results: when
                              set (or with RMIPS_FLAG_AUTOTUNE) the build ends
                              with rmips_index_tune(index, tune_cache) */
} rmips_build_opts;

/* rmips_build_opts.flags: run the batched filter on CUDA cores (float32 FMA)
   instead of tensor cores (TF32 tiles, used for float32 indexes with d <= 64). */
#define RMIPS_FLAG_BATCH_CUDA_CORES 1
/* rmips_build_index: select each user's candidate items on CUDA cores (float32
   FMA) instead of tensor cores (TF32 tiles, used when d <= 64). */
#define RMIPS_FLAG_BUILD_CUDA_CORES 2
/* rmips_build_index: switch the block filter (Lemma 3) off -- every block's
   bound is -inf, so no block is ever pruned.  Answers are unchanged; this is
   the "without blocks" ablation of the paper's evaluation. */
#define RMIPS_FLAG_NO_BLOCK_FILTER 4
/* rmips_build_index: run the autotuner (rmips_index_tune) at the end of the
   build, also without a tune_cache file. */
#define RMIPS_FLAG_AUTOTUNE 8

/* Optional restriction of a query to a subset of users. */
typedef struct {
  int32_t kind;       /* 0: all users, 1: ids in [begin, end), 2: id list,
                         3: a segment registered with a server (serving only;
                         begin = the handle of rmips_server_add_segment) */
  int32_t reserved;   /* must be 0 */
  int64_t begin, end; /* kind 1 */
  const int64_t* ids; /* kind 2: host array of n_ids distinct ids */
  int64_t n_ids;
} rmips_segment;

typedef struct {
  int64_t n, m;          /* |Q|, |P| */
  int32_t d, k_max;
  int32_t block_size, precision;
  int64_t n_blocks;
  int64_t p_prime;       /* items the bounds were built over */
  int64_t incomplete;    /* users whose candidate list could not be proven
                            complete (they fall back to a full scan) */
  int64_t device_bytes;  /* index footprint in device memory */
  double build_ms;       /* wall time of rmips_build_index (with tuning) */
  int32_t tuned;         /* 0 not tuned, 1 searched on the device, 2 read
                            from a tune cache */
  int32_t batch_stages;  /* query stages of the batched tensor-core filter
                            (0: as many as fit) */
  int32_t single_stages; /* row stages of the single-query kernel (0: as
                            many as fit) */
  int32_t build_kind;    /* operands of the build's tensor-core candidate
                            selection: 0 TF32, 1 BF16, 2 FP16, -1 CUDA cores */
  double tune_ms;        /* wall time of the tuning */
} rmips_index_info;

typedef struct {
  int64_t blocks_total, blocks_pruned;   /* Lemma 3 */
  int64_t users_tested;                  /* users of unpruned blocks */
  int64_t yes_fast;                      /* decided yes without a scan */
  int64_t todo;                          /* sent to recheck / Algorithm 2 */
  int64_t exact_calls;                   /* exact (integer) tie decisions */
  int64_t result;                        /* users returned */
} rmips_query_stats;

/*
 * rmips_build_index -- Algorithm 1 (Section 4.1, "Pre-processing").
 *
 * Q: n x d users, P: m x d items (float32, host or device).  Computes the
 * norms, sorts users and items by descending norm (ties by ascending id),
 * computes for every user bounds lo_j <= v_j <= hi_j on its j-th largest
 * inner product v_j over P' (j = 1..k_max), and the block arrays
 * L^j(B) = min_{u in B} lo_j(u) (Equation 1).  The index owns device copies
 * of everything it needs; the caller may free Q and P on return.
 * Errors: ARG (null pointer, n < 1, m < 1, d < 1 or d > 128, bad opts),
 * NONFINITE, OOM, CUDA.  On error *out is NULL.
 */
rmips_status rmips_build_index(const float* Q, int64_t n, const float* P, int64_t m,
                               int32_t d, const rmips_build_opts* opts, void* stream,
                               rmips_index** out);

/*
 * rmips_index_tune -- the autotuner (no counterpart in the paper, which
 * leaves the block size of Definition 4 at O(log n) and runs on CPU cores).
 *
 * Chooses the block size (32, 64, 128 or 256; the block arrays of Equation 1
 * are rebuilt from the index's bounds) and the pipeline depths of the batched
 * tensor-core filter and of the single-query kernel, by timing the index's
 * own filters on the device: 1,024 items of P spread over the norm order as
 * queries, k cycling through 1..k_max, then 64 single queries.  None of the
 * choices changes any answer.  tune_cache: NULL, or a text file; a line for
 * the same (n, m, d, k_max, precision, P', filter kind, GPU model) is used
 * instead of searching, and a search appends its result there.  The tuned
 * choices are saved with the index (rmips_index_save).  No query may run on
 * the index during the call.  Synchronises `stream`.
 * Errors: ARG, OOM, CUDA, TIMEOUT.
 */
rmips_status rmips_index_tune(rmips_index* index, const char* tune_cache, void* stream);

/*
 * rmips_query -- Algorithm 3 (Section 4.3, "Simpfer") for one query.
 *
 * q: d floats (host or device).  k: 1..k_max.  seg: NULL for all users.
 * out_ids: capacity int64 slots (host or device); receives the result ids in
 * ascending order.  *out_count (host) receives the result size, also when
 * the status is RMIPS_ERR_CAPACITY (then nothing is written to out_ids).
 * Synchronises `stream`.  Errors: ARG, K_RANGE, NONFINITE, CAPACITY, CUDA.
 */
rmips_status rmips_query(rmips_index* index, const float* q, int32_t k,
                         const rmips_segment* seg, int64_t* out_ids, int64_t capacity,
                         int64_t* out_count, void* stream);

/*
 * rmips_query_batch -- many queries in one call.
 *
 * qs: nq x d (host or device), ks: nq values of k (host or device), segs:
 * NULL or nq segments (host).  Results are concatenated in query order into
 * out_ids (capacity slots, host or device); out_offsets (host, nq + 1
 * entries) receives the CSR offsets, so query j's ids are
 * out_ids[out_offsets[j] .. out_offsets[j+1]).  On RMIPS_ERR_CAPACITY the
 * offsets are still filled (out_offsets[nq] is the size needed) and out_ids
 * is left unspecified.  Synchronises `stream`.
 * The batched filter lists the (user, query) pairs its O(1) tests leave
 * undecided; the list holds RMIPS_PAIR_LIST_CAP entries (an environment
 * variable read when a workspace is created; default 16,777,216).  A pass that
 * finds more is run again in passes of half the size, down to one query at a
 * time, so the results do not depend on the list size.
 */
rmips_status rmips_query_batch(rmips_index* index, const float* qs, int64_t nq,
                               const int32_t* ks, const rmips_segment* segs,
                               int64_t* out_ids, int64_t capacity, int64_t* out_offsets,
                               void* stream);

/*
 * rmips_query_batch_async -- rmips_query_batch for device-resident inputs and
 * outputs that does not wait for the GPU (Algorithm 3 for many queries, as
 * rmips_query_batch; no segments).
 *
 * qs [nq][d] float32, ks [nq] int32, out_ids [capacity] int64,
 * out_offsets [nq + 1] int64 and done [2] int64 are DEVICE pointers.  All work
 * is queued on `stream` and the call returns; when the stream passes it,
 * out_offsets holds the CSR offsets, done[0] an rmips_status (RMIPS_OK,
 * RMIPS_ERR_NONFINITE, RMIPS_ERR_K_RANGE, RMIPS_ERR_CAPACITY with
 * out_offsets[nq] = the size needed and out_ids unspecified,
 * RMIPS_ERR_OOM when the undecided-pair list overflowed -- this call cannot
 * re-run, so run that batch through rmips_query_batch or in smaller batches --,
 * RMIPS_ERR_TIMEOUT, RMIPS_ERR_INTERNAL) and done[1] the number of result
 * ids.  The returned status covers only what the host can check (arguments,
 * allocations, launches).  The buffers must stay valid until the stream has
 * passed the call.  Each call runs on a workspace of the index (scratch
 * buffers and captured graphs): the oldest one whose queued work has
 * finished, else a second one, so a call on another stream may run at the
 * same time as this one (the index itself is only read; consecutive batches
 * queued on two streams in turn overlap).  While both workspaces still have
 * work queued, a call waits on the device for the older one's work.  Filter
 * timing and kept pairs reach the profile when rmips_profile_read is called;
 * rmips_last_query_stats is not updated.
 */
rmips_status rmips_query_batch_async(rmips_index* index, const float* qs, int64_t nq, const int32_t* ks,
                                     int64_t* out_ids, int64_t capacity, int64_t* out_offsets,
                                     int64_t* done, void* stream);

/*
 * rmips_query_async -- rmips_query (Algorithm 3, Section 4.3, for one query)
 * for device-resident buffers, without waiting for the GPU.
 *
 * q [d] float32, out_ids [capacity] int64 and done [2] int64 are DEVICE
 * pointers of the index's GPU; no segment.  The work is queued on `stream`
 * (for a full-P index one kernel launch) and the call returns.  When the
 * stream passes it, out_ids holds the ascending result ids, done[0] an
 * rmips_status (RMIPS_OK, RMIPS_ERR_NONFINITE, RMIPS_ERR_CAPACITY with
 * out_ids unspecified, RMIPS_ERR_TIMEOUT, RMIPS_ERR_INTERNAL) and done[1] the
 * result size (the size needed on RMIPS_ERR_CAPACITY).  The returned status
 * covers only what the host can check.  The buffers must stay valid until the
 * stream has passed the call.  Workspaces are taken as for
 * rmips_query_batch_async, so calls queued back to back run one after the
 * other on their stream without host round trips.  Filter timing reaches the
 * profile when rmips_profile_read is called; rmips_last_query_stats is not
 * updated.
 */
rmips_status rmips_query_async(rmips_index* index, const float* q, int32_t k, int64_t* out_ids, int64_t capacity,
                               int64_t* done, void* stream);

/*
 * Index persistence.  rmips_index_save writes the index (sizes, options and
 * every device array) to a host file; rmips_index_load reads it back onto the
 * current device, answering exactly as the index that was saved.  The file
 * format belongs to this library build (native byte order); a file that does
 * not match its own header is refused with RMIPS_ERR_ARG.  The paper has no
 * counterpart.
 */
rmips_status rmips_index_save(const rmips_index* index, const char* path);
rmips_status rmips_index_load(const char* path, void* stream, rmips_index** out);

/*
 * rmips_index_rebuild -- Algorithm 1 again with another k_max (Section 4.1:
 * the index keeps k_max ranks; a query with a larger k needs a rebuild).
 * Builds a new index over the same users and items, with the same ids, block
 * size, P' and precision, taken from `index` itself (the caller's Q and P are
 * not needed).  `index` is unchanged; the caller frees both.
 */
rmips_status rmips_index_rebuild(const rmips_index* index, int32_t k_max, void* stream, rmips_index** out);

/*
 * rmips_topk_join -- k-MIPS (Definition 1) of every user over all items: the
 * join whose top-k_max part the index keeps.  out_ids [n][k] (host or device,
 * row = the caller's user id) receives the caller's ids of the user's k items
 * with the largest inner products, in descending order; equal products come
 * in ascending item id.  Needs a full-P index (p_prime = 0; otherwise
 * RMIPS_ERR_ARG); k in [1, min(k_max, m)] (otherwise RMIPS_ERR_K_RANGE).
 * Exact: products are ranked in float64 with their error bounds, and in exact
 * integer arithmetic where two bounds overlap.  Synchronises `stream`.
 */
rmips_status rmips_topk_join(const rmips_index* index, int32_t k, int64_t* out_ids, void* stream);

/* Per-kernel timing of the filter kernels (Lemmas 1-3), for roofline reports. */
typedef struct {
  int64_t filter_launches;   /* filter launches since profiling was enabled */
  double filter_ms;          /* summed CUDA-event durations of those launches,
                                events recorded on the launching stream */
  double filter_alg_bytes;   /* algorithmic bytes they had to move: 8 bytes of
                                block header and L^k(B) per block, plus per
                                tested user its row (d x element size), its
                                (lo, hi) pair (8 bytes), its norm (4 bytes,
                                where the filter reads it: the one-launch
                                query and P' indexes) and 4 bytes per listed
                                user */
  int64_t users_tested;      /* users of unpruned blocks */
  int64_t blocks_pruned;     /* blocks pruned by Lemma 3 */
  int64_t blocks_total;      /* blocks examined */
  int64_t mfilter_launches;  /* multi-query filter launches (rmips_query_batch) */
  double mfilter_ms;         /* their summed CUDA-event durations */
  int64_t mfilter_pairs;     /* (user, query) pairs kept by Lemma 3 */
  double mfilter_alg_flops;  /* 2 d flops per kept pair (the inner products
                                the per-user tests need) */
  int64_t mfilter_tiles;     /* 128-user x 128-query tensor-core items
                                multiplied (the padded work behind the kept
                                pairs) */
  double mfilter_wait[11];   /* SM clock cycles the tensor-core filter's roles
                                spent waiting, summed over CTAs: loader (free
                                tile slot), feeder (free query stage), MMA
                                (query tile landed), MMA (free accumulator),
                                epilogue warp 0 (accumulator ready), MMA (user
                                tile landed), epilogue warp 0 reading TMEM,
                                MMA thread issuing an item's MMAs, epilogue
                                warp 0 in per-pair tests; [9] is the number of
                                epilogue warp 0 items that needed them, [10]
                                the cycles of those tests spent appending
                                pairs */
  double mfilter_cycles[4];  /* cycles of each role from start to finish,
                                summed over CTAs: loader, feeder, MMA,
                                epilogue warp 0 */
  int64_t mfilter_active_tiles;  /* user tiles with at least one item */
} rmips_profile;

/* Turns filter timing on (resetting the counters) or off.  While on, every
   query records a CUDA event pair around each filter launch.  enable = 2 also
   fills the pipeline counters of the tensor-core batched filter
   (mfilter_tiles, mfilter_wait, mfilter_cycles, mfilter_active_tiles); that
   runs an instrumented copy of the kernel, so time with enable = 1. */
rmips_status rmips_profile_enable(rmips_index* index, int32_t enable);

/* Reads the accumulated filter timing. */
rmips_status rmips_profile_read(const rmips_index* index, rmips_profile* out);

/*
 * rmips_query_noalloc -- rmips_query for callers that must not allocate.
 * (The paper has no counterpart: this is an interface choice of the library.)
 *
 * Who needs it: code whose device memory belongs to another allocator (a
 * framework's caching allocator that has reserved the free memory, where a
 * cudaMalloc behind its back fails or fragments the pool), and
 * latency-critical serving threads, where cudaMalloc / cudaFree may
 * synchronise the device and stall every other stream.  This call performs no
 * allocation of any kind: its scratch (about 8.5 MB) is one fixed array in
 * device memory that exists on every GPU where the library is loaded, for the
 * life of the process.
 *
 * Limit: the index may hold at most 1,048,576 users (RMIPS_ERR_ARG beyond).
 * q: d floats, host or device.  out_ids: DEVICE memory, capacity int64 slots,
 * receives the ascending result ids.  *out_count (host) receives the result
 * size; on RMIPS_ERR_CAPACITY it is the size needed and out_ids is untouched.
 * The array belongs to a lazily loaded module of the library; building or
 * loading an index on a device loads it there (and looks up its address), so
 * the call itself only reads that cached address.  On an error return after
 * GPU work was queued, the call waits for that work before it releases the
 * lock.
 * All calls share the one array, so calls are serialised by a process-wide
 * lock held until the call's GPU work has finished; GPU work of two calls that
 * overlapped would race on the shared scratch.  Synchronises `stream`.
 * Errors: ARG, K_RANGE, NONFINITE, CAPACITY, CUDA.
 */
rmips_status rmips_query_noalloc(rmips_index* index, const float* q, int32_t k, int64_t* out_ids,
                                 int64_t capacity, int64_t* out_count, void* stream);

/*
 * Serving loop: continuous batching of reverse k-MIPS requests on one index
 * (no counterpart in the paper, whose queries arrive one at a time).
 *
 * A dispatcher thread takes the queued requests as a batch as soon as one
 * of `streams` CUDA streams is free and no batch is on the device; while
 * batches run, it closes a batch when it holds max_batch requests, when
 * their result reservations fill a slot's device result buffer, or when its
 * oldest request has waited max_wait_us.  So batches grow with the load and
 * up to `streams` of them overlap on the device.  A batch of at most
 * single_max requests runs as one-launch single queries on its stream, a
 * larger one through the batched filter.
 * Results are exactly those of rmips_query for the same request.  Every
 * segment kind is answered inside the batch (id ranges on the device; id
 * lists and registered segments, kind 3, by intersecting the request's exact
 * result with the list).
 *
 * Admission by device memory: each slot owns a device result buffer of
 * max_device_bytes / (8 x streams) ids; a queued or running request reserves
 * min(result_ids_per_request, its segment's size) of those ids.  A submission
 * whose reservation would exceed the buffers' total, or that would exceed
 * max_pending requests, is refused with RMIPS_ERR_BUSY (nothing is queued).
 * A batch whose results outgrow its buffer anyway (reservations are
 * estimates) is answered one request at a time, with the same results.
 * The index must outlive the server; no other server call may be in
 * progress when rmips_server_destroy is called.
 */
typedef struct rmips_server rmips_server;

typedef struct {
  int32_t max_batch;        /* requests per batch, 1..16384 (default 4096) */
  int32_t max_wait_us;      /* batch closing deadline while another batch is on
                               the device, in microseconds (default 200; with
                               the device idle a batch closes at once) */
  int32_t streams;          /* batches in flight, 1..16 (default 2) */
  int32_t single_max;       /* batches of at most this many requests run as
                               one-launch single queries (full-P index);
                               0 = 4, -1 = never, at most 64 */
  int64_t max_pending;      /* admission bound on queued + running requests
                               (default 1,048,576) */
  int64_t max_device_bytes; /* device memory of the result buffers; 0 = an
                               eighth of the free device memory at creation,
                               at most 256 MiB */
  int64_t result_ids_per_request;  /* result ids a request reserves (at most
                               its segment's size); 0 = 1,024 */
  int32_t spin_us;          /* the dispatcher, the completer and waiting callers
                               poll for up to this many microseconds before they
                               block (lower latency at light load, for busy
                               host cores); 0 = block at once (default),
                               at most 100,000 */
  int32_t reserved;         /* must be 0 */
} rmips_server_opts;

typedef struct {
  int64_t submitted, completed, rejected, pending;
  int64_t batches;
  double mean_batch;        /* requests per launched batch */
  double p50_ms, p99_ms, max_ms;   /* request latency, submit to completion */
  int64_t reserved_ids;     /* result ids reserved by pending requests */
  int64_t reservable_ids;   /* total ids of the result buffers (admission bound) */
  int64_t batches_one_by_one;  /* batches re-run one request at a time */
} rmips_server_stats;

/*
 * rmips_server_add_segment -- registers a user segment (host array of n_ids
 * ids, copied, duplicates dropped) with the server; requests refer to it as
 * rmips_segment{kind = 3, begin = *handle}, so that large subsets are not
 * copied with every request.  Handles stay valid for the server's lifetime.
 */
rmips_status rmips_server_add_segment(rmips_server* server, const int64_t* ids, int64_t n_ids, int32_t* handle);

/* opts may be NULL for the defaults.  Spawns two host threads. */
rmips_status rmips_server_create(rmips_index* index, const rmips_server_opts* opts, rmips_server** out);

/* Queues one request (q: d floats in HOST memory, copied).  Validates k,
   finiteness and the segment immediately.  *ticket identifies the request. */
rmips_status rmips_server_submit(rmips_server* server, const float* q, int32_t k, const rmips_segment* seg,
                                 int64_t* ticket);

/* Queues nq requests at once (all or none are admitted). */
rmips_status rmips_server_submit_many(rmips_server* server, const float* qs, int64_t nq, const int32_t* ks,
                                      const rmips_segment* segs, int64_t* tickets);

/* Waits up to timeout_ms (negative: forever, 0: poll) for a request; copies
   its ascending ids to out_ids (host or device, capacity slots), its size to
   *out_count and its latency to *latency_ms (may be NULL), then forgets the
   ticket.  RMIPS_ERR_TIMEOUT: not finished (ticket kept).
   RMIPS_ERR_CAPACITY: *out_count is the size needed (ticket kept). */
rmips_status rmips_server_wait(rmips_server* server, int64_t ticket, int64_t* out_ids, int64_t capacity,
                               int64_t* out_count, double* latency_ms, int32_t timeout_ms);

/* Waits for a set of requests and returns their results in CSR form:
   request i's ids are out_ids[out_offsets[i] .. out_offsets[i+1]) (out_offsets
   has nt + 1 entries, host); latency_ms (NULL or nt entries) receives each
   latency.  On success every ticket is forgotten; the first failing request's
   status is returned (its slice is empty).  RMIPS_ERR_TIMEOUT and
   RMIPS_ERR_CAPACITY (offsets filled) keep all tickets. */
rmips_status rmips_server_wait_many(rmips_server* server, const int64_t* tickets, int64_t nt, int64_t* out_ids,
                                    int64_t capacity, int64_t* out_offsets, double* latency_ms,
                                    int32_t timeout_ms);

/* Counters and latency percentiles of the requests completed so far. */
rmips_status rmips_server_get_stats(rmips_server* server, rmips_server_stats* out);

/* Stops the threads (queued requests fail), waits for running batches and
   releases everything. */
void rmips_server_destroy(rmips_server* server);

/* Sizes and build statistics of an index. */
rmips_status rmips_index_get_info(const rmips_index* index, rmips_index_info* out);

/* Counters of the most recent rmips_query on this index (host thread safe,
   but "most recent" is only meaningful without concurrent queries). */
rmips_status rmips_last_query_stats(const rmips_index* index, rmips_query_stats* out);

/*
 * rmips_index_export -- copy one index array to host memory (for tests and
 * inspection).  field: 0 permQ (int32 [n], sorted position -> original id),
 * 1 permP (int32 [m]), 2 lower bounds (float [k_max][n], sorted positions),
 * 3 upper bounds (float [k_max][n]), 4 block minima L^j(B) (float
 * [k_max][n_blocks]), 5 block headers (float [n_blocks], upper bound of the
 * first user's norm), 6 user norms rounded up (float [n]), 7 item norms
 * rounded up (float [m]), 8 incomplete flags (uint8 [n]).
 * bytes must equal the field's size.  Synchronises the index's device.
 */
rmips_status rmips_index_export(const rmips_index* index, int32_t field, void* host_dst,
                                int64_t bytes);

/* Releases every device and host resource of the index.  NULL is ignored. */
void rmips_free_index(rmips_index* index);

/* Static description of a status code. */
const char* rmips_status_string(rmips_status status);

/* Message of the last failing call on this host thread ("" if none). */
const char* rmips_last_error(void);

/*
 * rmips_exact_sign_host -- sign of u.a - u.b in exact arithmetic, computed on
 * the host with the same integer accumulator the device recheck uses.
 * Returns -1, 0 or +1.  Exposed so the tie-breaking arithmetic can be checked
 * without a GPU.  Ordinary host function; d in 1..256.
 */
int32_t rmips_exact_sign_host(const float* u, const float* a, const float* b, int32_t d);

/*
 * rmips_debug_tc_tile -- test hook for the tensor-core tiles of the batched
 * filter (no counterpart in the paper).  Runs one 128 x 64 x 64 tile through
 * the shared-memory layout, UMMA descriptors (always the filter's own layout
 * constants), tcgen05.mma and TMEM loads the batched filter uses:
 * D[128][64] = A[128][64] * B[64][64]^T.
 * kind: 0 TF32, 1 BF16, 2 FP16 (A and B rounded to nearest into that format).
 * A, B, D: device float32, row-major.  Synchronises `stream`.
 * Errors: ARG, TIMEOUT, CUDA.
 */
rmips_status rmips_debug_tc_tile(const float* A, const float* B, float* D, int32_t kind, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RMIPS_H */
