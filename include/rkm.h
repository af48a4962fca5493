/*
 * rkm.h -- C ABI of the GB300 reverse k-MIPS top-N library (librkm.so).
 *
 * Problem (Amagata et al., "How to Mine Potentially Popular Items? A Reverse
 * MIPS-based Approach", arXiv 2504.13445, Section 2.1):
 *   users U (n x d), items P (m x d); item id = row index of P.
 *   Definition 1 (k-MIPS): S_k(u) = the k items with the largest u.p.
 *   Definition 2 / Eq. 1 (reverse k-MIPS): T_k(p) = {u : p in S_k(u)}.
 *   Definition 3: the N items with the largest score(p) = |T_k(p)|.
 * The paper breaks ties "arbitrarily"; this library fixes the order
 *   i before j for user u  <=>  u.p_i > u.p_j  or  (u.p_i == u.p_j and i < j)
 * for S_k(u), and "larger score, then smaller id" for the top N.  With t_u the
 * k-th item of u under that order and tau_u = u.p_{t_u}:
 *   i in S_k(u)  <=>  u.p_i > tau_u  or  (u.p_i == tau_u and i <= t_u).
 *
 * Exactness: tau_u is the FP64 value of u.p_{t_u}.  For inputs on the grid
 * 2^e * q / 4096 (integer |q| <= 4096, one exponent e per row) that value is
 * exact and every output below is bit-identical to exact arithmetic.  For
 * other FP32 inputs inner products are evaluated as a left-to-right FP64 sum
 * of exact FP64 products, and membership is decided on that value.
 *
 * Conventions shared by every entry point:
 *  - Matrices are row-major FP32; `ld*` is the row stride in elements (>= d)
 *    and must keep every row 4-byte aligned.
 *  - Pointers marked "device" are CUDA device pointers owned by the caller;
 *    the library reads or writes them only during the call.  Pointers marked
 *    "host" are ordinary host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call enqueues its kernels on that stream and returns
 *    after its results are complete: it reads back a device status word
 *    after each pass (the thresholds, the counting pass, each retry), so it
 *    synchronises `stream` a few times.
 *  - The context owns its scratch memory (device workspace grown on demand
 *    and kept until rkm_destroy).  Calls on one context are thread-safe: a
 *    mutex inside the context serialises calls made from several host
 *    threads (for concurrency, give each thread its own context); distinct
 *    contexts are independent.  rkm_destroy must not race with other calls
 *    on the same context.
 *  - Inputs are not required to lie on the 2^-12 grid.  Each call detects
 *    whether they do (a device flag set while the rows are prepared) and
 *    picks the exact integer rescoring for grid inputs, the FP64 one
 *    otherwise; rkm_stats.exact_integer_path reports which ran.
 *  - Errors never trap on the device.  A call returns a status code and
 *    rkm_last_error() describes it.  On error the outputs are unspecified.
 */
#ifndef RKM_H
#define RKM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RKM_API __attribute__((visibility("default")))
#else
#define RKM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rkm_ctx rkm_ctx;

typedef enum {
    RKM_OK = 0,
    RKM_EINVAL = 1,     /* bad argument (null pointer, size, k, N, ld)          */
    RKM_ENOMEM = 2,     /* device workspace allocation failed                   */
    RKM_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed          */
    RKM_EOVERFLOW = 4,  /* a candidate or band buffer overflowed after retries  */
    RKM_ETIMEOUT = 5,   /* a bounded device wait gave up                        */
    RKM_ESTATE = 6,     /* call out of order (e.g. query before resident set)   */
    RKM_EINTERNAL = 7,  /* a device-side consistency check failed               */
    RKM_EBUSY = 8,      /* serving: the request queue is full; submit again later */
    RKM_EIO = 9         /* a state file could not be written or read, or is corrupt */
} rkm_status;

typedef enum {
    RKM_FP32 = 0,  /* FP32 CUDA-core products, FP64/integer exact rescoring       */
    RKM_BF16 = 1,  /* BF16 tensor-core (tcgen05) products, FP32 accumulate,
                      guard band + exact rescoring                               */
    RKM_FP8 = 2    /* FP8 e4m3 tensor-core products (users scaled by 2^(8-e) per row,
                      items per 256-item tile, e = the row's or tile's exponent),
                      FP32 accumulate, guard band + exact rescoring               */
} rkm_precision;

typedef struct {
    rkm_precision precision; /* default RKM_BF16                                   */
    int k_max;               /* largest k accepted; default and maximum 64        */
    int cand_capacity;       /* initial per-user candidate capacity (0 = auto)     */
    int64_t band_capacity;   /* initial band-queue capacity in pairs (0 = auto)    */
    int filter;              /* rkm_topn: 1 = Eq. 2 item filter (default), 0 = off */
    int profile;             /* 1 = time each phase with CUDA events (rkm_stats)   */
    int autotune;            /* rkm_topn_batch: 1 = tune the counting tiles per size
                                bucket on first sight (default 0)                    */
    const char* tune_cache;  /* file that keeps autotuned choices across runs, or NULL */
    int scores_from_topk;    /* rkm_topn: 1 = scores as the histogram of the exact S_k(u)
                                lists of the threshold pass (the first Section 2.2
                                baseline: n*k increments, no counting pass and no Eq. 2
                                filter); 0 = counting pass with the filter (default)    */
    int epilogue_groups;     /* tensor-core product kernels: warpgroups that read each
                                accumulator tile back (0 = auto, 2, or 4: four split every
                                tile's columns between two groups, doubling the reads in
                                flight).  Auto: 2 for the threshold pass; for the counting
                                pass 4 when a tile is one K-block deep (BF16 d <= 64, FP8
                                d <= 128), else 2.  The threshold pass takes 4 only when
                                asked and four per-user heaps of k bounds fit (k <= 32).   */
    int seed_order;          /* tensor-core threshold pass: 1 = first a pass over the 2,048
                                highest-norm items gives each user a lower bound of tau_u,
                                users are grouped into tiles by bound / ||u|| and the bound
                                seeds the selector, so each tile's Cauchy-Schwarz stop comes
                                sooner (default; used when the items span 16 tiles or more,
                                the users fit one launch and a tile's product is two K-blocks
                                deep or more, i.e. BF16 d > 64); 0 = users in input order  */
} rkm_opts;

/* Phases timed when rkm_opts.profile is set (indices of rkm_stats.phase_ms). */
enum {
    RKM_PHASE_PREP = 0,      /* K1: norms, grid codes, item sort, operand packs    */
    RKM_PHASE_THRESHOLD = 1, /* K2: threshold product + per-user selector          */
    RKM_PHASE_EXACT = 2,     /* K3: exact tau_u / t_u from the candidates          */
    RKM_PHASE_BOUNDS = 3,    /* K4: ratios tau_u/||u||, user bucket sort, packs    */
    RKM_PHASE_COUNT = 4,     /* K5: counting product + classification              */
    RKM_PHASE_BAND = 5,      /* K6: exact rescoring of band pairs                  */
    RKM_PHASE_TOPN = 6,      /* K7: top-N select and the filter cut                */
    RKM_PHASE_TRANSFER = 7,  /* host<->device copies of rkm_topn_host              */
    RKM_PHASES = 8
};

typedef struct {
    uint64_t pairs_total;       /* n*m (thresholds) plus n*m or n*q (counting)   */
    uint64_t pairs_evaluated;   /* user-item products actually computed (both passes) */
    uint64_t candidates;        /* threshold-pass candidates rescored exactly     */
    uint64_t band_pairs;        /* counting-pass pairs rescored exactly           */
    uint64_t items_counted;     /* items whose score was computed (rkm_topn)      */
    int32_t retries;            /* capacity-overflow retries in the last call     */
    int32_t exact_integer_path; /* 1 if the last call rescored with integers      */
    double last_ms;             /* wall time of the last call, milliseconds       */
    uint64_t kernel_launches;   /* kernels this library launched in the last call */
    uint64_t threshold_launches;/* launches of the threshold product kernel       */
    double phase_ms[RKM_PHASES];/* device time per phase (profile = 1), ms        */
    uint64_t threshold_pairs;   /* products computed by the threshold pass (n*m less
                                   the item tiles its Cauchy-Schwarz stop skipped)  */
} rkm_stats;

/* Fill `opts` with the defaults listed above. */
RKM_API void rkm_default_opts(rkm_opts* opts);

/* Create a context on CUDA device `device`.  `opts` may be NULL (defaults).
 * Returns RKM_EINVAL for a bad option, RKM_ECUDA if the device is unusable. */
RKM_API rkm_status rkm_create(rkm_ctx** out, const rkm_opts* opts, int device);

/* Free the context and its device workspace.  NULL is accepted. */
RKM_API void rkm_destroy(rkm_ctx* ctx);

/* Message for the last error on this host thread ("" if none). */
RKM_API const char* rkm_last_error(void);

/* Library version string. */
RKM_API const char* rkm_version(void);

/*
 * Thresholds -- Definition 1 for every user (the k-MIPS step of the first
 * Section 2.2 baseline, which Algorithm 1 approximates with A_i^k).
 *   U: device, n x d (stride ldu); P: device, m x d (stride ldp).
 *   1 <= k <= min(m, k_max); n >= 0 (n == 0 is a no-op); 1 <= d <= 256;
 *   n, m < 2^31.
 *   tau:  device, [n] double  -- tau_u (a zero threshold is +0.0).
 *   tid:  device, [n] int32   -- t_u, the k-th item of u.
 *   topk: device, [n * k] int32 or NULL -- S_k(u) in order, row u at u*k.
 */
RKM_API rkm_status rkm_thresholds(rkm_ctx* ctx, const float* U, int64_t n, int64_t ldu,
                          const float* P, int64_t m, int64_t ldp, int d, int k,
                          double* tau, int32_t* tid, int32_t* topk, void* stream);

/*
 * Scores -- Eq. 1 / the second Section 2.2 baseline: score(p_i) = |T_k(p_i)|
 * for every item, counted against given thresholds (tau, tid as produced by
 * rkm_thresholds for the same U, P, k).
 *   scores: device, [m] int32.
 */
RKM_API rkm_status rkm_scores(rkm_ctx* ctx, const float* U, int64_t n, int64_t ldu,
                      const float* P, int64_t m, int64_t ldp, int d,
                      const double* tau, const int32_t* tid, int32_t* scores,
                      void* stream);

/*
 * Top-N -- Definition 3: thresholds, then item scores (skipping, when the
 * filter option is on, every item whose Eq. 2 upper bound cannot reach the
 * N-th score, in the spirit of Algorithm 2), then the N best items.
 *   1 <= N <= min(m, 4096).  ids: device [N] int32; top_scores: device [N] int32, in
 *   order (score descending, id ascending).
 *   tau, tid: device [n] or NULL -- the thresholds computed on the way.
 */
RKM_API rkm_status rkm_topn(rkm_ctx* ctx, const float* U, int64_t n, int64_t ldu,
                    const float* P, int64_t m, int64_t ldp, int d, int k, int N,
                    int32_t* ids, int32_t* top_scores, double* tau, int32_t* tid,
                    void* stream);

/*
 * Top-N for any k <= kmax from one threshold pass -- the offline/online split of the
 * paper (Section 4: pre-processing done once, then queries for a given N and k; k_max, the
 * largest k, is fixed in Section 2.1).  Under the
 * order above S_k(u) is the first k entries of S_kmax(u), so with lists = the `topk`
 * output of rkm_thresholds at kmax, score_k(p) = #{u : p among the first k of u's list}
 * and Definition 3 follows without another product pass.
 *   lists: device [n * kmax] int32 (row u at u*kmax); 1 <= k <= min(kmax, m);
 *   1 <= N <= min(m, 4096); ids, top_scores: device [N] int32 as for rkm_topn.
 *   An id outside [0, m) in the first k entries of a row returns RKM_EINVAL.
 */
RKM_API rkm_status rkm_topn_from_topk(rkm_ctx* ctx, const int32_t* lists, int64_t n, int kmax, int k,
                                      int64_t m, int N, int32_t* ids, int32_t* top_scores, void* stream);

/* rkm_topn with HOST buffers: copies U and P to the device (inside the call),
 * runs rkm_topn and copies ids and top_scores back.  All pointers are host. */
RKM_API rkm_status rkm_topn_host(rkm_ctx* ctx, const float* U, int64_t n, int64_t ldu,
                         const float* P, int64_t m, int64_t ldp, int d, int k, int N,
                         int32_t* ids, int32_t* top_scores, void* stream);

/*
 * Item upper bounds -- Eq. 2 with A_i^k = tau_u (Section 4.1):
 * uscore[i] >= #{u : ||u|| ||p_i|| >= tau_u} >= score(p_i) (Theorem 2).
 * The count is taken over users bucketed by tau_u / ||u|| (rounded outward),
 * so it can exceed the exact count by the users of one bucket.
 *   uscore: device [m] int32.
 */
RKM_API rkm_status rkm_item_bounds(rkm_ctx* ctx, const float* U, int64_t n, int64_t ldu,
                           const float* P, int64_t m, int64_t ldp, int d,
                           const double* tau, int32_t* uscore, void* stream);

/*
 * Guard-band check -- the approximate products of the context's tensor-core path and their
 * error bounds, for validating the bound that makes the guarded paths exact (the paper's
 * algorithms are exact on the CPU and have no counterpart).  For every user u and item i,
 *   v[u * ldo + i] = the product the threshold and counting kernels compute for (u, i):
 *                    BF16 or FP8 e4m3 operands (FP8 scaled by powers of two per user row and
 *                    per 256-item tile of the norm-sorted items, then descaled), same TMA
 *                    boxes, swizzle, tcgen05 MMA shape and FP32 accumulation;
 *   E[u * ldo + i] = the bound E those kernels use for that pair, so that |v - u.p| <= E
 *                    must hold for every pair.
 *   U: device n x d (stride ldu), 0 <= n <= 65536; P: device m x d (stride ldp),
 *   0 <= m <= 2^20; v, E: device [n * ldo] float, ldo >= m.  RKM_EINVAL on the FP32 path.
 * The product kernels skip 64-column blocks of a tile on the row maximum that the TMEM load
 * instruction returns with the values (tcgen05.ld with .red.max); this call checks that
 * maximum against the values it loads and returns RKM_EINTERNAL if they ever differ.
 */
RKM_API rkm_status rkm_debug_products(rkm_ctx* ctx, const float* U, int64_t n, int64_t ldu,
                                      const float* P, int64_t m, int64_t ldp, int d,
                                      float* v, float* E, int64_t ldo, void* stream);

/*
 * Timeout-path check (no counterpart in the paper; a library service for failure handling).
 * Every wait inside this library's kernels gives up after a bounded number of SM clocks,
 * records the timeout in the context's status word and lets the kernel return, so a stalled
 * wait never hangs the device.  This call runs that bounded wait, with a limit of
 * `wait_cycles` clocks (1 <= wait_cycles <= 2^32), on a barrier that nothing completes: it
 * returns RKM_ETIMEOUT, and the context remains usable for later calls.
 */
RKM_API rkm_status rkm_debug_wait_timeout(rkm_ctx* ctx, int64_t wait_cycles, void* stream);

/*
 * Serving -- keep users and their thresholds resident, then score new
 * candidate items (Definition 2 for an item whose id exceeds every catalogue
 * id, so a tie at tau_u does not make it a member; the catalogue and the
 * thresholds are not updated).
 * rkm_resident_set copies what it needs from U, tau, tid into the context.
 */
RKM_API rkm_status rkm_resident_set(rkm_ctx* ctx, const float* U, int64_t n, int64_t ldu, int d,
                            const double* tau, const int32_t* tid, void* stream);

/*   Q: device, q x d (stride ldq), q >= 0.  counts: device [q] int32,
 *   counts[j] = #{u : u.Q_j > tau_u}.  Returns RKM_ESTATE without a resident set. */
RKM_API rkm_status rkm_query_new_items(rkm_ctx* ctx, const float* Q, int64_t q, int64_t ldq,
                               int32_t* counts, void* stream);

/*
 * Serving state on disk: the resident users and their thresholds (U, tau, tid as given to
 * rkm_resident_set), so that a serving process can restart without the threshold pass (the
 * paper's pre-processing is done once and reused, Section 4).  The file holds a header, the
 * three arrays and an FNV-1a hash of them; loading recomputes everything derived from them
 * (norms, grid codes, ratio order, operand packs) exactly as rkm_resident_set does.
 * rkm_state_save: RKM_ESTATE without a resident set, RKM_EIO when the file cannot be written.
 * rkm_state_load: replaces the context's resident set; RKM_EIO when the file cannot be read,
 * is not a state file, is truncated or fails its hash (the resident set is then unchanged);
 * RKM_ESTATE while a serving loop uses the context.  Synchronises `stream`.
 */
RKM_API rkm_status rkm_state_save(const rkm_ctx* ctx, const char* path);
RKM_API rkm_status rkm_state_load(rkm_ctx* ctx, const char* path, void* stream);

/* Counters of the last call. */
RKM_API rkm_status rkm_get_stats(const rkm_ctx* ctx, rkm_stats* out);

/* One problem of a batch: device inputs and outputs as for rkm_topn. */
typedef struct {
    const float* U;
    int64_t n, ldu;
    const float* P;
    int64_t m, ldp;
    int d, k, N;
    int32_t* ids;         /* device [N] */
    int32_t* top_scores;  /* device [N] */
} rkm_instance;

/*
 * Batch of independent top-N problems (Definition 3 for each).  The tensor-core threshold
 * products of all instances run in one persistent launch (work units = user tiles of every
 * instance, largest instances first); the whole sequence of kernels is captured into a CUDA
 * graph on the first call with a given batch layout (same pointers, sizes and options) and
 * replayed by later calls with that layout.  Results equal rkm_topn on each instance: an
 * instance whose candidate or band buffers overflow inside the graph is recomputed by the
 * retrying single-instance path (and the graph is rebuilt on the next call).  With
 * opts.autotune, the first sight of a size bucket (d, k, log2 n, log2 m) times the counting
 * pass's work-unit size and first-stage size on that instance and keeps the fastest (in
 * opts.tune_cache when given).  1 <= count <= 4096.  Synchronises `stream`.
 */
RKM_API rkm_status rkm_topn_batch(rkm_ctx* ctx, const rkm_instance* inst, int count, void* stream);

/*
 * Top-N of a score array without allocating device memory (the paper has no counterpart:
 * this is a library service).  For callers that cannot call cudaMalloc -- a process that
 * reserves all device memory up front and forbids later allocations, or code that runs
 * inside another library's memory manager with only the buffers it was given.
 *   scores: device [m] int32 (e.g. from rkm_scores), 1 <= m < 2^31; any int32 value,
 *   negative ones included, orders as a signed integer.
 *   ids, top_scores: device [N] int32, filled in order (score descending, id ascending),
 *   1 <= N <= min(m, 4096); a larger N returns RKM_EINVAL.
 * No context: the only scratch is a fixed 32 KB device array inside the library (one per
 * device that loads it, kept until the process exits); nothing is allocated or freed.  The
 * first call on a device looks up that array's address (a runtime call), so make it before
 * any stream capture on that device; the address is kept for the life of the process, so the
 * library must not be used on a device across a device reset.  Every call shares the array
 * and clears what it needs;
 * calls that overlap on the GPU race on it and must be serialised by the caller.  The call
 * synchronises `stream` to read its status word.
 */
RKM_API rkm_status rkm_topn_scores_noalloc(const int32_t* scores, int64_t m, int N, int32_t* ids,
                                           int32_t* top_scores, void* stream);

/*
 * Serving loop -- a request loop over the resident users and thresholds of a context (set by
 * rkm_resident_set), scoring new candidate items as rkm_query_new_items does.  Requests are
 * queued by rkm_serve_submit and served by `slots` worker threads, each with its own CUDA
 * stream and workspace.  A worker that becomes free takes the oldest waiting requests, as
 * many as fit both `max_batch_items` candidates and the free part of a device arena of
 * `memory_bytes` that holds the admitted requests' candidate rows and counts (continuous
 * batching: requests that arrive while other batches are on the GPU join the next batch
 * that a slot and memory allow), copies them to the device, runs one counting pass over the
 * users for the whole batch, and hands each request its counts.  Batches of different slots
 * overlap on the device.  A request's counts do not depend on which batch it joins.
 *
 * The server borrows the context: while it exists, the context's resident users must not be
 * replaced (rkm_resident_set returns RKM_ESTATE) and the context must not be destroyed.
 * Server calls are thread-safe; any host thread may submit and wait.
 */
typedef struct rkm_server rkm_server;

typedef struct {
    int slots;               /* concurrent batches (worker threads + streams); default 2, 1..16   */
    int64_t max_batch_items; /* candidates per batch, and the largest request; default 8192      */
    int64_t memory_bytes;    /* device arena for admitted requests' rows and counts; default
                                64 MiB.  A request needing more is rejected (RKM_EINVAL).         */
    int64_t max_pending;     /* requests queued (not yet admitted) before submit returns
                                RKM_EBUSY; default 1048576                                      */
} rkm_serve_opts;

typedef struct {
    uint64_t submitted;        /* requests accepted since the last reset                         */
    uint64_t completed;        /* requests finished, including failed ones                      */
    uint64_t failed;           /* requests finished with an error status                        */
    uint64_t items;            /* candidates scored by completed requests                       */
    uint64_t batches;          /* counting passes over the resident users                       */
    double mean_batch_items;   /* items / batches                                                */
    double p50_ms, p99_ms;     /* latency percentiles (nearest rank): submit -> counts written  */
    double mean_ms, max_ms;    /* mean and largest latency                                       */
    double mean_queue_ms;      /* submit -> admission into a batch, averaged                     */
    double window_ms;          /* first submission -> last completion                            */
    double items_per_s;        /* items / window                                                 */
    double pairs_per_s;        /* resident users * items / window                                */
    int64_t arena_peak_bytes;  /* most arena bytes held by admitted requests at once              */
    int32_t max_in_flight;     /* most batches admitted and not yet finished at once             */
    int32_t slots;             /* worker slots of the server                                      */
    uint64_t kernel_launches;  /* kernels launched by all slots since the last reset             */
} rkm_serve_stats;

/* Fill `opts` with the defaults listed above. */
RKM_API void rkm_serve_default_opts(rkm_serve_opts* opts);

/* Start a server on `ctx`, whose resident set must exist (else RKM_ESTATE).  `opts` may be
 * NULL.  Allocates the arena, each slot's workspace (sized by one warm-up pass of
 * max_batch_items zero candidates) and pinned staging, then starts the worker threads. */
RKM_API rkm_status rkm_serve_create(rkm_server** out, rkm_ctx* ctx, const rkm_serve_opts* opts);

/* Queue one request: Q host [q x d] FP32 (stride ldq >= d, d = the resident users' d),
 * 1 <= q <= max_batch_items; counts host [q] int32 receives #{u : u.Q_j > tau_u}.  Both
 * buffers are borrowed until rkm_serve_wait reports the ticket finished.  Returns RKM_EBUSY
 * when max_pending requests are waiting, RKM_ESTATE after the server started stopping. */
RKM_API rkm_status rkm_serve_submit(rkm_server* srv, const float* Q, int64_t q, int64_t ldq, int32_t* counts,
                                    uint64_t* ticket);

/* Wait for a request.  timeout_ms < 0 waits without limit.  Returns the request's own status
 * (its error message becomes this thread's rkm_last_error) and releases the ticket; returns
 * RKM_ETIMEOUT, keeping the ticket, if it has not finished in time; RKM_EINVAL for an unknown
 * ticket.  latency_ms (may be NULL) receives submit -> finish. */
RKM_API rkm_status rkm_serve_wait(rkm_server* srv, uint64_t ticket, double timeout_ms, double* latency_ms);

/* Block until no request is queued or running. */
RKM_API rkm_status rkm_serve_drain(rkm_server* srv);

/* Counters since creation or the last rkm_serve_reset_stats. */
RKM_API rkm_status rkm_serve_get_stats(rkm_server* srv, rkm_serve_stats* out);
RKM_API rkm_status rkm_serve_reset_stats(rkm_server* srv);

/* Finish every queued request, stop the workers and free the server (tickets not yet waited
 * for are released).  NULL is accepted. */
RKM_API void rkm_serve_destroy(rkm_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* RKM_H */
