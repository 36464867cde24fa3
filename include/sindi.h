/*
 * sindi.h — C ABI of the GB300 (sm_103a) implementation of SINDI's search
 * hot path (arXiv 2509.08395, "SINDI: an Efficient Index for Sparse Vector
 * Approximate Maximum Inner Product Search").
 *
 * What the library computes
 *   Build (Algorithm 3, with Algorithm 1 inside): every document x_i is cut
 *   to its alpha-mass subvector (Sec. 4.1, Definition "alpha-Mass
 *   Subvector"); the kept entries become value-storing inverted lists
 *   (Sec. 3.1) split into windows of lambda document ids, I_{j,w}
 *   (Sec. 3.3.1). The unpruned documents stay on the device for reordering.
 *   Search (Algorithm 4, with Algorithm 2 inside): for every window w and
 *   every query term q^j, A[i mod lambda] += q^j * x_i^j over I_{j,w}; the
 *   best gamma (score, id) pairs over all windows are the candidates; their
 *   exact inner products delta(x_i, q) (Definition 2) on the full vectors
 *   give the top-k.
 *
 * Conventions shared by every call
 *   - Sparse matrices are CSR: indptr int64[n+1] (indptr[0] = 0,
 *     non-decreasing), indices int32[nnz] (dims in [0, dim), unique within a
 *     row, any order), values float32[nnz] (finite). Explicit zeros are not
 *     entries (Definition 1) and are ignored.
 *   - Pointers may be host or device memory; the library asks the CUDA
 *     driver which. All inputs of one call must be of one kind, and all
 *     outputs of one kind.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   - Order of results: larger score first; equal scores: lower document
 *     id first (the paper does not fix tie order).
 *   - The caller owns every buffer it passes. The library owns the index
 *     and all scratch memory it allocates (stream-ordered, from a pool of
 *     its own that keeps freed blocks for reuse).
 *   - Errors: invalid arguments are reported before any device work with
 *     SINDI_ERR_INVALID_ARG. Malformed data is found on the device; it sets
 *     the index's error word, which sindi_build returns at once and which a
 *     search returns when it synchronises (host buffers) or on the next
 *     sindi_check. No exception crosses the ABI; sindi_last_error() holds a
 *     message for the calling thread.
 *   - An index is never modified by a search, so searches on different
 *     streams may run concurrently.
 */
#ifndef SINDI_H
#define SINDI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sindi_index sindi_index;

typedef enum {
    SINDI_OK = 0,
    SINDI_ERR_INVALID_ARG = 1,   /* bad pointer, size or parameter; nothing ran            */
    SINDI_ERR_INVALID_DATA = 2,  /* malformed CSR contents found on the device             */
    SINDI_ERR_OOM = 3,           /* device memory exhausted                                 */
    SINDI_ERR_CUDA = 4,          /* a CUDA call failed (message in sindi_last_error)        */
    SINDI_ERR_TIMEOUT = 5,       /* a bounded device wait gave up                           */
    SINDI_ERR_UNSUPPORTED = 6    /* valid but outside what this build handles              */
} sindi_status;

/* Storage type of posting values (the reduced-precision form; the paper
   stores full-precision values). Accumulation is FP32 in every case. */
typedef enum {
    SINDI_F32 = 0,
    SINDI_F16 = 1,      /* IEEE binary16, round to nearest even               */
    SINDI_F8E4M3 = 2    /* OCP FP8 E4M3 with one FP32 scale per list I_j:
                           scale_j = max|x| over I_j / 448; code = RNE(x / scale_j),
                           saturating; the stored value is code * scale_j    */
} sindi_dtype;

/* Search schedule. Both give the same results (within FP32 rounding). */
typedef enum {
    SINDI_MODE_PLAIN = 0,    /* one query per launch sequence                         */
    SINDI_MODE_BATCHED = 1   /* all queries of the call in shared launches             */
} sindi_mode;

/* Which entries of the documents become postings (Sec. 4.1 names three
   pruning methods and the ablation of Sec. 5 also combines two):
   - MASS (Mass Ratio Pruning, the method's own): every document keeps its
     alpha-mass subvector, the shortest prefix of its entries in pi order
     (|x| descending; equal |x|: lower dim first) whose |x| sum reaches
     alpha * mass(x).
   - VECTOR_NUMBER (Vector Number Pruning): every document keeps the first
     min(prune_n, nnz) entries in pi order.
   - LIST (List Pruning): every list I_j (all windows) keeps its prune_n
     entries of largest |x|; equal |x|: lower document id first.
   - MASS_LIST: MASS first, then LIST on the lists MASS leaves.
   The unpruned documents are kept for reordering in every case. */
typedef enum {
    SINDI_PRUNE_MASS = 0,
    SINDI_PRUNE_VECTOR_NUMBER = 1,
    SINDI_PRUNE_LIST = 2,
    SINDI_PRUNE_MASS_LIST = 3
} sindi_prune;

/* Parameters of Algorithm 3. A zero-filled struct with alpha = 1 is the
   unpruned index. */
typedef struct {
    uint32_t window;       /* lambda, documents per window (Sec. 3.3.1); 1..32768.
                              0 picks a default. A window's score array (4 bytes a
                              slot) lives in one thread block's shared memory.    */
    int32_t value_dtype;   /* sindi_dtype                                          */
    double alpha;          /* document pruning ratio in (0, 1]; 1 = no pruning.
                              Used by MASS and MASS_LIST, ignored otherwise      */
    int32_t prune;         /* sindi_prune                                          */
    uint32_t prune_n;      /* VECTOR_NUMBER: entries kept per document; LIST and
                              MASS_LIST: entries kept per list; >= 1 for those,
                              ignored by MASS                                     */
} sindi_build_params;

/* sindi_search_params.block_threads value of the pipelined window scan. */
#define SINDI_SCAN_PIPELINED 1u

/* The score window of the coarse scan (sindi_search_params.accumulator).

   F32: Alg. 2 as written: every product q_j * x_ij (FP32) is added into the
   window's FP32 score array (shared-memory FP32 atomicAdd).

   FIXED32: the window holds 32-bit integers in units of 2^-e. Each product is
   rounded to the nearest unit and added with an integer atomicAdd (native
   in shared memory, where an FP32 atomicAdd is a compare-and-swap loop); the
   sums are exact and do not depend on the order of the adds. The sums are
   converted to FP32 (times 2^-e) before the window's top-gamma cut, so the
   cut, merge and reorder are unchanged. Per (query, window):
     B = sum of |q_j| * vmax_j over the query's terms whose list I_{j,w} is
         not empty, vmax_j = the largest |stored value| of list I_j (all
         windows, after pruning; for E4M3 lists q_j includes the list scale),
     e = 30 - x, where 2^(x-1) <= B < 2^x (e = 0 when B = 0), clamped to
         [-126, 126] and so that |q_j| * 2^e stays below 2^127,
   so every window sum stays below 2^31 in magnitude. A coarse score of m
   products, a = the sum of their magnitudes, is then within
   2^-23 * a + m * 2^-(e+1) of the exact score (the FP32 rounding of each
   product and of the final conversion, plus half a unit per product); with e
   unclamped, m * 2^-(e+1) <= m * B * 2^-30.

   AUTO (the default): FIXED32 when the search reorders (gamma > 0; the
   window scores only choose the candidates that the exact FP32 reorder
   scores), F32 when the window scores are the answer (gamma = 0). The
   pipelined scan and the query-group scan always use F32. */
typedef enum {
    SINDI_ACCUM_AUTO = 0,
    SINDI_ACCUM_F32 = 1,
    SINDI_ACCUM_FIXED32 = 2
} sindi_accumulator;

/* Parameters of Algorithm 4. */
typedef struct {
    uint32_t k;            /* results per query, 1..1024                            */
    uint32_t gamma;        /* reorder pool size; 0 = no reordering (the coarse
                              top-k is the answer), else k <= gamma <= 8192        */
    double beta;           /* query pruning ratio in (0, 1]; 1 = off. With beta < 1
                              the coarse scan uses beta-mass(q) (Alg. 4) and
                              the reorder the full q. Supported by sindi_search;
                              plans, servers and sindi_search_noalloc return
                              SINDI_ERR_UNSUPPORTED for beta < 1                    */
    uint32_t mode;         /* sindi_mode                                           */
    uint32_t block_threads;/* window-scan shape: 0 = the default (one block of 512
                              threads per window); 256, 512 or 1024 = one block
                              of that many threads per window;
                              SINDI_SCAN_PIPELINED = one resident block per SM
                              that overlaps the scatter-add of one window with
                              the cut of the previous (lambda <= 16384; larger
                              windows take the default)                         */
    uint32_t group;        /* batched schedule: queries per scan block, 0..8. One
                              block owns a window for a group of this many queries
                              (their score windows side by side in shared memory)
                              and loads each posting of a list segment I_{j,w} once
                              for every query of the group that holds term j.
                              0 or 1 = one block per (query, window), the default.
                              A value larger than shared memory holds (its group's
                              windows and 36 KiB of tables within 207 KiB) is
                              reduced to what fits. Ignored by the plain schedule
                              and by SINDI_SCAN_PIPELINED                         */
    uint32_t accumulator;  /* sindi_accumulator; 0 = AUTO                          */
} sindi_search_params;

typedef struct {
    int64_t n_docs;        /* ||D||                                               */
    int32_t dim;           /* d                                                   */
    int32_t value_dtype;   /* sindi_dtype                                         */
    uint32_t window;       /* lambda                                              */
    uint32_t n_windows;    /* sigma = ceil(||D|| / lambda)                        */
    int64_t postings;      /* kept entries = sum of |alpha-mass(x_i)|             */
    int64_t doc_nnz;       /* entries of the unpruned documents                   */
    int64_t index_bytes;   /* device bytes of lists + offsets + scales            */
    int64_t doc_bytes;     /* device bytes of the unpruned documents              */
    double alpha;
    int32_t prune;         /* sindi_prune of the build                            */
    uint32_t prune_n;      /* its prune_n (0 for MASS)                            */
} sindi_index_info_t;

/* Counters of the calling index (for benchmarks). */
typedef struct {
    uint64_t launches;         /* kernels launched by searches on this index     */
    uint64_t scan_launches;    /* of which window-scan kernels                    */
    uint64_t queries;          /* queries searched                                */
    double scan_ms;            /* summed CUDA-event time of scan kernels while
                                  timing is on (see sindi_set_timing)              */
    uint64_t scan_timed;       /* scan launches included in scan_ms               */
} sindi_stats_t;

/*
 * Build an index (Algorithm 3: alpha-mass every document, then Algorithm 1
 * over the pruned documents, with the lists split into windows as in
 * Sec. 3.3.1). Postings are sorted by (dim, document) on the device and
 * stored as the 16-bit window-local id i mod lambda beside the value; inside
 * a list I_{j,w} they are ordered for the scan's shared-memory scatter-add
 * (the postings one warp instruction adds sit in different banks), which
 * changes scores only by FP32 rounding. With prune != MASS the other pruning
 * methods of Sec. 4.1 apply (see sindi_prune).
 *   indptr/indices/values: the documents (CSR, see conventions), n_docs rows,
 *       n_docs < 2^32 - 1, dims in [0, dim).
 *   params: see sindi_build_params. NULL = window 0, FP32, alpha 1.
 *   stream: the stream the build runs on; the call returns when it is done.
 *   out: receives the new index (owned by the caller, free with
 *       sindi_index_free). Untouched on error.
 * Returns SINDI_ERR_INVALID_DATA for a malformed CSR (decreasing indptr, dim
 * out of range, duplicate dim in a row, non-finite value) and
 * SINDI_ERR_UNSUPPORTED for a row with more than 16384 entries or more than
 * 2^32 - 4096 kept entries in total.
 */
sindi_status sindi_build(const int64_t* indptr, const int32_t* indices, const float* values,
                         int64_t n_docs, int32_t dim, const sindi_build_params* params,
                         void* stream, sindi_index** out);

/*
 * Search a batch of queries (Algorithm 4 per query, with Algorithm 2 for the
 * coarse stage and exact reordering of the gamma candidates).
 *   q_indptr/q_indices/q_values: the queries (CSR), n_queries rows (>= 0).
 *   params: see sindi_search_params (not NULL).
 *   out_ids:    uint32 [n_queries * k], row-major; document ids.
 *   out_scores: float  [n_queries * k]; delta(x_i, q) in FP32 when gamma > 0,
 *               else the coarse score. When the index has fewer than k
 *               documents, the tail of each row is id 0xFFFFFFFF, score -inf.
 *   stream: device inputs and outputs: the search is queued on the stream and
 *       the call returns at once. Host inputs or outputs: the call copies
 *       through device memory and returns when the results are in place.
 * Malformed queries (dim out of range, duplicate dim, non-finite value) set
 * the index's error word; they never read outside the index.
 * Plain schedule: several queries' launch chains run at once on streams of
 * the index (forked from and joined to `stream`). When the same call (same
 * buffers, n_queries, k, gamma and block shape; beta = 1; timing off; stream
 * not being captured) comes a second time, its launches are recorded as one
 * CUDA graph with working memory of its own (held until the index is freed
 * or another call is recorded); identical calls then launch the graph, which
 * reads the buffers' current contents. A plain call on a stream that is not
 * being captured first waits (on the GPU) for the graph's previous launch, so
 * launches from different streams never share its working memory at once.
 */
sindi_status sindi_search(const sindi_index* index, const int64_t* q_indptr, const int32_t* q_indices,
                          const float* q_values, int64_t n_queries, const sindi_search_params* params,
                          uint32_t* out_ids, float* out_scores, void* stream);

/*
 * The same search as sindi_search, for callers that cannot allocate device
 * memory while they run: an application that fixes its memory budget at start
 * and forbids later allocation, a host framework that owns every device
 * allocation itself, or a latency-critical loop in which the implicit
 * synchronisation of an allocation is not acceptable. The paper has no
 * counterpart to this call.
 *   All working memory comes from one static device array of 8 MiB
 *   (SINDI_NOALLOC_SCRATCH_BYTES) inside the library, which every GPU that loads
 *   the library holds until the process exits. The call allocates nothing:
 *   no cudaMalloc, no pool, no staging.
 *   Arguments and results are those of sindi_search, except that the queries
 *   and both outputs must be device memory (SINDI_ERR_INVALID_ARG otherwise).
 *   A search whose working memory for one query exceeds the array returns
 *   SINDI_ERR_UNSUPPORTED with the sizes in sindi_last_error(). One query
 *   needs, with g = min(gamma (k when gamma = 0), n_docs) and each term
 *   rounded up to 256 bytes: 16,404 bytes of counters and histogram, plus
 *   n_windows * 2 * min(g, window) * 8 bytes of window candidates, plus
 *   f * 8 bytes of merge filter (f = the smallest power of two >= 4096 and
 *   >= 2 g, at most 16384), plus 2 * g * 8 bytes of reorder keys (16 bytes
 *   when gamma = 0). Batched mode processes as many queries per launch group
 *   as fit.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current) and keeps it; make that
 *   first call before any stream capture.
 *   Every call uses the same array and clears the counters it starts from.
 *   Calls whose work overlaps on the GPU (other streams, other threads, other
 *   indexes) race on the array and give undefined results: order them on one
 *   stream or synchronise between them.
 */
#define SINDI_NOALLOC_SCRATCH_BYTES (8u << 20)
sindi_status sindi_search_noalloc(const sindi_index* index, const int64_t* q_indptr, const int32_t* q_indices,
                                  const float* q_values, int64_t n_queries, const sindi_search_params* params,
                                  uint32_t* out_ids, float* out_scores, void* stream);

/*
 * Merge the result rows of a document-sharded search (one index per range of
 * document ids, e.g. one per GPU): the top-k over all documents is the top-k
 * of the shards' top-k lists, because windows, and so shards aligned to
 * them, are independent (Sec. 3.3.1; Alg. 2 visits windows one by one and
 * its heap keeps the best over all of them).
 *   ids, scores: [n_shards][n_queries][k_in] device arrays, each shard's rows
 *       as sindi_search writes them (local ids, best first, padding id
 *       0xFFFFFFFF / score -inf, which is skipped).
 *   id_offset: int64 [n_shards] host array; shard s's local id i is global id
 *       id_offset[s] + i (0 <= id_offset[s] < 0xFFFFFFFF; the ranges must not
 *       overlap and global ids must stay below 0xFFFFFFFF).
 *   out_ids / out_scores: [n_queries][k] device arrays: the best k entries by
 *       (score desc, global id asc), padded when fewer exist.
 *   1 <= n_shards <= 64, n_shards * k_in <= 8192, 1 <= k <= 1024. Runs on the
 *   current device, queued on `stream`; SINDI_ERR_INVALID_ARG for sizes out
 *   of range or host pointers. The paper searches one machine; this call
 *   serves the multi-GPU split only.
 */
sindi_status sindi_merge_topk(const uint32_t* ids, const float* scores, int32_t n_shards, int64_t n_queries,
                              uint32_t k_in, const int64_t* id_offset, uint32_t k, uint32_t* out_ids,
                              float* out_scores, void* stream);

/*
 * Graph-captured batched search. Records the whole search of one query batch
 * (the batched schedule of sindi_search: every query of the batch in shared
 * launches) as a CUDA graph, so that each later run is one graph launch.
 *   The query and output device buffers given here are baked into the graph;
 *   the caller may change their contents between launches, but not their
 *   addresses, n_queries or the total number of query entries beyond what the
 *   buffers hold. Device pointers only; 1 <= n_queries <= 65535.
 *   The plan owns its workspace (allocated here, at most 4 GiB or what one
 *   query needs: a batch whose working memory exceeds that is recorded as
 *   several launch groups that reuse it, still replayed by one graph launch).
 *   Launches of one plan must not overlap each other on the GPU. The index
 *   must outlive the plan.
 */
typedef struct sindi_plan sindi_plan;
sindi_status sindi_plan_create(const sindi_index* index, const int64_t* q_indptr, const int32_t* q_indices,
                               const float* q_values, int64_t n_queries, const sindi_search_params* params,
                               uint32_t* out_ids, float* out_scores, sindi_plan** out);
/* Queue one run of the plan on `stream`. */
sindi_status sindi_plan_launch(sindi_plan* plan, void* stream);
void sindi_plan_free(sindi_plan* plan);

/* ---------------------------------------------------------------------------
 * Serving (continuous batching). The paper's algorithm is per query
 * (Algorithm 4); the server runs it for a stream of independent requests.
 * A worker thread inside the library takes queued requests in arrival order,
 * forms micro-batches of at most max_batch queries and starts each batch as
 * soon as a device slot is free. A slot is one CUDA stream with its own
 * pinned staging buffers, device query/result buffers and search workspace,
 * all allocated when the server is created. So requests that arrive while
 * others run are admitted as slots free up, and up to n_slots batches overlap
 * on the device. The index stays resident and is shared by all slots.
 * ------------------------------------------------------------------------- */
typedef struct sindi_server sindi_server;

typedef struct {
    uint32_t max_batch;        /* queries per micro-batch, 1..4096 (0 = 256)               */
    uint32_t max_slots;        /* batches in flight on the device, 1..64 (0 = 4)           */
    uint32_t max_query_nnz;    /* longest accepted query, 1..2048 (0 = 512)                */
    uint32_t max_wait_us;      /* how long a partial batch may wait for more requests while
                                  every slot is busy anyway (0 = do not wait)              */
    uint64_t memory_budget;    /* device bytes the slots may take (0 = no limit). Slots are
                                  admitted while they fit: fewer than max_slots if needed;
                                  SINDI_ERR_OOM if not even one fits                       */
    sindi_search_params search;/* k, gamma, beta of every request (mode is ignored)        */
} sindi_server_params;

typedef struct {
    uint64_t submitted, completed, failed, batches;
    uint32_t n_slots;          /* slots admitted by the memory budget                      */
    uint32_t peak_in_flight;   /* most batches seen on the device at once                  */
    uint64_t slot_bytes;       /* device bytes of one slot                                 */
    double mean_batch;         /* queries per batch                                        */
    double p50_ms, p99_ms, max_ms; /* request latency, submit -> results on the host,
                                  over requests completed since the last stats reset       */
} sindi_server_stats_t;

/* Create a server over `index` (which must outlive it). */
sindi_status sindi_server_create(const sindi_index* index, const sindi_server_params* params, sindi_server** out);

/* Queue one query: nnz entries (host arrays, copied before the call returns).
   *ticket identifies the request for sindi_server_poll. SINDI_ERR_INVALID_ARG
   if nnz exceeds max_query_nnz or the server is shutting down. */
sindi_status sindi_server_submit(sindi_server* server, const int32_t* q_indices, const float* q_values, int32_t nnz,
                                 uint64_t* ticket);

/* Wait up to wait_ms (0 = just look, < 0 = no limit) for a request. When it is
   done, copies its k ids and scores (as sindi_search writes one row) into the
   host buffers, sets *latency_ms if not NULL, forgets the ticket and returns
   SINDI_OK or the request's own error status (its reason then in
   sindi_last_error of the polling thread). Returns SINDI_ERR_TIMEOUT while
   it is still running, SINDI_ERR_INVALID_ARG for an unknown ticket. */
sindi_status sindi_server_poll(sindi_server* server, uint64_t ticket, int32_t wait_ms, uint32_t* ids, float* scores,
                               double* latency_ms);

/* Counters and latency percentiles; reset = 1 clears the latency record and counters. */
sindi_status sindi_server_stats(sindi_server* server, sindi_server_stats_t* out, int reset);

/* Stop accepting requests, finish the ones queued or in flight, free everything.
   No other call on the same server may run concurrently with it or after it. */
void sindi_server_destroy(sindi_server* server);

/* Synchronise `stream`, then return (and clear) the device error word of the
   index as a status: SINDI_ERR_INVALID_DATA if a malformed query or document
   was seen since the last check, SINDI_ERR_TIMEOUT if a bounded wait gave up. */
sindi_status sindi_check(const sindi_index* index, void* stream);

/* Sizes and parameters of an index. */
sindi_status sindi_index_info(const sindi_index* index, sindi_index_info_t* out);

/*
 * Write the index (parameters, lists and the unpruned documents) to the file
 * `path`, in host byte order, so that sindi_index_load can rebuild it without
 * a new build (checkpoint; the paper reports index sizes only, Sec. 5).
 * Waits for the device. Returns SINDI_ERR_INVALID_ARG if the file cannot be
 * written.
 */
sindi_status sindi_index_save(const sindi_index* index, const char* path);

/*
 * Read an index written by sindi_index_save onto the current device (working
 * on `stream`; the call returns when the index is ready). Every offset and
 * id the search kernels follow (list offsets, window ids < lambda, document
 * offsets, dims < dim) is checked on its way in; a file that is not an index
 * file of this version, is truncated or fails a check gives
 * SINDI_ERR_INVALID_DATA and no index. `out` receives the new index (free
 * with sindi_index_free).
 */
sindi_status sindi_index_load(const char* path, void* stream, sindi_index** out);

/*
 * Copy the index layout to host buffers (for inspection and tests).
 *   seg:   uint32 [dim * n_windows + 1]; list I_{j,w} is postings
 *          seg[j * n_windows + w] .. seg[j * n_windows + w + 1] - 1.
 *   ids:   uint16 [postings]; window-local id i mod lambda.
 *   vals:  [postings] of the value dtype (float / binary16 bits / E4M3 codes).
 *   scale: float [dim]; per-list E4M3 scale (1 for the other dtypes).
 *   kept:  uint32 [n_docs]; |alpha-mass(x_i)| for every document.
 * Any pointer may be NULL to skip that array.
 */
sindi_status sindi_index_export(const sindi_index* index, uint32_t* seg, uint16_t* ids, void* vals,
                                float* scale, uint32_t* kept);

/* Turn CUDA-event timing of scan kernels on (1) or off (0), and read or reset
   the index's counters. */
sindi_status sindi_set_timing(const sindi_index* index, int enable);
sindi_status sindi_get_stats(const sindi_index* index, sindi_stats_t* out);
sindi_status sindi_reset_stats(const sindi_index* index);

/* Free an index and everything it owns. NULL is ignored. Waits for work
   queued on the index's streams to finish. Plans and servers over the index
   must be freed first, and no search on it may still be running on a
   caller's stream. */
void sindi_index_free(sindi_index* index);

/* Message of the last failed call on this thread ("" if none). */
const char* sindi_last_error(void);

/* Library version string. */
const char* sindi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SINDI_H */
