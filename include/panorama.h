/*
 * panorama.h -- C-ABI of a GB300 (sm_103a) library for exact, level-wise
 * verification of approximate-nearest-neighbour candidates in the manner of
 * "Panorama: Fast-Track Nearest Neighbors" (arXiv 2510.00566).
 *
 * What the library computes (paper sections in brackets):
 *   * an orthogonal PCA transform T and centre mu fit in closed form
 *     [Section 4.1]; vectors are compared in the rotated space T(x - mu),
 *     where squared distances are unchanged [Eq. 1];
 *   * an IVF index: k-means centroids, lists of vectors [Section 6.1], each
 *     list stored level-major (the L slices of a chunk of vectors follow one
 *     another) together with per-vector cumulative tail norms [Section 6.5];
 *   * search: for every query the nprobe nearest lists form the candidate set
 *     Gamma [Problem 2]; candidates are refined level by level with the
 *     Cauchy-Schwarz lower bound of Eq. 3 and discarded as soon as it exceeds
 *     the running k-th distance [Algorithm 1, epsilon = 1], so the answer is
 *     the exact k nearest candidates [Problem 1].
 *
 * Conventions shared by every entry point:
 *   * Return value: PANO_OK (0) or a negative PANO_E* code.  The calling
 *     thread's last error message is available from panorama_last_error().
 *   * Matrices are row-major, FP32, one vector per row.
 *   * "device" pointers are CUDA device (or managed) memory of the current
 *     device; "host" pointers are ordinary process memory.  Entry points that
 *     accept either detect the kind with cudaPointerGetAttributes.
 *   * `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; temporary device memory is allocated
 *     and freed stream-ordered on it (cudaMallocAsync / cudaFreeAsync).
 *   * Squared Euclidean distances in the ORIGINAL space are reported.
 *   * Result rows are sorted ascending by (distance, id); a row with fewer
 *     than k candidates is padded with id -1 and distance +infinity.
 *   * Objects (pano_transform, pano_index) are owned by the library and freed
 *     with the matching panorama_free_* call; the caller owns every array it
 *     passes in.  An index may be searched from several host threads at once
 *     (searches only read it).
 */
#ifndef PANORAMA_H
#define PANORAMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ error codes */
#define PANO_OK 0
#define PANO_EINVAL (-1)   /* invalid argument (shape, range, null pointer)  */
#define PANO_ENOMEM (-2)   /* host or device allocation failed               */
#define PANO_ECUDA (-3)    /* a CUDA call failed (message has the cause)     */
#define PANO_ETIMEOUT (-4) /* a bounded device-side wait gave up             */
#define PANO_ECORRUPT (-5) /* index file malformed or checksum mismatch      */
#define PANO_ENODEV (-6)   /* no usable sm_103 device                        */

/* ------------------------------------------------------ storage precision */
#define PANO_FP32 0 /* level slices in FP32, SIMT partial products          */
#define PANO_BF16 1 /* level slices in BF16, tensor-core partial products   */
#define PANO_FP8 2  /* level slices in FP8 E4M3 with a per-vector power-of-
                       two scale, tensor-core partial products               */

typedef struct pano_transform pano_transform; /* opaque, library-owned */
typedef struct pano_index pano_index;         /* opaque, library-owned */

/* Build-time options.  Zero-initialise and set what you need; zero fields
 * take the documented defaults. */
typedef struct {
  int32_t n_levels;            /* L >= 1 (default 8; clamped to d)           */
  const int32_t* level_widths; /* host, L entries summing to d; NULL = equal
                                  widths (d must then be divisible by L)     */
  int32_t precision;           /* PANO_FP32 / PANO_BF16 / PANO_FP8           */
  int64_t fit_sample;          /* rows used for the PCA covariance
                                  (default min(n, 65536))                    */
  uint64_t seed;               /* k-means sampling / initialisation seed     */
  int32_t kmeans_iters;        /* Lloyd iterations (default 20)              */
  int64_t kmeans_sample;       /* training rows (default min(n, 256 nlist))  */
  int32_t identity_transform;  /* 1 = T = I, mu = 0 (raw axes)              */
  const float* centroids;      /* optional host nlist x d original-space
                                  centroids; when set k-means is skipped     */
} pano_build_opts;

/* Search-time options (pass NULL for the defaults). */
typedef struct {
  int32_t mode;        /* 0 = Panorama pruning (default); 1 = plain scan:
                          every candidate's full distance, no early pruning */
  int32_t synchronize; /* 1 (default when opts == NULL) = wait for the
                          search and report device-side errors; 0 = return
                          after enqueueing (errors surface on the next call
                          or via panorama_search_stats)                     */
  int32_t collect_stats; /* 1 = count pairs / levels / reranks (slower)     */
  int32_t query_group; /* max queries sharing one tile (0 = automatic)      */
  int32_t collect_timing; /* 1 = record CUDA events around each stage on
                             `stream` (stage_ms in the stats; implies a wait) */
  int32_t single_phase;   /* 0 (default) = automatic: each query's nearest
                             list first (phase A, which sets a tight
                             threshold) unless the index is BF16 and there
                             are fewer than 8 queries per list on average
                             (phase A's groups would fill few MMA columns);
                             1 = every probed list in one pass; 2 = two
                             phases always                                  */
  float epsilon;          /* 0 or 1 (default) = exact pruning with Eq. 3's
                             LB; in (0, 1): Eq. 4's relaxed LB_eps = A -
                             2 eps C prunes more and may lose true
                             neighbours (returned distances stay exact)    */
  int32_t test_every;     /* levels whose bound is tested (mode 0): level l
                             when l % test_every == 0, and always the last
                             level; with BF16 / FP8 storage a chunk of 128
                             candidates with at most 16 live rows is also
                             tested at every level (only a test that leaves
                             it no live row saves its copies and MMAs).
                             1 = every level, as Algorithm 1.  0 (default)
                             = the format's default: FP32 every level,
                             BF16 / FP8 every 4th.  panorama_autotune times
                             several.  The result is exact whatever the
                             value; only the work changes.               */
} pano_search_opts;

/* Counters of the most recent search through this index from this thread
 * (filled when collect_stats = 1). */
typedef struct {
  int64_t n_queries;
  int64_t pairs;          /* (query, candidate) pairs in all Gamma(q)        */
  int64_t pair_levels;    /* sum over pairs of levels whose partial product
                             was computed (dims scanned = sum of widths)     */
  int64_t dims_scanned;   /* sum over pairs of coordinates read            */
  int64_t tile_levels;    /* (query group, chunk, level) steps executed      */
  int64_t slice_bytes;    /* level-slice bytes staged into shared memory     */
  int64_t reranked;       /* pairs whose exact distance was computed         */
  int64_t work_items;     /* (list, query group, segment) work items         */
  int32_t device_error;   /* nonzero: a bounded wait or check failed         */
  int32_t pad_;
  /* device time per stage in ms (collect_timing = 1), measured with CUDA
   * events on the search stream: [0] transform + norms, [1] coarse probe,
   * [2] work inversion, [3] verify phase A (each query's nearest list),
   * [4] verify phase B (remaining lists), [5] result decode */
  float stage_ms[6];
  float pad2_[2];
  /* device cycles (summed over the verify CTAs' first threads, collect_stats
   * = 1).  Tensor-core path: [0] work-item prologue, [1] MMA issue, [2]
   * epilogues (bound tests), [3] next-level staging.  FP32 path: [0] item
   * and tile setup, [1] slice staging, [2] level-0 partial products and
   * tests, [3] the same for deeper levels.  Both: [4] last-level upper-bound
   * filter, [5] exact re-ranking, [6] whole kernel, [7] CTAs that ran. */
  int64_t section_cycles[8];
  int64_t dims_scanned_a; /* the part of dims_scanned read in phase A        */
  int64_t pairs_a;        /* the part of pairs in phase A (0 in one pass)    */
  int64_t section_cycles_a[8]; /* the part of section_cycles from phase A    */
  int64_t live_row_bytes; /* tensor-core path: sum over (query group, chunk,
                             level) steps of the candidates live for at
                             least one query of the group entering the
                             level x (level width x bytes per element + 4),
                             the slice and tail-norm bytes the method must
                             read; 0 on the FP32 path                        */
} pano_search_stats;

/* Description of a built index. */
typedef struct {
  int64_t n;
  int32_t d;
  int32_t nlist;
  int32_t n_levels;
  int32_t precision;
  int32_t chunk;        /* vectors per level-major chunk                     */
  int32_t max_level_width;
  int64_t n_chunks;
  int64_t device_bytes; /* device memory held by the index                   */
  double eta;           /* ||T~^T T~ - I||_F of the FP32 transform            */
} pano_index_info;

/* ---------------------------------------------------------------- transform
 * panorama_fit_transform -- PCA basis of a sample [Section 4.1].
 *   X: host or device, n x d FP32.  The first min(n, fit_sample) rows are
 *      used (pass a random subset if the rows are ordered).
 *   The covariance (1/n normalisation) and its eigen-decomposition are
 *   computed on the host in FP64; rows of T are eigenvectors ordered by
 *   eigenvalue descending, each with its largest-magnitude entry positive.
 *   opts may be NULL.  *out receives a new object.
 * Errors: PANO_EINVAL (n < 1, d < 1, null pointers), PANO_ENOMEM,
 *         PANO_ECUDA (copy of a device X failed). */
int panorama_fit_transform(const float* X, int64_t n, int32_t d,
                           const pano_build_opts* opts, pano_transform** out);

/* Copies the fitted transform out (any pointer may be NULL):
 *   T: d x d FP64 row-major, mu: d FP64, eigenvalues: d FP64 (descending). */
int panorama_transform_export(const pano_transform* t, double* T, double* mu,
                              double* eigenvalues);
int panorama_transform_dim(const pano_transform* t);
void panorama_free_transform(pano_transform* t);

/* ------------------------------------------------------------------- build
 * panorama_build_ivf -- IVF index with level-major lists [Section 6.1, 6.5].
 *   t:     transform from panorama_fit_transform (the index keeps a copy).
 *   X:     host or device, n x d FP32; vector i gets id i.
 *   nlist: number of lists (1 = flat index, every vector in one list).
 *   opts:  level split, precision, k-means settings (may be NULL).
 *   Steps (all on `stream`'s device): k-means (unless opts->centroids),
 *   nearest-centroid assignment (ties -> lower list id), transform of every
 *   vector, per-vector tail norms and rounding-error bounds, level-major
 *   packing in chunks, and an FP32 copy of the original rows for the exact
 *   re-ranking step.  Blocks until the index is complete.
 *   Level widths: PANO_BF16 needs 16, 32 or multiples of 64; PANO_FP8 32,
 *   64 or multiples of 128 (its tiles have the byte layout of bf16 tiles of
 *   half the width); both need d <= 8192.
 * Errors: PANO_EINVAL (d mismatch, nlist < 1 or > n, bad level split,
 *         unknown precision), PANO_ENOMEM, PANO_ECUDA, PANO_ENODEV. */
int panorama_build_ivf(const pano_transform* t, const float* X, int64_t n,
                       int32_t nlist, const pano_build_opts* opts,
                       void* stream, pano_index** out);

/* ------------------------------------------------------------------ search
 * panorama_search -- exact k nearest neighbours over each query's IVF
 * candidate set [Problems 1-2, Algorithm 1 with epsilon = 1].
 *   queries:  device, nq x d FP32.
 *   nprobe:   device, nq int32 (each in [1, nlist]); or NULL with
 *             nprobe_scalar in [1, nlist] for every query.
 *   k:        device, nq int32 (each in [0, k_max]); or NULL with k_scalar.
 *   k_max:    row stride of the outputs, 1..1024.
 *   out_ids:  device, nq x k_max int64; out_dists: device, nq x k_max FP32.
 *   Columns >= k of a row are filled with (-1, +inf).
 *   Every candidate whose exact distance can still be among the k smallest
 *   survives pruning (the bounds carry a rigorous rounding-error margin), and
 *   survivors are re-ranked with exact FP32 distances on the original rows,
 *   so ids equal those of an exact search except where two distances are
 *   within FP32 rounding of each other.
 * Errors: PANO_EINVAL (bad sizes, nprobe or k out of range when scalar),
 *         PANO_ENOMEM, PANO_ECUDA, PANO_ETIMEOUT (device wait gave up);
 *         out-of-range per-query nprobe/k values are clamped on the device.
 */
int panorama_search(const pano_index* idx, const float* queries, int64_t nq,
                    const int32_t* nprobe, int32_t nprobe_scalar,
                    const int32_t* k, int32_t k_scalar, int32_t k_max,
                    int64_t* out_ids, float* out_dists, void* stream);

/* panorama_search with options (opts may be NULL).  mode = 1 runs the plain
 * FP32 full-distance scan over the same candidate sets (the comparator). */
int panorama_search_ex(const pano_index* idx, const float* queries,
                       int64_t nq, const int32_t* nprobe,
                       int32_t nprobe_scalar, const int32_t* k,
                       int32_t k_scalar, int32_t k_max, int64_t* out_ids,
                       float* out_dists, void* stream,
                       const pano_search_opts* opts);

/* panorama_search_noalloc -- panorama_search without any device allocation.
 * The paper has no counterpart: this entry point serves callers that cannot
 * allocate device memory while searching (their memory is owned by another
 * allocator or pool, or they run on a path where an allocation, which can
 * synchronize or fail under fragmentation, is not allowed).  Arguments,
 * results and errors are those of panorama_search.  The workspace comes from
 * one 64 MiB array in the library's global memory (held by every GPU that
 * loads the library until the process exits) instead of cudaMallocAsync;
 * a call whose workspace would exceed it fails with PANO_EINVAL before any
 * work is queued (the workspace grows with nq x (d + nlist + nprobe + k_max)).
 * The array's device address is looked up on the first call on each device.
 * The call returns once the
 * search has finished: it synchronizes the stream and reads the device
 * error word, like panorama_search.  Every call reuses the same array, so
 * calls that overlap on the GPU race; serialise them on one stream. */
int panorama_search_noalloc(const pano_index* idx, const float* queries, int64_t nq,
                            const int32_t* nprobe, int32_t nprobe_scalar,
                            const int32_t* k, int32_t k_scalar, int32_t k_max,
                            int64_t* out_ids, float* out_dists, void* stream);

/* Counters of this thread's last search_ex with collect_stats = 1. */
int panorama_search_stats(pano_search_stats* out);
/* Status code of a device error word (pano_search_stats.device_error, or
 * the word a caller copied back itself): word & 1 (a bounded device-side
 * wait gave up; the top-k may be partial) -> PANO_ETIMEOUT; word & 4 (a
 * per-query value out of range was clamped, or an FP8 query exceeds the
 * format's range) -> PANO_EINVAL; otherwise PANO_OK (word & 2, a capacity
 * bound reached with the result still valid, is not an error).  Pure host
 * function; the serving loop maps each batch's word with it. */
int panorama_status_of_device_error(int32_t word);

/* ------------------------------------------------------------------ refine
 * panorama_build_flat -- flat index for refining candidate-id lists, the
 * paper's no-batch (B = 1) variant [Section 6.4 "IndexRefinePanorama",
 * Table 1]: every vector transformed and stored row-major (a candidate's
 * level slice is contiguous), with rounded-up tail norms, norms, error bounds
 * and the original FP32 rows for the exact re-ranking.
 *   t, X, n, opts: as panorama_build_ivf (opts: level split; precision must
 *   be PANO_FP32; no k-means).  Vector i gets id i.  panorama_search rejects
 *   a flat index; panorama_save / panorama_load keep it.
 * Errors: PANO_EINVAL, PANO_ENOMEM, PANO_ECUDA, PANO_ENODEV. */
int panorama_build_flat(const pano_transform* t, const float* X, int64_t n,
                        const pano_build_opts* opts, void* stream, pano_index** out);

/* panorama_refine -- exact k nearest neighbours of each query among its own
 * candidate ids (e.g. another index's top-k'), by Algorithm 1 with B = 1:
 * the first k candidates' exact distances seed the threshold, every other
 * candidate is refined level by level and abandoned at the first level
 * whose margined Eq. 3 lower bound exceeds the running k-th distance; the
 * rest are re-ranked exactly on the original rows.
 *   idx:       a flat index (panorama_build_flat).
 *   queries:   device, nq x d FP32 row-major.
 *   cand_ids:  device, nq x kprime int64; -1 = no candidate; an id may repeat
 *              (kept once).
 *   k:         1..1024.  epsilon: Eq. 4 (0 or 1 = exact; as search).
 *   out_ids / out_dists: device, nq x k, ascending (distance, id), padded
 *              with (-1, +inf) when a query has fewer than k distinct ids.
 *   Statistics of the call (pairs = candidates, dims_scanned, reranked) are
 *   read with panorama_search_stats.  Blocks until the results are written.
 * Errors: PANO_EINVAL (not a flat index, sizes, an id outside [-1, n)),
 *         PANO_ENOMEM, PANO_ECUDA, PANO_ENODEV. */
int panorama_refine(const pano_index* idx, const float* queries, int64_t nq,
                    const int64_t* cand_ids, int32_t kprime, int32_t k, int64_t* out_ids,
                    float* out_dists, float epsilon, void* stream);

/* panorama_probe -- the coarse step alone: the nprobe nearest lists of each
 * query by (original-space squared distance, list id) [Section 6.1].
 *   queries: device nq x d; out_lists: device nq x nprobe int32, ascending. */
int panorama_probe(const pano_index* idx, const float* queries, int64_t nq,
                   int32_t nprobe, int32_t* out_lists, void* stream);

/* ------------------------------------------------------------- batching
 * A plan is one search of a fixed batch shape captured into a CUDA graph:
 * workspace allocation, memsets, transform and probe GEMMs, work inversion,
 * the two persistent verify kernels and the decode replay with a single
 * cudaGraphLaunch.
 * panorama_plan_create runs the search once eagerly (so kernel attributes
 * are settled), then captures it on a private stream.  The device pointers
 * (queries, nprobe, k, out_ids, out_dists) are baked into the graph: every
 * launch reads their current contents and overwrites the outputs.  mode as
 * in pano_search_opts.  Device-side errors are not reported by launches;
 * use panorama_search_ex to diagnose.  The index must outlive the plan.
 * Errors: those of panorama_search, plus PANO_ECUDA for capture failures. */
typedef struct pano_plan pano_plan;
int panorama_plan_create(const pano_index* idx, const float* queries, int64_t nq,
                         const int32_t* nprobe, int32_t nprobe_scalar,
                         const int32_t* k, int32_t k_scalar, int32_t k_max,
                         int64_t* out_ids, float* out_dists, int32_t mode,
                         pano_plan** out);
/* The same with every search option (mode, test_every, epsilon, ...) taken
 * from opts (NULL = defaults); synchronize and collect_* are ignored. */
int panorama_plan_create_ex(const pano_index* idx, const float* queries, int64_t nq,
                            const int32_t* nprobe, int32_t nprobe_scalar,
                            const int32_t* k, int32_t k_scalar, int32_t k_max,
                            int64_t* out_ids, float* out_dists, const pano_search_opts* opts,
                            pano_plan** out);
int panorama_plan_launch(pano_plan* plan, void* stream);
void panorama_plan_free(pano_plan* plan);

/* panorama_autotune_levels -- picks the level split (L and widths, the
 * paper's L ablation of Section 7.5) that searches a sample fastest.
 *   X: host or device n x d rows to index (a sample of the data set);
 *   queries: device nq x d sample queries; nlist / nprobe / k / precision as
 *   in the build and search calls;
 *   widths: the candidates' widths concatenated, candidate c has
 *   n_levels[c] widths summing to d; repeats: timed searches per candidate
 *   (after one warm-up; the median counts).
 *   Every candidate is built with the centroids of the first one (k-means
 *   runs once) and timed with CUDA events on `stream`.  *best receives the
 *   fastest candidate's index, ms_out[c] (optional) its median ms (+inf when
 *   the split cannot be built, e.g. a bf16 width other than 16, 32 or a
 *   multiple of 64). */
int panorama_autotune_levels(const pano_transform* t, const float* X, int64_t n,
                             const float* queries, int64_t nq, int32_t nlist,
                             int32_t nprobe, int32_t k, int32_t precision,
                             const int32_t* widths, const int32_t* n_levels,
                             int32_t n_candidates, int32_t repeats, int32_t* best,
                             float* ms_out, void* stream);

/* panorama_autotune -- picks the storage precision and the level split
 * (the paper's L ablation of Section 7.5, extended to the precision of the
 * level slices) that search a sample fastest.
 *   X, queries, nlist, nprobe, k: as in panorama_autotune_levels;
 *   precisions: n_prec storage formats to try (PANO_FP32, PANO_BF16,
 *   PANO_FP8);
 *   widths / n_levels / n_candidates: candidate splits as in
 *   panorama_autotune_levels, tried with every precision; n_candidates = 0
 *   lets the tuner generate them per format: every uniform width (16, 32,
 *   64, 128, 256) dividing d that the format's kernels take, and
 *   front-loaded splits whose leading levels are narrow (16, 32 or 64) and
 *   double towards the widest width the format takes (BF16 128, FP8 and
 *   FP32 256), the last level taking the rest;
 *   trials (caller-owned, max_trials entries): one per (precision, split)
 *   pair in precision-major order, with its median search time over
 *   `repeats` timed searches (after one warm-up) at the fastest of the
 *   bound-test schedules test_every = 1, 2, 4 and n_levels (every level,
 *   every other, every fourth, the first and last only), and that
 *   schedule, or +inf
 *   when the pair cannot be built or staged; *n_trials and *best (index of
 *   the fastest) are written.  k-means runs once; every candidate is built with its
 *   centroids.  Errors: PANO_EINVAL for bad arguments, more pairs than
 *   max_trials, or no searchable pair; build / CUDA errors otherwise. */
typedef struct {
  int32_t precision;
  int32_t n_levels;
  int32_t widths[64];
  float ms;          /* at the fastest of the test schedules tried        */
  int32_t test_every; /* that schedule (pano_search_opts.test_every)      */
} pano_autotune_trial;
int panorama_autotune(const pano_transform* t, const float* X, int64_t n,
                      const float* queries, int64_t nq, int32_t nlist, int32_t nprobe,
                      int32_t k, const int32_t* precisions, int32_t n_prec,
                      const int32_t* widths, const int32_t* n_levels, int32_t n_candidates,
                      int32_t repeats, pano_autotune_trial* trials, int32_t max_trials,
                      int32_t* n_trials, int32_t* best, void* stream);

/* -------------------------------------------------------------- serving
 * A server batches single-query requests continuously over a device-resident
 * index.  A worker thread owns max_inflight slots (stream, pinned staging,
 * device buffers for max_batch queries); whenever a slot is free, requests
 * are queued and the memory budget admits the batch (estimated search
 * workspace + slot buffers, always admitted when nothing runs), up to
 * max_batch queued requests are copied in and searched on the slot's
 * stream.  Batches in different slots overlap on the device; requests that
 * arrive meanwhile go to the next free slot.  Each result is the exact top-k
 * of its own query (identical whatever it was batched with).  Latency is
 * measured from submit to results on the host. */
typedef struct pano_server pano_server;
typedef struct {
  int32_t max_batch;     /* queries per device batch (default 1024)           */
  int32_t max_inflight;  /* concurrent device batches (default 2, <= 16)      */
  int32_t k_max;         /* result row length (default 10)                    */
  int32_t pad_;
  int64_t memory_budget; /* device bytes for in-flight batches (default 1 GiB)*/
} pano_server_opts;
typedef struct {
  int64_t submitted, completed, batches;
  double mean_batch;     /* queries per launched batch                        */
  double p50_us, p99_us, max_us; /* request latency (last 10^6 requests)      */
  double qps;            /* completed / (last completion - first submit)      */
} pano_server_stats;
/* idx must outlive the server; opts may be NULL. */
int panorama_server_create(const pano_index* idx, const pano_server_opts* opts,
                           pano_server** out);
/* query: host, d FP32 values (copied); 1 <= nprobe <= nlist, 0 <= k <= k_max. */
int panorama_server_submit(pano_server* s, const float* query, int32_t nprobe,
                           int32_t k, uint64_t* ticket);
/* Blocks until the request is done (PANO_ETIMEOUT after timeout_ms; < 0 =
 * no limit) and copies k_max ids / distances (host) and its latency. */
int panorama_server_wait(pano_server* s, uint64_t ticket, int32_t timeout_ms,
                         int64_t* ids, float* dists, double* latency_us);
int panorama_server_stats(pano_server* s, pano_server_stats* out);
/* Open-loop replay: submits query i (host nq x d) at arrival_us[i]
 * microseconds after the call starts, then collects every result
 * (out_ids / out_dists host nq x k_max) and its latency (optional). */
int panorama_server_run_trace(pano_server* s, const float* queries, int64_t nq,
                              const double* arrival_us, const int32_t* nprobe,
                              const int32_t* k, int64_t* out_ids, float* out_dists,
                              double* latency_us);
/* Finishes queued work, then releases the server. */
void panorama_server_free(pano_server* s);

/* ------------------------------------------------------ index inspection */
int panorama_index_info(const pano_index* idx, pano_index_info* out);
/* host nlist x d FP32 original-space centroids */
int panorama_index_centroids(const pano_index* idx, float* out);
/* host n int32: the list of every vector id */
int panorama_index_assignment(const pano_index* idx, int32_t* out);

/* ------------------------------------------------------ persistence
 * panorama_save writes a versioned little-endian file with an FNV-1a 64-bit
 * checksum; panorama_load rebuilds the index on the current device.  Every
 * index kind is kept: IVF (FP32 / BF16 / FP8), flat, and IVFPQ
 * (panorama_pq.h).
 * Errors: PANO_EINVAL, PANO_ENOMEM, PANO_ECUDA, PANO_ECORRUPT (bad magic,
 *         version, sizes or checksum), and I/O failures as PANO_EINVAL. */
int panorama_save(const pano_index* idx, const char* path);
int panorama_load(const char* path, pano_index** out);
void panorama_free_index(pano_index* idx);

/* ------------------------------------------------------ list sharding
 * Host-side helpers of a search sharded by IVF lists over several GPUs
 * (each GPU holds the index of the vectors of its lists, with all
 * centroids, so its probes are the global ones; every candidate lives on
 * exactly one shard).  The paper's search is single-machine and has no
 * counterpart; the merge is the k-smallest selection of Problem 1 (§3) over
 * the union of the shards' candidate sets, which the shards' own top-k
 * lists contain.  Neither call touches the GPU.
 *
 * panorama_partition_lists: owner[c] in [0, n_shards) for every list, by
 * greedy bin packing (lists by decreasing size, ties by id, each to the
 * least-loaded shard, ties by shard id), so Σ sizes per shard is balanced.
 * list_size: host int32[nlist].  Errors: PANO_EINVAL (null pointer, nlist
 * < 1, n_shards < 1, negative size).
 *
 * panorama_merge_topk: n_parts partial results, part p at ids[p][nq][k] /
 * dists[p][nq][k] (host, contiguous: ids + (p * nq + i) * k), each row
 * sorted by (dist, id) and padded with (-1, +inf), as panorama_search
 * writes them.  Writes out_ids/out_dists [nq][k] (host): per query the k
 * smallest (dist, id) pairs over all parts, ascending, padded the same
 * way; an id in more than one part counts once, at its smallest distance.
 * Errors:
 * PANO_EINVAL (null pointer, n_parts < 1, nq < 0, k < 1). */
int panorama_partition_lists(const int32_t* list_size, int32_t nlist, int32_t n_shards,
                             int32_t* owner);
int panorama_merge_topk(const int64_t* ids, const float* dists, int32_t n_parts, int64_t nq,
                        int32_t k, int64_t* out_ids, float* out_dists);

/* Message of the calling thread's last failed call ("" if none). */
const char* panorama_last_error(void);
/* Library version string. */
const char* panorama_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PANORAMA_H */
