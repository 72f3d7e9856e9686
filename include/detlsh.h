/*
 * detlsh.h -- C ABI of a GB300 (sm_103a) implementation of DET-LSH
 * (Wei et al., "DET-LSH: A Locality-Sensitive Hashing Scheme with Dynamic
 * Encoding Tree for Approximate Nearest Neighbor Search", PVLDB 17(9), 2024).
 *
 * Every entry point returns 0 (DETLSH_OK) or a negative detlsh_status; on
 * error detlsh_last_error() describes the cause (thread-local string).
 * Pointers are plain host or device addresses, chosen per call by a `mem`
 * argument (DETLSH_MEM_HOST or DETLSH_MEM_DEVICE) that applies to every data
 * pointer of that call. The caller owns every buffer it passes; the library
 * owns the index it returns. `stream` is a cudaStream_t (NULL: the legacy
 * default stream); device work of a call is ordered on that stream and, with
 * host pointers, the call returns after its results reached host memory.
 * All computation of build and query runs in this library's CUDA kernels;
 * there is no CPU fallback: without a usable GPU every call returns
 * DETLSH_ECUDA.
 *
 * Limits: 1 <= K <= 16, 1 <= L <= 16, n_regions a power of two in [2, 256],
 * n_regions <= n_s <= n, 1 <= d <= 65536, n*L < 2^32, 1 <= k <= 1024.
 * Input values must be finite.
 */
#ifndef DETLSH_H_
#define DETLSH_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DETLSH_PENDING = 1,    /* detlsh_server_poll: the request has not finished */
  DETLSH_OK = 0,
  DETLSH_EINVAL = -1,    /* an argument is out of range or inconsistent   */
  DETLSH_ENOMEM = -2,    /* device or host allocation failed              */
  DETLSH_ECUDA = -3,     /* a CUDA call failed (no device, launch error)  */
  DETLSH_ETIMEOUT = -4,  /* a bounded device wait ran out                 */
  DETLSH_EADMIT = -5,    /* request refused by memory-based admission     */
  DETLSH_EINTERNAL = -6  /* an internal consistency check failed          */
} detlsh_status;

typedef enum { DETLSH_F32 = 0, DETLSH_U8 = 1 } detlsh_dtype;
typedef enum { DETLSH_MEM_HOST = 0, DETLSH_MEM_DEVICE = 1 } detlsh_mem;

/* projection arithmetic of the build (Eq. 1 for every point) */
typedef enum {
  DETLSH_PROJ_FP32 = 0,  /* FP32-faithful projections: on the tensor cores
                            as a TF32 split of points and hash vectors (FP32
                            points, d <= 256, d % 4 == 0, L*K <= 64) or as
                            uint8 points against the hash vectors in three
                            BF16 parts (d <= 256, d % 16 == 0, L*K <= 64),
                            both with a 16-byte aligned X; otherwise FP32
                            fused multiply-add on the CUDA cores. Exact
                            whenever the products and sums are exact in FP32;
                            else within about 1e-5 of sum |a x| (d <= 256). */
  DETLSH_PROJ_BF16 = 1   /* BF16 inputs (points and hash vectors rounded to
                            BF16; the index keeps a BF16 copy of X) on the
                            tensor cores with FP32 accumulation; needs
                            d % 8 == 0 and L*K <= 64. Codes are exact for
                            their BF16 inputs; queries are projected the same
                            way; the exact re-rank still uses FP32 X. */
} detlsh_proj_mode;

/* detlsh_params.flags */
#define DETLSH_BORROW_X 1  /* with DETLSH_MEM_DEVICE: keep a reference to the
                              caller's X instead of copying it; X must then
                              stay alive and unchanged until detlsh_free */
#define DETLSH_DEDUP_POS 2 /* index the query walk's duplicate test by each
                              point's position in the first tree's leaf order
                              (4*L bytes more per point). Chosen automatically
                              when the walk's per-CTA bitmaps of n bits do not
                              fit in L2 together; results are the same either
                              way. */

typedef struct detlsh_index detlsh_index;

/* Index parameters (Alg. 1-3 inputs; Sec. 5.2 and Sec. 6.1 give the paper's
 * defaults K=16, L=4, N_r=256, n_s=0.1n; max_size is not given there). */
typedef struct {
  int32_t K;            /* hash functions per projected space                */
  int32_t L;            /* projected spaces = DE-Trees                       */
  int32_t n_regions;    /* N_r: regions per projected dimension              */
  int32_t max_leaf;     /* max_size of Alg. 3 (>= 1)                         */
  int64_t sample_size;  /* n_s of Alg. 1: the number of entries of sample_ids,
                           or, when the library draws the sample, its size
                           (0: ceil(0.1*n), the paper's n_s = 0.1n, Sec. 6.1) */
  int32_t proj_mode;    /* detlsh_proj_mode                                  */
  int32_t flags;        /* DETLSH_BORROW_X | DETLSH_DEDUP_POS, or 0          */
  uint64_t seed;        /* seed of the draws the library makes when A or
                           sample_ids is NULL (detlsh_draw_hashes,
                           detlsh_draw_sample)                               */
} detlsh_params;

/* Launch shapes of the query pipeline (no counterpart in the paper). The
 * results do not depend on them; detlsh_autotune picks them by timing. Zero
 * fields take the defaults. */
typedef struct {
  int64_t batch;             /* queries per batch (0: sized from free device memory,
                                at most 16384)                                   */
  int32_t walk_ctas_per_sm;  /* bucket-walk CTAs per SM, 1..4 (0: as many as fit)  */
  int32_t dist_rows;         /* candidate rows per distance work item, a multiple
                                of 64 in [64, 8192] (0: 1024)                     */
  int32_t dist_ctas_per_sm;  /* persistent distance CTAs per SM, 1..4 (0: 4; 3 for
                                the BF16 gather of the shortlist mode)            */
  int32_t shortlist;         /* detlsh_autotune's pick for
                                detlsh_query_params.shortlist; the query ignores
                                this field                                        */
  int32_t streams;           /* 0 or 1: batches one after another on the call's
                                stream; 2: with several batches, batches
                                alternate between the call's stream and a
                                second one, each with its own scratch of half
                                the memory budget, so that one batch's kernels
                                may overlap the next one's. Plans run one batch
                                at a time.                                        */
  int32_t coarse_gather;     /* shortlist mode: 0 computes the coarse distances
                                leaf by leaf on the tensor cores (each leaf's rows
                                read once for up to 128 queries that activated
                                it); 1 gathers every candidate's row on the CUDA
                                cores                                             */
  int32_t id_bucket_log2;    /* the per-candidate distance gather takes the
                                batch's candidates grouped by point-id range, all
                                queries' candidates in ids [0, 2^x) first, then
                                [2^x, 2^(x+1)), ..., so that the rows read at the
                                same time lie in a few MB of X and stay in L2
                                (the points are candidates of many queries of a
                                batch). 0: x chosen for ranges of about 32 MB of
                                points, and the walk order kept where a point is
                                expected among fewer than 16 queries' candidates
                                (beta times the batch size); 10..31: that x;
                                -1: walk order (no grouping). The distances are
                                the same either way                               */
} detlsh_tuning;

/* Query parameters shared by a batch (Alg. 7 inputs besides q, k, c, r_min). */
typedef struct {
  double eps;         /* projected-radius factor of Lemma 3 (Eq. 2); <= 0 selects
                         detlsh_eps_lemma3(K, L)                            */
  double beta;        /* false-positive fraction: a query stops once its
                         candidate set holds ceil(beta*n + k) points (>= 0)  */
  uint32_t* cand_ids; /* optional [nq][cand_cap]: the candidate set S of each
                         query (unordered ids; the first |S| entries), in
                         the call's `mem` space; NULL to skip               */
  int64_t cand_cap;   /* capacity per query of cand_ids                      */
  int32_t shortlist;  /* 0: exact FP32 distances for every candidate. > 0
                         (index built with DETLSH_PROJ_BF16, at most 4096):
                         candidate distances from the BF16 copy of X (FP32
                         accumulation, used also by the "within c*r" test),
                         then the `shortlist` nearest are re-ranked with
                         exact FP32 distances before the top-k            */
  int32_t reserved;
  const detlsh_tuning* tuning;  /* launch shapes; NULL: defaults             */
  float* qproj;       /* optional [nq][L*K]: the projected queries q' (Alg. 7,
                         H_i(q)) in FP32 exactly as the query's later steps
                         read them, in the call's `mem` space; NULL to skip
                         (plans and detlsh_autotune take NULL)             */
} detlsh_query_params;

/*
 * detlsh_build -- encoding and indexing phases (Sec. 4.1-4.2: Eq. 1, Alg. 1,
 * Alg. 2, Alg. 3).
 *
 *   X           [n][d] row-major points, dtype DETLSH_F32 or DETLSH_U8 (uint8
 *               values are widened to FP32 inside the kernels).
 *   A           [L*K][d] row-major FP32 hash vectors of Eq. 1 (entries from
 *               N(0,1)); row r = i*K + j is a_ij, the j-th hash of projected
 *               space i. NULL: drawn by the library, detlsh_draw_hashes with
 *               params->seed (the paper's problem statement needs only the
 *               dataset and K, L, N_r).
 *   sample_ids  [n_s] distinct point ids in [0, n) whose projections select the
 *               breakpoints (Alg. 1: the sample of the n points), n_s =
 *               params->sample_size. NULL: drawn by the library,
 *               detlsh_draw_sample with params->seed, of params->sample_size
 *               points (0: ceil(0.1*n)).
 *   params      see detlsh_params.
 *   out         receives the new index (free it with detlsh_free).
 *
 * The index holds: A; per projected dimension N_r+1 breakpoints (minimum,
 * N_r-1 interior edges at sample ranks floor(n_s/N_r)*z, maximum); the 8-bit
 * region code of every point in every projected dimension; and L DE-Trees as
 * leaf tables (root split on the top code bit of all K dimensions, then
 * binary splits of the most evenly dividing dimension while a node holds more
 * than max_leaf points). It keeps a device copy of X (or the caller's X with
 * DETLSH_BORROW_X). The index is read-only afterwards; concurrent queries on
 * different streams are safe.
 * Errors: DETLSH_EINVAL for sizes or parameters outside the limits above,
 * DETLSH_ENOMEM, DETLSH_ECUDA, DETLSH_ETIMEOUT (a bounded wait of the
 * tensor-core kernel ran out).
 */
int detlsh_build(const void* X, int64_t n, int32_t d, int32_t dtype,
                 const float* A, const int64_t* sample_ids,
                 const detlsh_params* params, int32_t mem, void* stream,
                 detlsh_index** out);

/*
 * detlsh_query -- batched c^2-k-ANN queries (Alg. 7 with the optimised range
 * query of Sec. 6.2.2: a leaf whose lower-bound distance to q' is within the
 * projected radius eps*r joins the candidate set whole, leaves in order of
 * their lower bound; r grows r_min, c*r_min, c^2*r_min, ...).
 *
 *   Q           [nq][d] row-major queries, dtype as the index's X.
 *   k, c, r_min [nq] per query: result size (1 <= k <= k_max), approximation
 *               ratio (> 1), initial radius (<= 0 selects the square root of
 *               the smallest positive leaf lower bound divided by eps).
 *   k_max       row length of the outputs (1..1024).
 *   qp          see detlsh_query_params (NULL: eps from Lemma 3, beta = 0.1).
 *   out_ids     [nq][k_max] int64 ids of the k nearest candidates by
 *               (distance, id); -1 after the k-th or when |S| < k.
 *   out_dist    [nq][k_max] FP32 Euclidean distances (+inf padding).
 *   out_stats   optional [nq][4] int32: |S| at termination, rounds started,
 *               stop rule (1: |S| >= beta*n+k, 2: >= k candidates within c*r,
 *               3: every leaf active), and 0 (1 would flag an internal
 *               candidate-list overflow, which the list's sizing excludes).
 * Errors: DETLSH_EINVAL (bad sizes/parameters, dtype differs from the index),
 * DETLSH_ENOMEM, DETLSH_ECUDA.
 */
int detlsh_query(const detlsh_index* idx, const void* Q, int64_t nq, int32_t dtype,
                 const int32_t* k, const float* c, const float* r_min, int32_t k_max,
                 const detlsh_query_params* qp, int64_t* out_ids, float* out_dist,
                 int32_t* out_stats, int32_t mem, void* stream);

/* detlsh_free -- release an index and all its device memory (NULL is a no-op). */
void detlsh_free(detlsh_index* idx);

/*
 * detlsh_insert -- add m points (ids n .. n+m-1, rows of X [m][d] in the
 * index's dtype) to an index built with DETLSH_PROJ_FP32 (reading R14): their
 * Alg. 2 codes against the index's breakpoints (Alg. 1 is not run again), by
 * the projection kernel the build used, then the DE-Trees of all n+m points
 * as Alg. 3 bulk-loads them (reading R3: order-free, so the index equals one
 * built from all points with these breakpoints). The index then owns a copy
 * of all points (a borrowed X is no longer referenced). Plans and servers of
 * the index must be destroyed first; queries see the new points after the
 * call returns (it synchronizes `stream`). On an error other than
 * DETLSH_EINVAL the index must be freed.
 */
int detlsh_insert(detlsh_index* idx, const void* X, int64_t m, int32_t dtype, int32_t mem, void* stream);

/* What detlsh_export copies out (test introspection and persistence). */
typedef enum {
  DETLSH_EXPORT_A = 0,            /* float   [L*K][d]                          */
  DETLSH_EXPORT_EDGES = 1,        /* float   [L*K][N_r+1] breakpoints (Alg. 1) */
  DETLSH_EXPORT_CODES = 2,        /* uint8   [L][n][K] region codes (Alg. 2)   */
  DETLSH_EXPORT_LEAF_IDS = 3,     /* uint32  [L][n] point ids in leaf order     */
  DETLSH_EXPORT_LEAF_BASE = 4,    /* int64   [L+1] first leaf of each tree      */
  DETLSH_EXPORT_LEAF_RANGE = 5,   /* uint32  [n_leaves][2] start (within the
                                     tree's part of LEAF_IDS), count           */
  DETLSH_EXPORT_LEAF_PLEN = 6,    /* uint8   [n_leaves][K] prefix bits per dim  */
  DETLSH_EXPORT_LEAF_PREFIX = 7,  /* uint8   [n_leaves][K] prefix value per dim */
  DETLSH_EXPORT_SAMPLE_PROJ = 8,  /* float   [L*K][n_s] projections of the
                                     sampled points                            */
  DETLSH_EXPORT_SAMPLE_IDS = 9    /* int64   [n_s] the sampled point ids,
                                     ascending as given or drawn               */
} detlsh_export_what;

/* detlsh_export_size -- bytes detlsh_export needs for `what` (< 0 on error). */
int64_t detlsh_export_size(const detlsh_index* idx, int32_t what);

/* detlsh_export -- copy one index array into dst (`bytes` >= export size). */
int detlsh_export(const detlsh_index* idx, int32_t what, void* dst, int64_t bytes,
                  int32_t mem, void* stream);

/* detlsh_info -- index sizes: out[0..9] = n, d, dtype, K, L, n_regions,
 * max_leaf, n_s, total leaves, largest leaf. Returns the entries written. */
int detlsh_info(const detlsh_index* idx, int64_t* out, int32_t len);

/*
 * detlsh_project -- Eq. 1 for a batch of points: P[o][r] = sum_t A[r][t] X[o][t]
 * in FP32, X [n][d] (dtype), A [LK][d], P [n][LK] FP32. Same kernel as the
 * build's projection of the sample.
 */
int detlsh_project(const void* X, int64_t n, int32_t d, int32_t dtype,
                   const float* A, int32_t LK, float* P, int32_t mem, void* stream);

/*
 * detlsh_encode_values -- Alg. 2 on given projected values: codes[o][r] =
 * number of interior breakpoints E[r][z] (z = 1..N_r-1) with E[r][z] <= P[o][r]
 * (regions half-open [e_z, e_{z+1}), values below the first edge -> 0, at or
 * above the last -> N_r-1). P [n][LK] FP32, E [LK][N_r+1] FP32 sorted rows,
 * codes [n][LK] uint8. Same search routine as the build's fused kernel.
 */
int detlsh_encode_values(const float* P, int64_t n, int32_t LK, const float* E,
                         int32_t n_regions, uint8_t* codes, int32_t mem, void* stream);

/*
 * detlsh_select_breakpoints -- Alg. 1 (closed form of Sec. 4.1) on given sample
 * projections: for each row r of Ps [LK][n_s] (FP32), E[r][0] = minimum,
 * E[r][z] = the element of 0-based rank floor(n_s/N_r)*z (z = 1..N_r-1),
 * E[r][N_r] = maximum; E is [LK][N_r+1] FP32. Same kernels as the build.
 */
int detlsh_select_breakpoints(const float* Ps, int64_t n_s, int32_t LK, int32_t n_regions,
                              float* E, int32_t mem, void* stream);

/*
 * detlsh_rc_ann -- the (r,c)-ANN query of Alg. 6 on the index's L DE-Trees,
 * with the exact range query of Alg. 4/5: in tree i (in order) a leaf whose
 * lower-bound distance to q'_i exceeds eps*r is skipped, a leaf whose upper
 * bound does not is taken whole, and any other leaf gives the points whose own
 * projection lies within eps*r of q'_i (the outermost breakpoint edges count
 * as -inf/+inf in both bounds); the results are added to S. Once
 * |S| >= beta*n + 1 the point of S closest to q is returned; after the last
 * tree it is returned if it lies within c*r, else nothing (id -1).
 *
 * Q [nq][d] in the index's dtype, r [nq] and c [nq] (FP32), out_id [nq]
 * int64, out_dist [nq] FP64 (Euclidean; +inf when nothing is returned),
 * out_stats [nq][3] int32 (|S| at the end, trees range-queried, stop: 1 the
 * |S| bound, 2 within c*r, 0 nothing returned): all device pointers; the call
 * only enqueues work on `stream`. Every value is FP64 with a fixed operation
 * order, one CTA per query: a reference path for the paper's un-optimised
 * query semantics, not a throughput path. Temporary storage: n bits per query.
 */
int detlsh_rc_ann(const detlsh_index* idx, const void* Q, int64_t nq, int32_t dtype, const float* r,
                  const float* c, double eps, double beta, int64_t* out_id, double* out_dist,
                  int32_t* out_stats, void* stream);

/*
 * detlsh_select_breakpoints_noalloc -- detlsh_select_breakpoints for callers
 * that must not allocate device memory, e.g. a serving process that keeps a
 * fixed device-memory footprint (an allocation may fail under memory pressure
 * mid-request; freeing synchronizes the device) or an application whose own
 * allocator owns all device memory. The paper has no counterpart; the results
 * are those of detlsh_select_breakpoints.
 *
 * Ps [LK][n_s] and E [LK][N_r+1] must be device (or managed) pointers, else
 * DETLSH_EINVAL before any device work; the call only enqueues work on
 * `stream`. Temporary storage comes from one fixed 7 MiB array built into the
 * library (held by every GPU that loads it, until process exit), so n_s*LK
 * must not exceed DETLSH_NOALLOC_MAX_ITEMS (DETLSH_EINVAL otherwise). Each
 * call looks up that array's device address on the current device; the first
 * call on a device may load the library's device code there, so make it
 * before any stream capture. All calls share the array: calls whose GPU work
 * overlaps (e.g. on two streams) race and must be serialized by the caller.
 */
#define DETLSH_NOALLOC_MAX_ITEMS 262144
int detlsh_select_breakpoints_noalloc(const float* Ps, int64_t n_s, int32_t LK, int32_t n_regions,
                                      float* E, void* stream);

/*
 * Query plans (no counterpart in the paper: a serving form of detlsh_query).
 *
 * detlsh_plan_create -- allocates, once, the scratch of a batch of up to
 *   nq_max queries (or tuning->batch if smaller) with input and output staging,
 *   for results of k_max entries per query under qp (cand_ids must be NULL).
 *   flags: DETLSH_PLAN_GRAPH captures the batch's kernels in a CUDA graph (on a
 *   private stream) that every later batch replays with one launch; every
 *   kernel reads the batch size from device memory, so the graph serves any
 *   batch size up to the capacity. Synchronizes `stream`. The plan keeps a
 *   reference to idx, which must outlive it.
 * detlsh_plan_query -- the same results as detlsh_query for nq queries, run in
 *   chunks of the plan's capacity: each chunk's inputs are copied into the
 *   staging buffers, its size written to device memory, the batch run (graph
 *   launch or direct launches) and its outputs copied to out_*, all on
 *   `stream`, in the `mem` space of the arguments. No device allocation. With
 *   DETLSH_MEM_HOST the arguments are checked on the host and the call
 *   synchronizes and returns detlsh_plan_status. With DETLSH_MEM_DEVICE it
 *   returns after enqueueing: per-query arguments are checked on the device,
 *   a chunk with a bad one runs as an empty batch (its out_* rows are then
 *   unspecified) and detlsh_plan_status reports it. Calls on one plan must be
 *   serialized on one stream (they share the staging buffers).
 * detlsh_plan_status -- synchronizes `stream`; DETLSH_EINVAL if a chunk since
 *   the last status call had a bad per-query argument, DETLSH_ETIMEOUT if a
 *   bounded wait of the tensor-core projection ran out, else DETLSH_OK.
 * detlsh_plan_info -- out[0] batch capacity, [1] scratch bytes, [2] graph
 *   launches so far, [3] batches so far, [4] kernels in the captured graph.
 * detlsh_plan_destroy -- synchronizes the device and frees the plan.
 */
#define DETLSH_PLAN_GRAPH 1
typedef struct detlsh_plan detlsh_plan;
int detlsh_plan_create(const detlsh_index* idx, int64_t nq_max, int32_t k_max,
                       const detlsh_query_params* qp, int32_t flags, void* stream,
                       detlsh_plan** out);
int detlsh_plan_query(detlsh_plan* plan, const void* Q, int64_t nq, const int32_t* k,
                      const float* c, const float* r_min, int64_t* out_ids, float* out_dist,
                      int32_t* out_stats, int32_t mem, void* stream);
int detlsh_plan_status(detlsh_plan* plan, void* stream);
int detlsh_plan_info(const detlsh_plan* plan, int64_t* out5);
void detlsh_plan_destroy(detlsh_plan* plan);

/*
 * detlsh_autotune -- times the query pipeline on a sample of queries (the
 * arguments as for detlsh_query; qp->tuning, if set, is the starting point)
 * and writes the fastest launch shapes to *out: walk CTAs per SM, distance
 * rows per work item and distance CTAs per SM by coordinate descent, and the
 * batch size among the sizes that fit. For an index built with
 * DETLSH_PROJ_BF16 and min_agreement in (0, 1], out->shortlist is the
 * smallest shortlist in {64, 128, ..., 4096} (at least k_max) whose top-k
 * holds, averaged over the sample, at least min_agreement of the ids of the
 * exact FP32 top-k, if it is also faster than exact distances (else 0), and
 * out->coarse_gather is the faster of the two coarse-distance methods.
 * Synchronizes `stream`. Errors as detlsh_query.
 */
int detlsh_autotune(const detlsh_index* idx, const void* Q, int64_t nq, int32_t dtype,
                    const int32_t* k, const float* c, const float* r_min, int32_t k_max,
                    const detlsh_query_params* qp, double min_agreement, int32_t mem,
                    void* stream, detlsh_tuning* out);

/*
 * Continuous-batching server (no counterpart in the paper: Alg. 7 queries
 * that arrive one at a time, answered in batches against a resident index).
 *
 * A server admits requests into a fixed pool of queue_cap slots; a worker
 * thread forms batches of up to `slots` queries in arrival order and runs
 * each through one of `pipelines` query plans (own stream, preallocated
 * device buffers, CUDA-graph replay), so that consecutive batches overlap. A
 * batch starts when it is full, when no batch is running, or when its oldest
 * request has waited max_delay_us. Each query's result is the one
 * detlsh_query gives for it alone: it does not depend on the batch.
 */
typedef struct {
  int32_t k_max;           /* largest k of a request, 1..1024                     */
  int32_t slots;           /* queries per batch; 0: the largest power of two
                              <= 4096 whose buffers for all pipelines fit
                              mem_budget                                          */
  int32_t pipelines;       /* batches in flight, 1..4 (0: 2)                      */
  int32_t queue_cap;       /* requests admitted and not yet collected
                              (0: 4 * slots * pipelines)                          */
  int32_t max_delay_us;    /* wait of a partial batch while another runs (0: 200) */
  int32_t shortlist;       /* as detlsh_query_params.shortlist                    */
  double eps, beta;        /* as detlsh_query_params                              */
  int64_t mem_budget;      /* device bytes for the batch buffers of all pipelines
                              (0: 8 GiB); creation fails with DETLSH_EADMIT if
                              `slots` does not fit                                */
  const detlsh_tuning* tuning;  /* launch shapes (NULL: defaults)                */
  int32_t test_fail_batch; /* > 0: the N-th batch is reported failed
                              (DETLSH_ECUDA) without running, to exercise
                              failure handling on the host; 0 in service       */
  int32_t reserved;
} detlsh_server_config;
typedef struct detlsh_server detlsh_server;

/* detlsh_server_create -- plans, streams and the worker thread over idx (which
 * must outlive the server); errors as detlsh_plan_create, DETLSH_EADMIT as
 * above. */
int detlsh_server_create(const detlsh_index* idx, const detlsh_server_config* cfg,
                         detlsh_server** out);
/* detlsh_server_submit -- copies the query q (host memory, d values of the
 * index dtype) with its k, c and r_min into a free slot and queues it;
 * *ticket identifies it. DETLSH_EADMIT when every slot is in use (collect
 * finished requests with detlsh_server_poll), DETLSH_EINVAL on bad arguments. */
int detlsh_server_submit(detlsh_server* srv, const void* q, int32_t k, float c, float r_min,
                         uint64_t* ticket);
/* detlsh_server_poll -- waits up to wait_us for the request; DETLSH_PENDING if
 * it has not finished, else the batch's status (DETLSH_OK or an error) with
 * the results copied to ids/dist [k_max] and stats [4] (as detlsh_query; any
 * may be NULL) and *latency_us (optional) = completion - submission; the
 * ticket is then released. */
int detlsh_server_poll(detlsh_server* srv, uint64_t ticket, int32_t wait_us, int64_t* ids,
                       float* dist, int32_t* stats, double* latency_us);
/* detlsh_server_replay -- open-loop load: submits query i (host arrays) at
 * arrival_us[i] microseconds after the call starts (non-decreasing; a full
 * pool delays the submission), collects every result into out_ids/out_dist
 * [nq][k_max] and out_stats [nq][4] (each optional) and writes latency_us[i] =
 * completion - scheduled arrival (-1 for a failed request). Returns the first
 * error of any request, else DETLSH_OK. */
int detlsh_server_replay(detlsh_server* srv, const void* Q, int64_t nq, const int32_t* k,
                         const float* c, const float* r_min, const double* arrival_us,
                         int64_t* out_ids, float* out_dist, int32_t* out_stats,
                         double* latency_us);
/* detlsh_server_stats -- out[0] submitted, [1] completed, [2] rejected by
 * admission, [3] batches, [4] queries in batches, [5] largest batch,
 * [6] requests failed, [7] batch capacity. */
int detlsh_server_stats(detlsh_server* srv, int64_t* out8);
/* detlsh_server_destroy -- runs the queued requests, stops the worker and
 * frees the server (uncollected results are dropped). */
void detlsh_server_destroy(detlsh_server* srv);

/*
 * The random draws of the method from a seed (the paper fixes no generator;
 * these are the library's, documented so that others can reproduce them).
 * Both run on the host, write host memory and need no GPU. The generator is
 * splitmix64 (Steele, Lea, Flood, OOPSLA 2014): state += 0x9E3779B97F4A7C15;
 * z = state; z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;
 * z = (z ^ (z >> 27)) * 0x94D049BB133111EB; output z ^ (z >> 31).
 *
 * detlsh_draw_hashes -- the hash vectors of Eq. 1, A [LK][d] FP32 (row-major,
 *   row r = i*K + j): state = seed; entries in row-major order two at a time
 *   by Box-Muller in FP64 from two consecutive outputs z1, z2:
 *   u1 = ((z1 >> 11) + 1) * 2^-53, u2 = (z2 >> 11) * 2^-53,
 *   rho = sqrt(-2 ln u1), theta = (2 pi) u2, entries rho cos theta and
 *   rho sin theta (the second dropped past the end), each rounded to FP32.
 *   DETLSH_EINVAL unless 1 <= LK <= 256 and 1 <= d <= 65536.
 * detlsh_draw_sample -- the sample of Alg. 1, n_s distinct ids of [0, n)
 *   ascending: state = seed ^ 0x5A; a partial Fisher-Yates shuffle of the
 *   positions 0..n-1 where step i = 0..n_s-1 swaps positions i and
 *   i + ((z * (n - i)) >> 64) (z the next output, 128-bit product); the
 *   sample is the first n_s positions, sorted. DETLSH_EINVAL unless
 *   1 <= n_s <= n < 2^32.
 */
int detlsh_draw_hashes(uint64_t seed, int32_t LK, int32_t d, float* A);
int detlsh_draw_sample(uint64_t seed, int64_t n, int64_t n_s, int64_t* ids);

/* detlsh_eps_lemma3 -- eps of Lemma 3 (Eq. 2): eps^2 is the upper
 * alpha1-quantile of chi2(K), alpha1 = exp(-1/L). Returns < 0 on bad input. */
double detlsh_eps_lemma3(int32_t K, int32_t L);

/*
 * Tracing (no counterpart in the paper; its Fig. 4 reports a per-phase time
 * breakdown of the build, which this makes measurable on the GPU).
 * detlsh_trace_enable -- on != 0: every later build/query on the calling thread
 *   records CUDA events around its phases on its stream and synchronizes that
 *   stream before returning. Returns the previous setting.
 * detlsh_trace_get -- device milliseconds of the last build and the last query
 *   on this thread: out[0] sample projection, [1] breakpoint selection,
 *   [2] fused projection+encoding, [3] DE-Tree leaves, [4] query projection,
 *   [5] leaf lower bounds, [6] candidate distances, [7] number of distance
 *   launches, [8] number of lower-bound launches, [9] whole build, [10] whole
 *   query, [11] bucket walks, [12] stop test and top-k, [13] round table,
 *   leaf rounds and bucket lists, [14]-[16] the leaf build's root sort,
 *   gathers and level passes, [17] its number of level iterations, [18] the
 *   grouping of candidates by point-id range before the distances.
 *   Returns the number of entries written (<= len).
 * detlsh_launch_count -- kernels this library has launched in the process.
 */
int detlsh_trace_enable(int32_t on);
int detlsh_trace_get(double* out, int32_t len);
int64_t detlsh_launch_count(void);

/*
 * detlsh_memory_stats -- device memory in use by stream-ordered allocation on
 * the current device (no counterpart in the paper): out[0] bytes in use in the
 * library's own pool (index arrays and scratch), out[1] its high-water mark,
 * out[2] bytes in use in the device's default pool, out[3] its high-water
 * mark. With reset_peak != 0 both high-water marks are reset to the current
 * use after they are read. Returns the number of entries written (<= len).
 */
int detlsh_memory_stats(int32_t reset_peak, int64_t* out, int32_t len);

/*
 * detlsh_test_set_wait_limit_ns -- for tests of the failure path (no
 * counterpart in the paper): sets the limit of each bounded wait in the
 * tensor-core projection kernel for launches made after the call (default
 * 2,000,000,000 ns; 0 makes the first wait that does not succeed at once run
 * out) and returns the previous limit. A wait that runs out makes the kernel
 * wind down (its issued copies and MMAs completed, its tensor memory freed)
 * and the call return DETLSH_ETIMEOUT; later calls are unaffected once the
 * limit is restored. Process-wide; not for use while other threads run
 * builds or queries.
 */
uint64_t detlsh_test_set_wait_limit_ns(uint64_t ns);

/*
 * detlsh_check_status -- the checked build's record (no counterpart in the
 * paper). A library compiled with DETLSH_CHECKED checks the data-dependent
 * indices of its query kernels on the device (candidate positions, point
 * ids, bucket and list places, work items); a failed check skips the access
 * and is recorded. Synchronizes the current device, then writes out[0] the
 * number of failed checks since the previous call, out[1] the site of the
 * first one, out[2..3] its index (low, high 32 bits), and clears the record.
 * Returns 1 for a checked build (entries written: min(len, 4)), 0 for the
 * normal build (nothing written), DETLSH_ECUDA if the record cannot be read.
 */
int detlsh_check_status(uint32_t* out, int32_t len);

/* detlsh_strerror -- static text for a detlsh_status value. */
const char* detlsh_strerror(int status);

/* detlsh_last_error -- detail of the last error on the calling thread. */
const char* detlsh_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DETLSH_H_ */
