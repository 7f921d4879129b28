/*
 * d2.h -- C-ABI of the GB300 (sm_103a) assignment step of parallel
 * D2-clustering (Zhang, Wang & Li, "Parallel D2-Clustering: Large-Scale
 * Clustering of Discrete Distributions", arXiv 1302.0435).
 *
 * Objects and centroids are discrete distributions ("bags of weighted
 * vectors", Sec. 2, the notation above Eq. (D2opt)):
 *     v = {(v^(a), p^(a)) : a = 1..t},   v^(a) in R^d,  p^(a) >= 0.
 * The distance between a bag and a centroid is the Mallows distance: the
 * optimum of the transportation LP of Eq. (D2opt) with the centroid fixed,
 *     D^2(z, v) = min_w sum_{r,a} w_{r,a} ||z^(r) - v^(a)||^2
 *     s.t. sum_a w_{r,a} = p_z^(r),  sum_r w_{r,a} = p_v^(a),  w >= 0.
 * Every call returns D^2 (the squared distance); D itself is its root.
 *
 * Conventions common to every call
 *  - Status: every call returns an int, D2_OK (0) or a negative D2_E* code;
 *    d2_strerror() names it.  Nothing crosses this boundary as an exception
 *    or abort.  A call that fails leaves its outputs unspecified.
 *  - Weights: each bag's weights are divided by their sum in FP64 before use
 *    (the total-mass-one constraint of Eq. (D2opt)).  A bag with a negative,
 *    NaN or infinite weight, a zero total, or no support is rejected with
 *    D2_EINVAL.  Zero-weight supports are allowed.
 *  - Memory: the caller owns every buffer it passes.  Pointers may address
 *    device memory (cudaMalloc, torch CUDA tensors) or host memory (pageable
 *    or pinned); the library tells them apart with cudaPointerGetAttributes.
 *    Host inputs are copied to device scratch owned by the context and host
 *    outputs are copied back before the call returns.  The library never
 *    frees caller memory.
 *  - Streams: work is enqueued on the context's stream (d2_set_stream).
 *    d2_mallows_batch, d2_assign, d2_mallows_all and d2_update_locations
 *    return without waiting when all their outputs are device pointers and
 *    their bags declare max_support (with 0, a scan of the offsets waits
 *    first); the first call of a new launch shape may also wait for the
 *    autotuner, and BF16 batches screened with tensor-core tiles wait for
 *    their bin counts.  Outputs are valid after d2_sync() or an event
 *    recorded on that stream.  A call with any host output waits before it
 *    returns; so do the other calls.
 *  - Errors of calls that return without waiting (bad offsets or weights,
 *    pivot budgets, device timeouts) are raised on the device and reported
 *    by the next d2_sync(), or by the next call that waits, which then
 *    returns that code; a call that waits on entry (d2_set_centroids,
 *    d2_cost_matrix, d2_update_weights, d2_assign_multi, d2_segment,
 *    d2_cluster_level) returns such a pending code at once and does
 *    nothing else.  Reporting an error clears it.
 *  - Threads: one context per host thread; a context is not re-entrant.
 *  - Precision: see d2_config.precision.  D^2 outputs are FP64.
 */
#ifndef D2_H
#define D2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define D2_OK 0
#define D2_EINVAL (-1)          /* bad argument, offsets, sizes or weights */
#define D2_ENOMEM (-2)          /* device or host allocation failed */
#define D2_ENOTCONVERGED (-3)   /* a pair hit its pivot budget (see per-pair status) */
#define D2_ETIMEOUT (-4)        /* a device wait gave up (serving loop) */
#define D2_ECUDA (-5)           /* a CUDA runtime call failed */
#define D2_EUNSUPPORTED (-6)    /* size or dtype outside what the kernels support */
#define D2_ENOCENTROIDS (-7)    /* no resident centroid set */

/* element types */
#define D2_F64 0
#define D2_F32 1
#define D2_BF16 2

/* precision modes (d2_config.precision) */
#define D2_PREC_AUTO 0   /* FP64 for FP64 inputs, otherwise D2_PREC_FP32 */
#define D2_PREC_FP64 1   /* costs, duals, pricing and objective in FP64 */
#define D2_PREC_FP32 2   /* FP32 cost tile and FP32 pivots reach a basis; the
                            same tree and exact integer flows then continue on
                            an FP64 tile with FP64 potentials until no FP64
                            reduced cost is negative, and the objective is
                            summed in FP64.  d2_assign screens all centroids
                            with the FP32 solve alone and certifies in FP64
                            every centroid the FP32 error bound cannot rule
                            out, so labels and dist2 are FP64-exact. */

/* d2_cost_matrix only: the FP32 tile the tensor-core contraction gives
   (||x||^2 + ||y||^2 - 2 x.y over BF16 operands with FP32 accumulation),
   widened to FP64.  Needs BF16 objects and dim a multiple of 16 in 16..256. */
#define D2_PREC_TC 3

/* tensor-core ground costs for the FP32 screen of d2_assign (d2_config.cost_tc) */
#define D2_TC_AUTO 0  /* on for BF16 objects with dim a multiple of 16 in 64..256 */
#define D2_TC_OFF 1   /* the screen builds its FP32 tiles with SIMT FMAs */
#define D2_TC_ON 2    /* on for BF16 objects with dim a multiple of 16 in 16..256 */

/* cold-start basis of the simplex (d2_config.start_rule) */
#define D2_START_AUTO 0    /* the autotuner times both on large batches; otherwise
                              Vogel for centroids of 64 supports, else RANKED */
#define D2_START_RANKED 1  /* northwest staircase in principal-direction order */
#define D2_START_VOGEL 2   /* Vogel's approximation (largest-penalty line first) */

/* centroid update of d2_cluster_level's rounds (d2_config.centroid_update) */
#define D2_UPDATE_CONSTRAINED 0  /* Alg. 2 Step 3*: support weights fixed, locations by
                                    Eq. (WeightedUpdate) */
#define D2_UPDATE_ALG1 1         /* Alg. 1 (weighted D2-clustering, Alg. 3 Step 2): support
                                    weights by the joint LP (d2_update_weights), then the
                                    locations with flows at the new weights */

/* which screened pairs are certified in FP64 (d2_config.certify) */
#define D2_CERTIFY_CANDIDATES 0  /* only the centroids the FP32 error bound cannot rule
                                    out of the argmin (labels and dist2 stay FP64-exact) */
#define D2_CERTIFY_ALL 1         /* every (object, centroid) pair: the FP32-optimal basis
                                    of each pair gets an optimality certificate of FP64
                                    accuracy (the basic cells' costs in double-float,
                                    potentials corrected to them, the objective summed in
                                    FP64, reduced costs checked against a rounding bound
                                    and the few near the bound re-priced), so its
                                    D^2 is the FP64 objective of a feasible plan within
                                    max(2^-24 D^2, 2^-43 c_max) of the optimum; a pair that
                                    fails the check is solved to FP64 optimality */

/* segments of d2_cluster_level (d2_config.segmentation) */
#define D2_SEG_SLICES 0       /* contiguous slices of seg_size objects */
#define D2_SEG_CONSTRAINED 1  /* the binary constrained D2 splits of d2_segment */

/* Limits of the current kernels. */
#define D2_MAX_SUPPORT 64   /* supports per bag (objects and centroids) */
#define D2_MAX_DIM 256      /* vector dimension d */
#define D2_JOINT_MAX_ITER 4096  /* rounds of d2_update_weights */

/*
 * A ragged batch of bags in CSR form.  Bag b owns supports
 * [off[b], off[b+1]) of loc (row-major, dim values per support, element type
 * loc_dtype) and w (element type w_dtype, D2_F64 or D2_F32).  off has
 * count+1 entries, off[0] = 0, nondecreasing.  All three pointers must be in
 * the same memory space (all device or all host).
 * max_support: 0, or the caller's bound on every bag's support count
 * (1..D2_MAX_SUPPORT).  With a bound the calls need not read the offsets
 * back to size their kernels, so a call with device outputs returns without
 * waiting; the kernels check every bag against it (a bag with no support
 * or above the bound is reported as D2_EINVAL, by d2_sync for such calls).
 * With 0 the calls scan the offsets first, which waits for the stream.
 */
typedef struct {
    const void* loc;
    const void* w;
    const int64_t* off;
    int64_t count;
    int32_t dim;
    int32_t loc_dtype;
    int32_t w_dtype;
    int32_t max_support;
} d2_bags;

/* Context configuration; zero-initialise and set what you need. */
typedef struct {
    int32_t precision;          /* D2_PREC_* ; 0 = AUTO */
    int32_t pivot_budget;       /* pivots per pair = pivot_budget*(m+n); 0 = 64 */
    int32_t group_lanes;        /* lanes per pair: every pair is solved by one warp
                                   (32 lanes, one tree node per lane and bin).
                                   0 = the launch shape (threads per block, screening
                                   items per SM, cold-start rule) is autotuned per
                                   support bin on large batches; 32 = the default shape,
                                   no tuning; other values are rejected (D2_EINVAL) */
    int32_t cost_tc;            /* D2_TC_* ; 0 = AUTO */
    int32_t tile_budget_mib;    /* device memory for tensor-core cost tiles;
                                   0 = min(32 GiB, 40% of free memory) */
    int32_t start_rule;         /* D2_START_* ; 0 = AUTO */
    int32_t segmentation;       /* D2_SEG_* : how d2_cluster_level forms segments */
    int32_t split_iters;        /* update rounds per binary split of D2_SEG_CONSTRAINED;
                                   0 = 10 */
    double eps_tol;             /* d2_cluster_level: > 0 ends a level's rounds early once
                                   the objective sum_i omega_i D^2(v_i, z_C(i)) changes by
                                   at most eps_tol relative between rounds ("until epsilon
                                   converges", Alg. 2 Step 4); 0 = exactly `iters` rounds */
    int32_t centroid_update;    /* D2_UPDATE_* ; 0 = CONSTRAINED */
    int32_t joint_max_iter;     /* D2_UPDATE_ALG1: cutting-plane rounds per weight update;
                                   0 = 512 */
    double joint_tol;           /* D2_UPDATE_ALG1: relative gap of the weight LP; 0 = 1e-9 */
    int32_t certify;            /* D2_CERTIFY_* : d2_assign and d2_cluster_level;
                                   0 = CANDIDATES */
    int32_t tc_wait_probe;      /* diagnostic, 0 = off: > 0 makes the tensor-core kernel's
                                   first completion wait poll a barrier nothing arrives on
                                   (at most this many non-blocking polls), so it runs out
                                   and the call reports D2_ETIMEOUT after the kernel has
                                   waited for its issued MMAs and freed its tensor memory;
                                   tests of the timeout path use it */
    int32_t no_prune;           /* 0: d2_assign, d2_cluster_level and serving (without
                                   D2_CERTIFY_ALL) skip the pairs that cannot be an
                                   object's argmin: D^2 >= ||mean_P - mean_Q||^2 (Jensen),
                                   and the product plan bounds D^2 from above by that plus
                                   both bags' spreads, so a centroid whose lower bound
                                   exceeds the object's best upper bound is never solved
                                   (labels and distances unchanged); 1: every pair solved */
    int32_t joint_cold_start;   /* 0: each cutting-plane round of d2_update_weights (and of
                                   D2_UPDATE_ALG1 levels) restarts every member's LP from its
                                   optimal basis of the round before: only the centroid
                                   weights changed, so that basis stays dual feasible, and
                                   dual simplex pivots restore its flows (same optima); 1:
                                   every round solves every member from a cold start */
    int32_t warm_budget_mib;    /* device memory d2_cluster_level may take for the bases it
                                   keeps between rounds; 0 = 40% of the free memory.  The
                                   full store is 11 B per tree node and pair; when only its
                                   trees fit (3 B per node) the flows are recomputed on
                                   reload (same results, slower; not with
                                   D2_CERTIFY_ALL); below that the rounds start cold */
} d2_config;

/*
 * Optimal flows of solved pairs, one record of `stride` entries per pair:
 * entry e of pair t is (cell[t*stride+e], w[t*stride+e]) with
 * cell = (a << 16) | r (a: object support, r: centroid support) and w the
 * flow (mass moved from v^(a) to z^(r), total 1 per pair).  A pair uses
 * m+n-1 entries (its basis; some flows may be zero); unused entries have
 * cell = -1 and w = 0.  stride must be >= 2*D2_MAX_SUPPORT-1 or >= the
 * largest m+n-1 of the call.  Both arrays are caller-owned, device or host.
 */
typedef struct {
    int32_t* cell;
    double* w;
    int64_t stride;
} d2_flows;

typedef struct d2_ctx d2_ctx;

/* Create a context on CUDA device `device`.  cfg may be NULL (defaults).
 * A field outside its documented values (an unknown mode, a negative count
 * or budget) is rejected with D2_EINVAL before any device work.
 * Creates its own stream, a blocking one: it is ordered with the legacy
 * default stream, so device inputs written there (for instance by a
 * framework's default stream) are complete before the context's kernels
 * read them.  Work on other streams must be ordered by the caller (events,
 * or d2_set_stream).  Returns D2_ECUDA if the device cannot be used (no
 * GPU, or the library was not built for it). */
int d2_ctx_create(d2_ctx** out, int32_t device, const d2_config* cfg);
/* Destroy a context and free everything it owns (not caller buffers). */
int d2_ctx_destroy(d2_ctx* ctx);
/* Use the caller's cudaStream_t (NULL: back to the context's own stream). */
int d2_set_stream(d2_ctx* ctx, void* cuda_stream);
/* Wait for all work enqueued by this context; returns (and clears) the
 * first error its kernels raised since the last report, D2_OK if none. */
int d2_sync(d2_ctx* ctx);
/* Static description of a status code. */
const char* d2_strerror(int32_t status);
/* Version string of the library build. */
const char* d2_version(void);

/*
 * Set the resident centroid set z_1..z_K (Alg. 2 Step 1 hands in the
 * initial centroids; the paper draws them at random).  The bags are copied
 * into context-owned device memory and stay resident across calls; their
 * weights are normalised once.  loc_dtype decides the storage precision of
 * the centroid locations: d2_update_locations rounds its FP64 result to it.
 */
int d2_set_centroids(d2_ctx* ctx, const d2_bags* cents);
/* Read back the resident centroids: loc_out [sum n_j][dim] FP64, w_out
 * [sum n_j] FP64 (normalised), off_out [K+1] int64; any may be NULL.
 * Pointers may be host or device.  K and total supports via k_out/t_out. */
int d2_get_centroids(d2_ctx* ctx, double* loc_out, double* w_out, int64_t* off_out,
                     int64_t* k_out, int64_t* t_out);

/*
 * Symbol ground costs (the sequence variant of Eq. (D2opt)): with a table
 * set, supports are symbol ids (dim 1, integer values in [0, A)) and the
 * cost between symbols s and t is table[s*A + t] instead of the squared
 * Euclidean distance; Mallows distances, labels and plans are computed as
 * before.  table: [A][A] FP64, nonnegative and finite, host or device,
 * copied.  A = 0 (or table NULL) removes it.  The resident centroids, and
 * every later batch, must be symbol ids (else D2_EINVAL).  Symbolic
 * supports are not moved: d2_update_locations and d2_cluster_level return
 * D2_EUNSUPPORTED while a table is set.  A*A at most 2^26.
 */
int d2_set_cost_table(d2_ctx* ctx, const double* table, int32_t A);

/*
 * Ground-cost matrix of one pair (the objective coefficients of
 * Eq. (D2opt)): C[a*n_j + r] = ||v_i^(a) - z_j^(r)||^2 for object i of
 * `objs` and resident centroid j, as the kernels compute it in `precision`
 * (D2_PREC_FP64: FP64 explicit differences; D2_PREC_FP32: the FP32 tile the
 * FP32 solver prices with, widened to FP64; D2_PREC_TC: the tensor-core tile
 * the FP32 screen of d2_assign reads when cost_tc is on, D2_EUNSUPPORTED if
 * the objects are not BF16 or dim is not a multiple of 16 in 16..256).
 * C: m_i*n_j doubles.
 */
int d2_cost_matrix(d2_ctx* ctx, const d2_bags* objs, int64_t i, int64_t j, int32_t precision,
                   double* C);

/*
 * Mallows distance D^2 (Eq. (D2opt) with z fixed) for npairs listed pairs
 * (object pair_obj[t] of `objs`, resident centroid pair_cen[t]).
 * dist2[t]: FP64 result.  flows (may be NULL): optimal basis flows per pair.
 * status (may be NULL): per-pair D2_OK / D2_ENOTCONVERGED / D2_EINVAL.
 * Returns D2_ENOTCONVERGED if any pair hit its pivot budget (its dist2 is
 * then the cost of the last feasible plan, an upper bound).
 */
int d2_mallows_batch(d2_ctx* ctx, const d2_bags* objs, const int64_t* pair_obj,
                     const int64_t* pair_cen, int64_t npairs, double* dist2, d2_flows* flows,
                     int32_t* status);

/*
 * Alg. 2 Step 2: labels[i] = argmin_j D(v_i, z_j) over the resident
 * centroids (ties: smallest j), dist2[i] = D^2(v_i, z_labels[i]) in FP64.
 * omega (may be NULL = all ones): object weights omega_i of Eq. (WeightedD2).
 * eps_total (may be NULL): sum_i omega_i dist2[i], the objective of
 * Eq. (WeightedD2) at the current centroids (Alg. 1 Step 3 / Alg. 2 Step 4).
 * flows (may be NULL): optimal flows of each assigned pair (i, labels[i]),
 * which d2_update_locations can consume.
 */
int d2_assign(d2_ctx* ctx, const d2_bags* objs, const double* omega, int32_t* labels,
              double* dist2, double* eps_total, d2_flows* flows);

/*
 * Mallows distance of every (object, resident centroid) pair, Eq. (D2opt)
 * with z fixed for each z_j, and the argmin of Alg. 2 Step 2 over them:
 * dist2_all [count][K] (row-major: dist2_all[i*K + j] = D^2(v_i, z_j)),
 * labels [count] and dist2 [count] as d2_assign (either may be NULL).
 * Every value is certified in FP64 as with D2_CERTIFY_ALL (FP32 inputs),
 * or solved in FP64 throughout (FP64 inputs or D2_PREC_FP64): it lies
 * within max(2^-24 D^2, 2^-43 c_max) of the LP optimum, c_max the pair's
 * largest ground cost; values the argmin needs closer are solved to FP64
 * optimality.  Host or device pointers.
 */
int d2_mallows_all(d2_ctx* ctx, const d2_bags* objs, double* dist2_all, int32_t* labels,
                   double* dist2);

/*
 * Centroid location update, Eq. (WeightedUpdate) (Eq. (UpdateZ) when omega
 * is NULL), with the centroid weights held fixed as in Alg. 2 Step 3*:
 *     z_j^(r) <- sum_{i:C(i)=j} omega_i sum_a w^(i)_{r,a} v_i^(a)
 *               / sum_{i:C(i)=j} omega_i sum_a w^(i)_{r,a}
 * where w^(i) is the optimal flow of pair (i, labels[i]).  flows: the flows
 * d2_assign returned for these labels, or NULL to re-solve the N assigned
 * pairs.  Updates the resident centroids in place; a support whose
 * denominator is zero (empty cluster, no mass) keeps its location.
 * Summation order is fixed (objects in index order), so results are
 * deterministic run to run.
 */
int d2_update_locations(d2_ctx* ctx, const d2_bags* objs, const double* omega,
                        const int32_t* labels, const d2_flows* flows);

/*
 * Centroid weights of Alg. 1 Step 1: for every cluster j, with the support
 * locations z_j^(r) fixed, the weights p_j and all member flows that solve
 * the joint LP of Eq. (WeightedD2) under the constraints of Eq. (D2opt)
 * (omega NULL = 1):
 *     min_{p_j, w} sum_{i:C(i)=j} omega_i sum_{r,a} w^(i)_{r,a} c(z_j^(r), v_i^(a))
 *     s.t. sum_r p_jr = 1, sum_a w^(i)_{r,a} = p_jr, sum_r w^(i)_{r,a} = q_i^(a), p, w >= 0.
 * Replaces the resident centroid weights by the optimal p_j (d2_get_centroids
 * reads them back).  Given p_j the LP separates into the members' own
 * transportation LPs, so a following d2_update_locations (Alg. 1 Step 2,
 * Eq. (WeightedUpdate)) with the same labels moves the supports with
 * optimal flows of the joint LP.  Method: exact member solves give one
 * supporting cut of the objective per round (LP duality), and Kelley's
 * cutting-plane rounds choose the next p_j; a cluster stops when its best
 * objective and the cut model's lower bound agree within relative gap `tol`
 * (e.g. 1e-9), or after max_iter rounds (1..D2_JOINT_MAX_ITER) with the best
 * weights found.  labels: [count] cluster of every object (host or device;
 * labels outside [0, K) are ignored).  eps_out [K] (may be NULL): the
 * objective of Eq. (WeightedD2) at the new weights; iters_out [K] (may be
 * NULL): rounds used (0 for an empty cluster, whose weights are kept).
 * Works with a symbol cost table too (weights move, supports do not).
 * Device memory: about K * max_iter * (n_max + 1) doubles of cuts.
 * Returns D2_ENOTCONVERGED if any cluster was not certified within
 * max_iter rounds (its weights are still the best found), D2_EUNSUPPORTED
 * for centroids of more than 64 supports.
 */
int d2_update_weights(d2_ctx* ctx, const d2_bags* objs, const double* omega,
                      const int32_t* labels, int32_t max_iter, double tol, double* eps_out,
                      int32_t* iters_out);

/*
 * Nearest centroid under the combined distance of several bag types
 * (Eq. (imgdist)): object i is B bags, one per type, and
 * D^2(I_i, Z_j) = sum_b D^2(U_i^b, Z_j^b).  ctxs[b] holds type b's resident
 * centroids (all on one device, all with the same K; one context per type);
 * objs[b] holds type b's bag of every object (same count).  labels [count]
 * and dist2 [count] (the summed FP64 D^2; ties to the smallest j), host or
 * device.  Each type's FP32 screen bounds every pair; the candidates of the
 * summed bounds are solved exactly by every type.  Each type's centroids
 * are then updated on their own (d2_update_locations on ctxs[b] with these
 * labels).  B at most 8.
 */
int d2_assign_multi(d2_ctx* const* ctxs, int32_t B, const d2_bags* objs, int32_t* labels,
                    double* dist2);

/*
 * d2_cluster_level with the support weights of the result as well:
 * out_support_w [K*n] (host or device, may be NULL).  With the default
 * D2_UPDATE_CONSTRAINED they stay the resident set's; with D2_UPDATE_ALG1
 * every round of every level re-solves them (Alg. 1 Step 1) and the next
 * level's data carry them.  D2_ENOTCONVERGED when a weight LP was not
 * certified within joint_max_iter rounds (its best weights were used).
 */
int d2_cluster_level_ex(d2_ctx* ctx, const d2_bags* objs, const double* omega, int32_t K,
                        int64_t seg_size, int32_t iters, double* out_loc, double* out_support_w,
                        double* out_cent_weight, int32_t* labels);

/*
 * Initial data segmentation (Alg. 3 Step 1): split the bags into segments of
 * at most tau bags by repeated binary splits of the largest segment (ties:
 * the one formed first).  A split is a constrained D2-clustering with k = 2
 * (Alg. 2 with Step 3*): start centroids are the segment's first bag and
 * the bag with the largest D^2 to it (ties: the first), both with uniform
 * weights; then assign, and up to `iters` times update the locations with
 * the weights held fixed (Eq. (WeightedUpdate) with omega, NULL = 1) and
 * assign again, stopping when the labels repeat.  The first part keeps the
 * parent's place; a split with an empty side halves the segment instead.
 * seg_id [count] (host or device) receives the segment of every bag,
 * segments numbered by their smallest bag; *n_segments their number.
 * Needs no resident centroids.
 */
int d2_segment(d2_ctx* ctx, const d2_bags* objs, const double* omega, int64_t tau,
               int32_t iters, int32_t* seg_id, int64_t* n_segments);

/*
 * One hierarchical clustering job in the manner of Alg. 3 on one GPU:
 * the current data are split into contiguous segments of at most seg_size
 * (tau) objects; every segment starts from the resident centroid set (which
 * must hold K centroids) and runs `iters` rounds of (d2_assign,
 * d2_update_locations) -- all segments in one batched launch per step; the
 * labels are merged with Eq. (UpdateLabel) and Eq. (UpdateGlobalLabel); each
 * centroid's weight is the summed omega of its members; if more than one
 * segment was used the merged centroids become the next level's weighted
 * data, until a level fits in one segment.  seg_size must exceed K.
 * Outputs (caller-allocated, host or device):
 *   out_loc  [K*n][dim] FP64 final centroid locations (n = resident n),
 *   out_cent_weight [K] FP64 summed member weights,
 *   labels   [N] int32 final cluster of every object.
 * The resident centroid set is left unchanged.
 */
int d2_cluster_level(d2_ctx* ctx, const d2_bags* objs, const double* omega, int32_t K,
                     int64_t seg_size, int32_t iters, double* out_loc, double* out_cent_weight,
                     int32_t* labels);

/*
 * Serving: continuous batching of assignment requests (Alg. 2 Step 2)
 * against the context's resident centroid set.  A worker thread admits
 * queued requests into `slots` concurrent slots (one CUDA stream each) as
 * slots free up and as long as the device bytes of the requests in flight
 * stay within mem_budget_bytes (0 = 8 GiB; a request larger than the budget
 * is admitted alone).  Requests that arrive while others are on the GPU are
 * admitted at once and their kernels overlap on the device.  Every request
 * is solved by the same deterministic per-pair solver as d2_assign, so its
 * labels and distances are identical alone and in any mix.  The resident
 * centroid set must not change while a server exists.
 *
 * d2_server_submit copies a host request (objs: host pointers) and returns a
 * ticket at once.  d2_server_poll waits up to timeout_ms (<0: forever) for
 * a ticket, copies its labels [N] and dist2 [N] (host pointers, may be NULL)
 * and the submit-to-completion latency in ms, and forgets the ticket;
 * returns D2_ETIMEOUT if not done yet (the ticket stays valid).
 */
typedef struct d2_server d2_server;
int d2_server_create(d2_server** out, d2_ctx* ctx, int32_t slots, int64_t mem_budget_bytes);
int d2_server_submit(d2_server* srv, const d2_bags* objs, int64_t* ticket);
int d2_server_poll(d2_server* srv, int64_t ticket, int32_t* labels, double* dist2,
                   double* latency_ms, int32_t timeout_ms);
int d2_server_stats(d2_server* srv, int64_t* admitted, int64_t* completed, int64_t* peak_inflight,
                    int64_t* queued);
int d2_server_destroy(d2_server* srv);

/*
 * d2_update_locations_noalloc -- the location update of d2_update_locations
 * (the same kernels) for callers that cannot call cudaMalloc during the
 * call: for instance a framework that owns all device memory through its
 * own caching allocator and a fixed budget, so an outside allocation would
 * exceed or fragment it, or a latency-critical serving loop that must not
 * pay for the allocator's implicit device synchronisation.  It allocates
 * nothing: no cudaMalloc, cudaFree or allocating library routine.  The
 * paper has no counterpart; this is an integration variant only.
 *
 * Results: with at most 512*K bags, d2_update_locations sums each centroid
 * in one block, as this call always does, and the two give identical
 * centroids.  Beyond that d2_update_locations splits large clusters over
 * several blocks and adds the parts, a different summation order; the two
 * then agree to the rounding of those FP64 sums, i.e. within one unit in
 * the last place of the centroid location type (cent_loc_dtype) after the
 * final rounding to it.
 *
 * Scratch: a fixed array of about 3 MB in the library's own device memory
 * (a file-scope __device__ array), which every GPU that loads the library
 * holds until the process exits.  With lazy module loading the first call
 * on a device may be the one that loads the module and, with it, that
 * array.  Limits: at most 262,144 bags and 1,024 centroids per call; larger
 * calls return D2_EUNSUPPORTED.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress, once per device, with the
 * device current).  Every call shares the one array: calls whose work
 * overlaps on the GPU (other streams, other host threads) race and give
 * wrong results, so serialise them.  The sort counters and the offset check
 * words are cleared at the start of every call.
 *
 * Waiting: every call waits once on cuda_stream, to read back the check of
 * the bag offsets and the centroid offsets; it therefore cannot be
 * captured into a CUDA graph.  After that wait it enqueues the update and
 * returns without waiting for it.
 *
 * Arguments (all device pointers of the current device, caller-owned; host
 * pointers or another device's memory -> D2_EINVAL):
 *   objs (offsets checked on the device: off[0] = 0 and every bag
 *   1..D2_MAX_SUPPORT supports, else D2_EINVAL), omega (may be NULL = all
 *   ones), labels [N] int32 (centroid index in [0,K), others ignored), flows
 *   (required: the d2_assign flow records of the assigned pairs; entries
 *   that are not cells of their pair are ignored), cent_off [K+1] int64
 *   (centroid j owns supports [cent_off[j], cent_off[j+1]), 1..D2_MAX_SUPPORT
 *   of them, else D2_EINVAL), cent_loc64 [T][dim] FP64 centroid locations,
 *   updated in place, cent_loc32 [T][dim] FP32 mirror, rewritten where a
 *   location changes, cent_loc_dtype: the centroid location type the FP64
 *   result is rounded to (as d2_set_centroids' loc_dtype does for the
 *   resident set), cuda_stream: the stream to enqueue on (NULL = legacy
 *   default stream).
 */
int d2_update_locations_noalloc(const d2_bags* objs, const double* omega, const int32_t* labels,
                                const d2_flows* flows, int64_t K, const int64_t* cent_off,
                                int32_t cent_loc_dtype, double* cent_loc64, float* cent_loc32,
                                void* cuda_stream);

/*
 * Counters of this process's library activity (diagnostics, not a paper
 * quantity), monotonic since library load: kernels launched; pair LPs
 * solved on the FP32 screening path and their simplex pivots; pair LPs
 * solved to FP64 optimality and their pivots (FP32 warm start + FP64);
 * cutting-plane rounds of d2_update_weights (summed over calls) and the
 * pivots of its per-cluster master LPs; screened pairs whose FP32-optimal
 * basis passed the FP64 certificate of D2_CERTIFY_ALL (the others are
 * solved to FP64 optimality and counted in pairs_exact), and the cells the
 * certificate had to re-price in FP64.
 * Reading the device counters synchronises the current device.
 */
typedef struct {
    int64_t kernel_launches;
    int64_t pairs_screened;
    int64_t pivots_screened;
    int64_t pairs_exact;
    int64_t pivots_exact;
    int64_t joint_rounds;
    int64_t joint_master_pivots;
    int64_t pairs_certified;
    int64_t cells_checked;
} d2_stats;
int d2_get_stats(d2_stats* out);

#ifdef __cplusplus
}
#endif

#endif /* D2_H */
