/*
 * tsqbx.h -- C ABI of libtsqbx: the near-field target-specific QBX (TSQBX)
 * step of GIGAQBX (Wala & Kloeckner, arXiv:1811.01110), on one GB300 GPU.
 *
 * What one evaluation computes (Alg. 1 Stages 3, 5(a), 6(a); Sec. 2.6
 * eq. tsqbx; Appendix A).  For every target t with QBX center c = center(t),
 * and every source s listed in the pair list of c's group (List 1, List 3
 * close and List 4 close of c's owning box, given as half-open index ranges,
 * Sec. 3.2), the library adds w_s mu_s K^(p)(t, s) to the target's output,
 * where K^(p) is the p-th order target-specific expansion about c:
 *
 *   Laplace single layer   G^(p)   = 1/(4 pi) sum_{n<=p} |t-c|^n / |s-c|^{n+1} P_n(cos g)
 *   Laplace double layer   n_s . grad_s G^(p)                         (Appendix A)
 *   Helmholtz single layer G_k^(p) = ik/(4 pi) sum_{n<=p} (2n+1) j_n(k|t-c|)
 *                                     h_n(k|s-c|) P_n(cos g)         (Appendix A)
 *   Helmholtz double layer n_s . grad_s G_k^(p)
 *   S' (either kernel)     n_t . grad_t G^(p), n_t . grad_t G_k^(p), the
 *                          target-normal derivative with the center c held
 *                          fixed (Appendix A)
 *
 * g is the angle between s-c and t-c, j_n / h_n the spherical Bessel and
 * Hankel functions of the first kind.  The result is the near part
 * L^{qbx,near}_c(t) of the QBX local expansion at each target (Sec. 3.3); the
 * far part is the caller's.  Pair lists are summed exactly as given:
 * duplicated ranges count twice.
 *
 * Conventions for every entry point:
 *  - Status: 0 (TSQBX_OK) on success, TSQBX_PENDING (1) from tsqbx_poll while
 *    work is in flight, a negative TSQBX_E_* code on error.  No C++ exception
 *    crosses the ABI; tsqbx_strerror() names every code.
 *  - Arrays are structure-of-arrays: an "xyz [3][n]" array holds the n x
 *    coordinates, then the n y, then the n z coordinates (doubles).
 *  - Geometry pointers are HOST pointers, read only during tsqbx_plan_create
 *    and owned by the caller; the plan keeps its own device copies.
 *  - Density / output pointers may be host or device memory where stated.
 *  - Every entry point is thread-safe with respect to different plans; calls
 *    on one plan must not run concurrently from several host threads, except
 *    tsqbx_poll.
 */
#ifndef TSQBX_H
#define TSQBX_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TSQBX_API __attribute__((visibility("default")))
#else
#define TSQBX_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Highest expansion order accepted (the paper's experiments use p <= 9 for
 * Laplace and p = 4 for Helmholtz, Sec. 5). */
#define TSQBX_P_MAX 20

/* ---------------------------------------------------------------- status */
enum {
    TSQBX_OK = 0,
    TSQBX_PENDING = 1,         /* tsqbx_poll: still running                        */
    TSQBX_E_INVAL = -1,        /* bad sizes, null pointers, index out of range, p   */
    TSQBX_E_DIVERGENT = -2,    /* a listed pair has |t-c| >= |s-c| or s == c        */
    TSQBX_E_NOMEM = -3,        /* device or pinned-host allocation failed           */
    TSQBX_E_CUDA = -4,         /* a CUDA runtime call failed                        */
    TSQBX_E_TIMEOUT = -5,      /* tsqbx_poll: not done within the timeout           */
    TSQBX_E_BUSY = -6,         /* tsqbx_submit: every slot of the plan is in flight */
    TSQBX_E_NOTFOUND = -7,     /* unknown or already collected ticket               */
    TSQBX_E_KERNEL = -8,       /* a kernel flagged an out-of-range index            */
    TSQBX_E_UNSUPPORTED = -9,  /* kernel/layer/precision combination not provided   */
    TSQBX_E_TOO_LARGE = -10    /* tsqbx_eval_noalloc: more sources than its scratch */
};

/* ------------------------------------------------------------- options */
typedef enum { TSQBX_LAPLACE = 0, TSQBX_HELMHOLTZ = 1 } tsqbx_kernel;

/* layer mask: single layer, double layer (source-normal derivative
 * n_s . grad_s), and S' (target-normal derivative n_t . grad_t, Appendix A;
 * needs tgt_normal and the *_pk entry points, which take an S' output) */
enum { TSQBX_SLP = 1u, TSQBX_DLP = 2u, TSQBX_SP = 4u };

/* FP64: every step in double precision (results within 1e-12 relative of an
 *       FP64 reference).
 * MIXED (Laplace only): coordinates differenced in float-float, the
 *       recurrence and geometry ratios in FP32, per-lane sums Kahan-
 *       compensated in FP32 and per-target reduction in FP64 (results within
 *       1e-6 relative of an FP64 reference).
 * DF64 (Laplace only): every step in double-float arithmetic (pairs of FP32
 *       values, ~48-bit significands) on the FP32 pipes, geometry differenced
 *       in FP64 against a per-item reference point; results within the FP64
 *       bound (1e-12 relative).  On GPUs whose FP64 rate is a small fraction
 *       of FP32 (GB300: 1/61) this reaches FP64-class accuracy faster. */
typedef enum { TSQBX_FP64 = 0, TSQBX_MIXED = 1, TSQBX_DF64 = 2 } tsqbx_precision;

enum {
    TSQBX_FLAG_ALLOW_DIVERGENT = 1u,  /* accept pairs with |t-c| >= |s-c| (report only) */
    TSQBX_FLAG_SKIP_CHECK = 2u,       /* do not run the per-pair convergence check      */
    TSQBX_FLAG_USE_TUNED = 4u,        /* start from the process-wide tuning cache entry
                                         matching (kernel, precision, p, layers, list
                                         shape), if tsqbx_plan_autotune stored one      */
    /* Conventional QBX (Sec. 2.1 eqs. local-coeffs, local-expansion) for chosen
     * centers: the center's local coefficients L_n^m are formed from its
     * group's list (P2QBXL, (p+1)^2 per source) and evaluated at each of its
     * targets (QBXL2P, (p+1)^2 per target), instead of the target-specific
     * expansion ((p+1) per target and source).  The values are the same
     * truncated expansion (eq. tsqbx; Appendix A's addition theorem for
     * Helmholtz).  FP64 only (else TSQBX_E_UNSUPPORTED); such plans accept
     * per-call orders up to their own p.  Helmholtz: p <= 12 (with
     * CONVENTIONAL_ALL a larger p is TSQBX_E_UNSUPPORTED; CONVENTIONAL_AUTO
     * keeps every center target-specific). */
    TSQBX_FLAG_CONVENTIONAL_AUTO = 8u,  /* per center, whichever the cost model (Table 2
                                           form, GPU constants) says is cheaper        */
    TSQBX_FLAG_CONVENTIONAL_ALL = 16u,  /* every center takes the conventional path     */
    /* The plan's streams get a CUDA stream priority from the plan's work: the
     * listed pairs times a per-kernel/precision cost, one priority level per
     * decade above 1e5 pair-equivalents, the highest for the smallest plans.
     * When several plans run at once, pending thread blocks of short
     * evaluations are then dispatched before those of long ones.  Results
     * are unchanged.  See tsqbx_server_set_size_priority. */
    TSQBX_FLAG_SIZE_PRIORITY = 32u
};

typedef struct {
    tsqbx_kernel kernel;
    uint32_t layers;            /* TSQBX_SLP | TSQBX_DLP | TSQBX_SP                   */
    int p;                      /* expansion order, 0 <= p <= TSQBX_P_MAX             */
    double k;                   /* Helmholtz wavenumber (> 0); ignored for Laplace    */
    tsqbx_precision precision;
    int device;                 /* CUDA device ordinal                                */
    uint32_t flags;             /* TSQBX_FLAG_*                                       */
    int lanes_per_target;       /* 0 = chosen per group; 1..32 forces a value         */
    int n_slots;                /* concurrent submits per plan; 0 = 2                 */
    int max_item_iters;         /* cap on per-lane pair iterations of one warp item;
                                   longer lists are cut into source slices whose
                                   partial sums are added in slice order; 0 = automatic
                                   (32..512, scaled to the problem and the SM count) */
    int tile_depth;             /* sources a warp stages per shared-memory tile: 32, 64
                                   or 128; 0 = 64.  Results agree across depths to
                                   rounding (the order of the lanes' sums changes)     */
    int max_rhs;                /* densities one tsqbx_submit_multi_layers may carry,
                                   1..4; 0 = 1.  Above 1 only for Helmholtz
                                   single-layer plans and for Laplace plans in
                                   FP64 or double-float whose layers are the single
                                   and/or double layer (else TSQBX_E_UNSUPPORTED);
                                   each slot then holds scratch for that many
                                   densities                                        */
    int p_unroll;               /* how the order loop of the Laplace FP64 and mixed
                                   kernels is compiled: 0 = one kernel per order p
                                   with the recurrences fully unrolled (coefficients
                                   as immediates); 1, 2 or 4 = one kernel for every
                                   order, its loop over n unrolled by that factor
                                   and the coefficients read from constant memory.
                                   Other values: TSQBX_E_INVAL; nonzero for another
                                   kernel or precision: TSQBX_E_UNSUPPORTED.  Results
                                   are the same to rounding either way            */
    int fp64_share;             /* double-float (TSQBX_DF64) Laplace plans: work items
                                   whose index i has (i mod 20) < fp64_share run in
                                   native FP64 on the FP64 pipe, in the same launch as
                                   the double-float items on the FP32 pipes (GB300
                                   runs both pipes at once).  0..20; 0 = all
                                   double-float.  Each target's result comes from one
                                   fixed form, FP64 or double-float, both within the
                                   FP64 bar of 1e-12.  Out of range: TSQBX_E_INVAL;
                                   nonzero for another plan: TSQBX_E_UNSUPPORTED    */
} tsqbx_options;

/* ------------------------------------------------------------ geometry */
/* The problem statement of Sec. 3.3: quadrature sources with weights (and
 * normals for the double layer), QBX centers with radii, targets mapped to
 * centers, and per center group the pair list as a CSR of source ranges.
 * Centers of one group (e.g. the centers owned by one octree box) share the
 * list.  All pointers are host pointers, caller-owned, read during
 * tsqbx_plan_create only. */
typedef struct {
    int64_t n_src;
    const double *src_xyz;          /* [3][n_src]                                  */
    const double *src_weight;       /* [n_src] quadrature weight incl. Jacobian    */
    const double *src_normal;       /* [3][n_src] unit normals; NULL without DLP    */
    int64_t n_ctr;
    const double *ctr_xyz;          /* [3][n_ctr]                                  */
    const double *ctr_radius;       /* [n_ctr] ball radius (reported, may be NULL) */
    int64_t n_tgt;
    const double *tgt_xyz;          /* [3][n_tgt]                                  */
    const int32_t *tgt_center;      /* [n_tgt] center of each target              */
    int64_t n_group;
    const int32_t *ctr_group;       /* [n_ctr] group of each center                */
    const int64_t *group_range_start; /* [n_group+1] CSR offsets, [0] == 0         */
    const int32_t *range_begin;     /* [nnz] first source of each range            */
    const int32_t *range_end;       /* [nnz] one past the last source              */
    const double *tgt_normal;       /* [3][n_tgt] unit normals; NULL without S'    */
} tsqbx_geometry;

typedef struct tsqbx_plan_s *tsqbx_plan;

/* Counts describing a plan. */
typedef struct {
    int64_t n_src, n_ctr, n_tgt, n_group;
    int64_t n_pairs;           /* (target, source) pairs, duplicates counted        */
    int64_t n_pair_terms;      /* n_pairs * (p + 1): the throughput unit            */
    int64_t n_items;           /* warp work items                                   */
    int64_t n_divergent;       /* pairs with |t-c| >= |s-c| (0 if the check was off) */
    int64_t n_coincident;      /* pairs with s == c                                  */
    int64_t list_entries;      /* sum over groups of listed sources                  */
    double lane_utilisation;   /* active lanes / 32 averaged over items (by cost)    */
    size_t device_bytes;       /* device memory held by the plan                     */
    int64_t n_sliced;          /* target chunks whose list was cut into slices       */
    int launches_per_eval;     /* kernels one evaluation launches (prep, expansion,
                                  the slice combine when n_sliced > 0, and the two
                                  conventional kernels when n_conv_centers > 0)     */
    int64_t n_conv_centers;    /* centers on the conventional path                   */
    int64_t n_conv_targets;    /* their targets                                      */
    int64_t n_conv_items;      /* conventional coefficient-formation work items      */
} tsqbx_plan_stats;

/* Create a plan: validates the geometry and options, counts divergent pairs
 * on the device (unless TSQBX_FLAG_SKIP_CHECK), builds the work items and
 * uploads everything.  On success *out owns device memory until
 * tsqbx_plan_destroy.  Errors: TSQBX_E_INVAL, TSQBX_E_DIVERGENT (plan not
 * created; the counts are lost), TSQBX_E_NOMEM, TSQBX_E_CUDA,
 * TSQBX_E_UNSUPPORTED. */
TSQBX_API int tsqbx_plan_create(const tsqbx_geometry *geometry, const tsqbx_options *options,
                      tsqbx_plan *out);

/* Release a plan (waits for its in-flight work).  NULL is ignored. */
TSQBX_API void tsqbx_plan_destroy(tsqbx_plan plan);

/* Fill *stats.  Errors: TSQBX_E_INVAL. */
TSQBX_API int tsqbx_plan_info(tsqbx_plan plan, tsqbx_plan_stats *stats);

/* Device bytes held by the plan (geometry, lists, work items, slot buffers):
 * the admission unit of a serving loop.  Errors: TSQBX_E_INVAL. */
TSQBX_API int tsqbx_plan_footprint(tsqbx_plan plan, size_t *bytes);

/* Blocking evaluation: the near-field TSQBX sums of Alg. 1 Stages 3, 5(a)
 * and 6(a) (Sec. 2.6 eq. tsqbx, Appendix A; see the top of this file) for
 * one density, every layer of the plan's mask.  density: n_src doubles
 * (Laplace) or n_src complex doubles as interleaved (re, im) pairs
 * (Helmholtz), the mu_s of the sums (the plan applies the weights w_s).
 * out_slp / out_dlp: n_tgt doubles (Laplace) or n_tgt interleaved complex
 * values (Helmholtz), indexed by target; NULL for a layer not in the plan's
 * mask.  Each pointer may be host (pageable or pinned) or device memory.
 * Returns after the outputs are written.  Errors: TSQBX_E_INVAL,
 * TSQBX_E_CUDA, TSQBX_E_KERNEL. */
TSQBX_API int tsqbx_eval(tsqbx_plan plan, const void *density, void *out_slp, void *out_dlp);

/* tsqbx_eval / tsqbx_submit with the expansion order p (0..TSQBX_P_MAX) and,
 * for Helmholtz, the wavenumber k (> 0) chosen per call: the plan's geometry,
 * lists and schedule do not depend on them, so one plan serves every order
 * and wavenumber.  out_sp receives S' (n_t . grad_t G, layout as out_slp)
 * when the plan's mask has TSQBX_SP; it may be NULL, and then S' is not
 * formed.  tsqbx_eval, tsqbx_submit and tsqbx_eval_async form the single and
 * double layers only.  Errors as tsqbx_eval / tsqbx_submit. */
TSQBX_API int tsqbx_eval_pk(tsqbx_plan plan, int p, double k, const void *density, void *out_slp,
                            void *out_dlp, void *out_sp);
TSQBX_API int tsqbx_submit_pk(tsqbx_plan plan, int p, double k, const void *density, void *out_slp,
                              void *out_dlp, void *out_sp, uint64_t *ticket);

/* Asynchronous evaluation on DEVICE pointers only (same layouts as
 * tsqbx_eval), enqueued on `stream` (a cudaStream_t; NULL = the plan's own
 * stream).  Returns once the work is enqueued; the caller orders later work
 * on that stream.  Uses slot 0's scratch: concurrent calls on one plan must
 * be ordered on one stream.  Errors: TSQBX_E_INVAL, TSQBX_E_CUDA. */
TSQBX_API int tsqbx_eval_async(tsqbx_plan plan, const void *d_density, void *d_out_slp, void *d_out_dlp,
                     void *stream);
/* tsqbx_eval_async with the order p and wavenumber k chosen per call (as in
 * tsqbx_eval_pk) and an S' output (DEVICE pointer, may be NULL: S' is then
 * not formed).  Errors as tsqbx_eval_async. */
TSQBX_API int tsqbx_eval_async_pk(tsqbx_plan plan, int p, double k, const void *d_density, void *d_out_slp,
                                  void *d_out_dlp, void *d_out_sp, void *stream);

/* Submit an evaluation (the sums of tsqbx_eval: Alg. 1 Stages 3, 5(a), 6(a))
 * and return at once with a ticket, so that a serving loop overlaps
 * evaluations of many plans.  Pointers as for tsqbx_eval; host density is
 * copied before return, host outputs are written by the tsqbx_poll call that
 * reports completion, so they must stay valid until then.  Errors:
 * TSQBX_E_INVAL, TSQBX_E_BUSY (every slot in flight: poll first),
 * TSQBX_E_CUDA. */
TSQBX_API int tsqbx_submit(tsqbx_plan plan, const void *density, void *out_slp, void *out_dlp,
                 uint64_t *ticket);

/* Several densities in one evaluation: for the n densities density[0..n),
 * with order p and wavenumber k as in tsqbx_submit_pk, the single layer of a
 * Helmholtz plan, or the single and/or double layer of a Laplace plan in
 * TSQBX_FP64 or TSQBX_DF64 (no S'; created with max_rhs >= n; no
 * conventional centers).  The per-pair work of Appendix A's expansion --
 * geometry, 1/R, the Legendre (and Helmholtz: Hankel) recurrences, e^{ikR},
 * the sums over the orders -- depends on the geometry, p and k only, so the
 * densities share it and each adds only its own weight w_s mu_s (real for
 * Laplace, complex for Helmholtz): n densities cost little more than one.
 * out_slp[i] / out_dlp[i] (layout as tsqbx_submit) receive the layers of
 * density i; an array is read only when its layer is in the plan's mask and
 * may be NULL otherwise.  Each result is bit-identical to the evaluation of
 * density[i] alone on the same plan.  Pointers host or device as for
 * tsqbx_submit; one ticket covers all n results (tsqbx_poll).  Errors:
 * TSQBX_E_INVAL (n outside 1..max_rhs, NULL pointers, p or k),
 * TSQBX_E_UNSUPPORTED (not such a plan, or one with conventional centers),
 * TSQBX_E_BUSY, TSQBX_E_CUDA. */
TSQBX_API int tsqbx_submit_multi_layers(tsqbx_plan plan, int p, double k, int n, const void *const *density,
                                        void *const *out_slp, void *const *out_dlp, uint64_t *ticket);

/* tsqbx_submit_multi_layers without double-layer outputs: for plans whose
 * mask holds the single layer alone. */
TSQBX_API int tsqbx_submit_multi(tsqbx_plan plan, int p, double k, int n, const void *const *density,
                                 void *const *out_slp, uint64_t *ticket);

/* Wait up to timeout_us microseconds (0: just test, < 0: wait indefinitely)
 * for a ticket of tsqbx_submit / tsqbx_submit_pk / tsqbx_submit_multi(_layers)
 * (no counterpart in the paper: the completion side of the asynchronous
 * calls).  Returns TSQBX_OK once (the ticket is then retired), TSQBX_PENDING
 * if timeout_us == 0 and work is in flight, TSQBX_E_TIMEOUT if a positive
 * timeout expired, TSQBX_E_NOTFOUND for an unknown ticket, TSQBX_E_KERNEL /
 * TSQBX_E_CUDA on failure (ticket retired). */
TSQBX_API int tsqbx_poll(uint64_t ticket, int timeout_us);

/* Duration in milliseconds of the expansion kernel of the most recent
 * tsqbx_eval / tsqbx_eval_async on this plan, measured with CUDA events
 * recorded on the launching stream immediately before and after that kernel
 * (the per-evaluation w*mu preparation kernel is outside the interval).
 * Waits for that kernel to finish.  Errors: TSQBX_E_INVAL (no evaluation
 * yet), TSQBX_E_CUDA. */
TSQBX_API int tsqbx_plan_kernel_ms(tsqbx_plan plan, float *ms);

/* -------------------------------------------------------------- batches
 * Many plans evaluated in ONE persistent, load-balanced launch (the plans'
 * work items merged into one queue sorted by cost; resident warps pop items
 * with an atomic counter).  All plans must be Laplace FP64 or mixed (df64:
 * TSQBX_E_UNSUPPORTED), on one device, with the same precision and layer mask;
 * their orders p may differ.  A batch
 * snapshots the plans' schedules at creation and uses the plans' device
 * geometry, so the plans must outlive it; its scratch (w mu per plan, partial
 * sums, queue head) is its own, so batch and plan evaluations may interleave
 * on different streams.  Results are deterministic.  In single-layer mixed
 * batches up to four single-target items of one plan share a warp (8 or 16
 * lanes each), so their lane sums are reduced in another order than the plan
 * alone reduces them: the two agree to rounding (within the mixed error bar),
 * not bit for bit.  A batch stages sources at the default depth (64 per
 * tile) whatever a plan's own tile_depth, and runs the per-order kernels
 * whatever its p_unroll; otherwise it reproduces the results of each plan at
 * that depth bit for bit. */
typedef struct tsqbx_batch_s *tsqbx_batch;

typedef struct {
    int64_t n_plans, n_items, n_sliced, n_pairs, n_pair_terms;
    int grid_blocks;            /* persistent CTAs (one wave)                        */
    int graph;                  /* 1 if evaluations replay a captured CUDA graph     */
    int launches_per_eval;      /* kernels per evaluation                            */
    size_t device_bytes;        /* device memory held by the batch itself            */
} tsqbx_batch_stats;

/* use_graph != 0: capture the launch sequence (pointer-table copy, w mu
 * preparation of every plan, queue reset, persistent kernel, slice combine)
 * into a CUDA graph at creation and replay it per evaluation.
 * Errors: TSQBX_E_INVAL, TSQBX_E_UNSUPPORTED (non-Laplace), TSQBX_E_NOMEM,
 * TSQBX_E_CUDA. */
TSQBX_API int tsqbx_batch_create(const tsqbx_plan *plans, int n_plans, int use_graph, tsqbx_batch *out);
TSQBX_API void tsqbx_batch_destroy(tsqbx_batch batch);

/* Enqueue one evaluation of every plan on `stream` (NULL = the batch's own
 * stream).  d_density[i], d_out_slp[i], d_out_dlp[i]: DEVICE pointers for
 * plan i (layouts as tsqbx_eval; out arrays may be NULL for absent layers;
 * a batch forms the single and double layers only, never S').  Waits only
 * until the previous evaluation of this batch has read its pointer table.
 * Errors: TSQBX_E_INVAL, TSQBX_E_CUDA. */
TSQBX_API int tsqbx_batch_eval_async(tsqbx_batch batch, const void *const *d_density,
                                     void *const *d_out_slp, void *const *d_out_dlp, void *stream);

/* Waits for the last evaluation; *ms = device time from the queue reset to
 * the end of the combine (CUDA events in the launch sequence).  Returns
 * TSQBX_E_KERNEL if a kernel flagged an out-of-range index. */
TSQBX_API int tsqbx_batch_kernel_ms(tsqbx_batch batch, float *ms);
TSQBX_API int tsqbx_batch_info(tsqbx_batch batch, tsqbx_batch_stats *stats);

/* -------------------------------------------------------------- serving
 * A request-serving runtime: geometries are registered once; requests (one
 * evaluation of one geometry with a kernel variant and a density) arrive at
 * any time and are admitted as soon as their plan -- created on first use and
 * keyed by (geometry, kernel, layers, precision); p and k are per request --
 * has a free slot and
 * the resident plans fit the HBM budget (idle plans are evicted least recently
 * used).  Started requests run on their own plan slots and streams, so work
 * that arrives while other requests are on the GPU overlaps with them
 * (continuous batching).  Queued requests of the plans that
 * tsqbx_submit_multi_layers takes (Helmholtz single layer; Laplace single
 * and/or double layer in FP64 or double-float) with the same geometry,
 * layers, precision, order and (Helmholtz) wavenumber are started together,
 * up to four, as one multi-density evaluation: each result is bit-identical
 * to the request evaluated alone.  A worker thread owned by the server does
 * the admission and completion bookkeeping. */
typedef struct tsqbx_server_s *tsqbx_server;

typedef struct {
    double p50_ms, p99_ms, mean_ms, max_ms;  /* latency, arrival to completion   */
    int64_t completed, failed, rejected;     /* rejected: could never be admitted */
    int64_t queued, running;
    int64_t plans_resident, plans_created, plans_evicted;
    size_t resident_bytes;
    int64_t pair_terms_completed;
    double span_s;                           /* first arrival to last completion */
    int64_t merged;                          /* requests that ran inside another queued
                                                request's multi-density evaluation  */
} tsqbx_server_stats;

/* hbm_budget_bytes: cap on the device memory of resident plans; max_inflight:
 * cap on requests running at once.  Errors: TSQBX_E_INVAL, TSQBX_E_NOMEM. */
TSQBX_API int tsqbx_server_create(int device, size_t hbm_budget_bytes, int max_inflight, tsqbx_server *out);
/* Waits for running requests, stops the worker, frees every plan. */
TSQBX_API void tsqbx_server_destroy(tsqbx_server server);
/* Copies the geometry (host arrays, tsqbx_geometry layout); *geom_id names it. */
TSQBX_API int tsqbx_server_add_geometry(tsqbx_server server, const tsqbx_geometry *geometry, int *geom_id);
/* Builds (or refreshes in the LRU order) the plan for a variant ahead of
 * requests.  Errors: TSQBX_E_INVAL, TSQBX_E_NOMEM (larger than the budget),
 * TSQBX_E_BUSY (budget held by running work), plan-creation errors. */
TSQBX_API int tsqbx_server_prepare(tsqbx_server server, int geom_id, const tsqbx_options *options);
/* Queue one evaluation.  options: kernel, layers, p, k, precision (+ tuning
 * fields); device is the server's.  The density (host, layout as tsqbx_eval)
 * is copied before return; out_slp / out_dlp / out_sp (S', required when the
 * mask has TSQBX_SP) are HOST buffers written before the request reports
 * completion and must stay valid until then. */
TSQBX_API int tsqbx_server_submit(tsqbx_server server, int geom_id, const tsqbx_options *options,
                                  const void *density, void *out_slp, void *out_dlp, void *out_sp,
                                  uint64_t *request);
/* 0 once the request completed (its outputs written; the request is then
 * retired), TSQBX_PENDING (timeout_us == 0), TSQBX_E_TIMEOUT, or the
 * request's failure code (e.g. TSQBX_E_NOMEM if it could never fit). */
TSQBX_API int tsqbx_server_poll(tsqbx_server server, uint64_t request, int timeout_us);
TSQBX_API int tsqbx_server_get_stats(tsqbx_server server, tsqbx_server_stats *stats);
/* Clears latency samples and counters (e.g. after a warm-up phase). */
TSQBX_API int tsqbx_server_reset_stats(tsqbx_server server);
/* Scheduling policy for the plans the server builds from now on (plans that
 * are already resident keep theirs; build them with tsqbx_server_prepare
 * after this call).  on = 0 (the default): every plan's streams have the
 * default priority, so the GPU dispatches the blocks of concurrent requests
 * roughly in launch order.  on != 0: plans are built with
 * TSQBX_FLAG_SIZE_PRIORITY, so short evaluations overtake long ones -- a much
 * lower median latency for mixes of small and large requests, at the cost of
 * the largest requests' latency.  Errors: TSQBX_E_INVAL. */
TSQBX_API int tsqbx_server_set_size_priority(tsqbx_server server, int on);
/* How the server evaluates Laplace requests that ask for TSQBX_FP64, for the
 * requests submitted (and plans prepared) from now on: TSQBX_FP64 (the
 * default) on the FP64 kernels, or TSQBX_DF64 on the double-float kernels,
 * which meet the same FP64 bound (1e-12 relative) on the FP32 pipes at
 * several times the speed on GPUs whose FP64 rate is a small fraction of
 * their FP32 rate.  Such requests then share the DF64 plans of their
 * geometry.  Errors: TSQBX_E_INVAL. */
TSQBX_API int tsqbx_server_set_laplace_fp64_path(tsqbx_server server, int precision);

/* ------------------------------------------------------------- tuning
 * Work decomposition of a plan: lanes per target (0 = chosen per group from
 * its target and source counts), the cap on per-lane pair iterations of one
 * warp item (longer lists are cut into slices), the staging depth (sources
 * per shared-memory tile, as tsqbx_options.tile_depth) and the order-loop
 * form (as tsqbx_options.p_unroll). */
typedef struct {
    int lanes_per_target;
    int max_item_iters;
    float kernel_ms;            /* autotune: measured expansion time of this choice */
    int tile_depth;             /* 32, 64 or 128 (0 in tsqbx_plan_set_tuning: 64)   */
    int p_unroll;               /* 0, 1, 2 or 4; nonzero only for Laplace FP64 and
                                   mixed plans (else TSQBX_E_UNSUPPORTED)            */
    int fp64_share;             /* 0..20 as tsqbx_options.fp64_share; nonzero only
                                   for Laplace df64 plans (else TSQBX_E_UNSUPPORTED) */
} tsqbx_tuning;

/* Autotuner: times candidate decompositions of this plan (slice caps, then
 * lane policies, then tile depths, then, for Laplace FP64 and mixed plans, the
 * order-loop forms p_unroll 0, 1, 2, 4, and for Laplace df64 plans the FP64
 * shares 0, 1, 2, 3) with CUDA events on the plan's stream, evaluating the DEVICE
 * density d_density `repeats` times each (after one untimed run), keeps the
 * fastest, records it in the process-wide tuning cache (see
 * TSQBX_FLAG_USE_TUNED) and returns it in *chosen (may be NULL).  Uses the
 * plan's slot-0 buffers; do not overlap with other evaluations of the plan.
 * Errors: TSQBX_E_INVAL, TSQBX_E_NOMEM, TSQBX_E_CUDA. */
TSQBX_API int tsqbx_plan_autotune(tsqbx_plan plan, const void *d_density, int repeats,
                                  tsqbx_tuning *chosen);

/* Install a decomposition (e.g. one found by the autotuner) / read the current
 * one (kernel_ms = 0).  Errors: TSQBX_E_INVAL, TSQBX_E_UNSUPPORTED (p_unroll
 * nonzero for a plan other than Laplace FP64 or mixed, fp64_share nonzero
 * for a plan other than Laplace df64), TSQBX_E_NOMEM, TSQBX_E_CUDA. */
TSQBX_API int tsqbx_plan_set_tuning(tsqbx_plan plan, const tsqbx_tuning *tuning);
TSQBX_API int tsqbx_plan_get_tuning(tsqbx_plan plan, tsqbx_tuning *tuning);

/* ------------------------------------------------ no-allocation evaluation
 * The paper has no counterpart: this entry point serves callers that cannot
 * call cudaMalloc -- e.g. a program whose device memory is owned by its own
 * pool or arena, or a latency-critical loop that cannot accept cudaMalloc's
 * implicit synchronisation.  Such callers cannot create a plan (that
 * allocates), so everything is passed as DEVICE arrays and nothing is
 * allocated: the scratch it needs (w_s mu_s per source and a status word)
 * lives in one fixed __device__ array of 8 MiB inside the library, which every
 * GPU that loads the library holds until the process exits.
 *
 * Computes the same quantities as tsqbx_eval for a plan with the same
 * geometry, p and layers (the Laplace single and/or double layer, FP64), to
 * FP64 roundoff (about 1e-12 relative): its recurrence and lane reduction are
 * its own, so the two agree to rounding, not bit for bit.
 *  d_geometry: a HOST struct whose counts are sizes and whose pointer fields
 *              are all DEVICE pointers in the tsqbx_geometry layout;
 *              group_range_start must hold n_group + 1 entries, and
 *              range_begin / range_end must be non-NULL when n_group > 0
 *              (even if every list is empty); ctr_radius is ignored;
 *              src_normal is required for TSQBX_DLP.
 *  d_density:  n_src doubles (device).  d_out_slp / d_out_dlp: n_tgt doubles
 *              (device) for the requested layers.
 *  stream:     cudaStream_t (NULL = legacy default stream); the call blocks
 *              until the work on that stream is done.
 * Limits and sharing: n_src <= TSQBX_NOALLOC_MAX_SRC (else TSQBX_E_TOO_LARGE).
 * Every call on a device shares the one scratch array, which keeps the last
 * call's contents (the status word is cleared and w mu rewritten by each
 * call): calls that overlap on the GPU race and must be serialised.  The
 * first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Index ranges are checked on the device: an
 * out-of-range index is skipped and reported as TSQBX_E_KERNEL, and so is a
 * listed source that sits exactly on its center (|s-c| = 0, where the
 * expansion does not exist): that pair is skipped.  Unlike
 * tsqbx_plan_create, this entry point does NOT look for divergent pairs
 * (|t-c| >= |s-c|); such a pair is summed like any other and its terms grow
 * with p.  Errors: TSQBX_E_INVAL, TSQBX_E_TOO_LARGE, TSQBX_E_KERNEL,
 * TSQBX_E_CUDA. */
#define TSQBX_NOALLOC_MAX_SRC 1048544
TSQBX_API int tsqbx_eval_noalloc(const tsqbx_geometry *d_geometry, int p, uint32_t layers,
                                 const double *d_density, double *d_out_slp, double *d_out_dlp,
                                 void *stream);

/* ------------------------------------------------------------- octree
 * The GIGAQBX octree over sources and QBX centers and the near-field pair
 * lists, built on the GPU (Sec. 3.1-3.2, Defs. 1-9; the list building of
 * Alg. 1 Stage 1).  Rules: the root is the smallest power-of-two cube holding
 * every source and QBX ball, centered on the grid of spacing H/1024; a box
 * with more than n_max owned sources + centers splits, sources moving to their
 * octant's child and a center only if its ball fits that child's target
 * confinement region (radius sqrt(3) h (1 + t_f)); empty children are not
 * created.  Boxes are numbered breadth first (children in octant order),
 * sources ordered depth first.  For every box owning a center the result is
 * the sorted, merged source ranges of List 1 + List 3 close + List 4 close
 * (List 3 boxes separated from the box's confinement region with at least
 * n_mpole sources are "far" and excluded), in the depth-first source order:
 * exactly the pair lists tsqbx_geometry takes (groups = boxes owning centers),
 * so no host preprocessing precedes tsqbx_plan_create. */
typedef struct tsqbx_octree_s *tsqbx_octree;
typedef struct {
    int64_t n_boxes, n_leaves, max_level;
    int64_t n_target_boxes;     /* boxes owning at least one center                  */
    int64_t near_nnz;           /* merged near-field ranges over all target boxes    */
    int64_t center_source_pairs;/* sum over centers of their near-field source count  */
    double build_ms;            /* wall time of tsqbx_octree_build (host view)        */
    double upload_ms, tree_ms, order_ms, lists_ms, download_ms;   /* its phases     */
} tsqbx_octree_stats;

/* Build.  src_xyz [3][n_src], ctr_xyz [3][n_ctr] (HOST pointers), ctr_radius
 * [n_ctr] >= 0, all finite; n_max >= 1, t_f >= 0, n_mpole >= 0.  Errors:
 * TSQBX_E_INVAL, TSQBX_E_TOO_LARGE (deeper than 30 levels: too many
 * coincident points), TSQBX_E_NOMEM, TSQBX_E_CUDA. */
TSQBX_API int tsqbx_octree_build(int64_t n_src, const double *src_xyz, int64_t n_ctr, const double *ctr_xyz,
                                 const double *ctr_radius, int n_max, double t_f, int n_mpole, int device,
                                 tsqbx_octree *out);
TSQBX_API void tsqbx_octree_destroy(tsqbx_octree tree);
TSQBX_API int tsqbx_octree_info(tsqbx_octree tree, tsqbx_octree_stats *stats);
/* Host copies (any pointer may be NULL): per box, n_boxes entries (center:
 * [3][n_boxes]); src_begin/src_end: the box's sources in depth-first order. */
TSQBX_API int tsqbx_octree_boxes(tsqbx_octree tree, int32_t *level, double *center, double *halfwidth,
                                 int32_t *parent, int32_t *src_begin, int32_t *src_end, int32_t *n_owned_ctr,
                                 int32_t *is_leaf);
/* src_perm[i]: input index of the i-th source in depth-first order;
 * ctr_box[c]: the box owning center c. */
TSQBX_API int tsqbx_octree_order(tsqbx_octree tree, int32_t *src_perm, int32_t *ctr_box);
/* Near-field ranges: box b's are near_begin/near_end[near_start[b] ..
 * near_start[b+1]) (half-open, depth-first source positions); near_start has
 * n_boxes + 1 entries, the ranges stats.near_nnz. */
TSQBX_API int tsqbx_octree_near(tsqbx_octree tree, int64_t *near_start, int32_t *near_begin, int32_t *near_end);

/* ------------------------------------------------------- measurement aid
 * The paper has no counterpart (its timings are CPU process times, Sec. 4):
 * the expansion kernels are bound by the FP64 pipe (FP64 and Helmholtz) or
 * the FP32 pipe (mixed and df64), so their rooflines divide by these pipes'
 * throughput, measured here on the device itself.  Register-only fused
 * multiply-add chains (no memory traffic); per pipe, nine launch shapes (4, 8
 * or 16 chains per thread, 2, 4 or 8 blocks of 256 threads per SM) are timed
 * briefly and the fastest again at about 150 ms per launch, with CUDA events
 * (best of 3); an FMA counts as two flops.  Runs a few seconds in all and
 * changes no setting of the GPU.  Errors: TSQBX_E_INVAL (bad device or NULL),
 * TSQBX_E_CUDA. */
typedef struct {
    double fp64_tflops;         /* DFMA                                               */
    double fp32_tflops;         /* scalar FFMA                                        */
    double fp32x2_tflops;       /* packed fma.rn.f32x2 (two FMAs per instruction)     */
    int sm_count;               /* the device's multiprocessors                       */
    float ms_fp64, ms_fp32, ms_fp32x2;   /* duration of the best timed launch        */
} tsqbx_pipe_peaks;
TSQBX_API int tsqbx_measure_pipe_peaks(int device, tsqbx_pipe_peaks *out);

/* Name of the last CUDA runtime error that a libtsqbx call made on the
 * calling thread ran into (the detail behind TSQBX_E_CUDA / TSQBX_E_NOMEM);
 * "no error" if none. */
TSQBX_API const char *tsqbx_last_error(void);

/* Static description of a status code. */
TSQBX_API const char *tsqbx_strerror(int status);

/* Version of this ABI (major * 10000 + minor * 100 + patch).  1.3 added
 * tsqbx_options.p_unroll / .fp64_share and tsqbx_tuning.p_unroll /
 * .fp64_share (appended: callers built against 1.2 pass structs of the old
 * size and must be rebuilt).  1.4 accepts max_rhs > 1, and so
 * tsqbx_submit_multi, for Laplace single-layer plans in FP64 and
 * double-float (no struct changed).  1.5 adds tsqbx_submit_multi_layers
 * (Laplace double layer with several densities). */
TSQBX_API int tsqbx_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TSQBX_H */
