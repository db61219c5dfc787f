/*
 * hp.h — C ABI of the hierarchical loop-nest executor for GB300 (sm_103a).
 *
 * A nest is a depth-d loop nest, rectangular or ragged (CSR), with a body
 * evaluated once per iteration and a reduction at any level.  Each nest level
 * is bound to one level of the GPU's hardware hierarchy (grid, thread-block
 * cluster, CTA, warp, sub-warp, lane, sequential), the way the paper's
 * level(...) clause selects "where to get the new parallelism from" (Sec. 3.1),
 * and each reduction is carried out on the level it is bound to with that
 * level's own means of communication (Sec. 2: shuffles at warp level, shared
 * memory at CTA level, distributed shared memory at cluster level, a
 * deterministic two-pass combine at grid level).
 *
 * Conventions for every entry point:
 *   - Calls return an hp_status and never abort or exit.  On failure,
 *     hp_last_error() returns a message for the calling thread.
 *   - "device pointer" means memory of the current CUDA device (e.g. from
 *     torch or cudaMalloc); "host pointer" means ordinary host memory.
 *     The caller owns every buffer it passes; the library owns its own scratch
 *     and frees it in the matching destroy call.
 *   - stream is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Runs are asynchronous on that stream: inputs must stay valid,
 *     and outputs must not be read, until the stream's work completes.
 *   - The library performs no CPU fallback: when no GB300 is present, runs
 *     fail with HP_ECUDA.
 */
#ifndef HP_H
#define HP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HP_MAX_DEPTH 5

typedef enum hp_status {
    HP_OK = 0,
    HP_EINVAL = 1,          /* invalid argument or illegal level map */
    HP_ENOMEM = 2,          /* device or host allocation failed, or over budget */
    HP_EBUSY = 3,           /* resource (serving slot, stream) in use */
    HP_EAGAIN = 4,          /* not finished yet (serving poll) */
    HP_ETIMEOUT = 5,        /* a bounded wait ran out (host or device side) */
    HP_ECUDA = 6,           /* a CUDA call failed; message in hp_last_error() */
    HP_EUNSUPPORTED = 7     /* legal request this build does not implement */
} hp_status;

/*
 * Hardware levels (Sec. 3.1, level clause; Fig. 1 hierarchy, reduced to the
 * levels CUDA exposes on GB300).  A nest level bound to level X has its
 * iterations spread over the members of one X: GRID spreads over the clusters
 * (or CTAs) of the grid, CLUSTER over the CTAs of a cluster, CTA over the
 * warps of a CTA, WARP over the 32 lanes of a warp (or over its sub-warp
 * groups when a deeper nest level is bound to SUBWARP), SUBWARP over the
 * sub_width lanes of a sub-warp group (Sec. 3.8, level partitioning), LANE over
 * the vector slots of one thread's 128-bit registers (the SIMD-in-register
 * level at the bottom of Fig. 1), SEQ runs sequentially in one thread.
 * Iterations left over after the members are used up are strip-mined: each
 * member loops over its share (Sec. 3.4, "SPMD mode").
 * A nest level also covers the hardware levels below its own down to the next
 * nest level's (collapse, Sec. 3.1); consecutive nest levels bound to the same
 * hardware level are collapsed into one.
 */
typedef enum hp_hw {
    HP_HW_GRID = 0,
    HP_HW_CLUSTER = 1,
    HP_HW_CTA = 2,
    HP_HW_WARP = 3,
    HP_HW_SUBWARP = 4,
    HP_HW_LANE = 5,
    HP_HW_SEQ = 6,
    HP_HW_AUTO = 7          /* let the planner choose (all levels must be AUTO) */
} hp_hw;

typedef enum hp_red_op {
    HP_RED_SUM = 0,
    HP_RED_MAX = 1,
    HP_RED_MIN = 2,
    HP_RED_HIST_COUNT = 3,  /* CSR nests only: count histogram of col >> shift */
    HP_RED_AFFINE_COMPOSE = 4, /* non-commutative: composition of affine maps in
                                  iteration order (below) */
    HP_RED_MAT2_PRODUCT = 5,   /* non-commutative: product of 2x2 matrices in
                                  iteration order (below) */
    HP_RED_LAST_VALID = 6      /* non-commutative: the last value that is not NaN
                                  (below) */
} hp_red_op;

/*
 * HP_RED_AFFINE_COMPOSE (Sec. 2: a reduction combines the results of sibling
 * tasks on each level; OpenMP's reduction clause does not allow
 * non-commutative user-defined operators, a hierarchy that combines siblings in
 * order does).  Rectangular nests, prec HP_F32, body HP_BODY_LOAD with
 * in_dev = {a, b}, two FP32 arrays of the nest's shape.  Iteration x of an
 * output contributes f_x(y) = a[x] * y + b[x]; the output is the composition in
 * iteration order F = f_{R-1} o ... o f_0, written as the pair (A, B) with
 * F(y) = A * y + B: B is the last value of the recurrence y_x = a_x y_{x-1} + b_x
 * from y = 0, A the product of the a_x.  out_dev: 2 floats per output (A, B).
 * Every warp folds a contiguous range of iterations in rounds of 32
 * consecutive pieces, one per lane (A <- a A, B <- fma(a, B, b) within a
 * piece); pieces, rounds, warps and grid parts are combined in iteration
 * order: (A2, B2) after (A1, B1) gives (A2 A1, fma(A2, B1, B2)).  Level map: outputs on GRID,
 * the reduced levels on WARP (a warp per output), CTA (sub_width warps per
 * output) or GRID (tile > 0 on the first reduced level: parts of tile x the
 * deeper extents, one CTA each, folded in part order), or AUTO.  Not batched,
 * served, tuned or run from host buffers (HP_EUNSUPPORTED).
 *
 * HP_RED_MAT2_PRODUCT: the same lowering with 2x2 matrices.  in_dev = {m}, one
 * FP32 array of 4 entries per iteration (row-major m00 m01 m10 m11, iteration
 * x of the flat nest at m[4x .. 4x+3]); the output is M_{R-1} ... M_1 M_0 (the
 * later matrix on the left), 4 floats per output.  Combining E then L gives
 * L E, each entry as fma(l_i0, e_0j, l_i1 * e_1j).  Second-order linear
 * recurrences y_x = p_x y_{x-1} + q_x y_{x-2} take the step [[p, q], [1, 0]];
 * the affine maps are the case [[a, b], [0, 1]].
 *
 * Error bound of both (hp_nest_error_bound): gamma_{2(R-1)} relative to the
 * product of the |M_x| (for affine maps: |A| and sum |b_x| prod_{z>x} |a_z|).
 * R maps make R - 1 combines in any tree and the relative errors of all of them
 * add (for products the count, not the depth of the tree, decides); infinite
 * once 2 (R - 1) u >= 1.  Typical errors grow like sqrt(R) u.
 *
 * HP_RED_LAST_VALID: in_dev = {v}, one FP32 array of the nest's shape; NaN
 * marks an iteration without a value.  The output (1 float) is the value of
 * the last iteration in order that is not NaN, copied bit for bit, or the
 * quiet NaN 0x7fc00000 when there is none (the final value of a forward fill).
 * Exact (error bound 0).  Inputs 32-byte aligned with R (and grid parts) a
 * whole number of 256-bit loads use them; 16-byte aligned, 128-bit loads;
 * otherwise scalar loads, for every ordered operator.
 */

/*
 * Arithmetic of body and reduction.
 *   HP_F32       FP32 inputs, plain FP32 accumulation (deterministic tree).
 *   HP_F32_COMP  FP32 inputs, compensated FP32 accumulation at every level
 *                (error-free product and sum transformations; Ogita-Rump-
 *                Oishi Dot2); grid parts are combined as double-float
 *                numbers (no FP64 on the GPU: a dependent FP64 operation
 *                costs about 14 FP32 ones on this GPU).
 *   HP_I32       int32 inputs, int32 accumulation: sums are exact modulo 2^32.
 *   HP_I64       int32 inputs widened to int64, int64 accumulation.
 * Outputs: float for the FP precisions, int32_t / int64_t for the integer ones.
 */
typedef enum hp_prec {
    HP_F32 = 0,
    HP_F32_COMP = 1,
    HP_I32 = 2,
    HP_I64 = 3,
    HP_I8 = 4,    /* int8 inputs, SIMD-in-register sub-lanes (below) */
    HP_I16 = 5    /* int16 inputs, SIMD-in-register sub-lanes (below) */
} hp_prec;

/*
 * HP_I8 / HP_I16 (App. A: CUDA's SIMD intrinsics treat a 32-bit register as 2
 * x 16-bit or 4 x 8-bit lanes; Sec. 3.8: a level below the lanes).  Rectangular
 * nests, body LOAD (SUM, MAX, MIN) or DOT_BCAST (HP_I8 only, SUM: int8 x int8
 * products), in_dev arrays of int8_t / int16_t.  Each thread's 128-bit loads
 * hold 16 (8) elements, 4 sub-lanes (2) in each 32-bit register: sums and
 * dot products accumulate into int32 with __dp4a / __dp2a_lo (exact modulo
 * 2^32), MAX / MIN keep packed running registers (__vmaxs4 / __vmins4,
 * __vmaxs2 / __vmins2) folded over their sub-lanes at the end.  Outputs int32_t
 * per output: the sum modulo 2^32, or the max / min value; an empty reduction
 * gives 0 (SUM) or the type's minimum (MAX) / maximum (MIN).  Level map:
 * outputs on GRID, the reduced levels on WARP, CTA (sub_width warps) or GRID
 * (tile > 0: parts combined after a ticket), or AUTO.  Rows whose length or
 * base is not 16-byte aligned take per-element loads (same results).  Not
 * batched, served, tuned or run from host buffers.
 */

/*
 * Bodies (flat = row-major index over all levels, rflat = row-major index over
 * the reduced levels red_level..depth-1):
 *   LOAD        A[flat]                            in_dev = {A}
 *   DOT_BCAST   A[flat] * w[rflat]                 in_dev = {A, w}
 *   CSR_GATHER  val[e] * x[col[e]]  (CSR nests)    in_dev = {offsets, col, val, x [, hist_out]}
 *   AFFINE      a + b * (flat mod m)               no inputs; hp_affine_params
 *   GEOMETRIC   fl32(q^(flat mod m))  (FP sums)    no inputs; hp_geometric_params
 * AFFINE and GEOMETRIC read no memory: they exercise a mapping at any size
 * against closed forms.
 */
typedef enum hp_body {
    HP_BODY_LOAD = 0,
    HP_BODY_DOT_BCAST = 1,
    HP_BODY_CSR_GATHER = 2,
    HP_BODY_AFFINE = 3,
    HP_BODY_GEOMETRIC = 4
} hp_body;

/* One entry per nest level.
 *   hw         an hp_hw value.
 *   sub_width  level-specific width: CLUSTER = CTAs per cluster (1..16),
 *              CTA = warps per CTA (1..32), SUBWARP = lanes per group
 *              (1, 2, 4, 8, 16, 32), LANE = vector slots (1 or 4);
 *              0 = default (8, 8, -, 4).
 *   tile       GRID level of a reduction: iterations per grid part (0 = auto);
 *              ignored elsewhere. */
typedef struct hp_level_map {
    int32_t hw;
    int32_t sub_width;
    int64_t tile;
} hp_level_map;

typedef struct hp_affine_params {
    int64_t a, b, m;        /* m >= 1 */
} hp_affine_params;

typedef struct hp_geometric_params {
    double q;               /* the body is fl32(q^k), q^k formed in FP64 */
    int64_t m;              /* 1 <= m <= 1024 */
} hp_geometric_params;

/* CSR nests: offsets int64[n_rows + 1] (device), col int32[nnz] (device),
 * val float[nnz] (device), x float[n_cols] (device). */
typedef struct hp_csr_params {
    int64_t nnz;
    int64_t n_cols;
    int32_t hist_shift;     /* histogram bin of entry e: col[e] >> hist_shift */
    int32_t fuse_hist;      /* SUM nests: 1 = also count the histogram in the same sweep into in_dev[4] */
    int64_t n_bins;         /* histogram bins (col >> shift must be < n_bins) */
} hp_csr_params;

typedef struct hp_nest hp_nest;
typedef struct hp_server hp_server;

/*
 * Create a nest and its execution plan (host only; touches no GPU).
 *   depth        1..HP_MAX_DEPTH for rectangular nests, 2 for CSR nests.
 *   extents      int64[depth], each >= 0 (host pointer); NULL for CSR nests.
 *   csr_offsets  NULL for rectangular nests; for CSR nests any non-NULL value
 *                marks the nest as ragged (the offsets themselves are passed
 *                at run time in in_dev[0]).
 *   n_rows       CSR nests: number of outer rows; ignored otherwise.
 *   map          hp_level_map[depth] (host pointer), or NULL to let the
 *                planner choose (same as all HP_HW_AUTO).
 *   op           reduction operator; red_level r in [0, depth]: levels
 *                0..r-1 index the outputs, levels r..depth-1 are reduced
 *                (r == depth: pure map, one output per iteration).
 *   body_params  hp_affine_params / hp_geometric_params / hp_csr_params for
 *                those bodies, else NULL (copied; host pointer).
 * Output layout: row-major over levels 0..r-1 (float / int32 / int64 per prec).
 * Errors: HP_EINVAL for an illegal shape or map (message names the rule),
 * HP_EUNSUPPORTED for a legal combination this build does not implement,
 * HP_ENOMEM if the host object cannot be allocated.
 */
hp_status hp_nest_create(int depth, const int64_t *extents, const int64_t *csr_offsets, int64_t n_rows,
                         const hp_level_map *map, hp_red_op op, int red_level, hp_prec prec, hp_body body,
                         const void *body_params, hp_nest **out);

/*
 * Run a nest on a stream (Sec. 2 reduction, executed as planned).
 *   in_dev   array of device pointers (host array), per the body's list.
 *            Memory-reading bodies need 16-byte aligned inputs when the plan
 *            uses 128-bit loads (hp_nest_describe reports "vec").
 *   out_dev  device pointer to the outputs (overwritten, never accumulated).
 * The first run on a device allocates the nest's scratch; later runs allocate
 * nothing.  Asynchronous: returns after enqueueing.  Device-side errors
 * (a bounded wait that ran out) are reported by hp_nest_check.
 * Concurrency: runs of one nest share its scratch (grid-part partials and,
 * for ordered and narrow nests split over parts, per-output tickets), so
 * runs of the same nest must be ordered (one stream, or events between
 * streams); different nests may run concurrently on any streams.  A nest
 * object is not thread-safe; give each host thread its own, or lock.
 */
hp_status hp_nest_run(hp_nest *n, const void *const *in_dev, void *out_dev, void *stream);

/*
 * hp_nest_run of a compensated FP32 sum (HP_F32_COMP, HP_RED_SUM, rectangular)
 * that also writes, for each output, the FP32 compensation of its final
 * rounding: comp_dev[o] is the exact error of out_dev[o] against the
 * two-word sum s + c the reduction tree reached (Sec. 2's recursive
 * reduction, carried in Ogita-Rump-Oishi double-word form), also when the
 * plan combines grid parts (their double-float sum).  out + comp then carries
 * the result to about 2^-48 relative; |comp|
 * is what the FP32 output gave away, for a caller's own error report.
 *   comp_dev  device pointer, one float per output (same layout as out_dev).
 * out_dev holds the same bits as hp_nest_run's.  HP_EUNSUPPORTED for other
 * nests; otherwise as hp_nest_run.
 */
hp_status hp_nest_run_comp(hp_nest *n, const void *const *in_dev, void *out_dev, void *comp_dev, void *stream);

/*
 * End-to-end run with HOST buffers: copies the inputs to device staging
 * buffers owned by the nest, runs, copies the outputs back, and waits for the
 * stream.  in_host / out_host are host pointers (pinned memory is fastest).
 * When the first (streamed) input is page-locked host memory that the device
 * maps (cudaHostAlloc / cudaMallocHost, or registered memory) and the option
 * "host_zero_copy" is 1 (the default), the kernel reads it in place over the
 * host link instead of after a staging copy; results are the same bits.
 * CSR nests are not supported here (HP_EUNSUPPORTED).
 */
hp_status hp_nest_run_host(hp_nest *n, const void *const *in_host, void *out_host, void *stream);

/*
 * Run a rectangular nest without allocating any memory.  The paper has no
 * counterpart to this entry point.  It is for callers that cannot allocate
 * device memory at run time: latency-critical serving loops (cudaMalloc and
 * cudaFree synchronise the whole device), services that handed out their
 * whole device-memory budget at start-up, and code that runs while a
 * framework holds its allocator.
 *   Same kernels, same reduction tree and same results as hp_nest_run.  The
 *   partials of a reduction split over grid parts live in one file-scope
 *   device array of 8 MiB instead of per-nest scratch; every GPU that loads
 *   the library holds that array until the process exits.  A plan that needs
 *   more than 8 MiB of partials returns HP_EINVAL.
 *   The first call on a device looks up the array's device address (with that
 *   device current); make that first call before any stream capture.
 *   All calls share the array and it keeps what the last call left: calls
 *   whose work overlaps on the GPU (other streams or host threads) race.
 *   CSR nests and the GEOMETRIC body (which needs a device table): HP_EUNSUPPORTED.
 */
hp_status hp_nest_run_static(hp_nest *n, const void *const *in_dev, void *out_dev, void *stream);

/*
 * Run many independent nests in one persistent launch per arithmetic
 * (replayed from a cached CUDA graph; the arithmetics' kernels are parallel
 * branches of it).  nests[i], in_dev[i], out_dev[i] as for hp_nest_run.  All
 * nests must be rectangular.  Each nest's outputs equal those of hp_nest_run
 * on the same nest bit for bit (same reduction tree).  Nests whose plan is a
 * cluster of CTAs (or a CTA of more than 8 warps), which the persistent
 * kernel's single CTAs cannot run, are run with their own launches on the
 * same stream after it.
 */
hp_status hp_nest_run_batch(hp_nest *const *nests, const void *const *const *in_dev, void *const *out_dev,
                            int count, void *stream);

/*
 * Autotune the level -> hardware binding of a rectangular nest (Sec. 3.2
 * selects levels by property, Sec. 3.3 compiles a region for several
 * candidate levels and picks one at run time; here the pick is timed).
 * Candidates keep the output levels on the grid and bind every reduced level
 * to one hardware level (CTA of 4 or 8 warps, warp, sub-warp group of 2..16
 * lanes, the vector slots of a thread, a thread, or a split over grid parts),
 * or, for long reductions, the first reduced level to a cluster of 2, 4 or 8
 * CTAs and the inner ones to a CTA (not in batched timing), or, with several
 * reduced levels, the first to the warps of a CTA (or to grid parts) and the
 * inner ones to the lanes of each warp (or to a CTA);
 * each is run on in_dev / out_dev, once on `stream`, then (after `stream`
 * is synchronized) as a CUDA graph of back-to-back runs on a private stream,
 * timed with CUDA events, best of three (device time, not launch rate).
 * The fastest is installed in n and stored for the nest's shape class (log2
 * of the output count and of the reduced size, 128-bit divisibility, body,
 * precision, operator); nests created later with map == NULL take it.
 * flags bit 0: re-time even if the class is already tuned.
 * flags bit 1: time every candidate, and the planner's own map, in the
 *   batched executor (hp_nest_run_batch on as many copies of the nest as give
 *   about 2^24 iterations, at most 64, all reading in_dev and writing the same
 *   values to out_dev), keeping the planner's map unless another is 3% faster:
 *   the choice for nests that will run in batches or under a server.
 * Synchronous (waits for the stream).  On return out_dev holds the installed
 * plan's result.  The GEOMETRIC body is not tuned.  Tune a nest before
 * passing it to hp_nest_run_batch or a server; batches built earlier with it
 * are rebuilt on their next call.
 */
hp_status hp_nest_tune(hp_nest *n, const void *const *in_dev, void *out_dev, void *stream, int32_t flags);

/* A-priori bound on the normalized error of each FP result of this nest
 * (|got - exact| / max(|exact|, scale), scale as reported by the tests):
 * 0 for integer precisions and MAX/MIN. */
hp_status hp_nest_error_bound(const hp_nest *n, double *rel_bound);

/* Write the plan as one line of JSON (levels, hardware binding, team, grid,
 * vector width, kernels) into buf[len]; truncated if too small. */
hp_status hp_nest_describe(const hp_nest *n, char *buf, size_t len);

/* Wait for the stream, then read the nest's device error word (0 = none;
 * 1 = a device-side bounded wait ran out; 2 = CSR offsets or column indices
 * outside the sizes declared at create, whose entries were skipped; 3 = a
 * wait of the batched executor's shared-memory stage ring ran out of time
 * (1 s) while a tile of this nest ran; the batch's outputs are then invalid).
 * Returns HP_ETIMEOUT if the word is set, HP_OK otherwise. */
hp_status hp_nest_check(hp_nest *n, void *stream, int32_t *device_error);

void hp_nest_destroy(hp_nest *n);

/*
 * Measurement aid for the roofline of ragged nests (not a step of the method):
 * one kernel that reads n_gathers random 4-byte elements of x_dev[0 .. n_x)
 * (indices uniform from a counter hash of (index, seed)) through the same
 * loads as the CSR executor's x gathers (cached in L2 only), 8 independent
 * reads in flight per thread, and writes their FP32 sum to *sum_dev (one
 * float, device memory; zeroed first).  Timing it gives the rate at which
 * this GPU serves random 32-byte L2 sectors to one 4-byte use each: the bound
 * of the CSR body's x[col[e]] reads once x fits L2.  Asynchronous on stream;
 * allocates nothing.  HP_EINVAL for n_x outside [1, 2^32) or NULL pointers.
 */
hp_status hp_probe_gather(const float *x_dev, int64_t n_x, int64_t n_gathers, uint32_t seed, float *sum_dev,
                          void *stream);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of nest requests under a device-memory budget.
 *
 * A scheduler thread admits submitted requests in arrival order while a slot
 * is free and the admitted requests' inputs, outputs and grid-split scratch
 * fit the budget, packs every admitted request that is not yet running into
 * one step, and launches it on a free stream with the batched persistent
 * kernels (so steps on different streams overlap, and requests arriving while
 * others run join the next step).  A request runs its nest's own plan with the
 * single-run reduction tree: its result is the same alone and in any mix, bit
 * for bit.  With hp_set_option("serve_batching", 0) servers created afterwards
 * launch every admitted request alone with the single-nest kernels (the plain
 * per-request baseline).  Completion is observed on the host by event queries:
 * while steps are in flight, and for 2 ms after its last activity, the
 * scheduler thread polls without sleeping (it occupies one host core); idle
 * longer, it sleeps until a submission wakes it.
 *
 * With hp_set_option("serve_batching", 2) servers created afterwards keep the
 * batched persistent kernel resident instead: while the server has work, one
 * instance of it runs with (resident CTAs per SM - 1) CTAs on every SM (room
 * for one more CTA of other kernels stays free), and its producer warps take
 * the tiles of newly admitted requests from a ring in mapped page-locked host
 * memory that the scheduler fills; a request then reaches the GPU without a
 * kernel launch, and the CTA that finishes its last tile writes its
 * completion to a mapped host word that the scheduler polls.  Results are
 * bit-identical to hp_nest_run as in the batched mode.  An instance takes new
 * tiles for 100 ms of host time, then the scheduler stops it and starts the
 * next (they overlap while the old one drains); 2 ms after the server's last
 * activity it stops the instance and starts a new one on the next admission.
 * Device waits for tiles are bounded (2 s per wait; the instance then leaves
 * with an error status, which fails the server's live requests).  A resident
 * server runs one arithmetic, set by its first request (FP32 sum, compensated
 * sum, max, min or int32 sum, max, min); other requests get HP_EUNSUPPORTED.
 * Other kernels on the GPU share it with the instance while it runs.  A
 * resident server prepares nothing of a submitted nest on the device (its
 * requests report device errors through the server's own error word), so that
 * no allocation in hp_serve_submit can wait for the running instance. */

/* mem_budget_bytes: admission budget (inputs + outputs + scratch of admitted
 * requests); max_slots: requests resident at once; n_streams (1..64): CUDA
 * streams the scheduler launches steps on.  Needs a GPU (HP_ECUDA otherwise). */
hp_status hp_serve_create(size_t mem_budget_bytes, int max_slots, int n_streams, hp_server **out);

/* Submit one request: a nest (shape and plan), its device inputs and output.
 * Returns a ticket.  The inputs and the output must be ready when the call is
 * made: the server orders its work after nothing on the caller's streams, so
 * writes to them still pending there (a fill, a copy) must be synchronized
 * first.  The server prepares the nest's device state and its
 * launch configuration on first use, from the scheduler thread, so from
 * submission until every ticket on it is polled done the caller must not run,
 * tune or destroy that nest (hp_nest_run*, hp_nest_tune*, hp_nest_destroy):
 * those calls would race with the scheduler on the nest's state. */
hp_status hp_serve_submit(hp_server *s, const hp_nest *shape, const void *const *in_dev, void *out_dev,
                          uint64_t *ticket);

/* The serving clock: microseconds of the monotonic clock that the latency
 * statistics use.  Host only; needs no GPU. */
double hp_serve_clock_us(void);

/* hp_serve_submit for a request whose arrival was scheduled at arrival_us (on
 * the serving clock, not later than the call).  Its latency counts from
 * arrival_us instead of from the call, so that a client that falls behind
 * its arrival schedule does not hide the lag from the percentiles (open-loop
 * load: latency from scheduled arrival to observed completion).  HP_EINVAL if
 * arrival_us is negative or in the future. */
hp_status hp_serve_submit_at(hp_server *s, const hp_nest *shape, const void *const *in_dev, void *out_dev,
                             double arrival_us, uint64_t *ticket);

/* HP_OK when the request finished (its output is valid), HP_EAGAIN while
 * pending, HP_ETIMEOUT if timeout_us elapsed (timeout_us < 0 waits without limit
 * on the host; the device side never spins), or an error. */
hp_status hp_serve_poll(hp_server *s, uint64_t ticket, int timeout_us);

/* Latency percentiles (microseconds, arrival to observed completion; arrival
 * is the scheduled time given to hp_serve_submit_at, else the submit call) and
 * throughput (requests/s) over all completed requests. */
hp_status hp_serve_stats(const hp_server *s, double *p50_us, double *p99_us, double *p999_us,
                         double *nests_per_s);

/* Counters: completed requests, launched steps (resident form: kernel
 * instances started), peak admitted bytes and peak admitted requests (both
 * stay within the budget and max_slots). */
hp_status hp_serve_counters(const hp_server *s, uint64_t *completed, uint64_t *steps, size_t *peak_bytes,
                            int32_t *peak_slots);

/* Stops the scheduler after the steps in flight complete; requests still
 * queued are dropped.  Nests and buffers stay the caller's. */
void hp_serve_destroy(hp_server *s);

/* ---------------------------------------------------------------------- */
/* Selecting levels by property (Sec. 3.2: a construct states the features it
 * needs, `sync(...)`, and the runtime picks the hardware level; Sec. 3.3: a
 * construct reserves, `reserve(...)`, what its nested constructs need).
 *
 * Properties of a hardware level (the paper's table of level properties, as
 * GB300 provides them to this executor):
 *   BARRIER    a barrier across the level's tasks (cluster.sync, __syncthreads,
 *              __syncwarp; the grid has none: no kernel here waits for the grid)
 *   CRITICAL   mutual exclusion among the level's tasks is implementable
 *   ATOMIC     atomic read-modify-write on memory the tasks share
 *   SHUFFLE    register exchange among the tasks (Sec. 3.7: warp lanes)
 *   OVERSUB    more tasks than run at once (time-shared: grid CTAs)
 *   DYNAMIC    non-static schedules (Sec. 3.5: an atomic work queue)
 *   LOCKSTEP   the tasks execute in lockstep (vector slots of one thread)
 *   PROGRESS   forward progress between tasks (independent thread scheduling)
 *   GLOBALMEM  the global address space is accessible
 *   LOCALMEM   memory shared by the level's tasks only (DSMEM, shared memory)
 *   GROUPMEM   memory private to each task (registers, local memory)
 *   CACHE      a transparent cache at the level (L2, L1)
 */
typedef enum hp_prop {
    HP_PROP_BARRIER = 1u << 0,
    HP_PROP_CRITICAL = 1u << 1,
    HP_PROP_ATOMIC = 1u << 2,
    HP_PROP_SHUFFLE = 1u << 3,
    HP_PROP_OVERSUB = 1u << 4,
    HP_PROP_DYNAMIC = 1u << 5,
    HP_PROP_LOCKSTEP = 1u << 6,
    HP_PROP_PROGRESS = 1u << 7,
    HP_PROP_GLOBALMEM = 1u << 8,
    HP_PROP_LOCALMEM = 1u << 9,
    HP_PROP_GROUPMEM = 1u << 10,
    HP_PROP_CACHE = 1u << 11
} hp_prop;

/* The properties of hardware level hw (GRID, CLUSTER, CTA, WARP, SUBWARP,
 * LANE, SEQ) and num = how many tasks of it run in parallel within one unit
 * of the enclosing level (`num(c)`; the grid: CTAs resident on the device at
 * 256 threads).  No GPU needed (the device's SM count, if a device is present;
 * else GB300's 152). */
hp_status hp_level_properties(hp_hw hw, uint32_t *props, int64_t *num);

/* One nest level's requirements: the `sync` set it needs, the `reserve` set
 * it must leave to its nested levels, and min_num, the fewest parallel tasks
 * it needs at its level (0: any). */
typedef struct {
    uint32_t sync;
    uint32_t reserve;
    int64_t min_num;
} hp_level_req;

/* Pick a level map for a nest of `depth` levels from their requirements:
 * level l (outermost first) takes the coarsest hardware level at or below the
 * previous level's that has req[l].sync and at least req[l].min_num tasks,
 * such that every inner level can still be placed.  With req[l].reserve set,
 * the level's own hardware level must lack the reserved properties, a strictly
 * finer one must have them, and the inner levels start strictly below it (the
 * level uses every level except those it reserves).  A level with no
 * requirement stays on its enclosing level (collapse) or, outermost, takes GRID.
 * At the warp's level, 0 < min_num < 32 asks for a sub-warp partition (Sec.
 * 3.8): the narrowest power-of-two width >= min_num whose inner levels can
 * still be placed (up to the whole warp); an inner level that collapses onto
 * a sub-warp partition keeps its width.  HP_EINVAL (with the level that could
 * not be placed) when no map satisfies them: selection succeeds exactly when
 * some map passes hp_level_check. */
hp_status hp_level_select(int depth, const hp_level_req *req, hp_level_map *map_out);

/* Does `map` (depth entries, no AUTO) meet the requirements `req`, under the
 * rules of hp_level_select?  Each level must be at or below its enclosing
 * level's hardware level (strictly below one that reserves), have the sync
 * properties, at least min_num tasks (the team size the map gives a CTA,
 * sub-warp or vector level, else the level's capacity) and, with a reserve
 * set, lack those properties while a finer level has them.  HP_OK, or
 * HP_EINVAL with the first level that fails in hp_last_error.  Host only. */
hp_status hp_level_check(int depth, const hp_level_req *req, const hp_level_map *map);

/* hp_nest_tune with requirements as its constraint language (Sec. 3.2: a
 * construct states what it needs and the implementation picks the level):
 * req[depth] as for hp_level_select.  Only candidate maps that meet them are
 * timed (hp_level_check), with the map hp_level_select derives from them
 * first; flags as for hp_nest_tune.  The winner is cached for the shape class
 * under this set of requirements only: nests created later with map == NULL
 * never take it.  HP_EINVAL when no candidate meets the requirements (a nest
 * whose levels are all outputs: when its map does not). */
hp_status hp_nest_tune_req(hp_nest *n, const hp_level_req *req, const void *const *in_dev, void *out_dev,
                           void *stream, int32_t flags);

/* ---------------------------------------------------------------------- */
/* Stencil nests with ghost zones.
 *
 * Sec. 2: stencils can be tiled to any level that has local memory, a region
 * chosen so that its input region fits that memory; Sec. 4: a level maps each
 * of its units an array section, the `to` sections overlapping by a ghost
 * surface, the `from` sections partitioning the array.
 *
 * One step of a 2-D stencil of radius r (0..4) over the ny x nx FP32 array v
 * (row-major) is the cross-correlation
 *     (S v)[y][x] = sum_{dy,dx = -r..r} c[dy+r][dx+r] * v[y+dy][x+dx],
 * with v = 0 outside the array.  A nest of `steps` steps (1..8) computes
 * S^steps(A), each point of each step as one FP32 fused multiply-add chain
 * over the window in row-major (dy, dx) order, starting from 0, every step's
 * values rounded to FP32: a run with steps = T gives bit for bit the result of
 * T runs with steps = 1.
 *
 * Two levels: the GRID level's map sections (section_y x section_x points,
 * whole tiles; 0 = the whole array) order the work, section after section, so
 * that neighbouring tiles share their ghost rows through L2; the CTA level's
 * tiles (tile_y x tile_x, tile_x a multiple of 4; 0 = automatic) are mapped
 * into shared memory with a ghost border of r * steps points (one 2-D tensor
 * copy, out-of-array points read as 0), all steps run there, and the CTA
 * writes back its tile.
 */
typedef struct hp_stencil hp_stencil;
typedef struct {
  int64_t section_y, section_x;   /* GRID-level sections (multiples of the tile; 0 = whole array) */
  int32_t tile_y, tile_x;         /* CTA-level tiles (0 = automatic) */
} hp_stencil_map;

/* Plan a stencil nest (host only, no GPU needed).  coeffs: (2r+1)^2 host
 * floats, row-major over (dy, dx), copied.  map may be NULL (automatic).
 * HP_EINVAL for sizes out of range or a tile whose ghost-bordered box does not
 * fit one CTA's shared memory (226 KB) or one tensor copy (256 x 256 points). */
hp_status hp_stencil_create(int64_t ny, int64_t nx, int radius, const float *coeffs, int steps,
                            const hp_stencil_map *map, hp_stencil **out);

/* Run on `stream` (asynchronous).  in_dev / out_dev: device arrays of ny x nx
 * FP32, row-major, not overlapping.  Rows whose pitch (4 nx bytes) or base is
 * not 16-byte aligned are loaded with plain loads instead of tensor copies
 * (same results).  Device-side waits are bounded; hp_stencil_check reports. */
hp_status hp_stencil_run(hp_stencil *s, const float *in_dev, float *out_dev, void *stream);

/* The plan as one line of JSON: sizes, tile, ghost widths, tensor box,
 * shared memory, tiles, and the GRID-level sections' `to` / `from` boxes
 * (when there are at most 64 sections). */
hp_status hp_stencil_describe(const hp_stencil *s, char *buf, size_t len);

/* Wait for the stream, read the stencil's device error word (0 = none, 1 = a
 * tensor-copy wait ran out of time); HP_ETIMEOUT if set. */
hp_status hp_stencil_check(hp_stencil *s, void *stream, int32_t *device_error);

void hp_stencil_destroy(hp_stencil *s);

/*
 * Process-wide planner options, read when a nest is created (existing nests
 * keep their plan).  Names:
 *   "pipeline"  1 (default): block teams whose element groups allow it stream
 *               their inputs through per-thread cp.async rings; 0: plain loads.
 *               Both give bit-identical results (same reduction tree).
 *   "serve_batching"  1 (default): servers pack admitted requests into
 *               batched steps; 0: servers launch each request alone.
 *   "tune_log"  0 (default); 1: hp_nest_tune* write every candidate's map,
 *               kernel and time to stderr.
 *   "host_zero_copy"  1 (default): hp_nest_run_host reads a mapped page-locked
 *               first input in place; 0: always through a staging copy.
 * HP_EINVAL for an unknown name.
 */
hp_status hp_set_option(const char *name, int64_t value);
hp_status hp_get_option(const char *name, int64_t *value);

/* Message of the last failed call on this thread ("" if none). */
const char *hp_last_error(void);

/* ABI version (major * 100 + minor). */
int hp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HP_H */
