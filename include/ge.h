/*
 * ge.h -- C ABI of the GB300 group explicit (GE) solver for the transient
 * diffusion equation u_t = u_xx on [0, 1] (Parand, Zafarvahedian, Hossayni,
 * arXiv:1310.3422, Sec. 2; Tavakoli's unconditionally stable alternating
 * Saul'yev scheme, sub-domain width 1).
 *
 * Problem (Sec. 2, problem statement):
 *   u_t = u_xx,  u(x, 0) = phi(x),  u(0, t) = beta_l,  u(1, t) = beta_r.
 *   The paper has one wall value beta; two independent values are a superset.
 * Mesh (Sec. 2): n interior points, h = 1/(n+1), x_i = (i+1) h for the 0-based
 *   array index i = 0..n-1, tau = r h^2, r = tau / h^2 the mesh ratio.
 * Step (Sec. 2, Eqs. (aa), (bb), (cc), (dd)): with parity p = s mod 2 of the
 *   global step counter s, p = 0 couples the points in groups (0,1),(2,3),...
 *   and p = 1 in groups (1,2),(3,4),...; a point without a partner at either
 *   end is a singleton.  Each group's 2x2 system (Saul'yev B at its left
 *   member, A at its right member) is solved by Eqs. (cc)/(dd) with the
 *   prefactor 1/(1+2r); a singleton uses Saul'yev A at the left wall and B at
 *   the right wall, the wall value standing in for the new-level neighbour.
 *
 * Conventions for every entry point:
 *   - Element type: double for GE_F64, float for GE_F32 and GE_F32_COMP.
 *   - "_dev" pointers are CUDA device pointers (or managed memory) on the
 *     current device; "_host" pointers are host memory.  The caller owns
 *     every buffer it passes; the library never frees or retains them past
 *     the call (asynchronous calls read/write them in stream order).
 *   - `stream` is a cudaStream_t passed as void*; NULL selects the legacy
 *     default stream.  Work is enqueued asynchronously on that stream unless
 *     stated otherwise.
 *   - Every call returns a ge_status and never throws; a thread-local text
 *     for the last failure is available from ge_last_error().
 *   - Device-side failures (a bounded wait that ran out) are recorded in a
 *     device word and reported by ge_sync() or the next synchronising call.
 */
#ifndef GE_H
#define GE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GE_OK = 0,
    GE_EINVAL = 1,      /* invalid argument (see each entry point)           */
    GE_ENOMEM = 2,      /* a device or pinned-host allocation failed         */
    GE_ECUDA = 3,       /* a CUDA runtime or driver call failed              */
    GE_ETIMEOUT = 4,    /* a bounded device-side wait gave up                */
    GE_ENONFINITE = 5   /* the checked state holds NaN or Inf                */
} ge_status;

typedef enum {
    GE_F64 = 0,         /* FP64 storage and arithmetic                        */
    GE_F32 = 1,         /* FP32 storage and arithmetic                        */
    GE_F32_COMP = 2     /* FP32 storage; each point's updates are summed with
                           a compensation word (Kahan) kept on chip within a
                           launch                                            */
} ge_precision;

typedef enum {
    GE_KERNEL_AUTO = 0,      /* GE_KERNEL_TEMPORAL with the built-in depth    */
    GE_KERNEL_CANONICAL = 1, /* one launch per step; Eqs. (cc)/(dd), (aa)/(bb)
                                evaluated literally with fused multiply-adds
                                in the order the equations print their terms
                                (GE_F64: bit-identical to a serial FP64
                                evaluation in that order); GE_F64/GE_F32 only */
    GE_KERNEL_ONESTEP = 2,   /* one launch per step on the group systems'
                                right-hand sides (see GE_KERNEL_TEMPORAL)     */
    GE_KERNEL_TEMPORAL = 3,  /* `depth` steps per launch: a tile plus a halo
                                of depth+1 points per side is staged in shared
                                memory by TMA and advanced on chip.  Between
                                steps it carries the right-hand side of each
                                group's 2x2 system, w = (I - r G') u + wall
                                terms, so one step is the block map
                                (I - r G)(I + r G)^{-1} = [[1,2r],[2r,1]]/(1+2r)
                                on each group: the same scheme, reassociated */
    GE_KERNEL_TEMPORAL_DF = 4 /* GE_KERNEL_TEMPORAL for GE_F64 contexts with
                                the steps evaluated on the FP32 pipes in
                                double-float arithmetic: every value an
                                unevaluated sum of two floats (about 48
                                significant bits), each step built from
                                error-free transformations (TwoProd by FMA,
                                TwoSum, Fast2Sum).  Storage, API and HBM bytes
                                stay FP64; each call prescales by the power of
                                two that brings max |u| and the wall values
                                below 1, so any double data are in range.
                                Rounding is about 2^-48 per step instead of
                                2^-53: within 1e-12 of a serial FP64
                                evaluation at moderate r, but at very large r
                                (where FP64 itself loses digits to
                                conditioning) some 30x further off than FP64.
                                GE_F64 only; r <= 2^20; width k = 1 */
} ge_kernel;

typedef struct ge_ctx ge_ctx;  /* opaque; owned by the library */

/* Create a solver for one problem.
 *   out        receives the new context (set to NULL on failure).
 *   n          number of interior points, n >= 1.
 *   r          mesh ratio tau/h^2, finite and > 0.
 *   beta_l/r   wall values u(0,t), u(1,t), finite.
 *   prec       GE_F64, GE_F32 or GE_F32_COMP.
 *   u0_dev     n elements of phi(x_i) (device memory, caller-owned, copied
 *              before the call returns); NULL starts from zeros.
 *   stream     stream all later work of this context is enqueued on.
 * The context owns two device buffers of n elements (padded to whole
 * 128-byte rows).  The step counter starts at 0 (next step has parity 0).
 * The tiled kernel's steps per launch start at the built-in default, or at
 * the first line of the tuning table named by the environment variable
 * GE_TUNE_TABLE that matches: lines "<f64|f32|f32c> <n_min> <n_max>
 * <depth>", '#' comments, malformed lines skipped (ge_tune writes what to
 * put there).
 * Errors: GE_EINVAL (bad n, r, beta, prec, out == NULL), GE_ENOMEM, GE_ECUDA. */
ge_status ge_create(ge_ctx **out, int64_t n, double r, double beta_l, double beta_r,
                    ge_precision prec, const void *u0_dev, void *stream);

/* Select the kernel used by later ge_step_n calls.  depth: steps per launch
 * for GE_KERNEL_TEMPORAL and GE_KERNEL_TEMPORAL_DF, 1..1023 (0 = built-in
 * default); ignored otherwise.
 * Errors: GE_EINVAL (NULL ctx, unknown kernel, depth out of range,
 * GE_KERNEL_CANONICAL with GE_F32_COMP, GE_KERNEL_TEMPORAL_DF with a
 * precision other than GE_F64 or with r > 2^20). */
ge_status ge_set_kernel(ge_ctx *ctx, ge_kernel kernel, int32_t depth);

/* The kernel in use and the tiled kernel's steps per launch (the default
 * resolved).  Errors: GE_EINVAL. */
ge_status ge_get_kernel(const ge_ctx *ctx, ge_kernel *kernel, int32_t *depth);

/* Autotune the tiled kernel's steps per launch: times `steps` steps from the
 * current state at each candidate depth (FP64: 24, 32, 48, 64, 96; FP32:
 * 64 ... 256; double-float: 32 ... 128), keeps the fastest (returned in *best_depth, may be NULL) and
 * leaves the state and the step counter as they were.  A context on the
 * canonical, one-step or width-k path keeps its setting.  Synchronous;
 * allocates one scratch copy of the state.  Errors: GE_EINVAL, GE_ENOMEM,
 * GE_ECUDA. */
ge_status ge_tune(ge_ctx *ctx, int64_t steps, int32_t *best_depth);

/* Sub-domain width k (Sec. 2: odd sub-domains [x_{2ik}, x_{2ik+k-1}], even
 * sub-domains [x_{2ik+k}, x_{2(i+1)k-1}] of the paper's nodes x_0..x_{n+1}).
 * k = 1 (the default) is the 2-point group scheme every kernel above runs.
 * For k > 1 each step couples the two wall nodes of every confluence of a B
 * sub-domain with the A sub-domain to its right by Eqs. (cc)/(dd) and sweeps
 * Saul'yev A runs to the right and B runs to the left (paper node j uses A
 * at parity p iff floor(j/k) + p is even), one thread per confluence unit.
 * With GE_KERNEL_AUTO / GE_KERNEL_TEMPORAL ge_step_n then runs `depth` steps
 * per launch (ge_set_kernel; default 8) on tiles kept in shared memory,
 * falling back to one launch per step when fewer than 64 units of 2k nodes
 * fit a CTA's shared memory; GE_KERNEL_CANONICAL / GE_KERNEL_ONESTEP run one
 * launch per step.  Both are bit-identical to a serial FP64 evaluation.
 * Errors: GE_EINVAL (NULL ctx, k < 1, k > 1 with GE_F32_COMP). */
ge_status ge_set_subdomain_width(ge_ctx *ctx, int64_t k);

/* Advance the state by `steps` GE time steps (steps >= 0), continuing the
 * parity of the step counter, which increases by `steps`.  Asynchronous on
 * the context's stream; may be captured in a CUDA graph once the context
 * exists.  Errors: GE_EINVAL (NULL ctx, steps < 0), GE_ECUDA (launch). */
ge_status ge_step_n(ge_ctx *ctx, int64_t steps);

/* Copy the current n values into out_dev (device, n elements of the
 * context's type).  Asynchronous.  Errors: GE_EINVAL, GE_ECUDA. */
ge_status ge_read_state(ge_ctx *ctx, void *out_dev);

/* Replace the state by in_dev (n elements) and set the step counter to
 * step_count >= 0 (resume from a checkpoint).  Also clears a recorded
 * device failure (the state it spoiled is replaced).  Asynchronous.
 * Errors: GE_EINVAL, GE_ECUDA. */
ge_status ge_write_state(ge_ctx *ctx, const void *in_dev, int64_t step_count);

/* Copy points [offset, offset + count) of the current state to out_dev
 * (device, count elements of the context's type, caller-owned), or replace
 * them by in_dev.  The step counter and any recorded device failure stay as
 * they are.  These move the halos of a solve split over ranks: after S steps
 * a point depends only on the points within S + 1 of it (the dependency cone
 * of the step of Sec. 2), so refreshing a range's halos every S steps keeps
 * its inner points exact.  Asynchronous on the context's stream.
 * Errors: GE_EINVAL (NULL buffer, range outside 0..n), GE_ECUDA. */
ge_status ge_read_range(ge_ctx *ctx, int64_t offset, int64_t count, void *out_dev);
ge_status ge_write_range(ge_ctx *ctx, int64_t offset, int64_t count, const void *in_dev);

/* Query the step counter.  Errors: GE_EINVAL. */
ge_status ge_get_step(const ge_ctx *ctx, int64_t *step_count);

/* Wait for the context's stream and report deferred device errors
 * (GE_ETIMEOUT) and launch errors (GE_ECUDA).  A GE_ETIMEOUT stays reported
 * (the state is not valid) until ge_write_state replaces the state. */
ge_status ge_sync(ge_ctx *ctx);

/* Diagnostic (failure handling without a GPU fault): with cycles > 0 every
 * tile-load wait of the context's tiled launches polls a barrier that
 * nothing arrives on, gives up after `cycles` SM clock cycles, and takes the
 * path of a tile load that never completes: the kernel records GE_ETIMEOUT,
 * lets its own copies in flight land (each within the normal limit of about
 * 2 s) and returns, so the context stays usable.  cycles = 0 turns it off.
 * Errors: GE_EINVAL (NULL ctx, cycles < 0). */
ge_status ge_debug_stall(ge_ctx *ctx, int64_t cycles);

/* Release the context and its buffers (after finishing its stream's work).
 * NULL is a no-op. */
void ge_destroy(ge_ctx *ctx);

/* One-shot solve from HOST memory (the end-to-end path): copies u0_host
 * (n elements) to the device, advances `steps` steps from step counter 0
 * with the given kernel/depth, and copies the result to u_out_host.
 * Synchronous.  Both host buffers may be pageable or pinned, and may alias.
 * Errors: as ge_create / ge_set_kernel / ge_step_n, plus GE_EINVAL for NULL
 * host buffers. */
ge_status ge_solve(int64_t n, double r, double beta_l, double beta_r, ge_precision prec,
                   ge_kernel kernel, int32_t depth, int64_t steps, const void *u0_host,
                   void *u_out_host, void *stream);

/* ---- Batched solves: many independent problems, one packed buffer ---------
 * Each problem b is the problem of Sec. 2 with its own n[b] interior points,
 * mesh ratio r[b] and wall values beta_l[b], beta_r[b]; all share the step
 * count and start from step counter 0.  Its n[b] values sit at u_dev[offsets[b]
 * .. offsets[b] + n[b]) of one caller-owned device buffer of `total` elements
 * (type as for ge_create).  offsets[b] must be a multiple of 128 bytes (16
 * doubles / 32 floats) and problems may not share a 128-byte row; the values
 * between problems are left untouched.  The batched kernel runs the tiled
 * right-hand-side scheme of GE_KERNEL_TEMPORAL, each thread taking its
 * problem's constants, `depth` steps per launch.  GE_F64 and GE_F32 run it
 * in the scaled form x <- x + 2r x_partner on each problem minus its linear
 * wall profile (a fixed point of the step, so the shifted problem has zero
 * walls), with per-problem power-of-two rescalings and the inverse scale
 * applied at each launch end (the same data range as ge_create's tiled
 * kernel); GE_F32_COMP runs the normalised form
 * x <- x + 2r/(1+2r) (x_partner - x) with Kahan-summed updates. */
typedef struct ge_batch ge_batch;   /* opaque plan, owned by the library */

/* Build a plan: checks the layout and uploads the per-problem table (host
 * arrays, copied).  The plan owns two working copies of the packed buffer
 * (padded to whole rows), a row -> problem table and the device error word.
 * Errors: GE_EINVAL (n_problems < 1, NULL array, n[b] < 1, r[b] not finite
 * and > 0, unaligned or out-of-range offset, overlapping problems),
 * GE_ENOMEM, GE_ECUDA. */
ge_status ge_batch_create(ge_batch **out, int32_t n_problems, const int64_t *n, const double *r,
                          const double *beta_l, const double *beta_r, const int64_t *offsets,
                          int64_t total, ge_precision prec, void *stream);

/* Steps per launch (1..512, 0 = built-in default).  Errors: GE_EINVAL. */
ge_status ge_batch_set_depth(ge_batch *plan, int32_t depth);

/* Kernel of later ge_batch_run calls: GE_KERNEL_AUTO / GE_KERNEL_TEMPORAL
 * (the default), or for a GE_F64 plan GE_KERNEL_TEMPORAL_DF.  The
 * double-float kernel keeps the plan's FP64 storage and evaluates the steps
 * as pairs of floats (see GE_KERNEL_TEMPORAL_DF): each call prescales every
 * problem by the power of two above its largest |u| and wall value, and
 * padding between problems comes back bit for bit.  Every distinct launch
 * length of a plan takes one of its 64 end-factor slots; the FP64 kernel
 * falls back to its normalised form past them, the double-float kernel has
 * none, so there ge_batch_run fails with GE_EINVAL.  Synchronous (waits for
 * the plan's stream, recomputes the rescaling table).
 * Errors: GE_EINVAL (NULL plan, another kernel, GE_KERNEL_TEMPORAL_DF on a
 * GE_F32 / GE_F32_COMP plan or with some r > 2^20), GE_ENOMEM, GE_ECUDA. */
ge_status ge_batch_set_kernel(ge_batch *plan, ge_kernel kernel);
ge_status ge_batch_get_depth(const ge_batch *plan, int32_t *depth);

/* Tile geometry of later ge_batch_run calls: rows per tile (256, the
 * default, or 128: the tile width W of the 2D TMA box; 0 = 256) and CTAs per
 * SM of the persistent grid (1 .. what fits, 0 = as many as fit; 256-row
 * tiles fit 2 per SM, 128-row tiles 4).  The double-float kernel has
 * 256-row tiles only.  Errors: GE_EINVAL (NULL plan, other values). */
ge_status ge_batch_set_geometry(ge_batch *plan, int32_t tile_rows, int32_t ctas_per_sm);
/* The geometry in use (0 values resolved).  Errors: GE_EINVAL. */
ge_status ge_batch_get_geometry(const ge_batch *plan, int32_t *tile_rows, int32_t *ctas_per_sm);

/* Persistent launch (on = 1) for a plain FP32 plan: a ge_batch_run of more
 * than `depth` steps runs as ONE launch that advances every tile round by
 * round (rounds of `depth` steps, the same cut and arithmetic as one launch
 * per round, so the same bits).  A tile of round k + 1 starts once its own
 * and its two neighbouring tiles of round k are written: per-tile counters in
 * device memory, acquire / release ordered, each wait bounded (GE_ETIMEOUT).
 * There is no launch boundary, so the tail of one round overlaps the start
 * of the next.  Other plans (FP64, compensated FP32, double-float) keep one
 * launch per round.  on = 0 (the default): one launch per `depth` steps.
 * Errors: GE_EINVAL, GE_ENOMEM (its counters, n_rows ints, on first use). */
ge_status ge_batch_set_persistent(ge_batch *plan, int32_t on);
ge_status ge_batch_get_persistent(const ge_batch *plan, int32_t *on);

/* Autotune the launches on the caller's data: times `steps` steps of the
 * data in u_dev (which is not modified) for each candidate, by coordinate
 * search: the depth T (16, 32, 48, 64, 96, 128, 192, 256 steps per launch)
 * at the plan's geometry, then the geometry (rows per tile W in {256, 128}
 * x CTAs per SM) at that depth, then the depth again, and for a plain FP32
 * plan the persistent launch against one launch per depth steps.  Keeps the
 * fastest (see ge_batch_get_depth, ge_batch_get_geometry,
 * ge_batch_get_persistent) and returns its depth in
 * *best_depth (may be NULL).  This is the counterpart of the paper's tuning
 * of its block count (Sec. 4) for the batched kernel.  Synchronous.
 * Errors: GE_EINVAL, GE_ECUDA. */
ge_status ge_batch_tune(ge_batch *plan, const void *u_dev, int64_t steps, int32_t *best_depth);

/* Advance every problem of the batch by `steps` steps, in place in u_dev.
 * Asynchronous on the plan's stream; launches and device-to-device copies
 * only, so a CUDA graph may capture it.  Errors: GE_EINVAL, GE_ECUDA. */
ge_status ge_batch_run(ge_batch *plan, void *u_dev, int64_t steps);

/* Wait for the plan's stream; report deferred device errors (GE_ETIMEOUT),
 * then clear them (every run starts again from the caller's buffer). */
ge_status ge_batch_sync(ge_batch *plan);

/* Scan the packed buffer u_dev (the plan's layout and type) for NaN and Inf:
 * status_dev[b] (device, n_problems int32, caller-owned) receives GE_OK or
 * GE_ENONFINITE for problem b.  Only values inside problems are read.
 * Asynchronous on the plan's stream.  Errors: GE_EINVAL, GE_ECUDA. */
ge_status ge_batch_check(ge_batch *plan, const void *u_dev, int32_t *status_dev);

/* Diagnostic, as ge_debug_stall for the plan's launches. */
ge_status ge_batch_debug_stall(ge_batch *plan, int64_t cycles);

/* Release the plan (NULL is a no-op). */
void ge_batch_destroy(ge_batch *plan);

/* One-shot: ge_batch_create + ge_batch_run [+ ge_batch_check into
 * status_dev, n_problems int32 on the device, when not NULL] +
 * ge_batch_sync + ge_batch_destroy.  Synchronous. */
ge_status ge_solve_batch(int32_t n_problems, const int64_t *n, const double *r, const double *beta_l,
                         const double *beta_r, const int64_t *offsets, int64_t total, void *u_dev,
                         int32_t *status_dev, int64_t steps, ge_precision prec, void *stream);

/* The tiled solve (GE_KERNEL_TEMPORAL) for callers that may not allocate
 * device memory: a plug-in inside a host application or server that owns all
 * device memory through its own pool, a real-time loop that cannot take
 * cudaMalloc's implicit synchronisation, or a sandbox without driver
 * allocations after start-up.  The paper has no counterpart; it is a
 * deployment variant of the same kernel.
 *   u0_dev      n elements of the initial state (device, caller-owned).
 *   u_out_dev   n elements receiving the state after `steps` steps from
 *               step counter 0 (device, caller-owned; may alias u0_dev).
 *   depth       steps per launch, 0 = built-in default, up to 1023.
 * It allocates nothing: its working memory (two padded state buffers and the
 * device error word) is one static device array of 16 MiB + 256 bytes, held
 * on a device from its creation until exit, so n is limited to 1,048,576
 * points (GE_EINVAL beyond).  The first call on a device does the set-up,
 * with that device current: it looks the array's address up, and under
 * CUDA's default lazy module loading the driver then loads the library's
 * modules and creates the array -- driver allocations.  A caller that must
 * not allocate later therefore makes one warm-up call at start-up on each
 * device, for each precision it uses, with steps >= 1 (or sets
 * CUDA_MODULE_LOADING=EAGER); make it before any stream capture.  Every call
 * on a device shares the array: calls whose GPU work overlaps (other
 * streams, other host threads) race, so serialise them.
 * Synchronous: returns once u_out_dev holds the result (it synchronises the
 * stream).
 * Errors: GE_EINVAL (n out of range, bad r, beta, prec, depth, steps, NULL
 * buffer), GE_ECUDA, GE_ETIMEOUT (a bounded device wait gave up). */
ge_status ge_solve_noalloc(int64_t n, double r, double beta_l, double beta_r, ge_precision prec,
                           int32_t depth, int64_t steps, const void *u0_dev, void *u_out_dev,
                           void *stream);

/* Whether the FP64 tiled kernel of this context computes part of its
 * interior updates as exact FP64 multiply-adds on the integer pipes (on = 1,
 * the default; see ge_fp64_int_share) or all of them on the FP64 unit
 * (on = 0).  The results are the same bits either way; the switch exists to
 * compare the two.  Affects later GE_KERNEL_TEMPORAL / ONESTEP steps of
 * GE_F64 contexts.  Errors: GE_EINVAL (NULL ctx, on not 0 or 1). */
ge_status ge_set_int_pipes(ge_ctx *ctx, int32_t on);

/* Build information: the fraction of the FP64 tiled kernel's interior
 * updates (GE_KERNEL_TEMPORAL and ONESTEP, GE_F64, threads whose points and
 * partners all lie inside the grid; the batched FP64 kernel of ge_batch_*
 * takes the same share in its interior warps) computed as exact FP64
 * multiply-adds on the integer pipes instead of the FP64 unit (the scaled
 * block step of Sec. 2, x <- x + 2r x_partner; same bits either way).  A warp whose emulated
 * updates leave the integer fast path in a step (zeros, subnormals, far-apart
 * magnitudes) recomputes them on the FP64 unit, so the realised share can
 * be lower.  *share (host) receives the build's share, 0 when disabled.
 * Errors: GE_EINVAL (NULL share). */
ge_status ge_fp64_int_share(double *share);

/* Diagnostic: checks the integer-pipe FP64 multiply-add of the FP64 tiled
 * kernel (the scaled block step x + g p, Sec. 2) against the FP64 unit's fma
 * on n inputs p_dev[i], x_dev[i] (device, caller-owned, n doubles each).
 * counts_dev (device, 3 uint64, overwritten): [0] inputs where the integer
 * form reported its fast path but gave other bits than the FP64 unit (0 in
 * a correct build), [1] inputs its general fast path took, [2] inputs its
 * addition-only form took.  Asynchronous on `stream`.  Errors: GE_EINVAL
 * (NULL buffer, n < 0), GE_ECUDA. */
ge_status ge_emu_fma_check(double g, const double *p_dev, const double *x_dev, int64_t n, uint64_t *counts_dev,
                           void *stream);

/* Diagnostic: register-only fused multiply-add throughput probe, the
 * measured ALU ceiling the tiled kernels are read against (the paper has no
 * counterpart).  Launches `blocks` CTAs of 256 threads on `stream`; every
 * thread runs `chains` (4, 8, 16 or 32) independent chains x <- x * a + b
 * for `iters` iterations in registers (prec GE_F64: DFMA, GE_F32: FFMA),
 * then stores one value to sink_dev (device, caller-owned, blocks * 256
 * elements of the precision's type).  Multiply-adds done:
 * blocks * 256 * chains * iters.  Asynchronous; the caller times it on the
 * stream.  Errors: GE_EINVAL, GE_ECUDA. */
ge_status ge_probe_fma(int32_t prec, int32_t blocks, int32_t chains, int64_t iters, void *sink_dev,
                       void *stream);

/* Name of a status code (static string). */
const char *ge_status_str(ge_status status);

/* Text describing the last failure on the calling thread (static storage,
 * valid until the next failing call on this thread); "" if none. */
const char *ge_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GE_H */
