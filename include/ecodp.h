/*
 * ecodp.h -- C ABI of the GB300 dynamic-programming solver for look-ahead
 * eco-driving (Zhu, Gupta, Pivaro, Deshpande, Canova: "A GPU Implementation
 * of a Look-Ahead Optimal Controller for Eco-Driving Based on Dynamic
 * Programming", ECC 2021).
 *
 * The solver computes, on one GPU and in FP32, the backward recursion of
 * Eq. (9a)-(9d) over the three-state grid x = [v, SoC, t] (Eq. 4a) with
 * controls u = [T_eng, T_bsg] plus a brake flag (Eq. 4b), the dynamics of
 * Eq. (5a)-(5c), the stage cost of Eq. (1)/(6) and the constraints of
 * Eq. (7)/(8), followed by a forward rollout that extracts the optimal
 * speed/SoC/time trajectory.
 *
 * Conventions (all entry points):
 *   - Every call returns a dp_status; none aborts, exits or prints.  The
 *     message of the last failure on the calling thread is dp_last_error().
 *   - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls that take a stream enqueue their GPU work on it and
 *     return before it finishes unless they copy results to host memory.
 *   - Arrays are C order.  Value arrays are float32 [n_v][n_soc][n_t] (t
 *     fastest); infeasible states hold +INFINITY.  Policies are int16 of the
 *     same shape holding the control index u = (i_eng * n_tm + i_bsg) *
 *     n_brake + brake, or -1 where the state is infeasible.
 *   - A problem object owns all its device memory (allocated through the
 *     caller's allocator when one is given) and frees it in
 *     dp_problem_destroy.  The caller owns descriptors and output buffers.
 *   - After DP_ERR_CUDA the problem object must only be destroyed.
 */
#ifndef ECODP_H
#define ECODP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DP_OK = 0,
    DP_ERR_INVALID_ARG = 1, /* a descriptor field or argument is out of range */
    DP_ERR_OOM = 2,         /* the allocator returned NULL */
    DP_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    DP_ERR_INFEASIBLE = 4,  /* no feasible control at some rollout stage */
    DP_ERR_NOT_SOLVED = 5,  /* results requested before dp_solve_backward */
    DP_ERR_TIMEOUT = 6,     /* a bounded device wait gave up */
    DP_ERR_INTERNAL = 7     /* a kernel reported an inconsistency */
} dp_status;

/* Device-memory allocator supplied by the caller (for example a wrapper of
 * PyTorch's caching allocator).  alloc returns a device pointer or NULL;
 * free releases it.  Both are called on the creating thread, with the
 * stream given to dp_problem_create.  A NULL allocator makes the library use
 * cudaMallocAsync / cudaFreeAsync on that stream. */
typedef struct dp_allocator {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, void *stream, void *ctx);
    void *ctx;
} dp_allocator;

/* One receding-horizon problem (Eq. 6) in SI units.  All grids are uniform
 * with inclusive ends: node i of an n-point grid over [lo, hi] is
 * lo + (hi - lo) * i / (n - 1).  Copied at create/update; the caller keeps
 * ownership of the arrays. */
typedef struct dp_problem_desc {
    int32_t n_stages;     /* N distance steps of ds metres (Eq. 1) */
    double ds;            /* distance step Delta d, m (Eq. 2) */
    const double *grade;  /* [n_stages] road grade per step, fraction (Eq. 5a) */
    double v_lo, v_hi;    /* speed grid, m/s; its ends are the limits of Eq. 7a */
    int32_t n_v;          /* >= 2 */
    double soc_lo, soc_hi; /* SoC grid, fraction; limits of Eq. 7b */
    int32_t n_soc;        /* >= 2 */
    double t_lo, t_hi;    /* time grid, s; t_hi is the horizon's t_f (Eq. 8) */
    int32_t n_t;          /* >= 2 */
    double te_lo, te_hi;  /* engine torque grid, Nm (Eq. 7e); te_lo >= 0 */
    int32_t n_te;         /* >= 1 */
    double tm_lo, tm_hi;  /* BSG torque grid, Nm (Eq. 7f) */
    int32_t n_tm;         /* >= 1 */
    int32_t n_brake;      /* 1 = no brake control, 2 = brake flag {0, 1} */
    double brake_decel;   /* deceleration added by the brake flag, m/s^2 */
    double a_min, a_max;  /* comfort acceleration limits, m/s^2 (Eq. 7d) */
    double mass, cda, crr, rho, g; /* road load (Eq. 5a) */
    double r_wheel, gear;          /* one total ratio gear / r_wheel, 1/m */
    double eta_motor;              /* constant BSG efficiency in (0, 1] */
    double voc, r0, capacity_As;   /* zeroth-order battery (Eq. 5b) */
    double fuel_coef[6];  /* mdot = s (c0 + c1 w + c2 T + c3 w T + c4 w^2 + c5 T^2) g/s, T > 0 */
    double fuel_scale;    /* s */
    double gamma;         /* fuel/time weight of Eq. 1 in [0, 1] */
    double soc_ref, w_soc, v_ref, w_v; /* terminal cost w_soc max(0, soc_ref - soc) + w_v (v - v_ref)^2 */
    int32_t n_lights;     /* traffic lights (Fig. 3) */
    const int32_t *light_stage; /* [n_lights] distinct nodes in [1, n_stages - 1] */
    const double *cycle, *red, *offset; /* [n_lights] s; red iff ((t - offset) mod cycle) < red */
    /* Paper variants; 0 selects the default reading. */
    int32_t light_model;  /* 0: an arrival at a light node with v' > 0 is checked at its continuous
                             time, and a vehicle standing at the line waits for green;
                             1: the green indicator sampled on the time grid (Sec. III, Eq. 8):
                             at a light node every state with v > 0 at a red time node is
                             infeasible, and arrivals are not checked otherwise;
                             2: the literal standstill step of Eq. 5c: standing at a light node,
                             a control without forward acceleration and with T_eng = 0 makes the
                             distance step at zero speed while the clock jumps to the end of red
                             (zero time during green), at the cost (1 - gamma) t_RG; a departure
                             needs green */
    int32_t torque_limits; /* 0: the torque grids are the limits; 1: speed-dependent limits
                              (Eq. 7e, 7f) at the stage-start crank speed w = v gear / r_wheel */
    double te_max_coef[3]; /* torque_limits = 1: T_eng <= c0 + c1 w + c2 w^2 (Nm, w in rad/s) */
    double bsg_power_max;  /* torque_limits = 1: |T_bsg| w <= bsg_power_max (W, >= 0) */
} dp_problem_desc;

typedef struct dp_problem *dp_problem_t;

/* Rollout output: caller-owned HOST arrays. */
typedef struct dp_trajectory {
    double *v, *soc, *t; /* [n_stages + 1] states along the route */
    int32_t *u;          /* [n_stages] applied control index */
    double *dt;          /* [n_stages] driving time of each step, s */
    double *wait;        /* [n_stages] standstill at a red light before the step, s */
    double *fuel;        /* [n_stages] fuel burnt in each step, g */
    double fuel_g;       /* out: total fuel, g */
    double time_s;       /* out: total time, s */
    double J;            /* out: total cost including the terminal cost */
    int32_t fail_stage;  /* out: first stage without a feasible control, or -1 */
} dp_trajectory;

/* Validate desc, allocate the problem's device state (value function for
 * all N+1 stages, policy for N stages, per-stage scratch) and copy the
 * problem tables to the device on `stream`.  Errors: DP_ERR_INVALID_ARG
 * (sizes < limits above, non-finite parameters, lights not at distinct
 * nodes in [1, N-1], n_te * n_tm * n_brake > 32767), DP_ERR_OOM,
 * DP_ERR_CUDA. */
dp_status dp_problem_create(const dp_problem_desc *desc, const dp_allocator *alloc, void *stream,
                            dp_problem_t *out);

/* Replace the problem's route data and parameters (grade, lights, model
 * constants, grid ranges; Eq. 5-8) with those of desc, which must have the
 * same sizes (stages, grid points, controls, torque classes); the number of
 * lights may change.  Asynchronous on stream (the host tables are copied
 * before the call returns).  Previously computed results become stale
 * (DP_ERR_NOT_SOLVED). */
dp_status dp_problem_update(dp_problem_t p, const dp_problem_desc *desc, void *stream);

/* Free everything (through the caller's allocator). NULL is accepted. */
dp_status dp_problem_destroy(dp_problem_t p);

/* Backward recursion of Eq. (9a)-(9d): J_N = c_T on the grid, then for
 * k = N-1 .. 0 the per-state minimum over all controls of the stage cost
 * plus the trilinearly interpolated J_{k+1} at the successor, with the
 * argmin.  Controls with the same total torque T_eng + T_bsg and brake flag
 * (a torque class) and the same SoC cell shift read the same two SoC rows of
 * J_{k+1}; their values are lines c + f D in the difference D of those rows,
 * and only the lines on the lower envelope of each such group are evaluated
 * (the FP32 minimum is that of all controls, see dp_set_envelopes).  Successor
 * times never precede the state's own time, so a state whose time node lies
 * beyond the last time column of J_{k+1} holding a feasible value reads only
 * infeasible values: the sweep writes such states infeasible without
 * evaluating them, and the GPU threads that frees share the class lists of
 * the remaining states (the results are the same).  Exact FP32 ties
 * are broken in the order (torque class, control index): the first class,
 * ordered by brake flag and then by ascending total torque, that reaches the
 * minimum, then the lowest control index inside that class.  Asynchronous on stream;
 * results stay on the device.  The sweep's launches (terminal values, the
 * per-stage tables of all stages, then the N Bellman stages) are captured in a
 * CUDA graph on the first call and replayed afterwards. */
dp_status dp_solve_backward(dp_problem_t p, void *stream);

/* Copy J_stage (stage in [0, N]) or pi_stage (stage in [0, N-1]) into
 * `out` (device memory, or host memory when out_is_host; the host copy
 * synchronises the stream).  DP_ERR_NOT_SOLVED before a solve. */
dp_status dp_get_value(dp_problem_t p, int32_t stage, float *out, int32_t out_is_host, void *stream);
dp_status dp_get_policy(dp_problem_t p, int32_t stage, int16_t *out, int32_t out_is_host, void *stream);

/* One stage of the recursion in isolation: J_k and pi_k from a given J_{k+1}
 * (float32 [n_v][n_soc][n_t], +INFINITY = infeasible), device or host
 * memory as flagged.  Outputs go to v_out / pi_out (either may be NULL)
 * with the same location flag.  Used to compare single stages; it does not
 * change the stored solution. */
dp_status dp_solve_stage(dp_problem_t p, int32_t k, const float *v_next, int32_t v_next_is_host, float *v_out,
                         int16_t *pi_out, int32_t out_is_host, void *stream);

/* Forward rollout from x0 = {v, soc, t} (host array) through the stored
 * J_1..J_N: at each stage every control is evaluated at the continuous
 * state, the argmin (lowest index on ties) is applied, and fuel and time are
 * summed in FP64 on the device.  Fills the caller's host trajectory and
 * synchronises the stream.  Called right after dp_solve_backward on the same
 * stream (no other call on the problem in between, no checkpointing), the
 * rollout starts as soon as J_1 is written, beside the sweep's last stage,
 * on a stream of the problem's own that the caller's stream then waits for;
 * the result is the same.  DP_ERR_INFEASIBLE if a stage has no feasible
 * control (traj->fail_stage tells which); DP_ERR_NOT_SOLVED before a solve. */
dp_status dp_rollout(dp_problem_t p, const double x0[3], dp_trajectory *traj, void *stream);

/* Bounds-check report (a debugging aid; no counterpart in the paper).  The
 * library ships in two builds from the same sources: libecodp.so and the
 * bounds-checked libecodp_checked.so, in which every index the kernels
 * compute into shared or global memory is compared with its array's extent
 * before the access.  A failed check never traps: the kernel records the
 * first failure (source tag, line, index) in a device word, skips the
 * access and goes on, and the host reports it as DP_ERR_INTERNAL.
 *   enabled: (host, may be NULL) 1 in the checked build, 0 otherwise; set
 *            without touching the device
 *   site:    (host, may be NULL) receives the first recorded failure
 *            (tag << 48 | line << 32 | index), 0 if none; the record is then
 *            cleared.  Reading it synchronises the device.
 * Returns DP_ERR_INTERNAL (with the site in dp_last_error) when a failure was
 * recorded, DP_OK otherwise (always in the production build).  In the
 * checked build dp_rollout, dp_adjoint, dp_multi_wait, dp_multi_rollout and a
 * completed dp_batch_poll check the record themselves and return
 * DP_ERR_INTERNAL instead of their result when it is set. */
dp_status dp_debug_checks(int32_t *enabled, uint64_t *site);

/* FP32 FMA throughput probe (a measurement aid; no counterpart in the
 * paper).  The Bellman kernels are bound by FP32 issue and their roofline is
 * quoted against SMs x 128 FP32 lanes x 2 FLOP x SM clock; this call times
 * `repeats` launches (after one warm-up) of a kernel that keeps every SM's
 * FP32 pipes busy with independent packed FMAs, on the current device and
 * stream, and returns the fastest launch's rate.
 *   repeats: >= 1
 *   tflops:  (host) FP32 FLOP/s of the fastest launch / 1e12, 2 FLOP per FMA
 *   ms:      (host) that launch's milliseconds
 * Allocates a few KB on the stream (cudaMallocAsync) and synchronises it.
 * DP_ERR_INVALID_ARG for NULL outputs or repeats < 1, DP_ERR_CUDA on a CUDA
 * failure. */
dp_status dp_measure_fp32_peak(int32_t repeats, double *tflops, double *ms, void *stream);

/* On-chip load bandwidth probes, the measured peaks beside the Bellman
 * kernel's rates (a measurement aid; the paper has no counterpart).  Every
 * thread of SMs x 6 CTAs of 256 threads keeps 8 independent 16-byte loads in
 * flight:
 *   kind 0: shared memory (32 KB per CTA, conflict-free);
 *   kind 1: L1 (each CTA re-reads its own 16 KB of a global buffer with
 *           ld.global.ca; after the first pass every load hits);
 *   kind 2: L2 (a 64 MB buffer, inside the L2, streamed with L2-only loads).
 * Each kind runs one warm-up launch and `repeats` timed launches on stream
 * and reports the fastest: *gbs = bytes loaded / time in GB/s (1e9 B/s),
 * *ms = that launch's time.  Allocates and frees (stream-ordered) at most
 * 64 MB; synchronises stream.  DP_ERR_INVALID_ARG for a null output,
 * repeats < 1 or another kind.
 */
dp_status dp_measure_onchip_bw(int32_t kind, int32_t repeats, double *gbs, double *ms, void *stream);

/* One stage of the recursion, like dp_solve_stage, for callers that cannot
 * allocate GPU memory.  The paper has no counterpart; this entry point exists
 * for integrations whose memory is fixed after start-up: a controller task
 * that runs under a hard real-time budget (cudaMalloc and cudaFree may block
 * and synchronise the whole device), or code embedded in a host framework
 * that owns every device allocation and forbids others.  Such callers cannot
 * create a dp_problem (it allocates), so this call takes the descriptor
 * directly and allocates nothing: its working memory is one static device
 * array of about 12 MB built into the library, present on every GPU that
 * loads it until the process exits.
 *   desc:    the problem (host memory); only stage k's grade and lights are used
 *   v_next:  J_{k+1}, float32 [n_v][n_soc][n_t] in DEVICE memory, +INFINITY =
 *            infeasible
 *   v_out:   J_k, same layout, DEVICE memory (caller-owned)
 *   pi_out:  pi_k, int16 same shape, DEVICE memory (caller-owned)
 * Results equal those of dp_solve_stage on the same inputs.  Limits: n_v <= 64,
 * n_soc <= 64, n_t <= 255, at most 2048 controls and 256 torque classes;
 * larger problems get DP_ERR_INVALID_ARG.  Asynchronous on stream.  Each call
 * looks up the array's address on the current device; the first call on a
 * device also loads the library's device code there (a set-up step), so make
 * that first call before any stream capture begins.  Every
 * call on a device shares that device's one array, so calls whose GPU work
 * can overlap (issued on different streams or from different host threads)
 * race and corrupt each other's results: order them on one stream.  Each
 * call re-initialises what it reads from the array. */
dp_status dp_solve_stage_static(const dp_problem_desc *desc, int32_t k, const float *v_next, float *v_out,
                                int16_t *pi_out, void *stream);

/* Gradient of the optimal cost J_0(x0) (the interpolated value function at
 * x0 = {v, soc, t}, host array) with respect to theta = (mass, CdA, Crr, R0,
 * fuel-map scale), written to the host array dJ_dtheta[5]; J0 (host, may be
 * NULL) receives J_0(x0).  Envelope theorem: with the stored argmins fixed,
 * dJ_0/dtheta = sum_k sum_s lam_k(s) (dc/dtheta + grad J_{k+1} . df/dtheta),
 * with lam propagated forward from x0 through the argmins and the
 * interpolation weights; the step derivatives follow Eq. (2), (5a), (5b), (6).
 * FP32 per-state terms, FP64 weights and reduction.  Synchronises the
 * stream.  DP_ERR_NOT_SOLVED before a solve, DP_ERR_INFEASIBLE if x0 is
 * outside the grid or infeasible.  The derivative is one-sided information
 * where an argmin or an interpolation cell changes with theta. */
dp_status dp_adjoint(dp_problem_t p, const double x0[3], double dJ_dtheta[5], double *J0, void *stream);

/* Value-function storage (the adjoint's checkpointing).  every = 0 or 1:
 * J_k of every stage stays on the device after a solve (the default).
 * every = K >= 2: the backward sweep keeps only J_0, J_K, J_2K, ... and J_N;
 * dp_rollout, dp_adjoint and dp_get_value recompute the stages between two
 * checkpoints, one segment at a time, with the same kernels and per-stage
 * tables (results bit-identical to the default; the adjoint's FP64 sums may
 * differ in the last bits from a different atomic order).  The recompute
 * costs about one extra backward sweep per rollout or adjoint call; value
 * memory drops from N+1 stages to about N/K + K + 2.  Waits for the device
 * to be idle, replaces the storage and marks the problem unsolved.
 * DP_ERR_INVALID_ARG unless 0 <= every <= n_stages. */
dp_status dp_set_checkpointing(dp_problem_t p, int32_t every);

/* Human-readable name of a status, and the last error message of the
 * calling thread (empty string if none). */
const char *dp_status_string(dp_status s);
const char *dp_last_error(void);

/* Sizes of the problem (for marshalling): fills n_stages, n_v, n_soc, n_t,
 * n_controls. */
dp_status dp_problem_sizes(dp_problem_t p, int32_t sizes[5]);

/* Select the Bellman kernel of later solves: 1 = tiled (default: torque
 * classes, register windows, shared-memory tables; on grids whose tiles cannot
 * fill the GPU each tile's classes are split over several CTAs and joined; a
 * lane holds 8 SoC rows, or 6 where that fills the lanes at least 15 % better),
 * 2 / 3 = tiled with 8 / 6 SoC rows per lane forced, 0 = direct (one thread per
 * state, every kept control read separately; the layout of the paper's second
 * kernel, Sec. IV).  All return bit-identical values and policies; the direct
 * one exists for cross-checking.  DP_ERR_INVALID_ARG otherwise. */
dp_status dp_set_kernel_variant(dp_problem_t p, int32_t variant);

/* Lower envelopes of the stage tables (Sec. IV's per-(v, u) table, reduced):
 * within one torque class and SoC-shift bucket every control's value at a
 * state is G + (c_u + f_u D) for the same two blended values of J_{k+1}
 * (Eq. 9b), a line in D, so only the lines on the bucket's lower envelope can
 * be the minimum.  on = 1 (default) keeps only those lines (a line is dropped
 * only when it lies above two others by a clear margin); on = 0 keeps every
 * feasible control, a cross-check: the values and policies of a solve are the
 * same either way (FP32 evaluations of a dropped line never fall below the
 * kept ones).  Takes effect at the next solve; call it between solves, not
 * while one runs.  Synchronous; DP_ERR_INVALID_ARG for another value. */
dp_status dp_set_envelopes(dp_problem_t p, int32_t on);

/* Profiling hook: run one backward sweep (same work and results as
 * dp_solve_backward) with direct launches and CUDA events around every
 * kernel, synchronise, and report milliseconds: ms[0] terminal values,
 * ms[1] all N precompute launches, ms[2] all N Bellman launches, ms[3] the
 * whole sweep. */
dp_status dp_profile_sweep(dp_problem_t p, void *stream, float ms[4]);

/* Counters of the last sweep (synchronises the stream): out[0] = state x
 * control evaluations whose control passed the per-(speed, control) checks
 * (effective evaluations, summed over stages and over every state), out[1] =
 * state x torque-class pairs evaluated, out[2] = bytes one dp_problem_update
 * copies host to device, out[3] = bytes one dp_rollout copies device to
 * host, out[4] = reserved (0), out[5] = feasible states whose argmin the
 * tiled kernel recovered, out[6] = state x control pairs the Bellman kernels
 * evaluate: per torque class and SoC shift only the controls on the lower
 * envelope of their values, out[7] = (state, stage) pairs written infeasible
 * without evaluation because their time lies beyond J_{k+1}'s last feasible
 * time column (out[1] and out[6] exclude them; see dp_solve_backward).
 * DP_ERR_NOT_SOLVED before a sweep. */
dp_status dp_sweep_stats(dp_problem_t p, int64_t out[8], void *stream);

/* ---- Batches of independent problems ------------------------------------
 *
 * The paper solves one horizon at a time (Sec. IV-V).  A batch solves many
 * independent problems -- each its own recursion of Eq. (9a)-(9d), with its
 * own horizon, grids, controls and lights -- in one persistent Bellman
 * launch.  Every instance's values and policies are bit-identical to those
 * of dp_solve_backward on the same descriptor (same arithmetic, same tie
 * order), whatever the batch and the configuration.  A batch owns the device
 * memory of all its instances (through the caller's allocator when one is
 * given) until dp_multi_destroy.  After DP_ERR_CUDA the batch must only be
 * destroyed. */
typedef struct dp_multi *dp_multi_t;

typedef struct dp_multi_opts {
    int32_t rows_per_lane; /* SoC rows per lane of a Bellman tile: 4 or 8 (0 = 8) */
    int32_t ctas_per_sm;   /* resident CTAs per SM of the persistent launch (0 = as many as fit) */
    int32_t wait_limit_ms; /* bound of one dependency wait of the persistent launch (0 = 10000) */
} dp_multi_opts;

/* Validate descs[0..n-1] (the rules of dp_problem_create, instance by
 * instance), allocate every instance's value function, policy and per-stage
 * tables, and upload the route tables on `stream` (synchronised before
 * returning).  opts may be NULL (defaults).  Errors: DP_ERR_INVALID_ARG (the
 * message names the instance), DP_ERR_OOM, DP_ERR_CUDA. */
dp_status dp_multi_create(const dp_problem_desc *descs, int32_t n, const dp_multi_opts *opts,
                          const dp_allocator *alloc, void *stream, dp_multi_t *out);

/* Free everything.  NULL is accepted. */
dp_status dp_multi_destroy(dp_multi_t m);

/* Change the tile configuration (rows_per_lane in {0, 4, 8}, ctas_per_sm in
 * [0, the number that fit]) and select the persistent launch; synchronises
 * the creation stream.  Results of earlier solves become stale
 * (DP_ERR_NOT_SOLVED). */
dp_status dp_multi_set_config(dp_multi_t m, int32_t rows_per_lane, int32_t ctas_per_sm);

/* Select the per-instance mode (streams in [1, 16]) or return to the
 * persistent launch (streams = 0).  Per instance: the single-problem sweep
 * (terminal values, corner quads, tables, one Bellman launch per stage, the
 * kernels of dp_solve_backward, results bit-identical to it) captured as its
 * own CUDA graph on the batch's buffers; a solve forks `streams` internal
 * streams from the caller's stream, deals the instances over them by
 * decreasing work (each to the stream with the least so far) and joins them
 * back, so it stays asynchronous on that stream.  The first switch allocates
 * each instance's two corner-quad slots and captures the graphs (a few ms
 * per instance); synchronises the creation stream.  Results of earlier
 * solves become stale. */
dp_status dp_multi_set_streams(dp_multi_t m, int32_t streams);

/* Solve every instance.  Persistent launch: terminal values and per-stage
 * tables of all instances (one launch each), then one persistent launch over
 * (instance, stage, tile) work items in wavefront order, each tile of stage
 * k waiting for the tiles of stage k+1 of its instance; captured in a CUDA
 * graph on the first call (and after dp_multi_set_config) and replayed on
 * `stream`; a dependency wait that gives up (after 10 s) is reported by the
 * next synchronising call as DP_ERR_TIMEOUT.  Per-instance mode
 * (dp_multi_set_streams): the instances' graphs on the internal streams,
 * joined back into `stream`.  Asynchronous either way. */
dp_status dp_multi_solve(dp_multi_t m, void *stream);

/* Synchronise `stream` and report DP_ERR_TIMEOUT if the last solve's
 * persistent launch gave up a dependency wait. */
dp_status dp_multi_wait(dp_multi_t m, void *stream);

/* One solve with direct launches and CUDA events (same work and results as
 * dp_multi_solve); synchronises and reports ms[0] terminal + precompute
 * launches, ms[1] the persistent Bellman launch, ms[2] the whole solve (in
 * the per-instance mode ms[0] = 0 and ms[1] = ms[2], the instances' graphs
 * interleaving on the streams). */
dp_status dp_multi_profile(dp_multi_t m, void *stream, float ms[3]);

/* Autotuner: time every persistent configuration (rows_per_lane in {4, 8}
 * x every ctas_per_sm that fits) and the per-instance mode on 2, 4 and 8
 * streams, `repeats` timed solves each after one warm-up, keep the fastest
 * (minimum whole-solve time) and set it.  best[0] = rows_per_lane, best[1] =
 * ctas_per_sm, best[2] = streams (0: the persistent launch won; then best[0]
 * and best[1] are its configuration, else both 0); *best_ms (may be NULL)
 * its time.  Synchronises; leaves the batch solved. */
dp_status dp_multi_autotune(dp_multi_t m, void *stream, int32_t repeats, int32_t best[3], float *best_ms);

/* Test hook for the timeout path: raise instance b's per-stage completion
 * target by one, so that every dependency wait on b's stages runs out
 * (bounded by wait_limit_ms each) and the next synchronising call reports
 * DP_ERR_TIMEOUT; the results of b are then meaningless.  dp_multi_set_config
 * restores the target.  DP_ERR_INVALID_ARG for a bad index. */
dp_status dp_multi_debug_stall(dp_multi_t m, int32_t b);

/* out[0] instances, out[1] work items of the persistent launch, out[2] its
 * CTAs, out[3] rows_per_lane, out[4] CTAs per SM, out[5] nominal state x
 * control evaluations of one solve (sum of N n_v n_soc n_t n_controls),
 * out[6] device bytes held, out[7] the longest horizon, out[8] streams of
 * the per-instance mode (0: the persistent launch is selected). */
dp_status dp_multi_info(dp_multi_t m, int64_t out[9]);

/* J_stage / pi_stage of instance b, as dp_get_value / dp_get_policy (dense
 * [n_v][n_soc][n_t] of that instance, device or host memory as flagged).
 * Synchronise the stream. */
dp_status dp_multi_get_value(dp_multi_t m, int32_t b, int32_t stage, float *out, int32_t out_is_host, void *stream);
dp_status dp_multi_get_policy(dp_multi_t m, int32_t b, int32_t stage, int16_t *out, int32_t out_is_host,
                              void *stream);

/* Forward rollout of every instance (one CTA each, the arithmetic of
 * dp_rollout): x0 is a host array [n][3], traj an array of n caller-owned
 * trajectories sized for their instances.  Synchronises.  DP_ERR_INFEASIBLE
 * if any instance has a stage without a feasible control (every
 * trajectory's fail_stage tells which). */
dp_status dp_multi_rollout(dp_multi_t m, const double *x0, dp_trajectory *traj, void *stream);

/* ---- Serving: continuous batching of receding-horizon re-solves ---------
 *
 * The paper's controller re-solves the look-ahead problem as the vehicle
 * advances (receding horizon, Sec. III); a server re-solves for many
 * vehicles at once.  A dp_batch holds up to max_slots slots; each is a
 * resident problem with its own CUDA stream, so requests submitted while
 * others are on the GPU run concurrently with them.  A request's result is
 * identical to dp_solve_backward + dp_rollout of the same descriptor alone
 * (same kernels, same arithmetic, no cross-request state).
 *
 * Memory: a slot's device memory (value function, policy, tables) stays
 * allocated after its request is collected; the next request whose sizes
 * match re-uses it through an in-place table update (dp_problem_update).
 * New slots are created only while the sum of the slots' device bytes stays
 * within mem_budget.  Slots and results are owned by the batch; trajectories
 * by the caller.  Calls on one batch are serialised by an internal lock. */
typedef struct dp_batch *dp_batch_t;

/* Errors: DP_ERR_INVALID_ARG (max_slots outside [1, 4096], mem_budget 0,
 * allocator with a NULL function), DP_ERR_OOM. */
dp_status dp_batch_create(int32_t max_slots, size_t mem_budget, const dp_allocator *alloc, dp_batch_t *out);

/* Wait for every slot's work and free all device and pinned memory. NULL is
 * accepted.  Uncollected results are discarded. */
dp_status dp_batch_destroy(dp_batch_t b);

/* Admit one request: the problem desc (validated as in dp_problem_create)
 * and the rollout start x0 = {v, soc, t} (host).  Non-blocking: enqueues the
 * backward sweep (Eq. 9), the forward rollout and the copy of its result on
 * the slot's stream and returns a ticket.  DP_ERR_OOM when no slot is free
 * and no new slot fits in the budget (the request is not admitted: collect
 * finished requests with dp_batch_poll and submit again). */
dp_status dp_batch_submit(dp_batch_t b, const dp_problem_desc *desc, const double x0[3], uint64_t *ticket);

/* Collect a request: DP_ERR_NOT_SOLVED while it is still running (nothing
 * written); otherwise fills the caller's trajectory (host arrays sized for
 * the request's n_stages), frees the slot and returns DP_OK, or
 * DP_ERR_INFEASIBLE when the rollout found a stage without a feasible
 * control.  DP_ERR_INVALID_ARG for a ticket that is unknown or collected. */
dp_status dp_batch_poll(dp_batch_t b, uint64_t ticket, dp_trajectory *traj);

/* out[0] slots, out[1] busy slots, out[2] device bytes held, out[3]
 * requests admitted, out[4] collected, out[5] submit attempts refused with DP_ERR_OOM,
 * out[6] slot creations, out[7] admissions that re-used a slot's memory. */
dp_status dp_batch_stats(dp_batch_t b, int64_t out[8]);

#ifdef __cplusplus
}
#endif

#endif /* ECODP_H */
