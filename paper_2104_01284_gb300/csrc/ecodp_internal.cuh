// Internal types and FP32 device arithmetic shared by the ecodp kernels.
//
// Paper: Zhu et al., "A GPU Implementation of a Look-Ahead Optimal
// Controller for Eco-Driving Based on Dynamic Programming", ECC 2021.
//
// Data layout in HBM (per problem):
//   V   float [N+1][n_v][n_soc+2][ld_t]   value function of every stage.  Soc
//       rows 0 and n_soc+1 and time columns >= n_t are padding that always
//       holds V_BIG, so an interpolation corner that falls outside the grid
//       reads an "infeasible" value without a branch.  ld_t = round_up(n_t+2,
//       4) keeps every row 16-byte aligned and leaves the column after the
//       first padding column inside the row (a clamped lower time corner at
//       n_t still has its upper neighbour there).
//   pi  int16 [N][n_v][n_soc][n_t]        argmin control index, -1 infeasible.
//   per-stage tables (written for every stage by the precompute kernel):
//       ClassRec  [N][n_v][n_cls]  speed/time transition of every torque class
//       ClassEntry[N][n_v][n_cls]  the feasible classes of each speed row
//       SplitRec  [N][n_v][n_u]    per-control record (cost, SoC shift, weights, u)
//
// Infeasibility is carried as the finite sentinel V_BIG instead of +inf: an
// interpolation weight of exactly 0 (a snapped fraction) then contributes
// exactly 0, and any non-zero weight (>= 1e-5 per axis, so >= 1e-15 for a
// trilinear corner) lifts the sum above V_FEAS_MAX.  Results >= V_FEAS_MAX are
// stored as V_BIG and reported to callers as +inf.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

// Bounds-checked build (compiled with -DECODP_CHECKS into a second library,
// libecodp_checked.so).  Every index a kernel computes into shared or global
// memory is compared with its array's extent before the access, through
// DP_IN(index, extent).  A failed check records the first failure -- the
// source file's tag (ECODP_FILE_TAG, set per file), the line and the index --
// in the translation unit's device word, skips the access (the code takes a
// safe fallback) and never traps; the host reads the words and reports
// DP_ERR_INTERNAL.  In the production build DP_IN is the constant true and
// costs nothing.
#ifndef ECODP_FILE_TAG
#define ECODP_FILE_TAG 0
#endif

namespace ecodp {

#ifdef ECODP_CHECKS
static __device__ unsigned long long g_check_word;  // one per translation unit

__device__ __forceinline__ bool dp_in_range(long long i, long long n, unsigned line, unsigned tag)
{
    if (i >= 0 && i < n)
        return true;
    const unsigned long long site = ((unsigned long long)((tag << 16) | (line & 0xffffu)) << 32) | (unsigned)i;
    atomicCAS(&g_check_word, 0ull, site);
    return false;
}
#define DP_IN(i, n) ::ecodp::dp_in_range((long long)(i), (long long)(n), __LINE__, ECODP_FILE_TAG)
// Host: this translation unit's word (first failure, 0 if none), then cleared.
#define ECODP_CHECK_ACCESSOR(name)                                                       \
    cudaError_t name(unsigned long long *w)                                              \
    {                                                                                    \
        cudaError_t e = cudaMemcpyFromSymbol(w, g_check_word, sizeof *w);                \
        if (e != cudaSuccess || *w == 0)                                                 \
            return e;                                                                    \
        const unsigned long long zero = 0;                                               \
        return cudaMemcpyToSymbol(g_check_word, &zero, sizeof zero);                     \
    }
#else
#define DP_IN(i, n) true
#define ECODP_CHECK_ACCESSOR(name)          \
    cudaError_t name(unsigned long long *w) \
    {                                       \
        *w = 0;                             \
        return cudaSuccess;                 \
    }
#endif

// the check words of the kernel translation units (all 0 in the production build)
cudaError_t check_word_precompute(unsigned long long *w);
cudaError_t check_word_bellman(unsigned long long *w);
cudaError_t check_word_rollout(unsigned long long *w);
cudaError_t check_word_adjoint(unsigned long long *w);
cudaError_t check_word_batch(unsigned long long *w);

constexpr float V_BIG = 1e30f;
constexpr float V_FEAS_MAX = 1e12f;
constexpr float SNAP = 1e-5f;

struct DevParams {
    // sizes
    int N, n_v, n_xi, n_t, n_te, n_tm, n_b, n_u;
    int n_cls;      // torque classes (see ClassRec)
    int class_sum;  // 1: classes are the sums i_e + i_m (equal torque steps)
    int ld_t, xi_rows;
    int n_lights;
    // grids: node i = lo + (span * i) / (n - 1)
    float v_lo, v_span, xi_lo, xi_span, t_lo, t_span, te_lo, te_span, tm_lo, tm_span;
    float h_v, h_xi, h_t;
    float ds;
    // model
    float mass, g, crr, half_rho_cda, ratio, brake_force, a_min, a_max, eta, voc, r0, cap;
    float half_rho;  // rho / 2 (for the CdA derivative of the adjoint)
    float fc[6];
    float fuel_scale, gamma;
    float soc_ref, w_soc, v_ref, w_v;
    // paper variants (see dp_problem_desc)
    int light_model;    // 1: green indicator sampled on the time grid
    int torque_limits;  // 1: speed-dependent torque limits
    float te_max_c[3], bsg_pmax;
    int all_lines;  // 1: the tables keep every feasible control of each SoC-shift bucket (no envelope)
};

// Speed-dependent torque limits (Eq. 7e, 7f) at crank speed w; true if the
// control (Te, Tm) is allowed.
__device__ __forceinline__ bool torque_allowed(const DevParams &P, float w, float Te, float Tm)
{
    if (!P.torque_limits)
        return true;
    const float te_max =
        __fadd_rn(__fadd_rn(P.te_max_c[0], __fmul_rn(P.te_max_c[1], w)), __fmul_rn(__fmul_rn(P.te_max_c[2], w), w));
    return !(Te > te_max) && !(__fmul_rn(fabsf(Tm), w) > P.bsg_pmax);
}

// A torque class: all controls with the same total torque T_eng + T_bsg and
// brake flag share the speed update (Eq. 5a) and the step time (Eq. 2), hence
// the speed-axis and time-axis interpolation of J_{k+1}.
struct __align__(16) ClassRec {
    int ok;     // feasible at class level (Eq. 7a, 7d, stopping rule)
    int iv;     // lower speed node of v'
    float fv;   // snapped weight of node iv + 1
    float v1;   // v'
    float dt;   // driving time of the step
    int st;     // floor(dt / h_t) after snapping
    float ft;   // snapped fraction of dt / h_t
    int pad;
};

// One control of a row's table: its stage cost c (Eq. 1/6), the SoC-axis
// cell shift d and fraction f of xi' = xi - dt I / C_nom (Eq. 5b), and its
// index u, packed as bits = u | d << 16.  Its interpolated value at SoC row j
// is G(j + d) + (c + f (G(j + d + 1) - G(j + d))) with G the speed/time
// blend of J_{k+1}.  16 bytes: one vector load.
struct __align__(16) SplitRec {
    float c, f;
    unsigned bits;
    unsigned pad;
};

struct __align__(16) ClassEntry {
    int cls;    // class index
    int off;    // first split record of this class in the row's split array
    int nb[4];  // lower-envelope controls with soc shift d = -2, -1, 0, +1
    int n_other;  // every control with any other shift (after the four buckets)
    int n_total;
};

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

__device__ __forceinline__ float node_val(float lo, float span, int i, int n)
{
    return n > 1 ? __fadd_rn(lo, __fdiv_rn(__fmul_rn(span, (float)i), (float)(n - 1))) : lo;
}

// Position inside a light cycle in [0, cycle): red iff < red duration.
__device__ __forceinline__ float phase_pos(float t, float offset, float cycle)
{
    float x = __fsub_rn(t, offset);
    float ph = __fsub_rn(x, __fmul_rn(cycle, floorf(__fdiv_rn(x, cycle))));
    if (ph < 0.f)
        ph = __fadd_rn(ph, cycle);
    if (ph >= cycle)
        ph = __fsub_rn(ph, cycle);
    return ph;
}

// Snap a fraction: below SNAP -> 0, above 1 - SNAP -> next node.
__device__ __forceinline__ void snap_split(float q, int &i, float &f)
{
    float fl = floorf(q);
    i = (int)fl;
    f = __fsub_rn(q, fl);
    if (f < SNAP) {
        f = 0.f;
    } else if (f > 1.f - SNAP) {
        f = 0.f;
        i += 1;
    }
}

// Engine torque and BSG torque of control u = (ie * n_tm + im) * n_b + b.
__device__ __forceinline__ void decode_u(const DevParams &P, int u, int &ie, int &im, int &b)
{
    b = u % P.n_b;
    int r = u / P.n_b;
    im = r % P.n_tm;
    ie = r / P.n_tm;
}

// ---- model pieces (FP32) ----------------------------------------------------

// Road load at speed v on a slope with sin/cos theta (Eq. 5a).
__device__ __forceinline__ float road_load(const DevParams &P, float v, float sin_th, float cos_th)
{
    float roll_grade = __fmul_rn(__fmul_rn(P.mass, P.g), __fadd_rn(__fmul_rn(P.crr, cos_th), sin_th));
    return __fadd_rn(roll_grade, __fmul_rn(P.half_rho_cda, __fmul_rn(v, v)));
}

// Speed update and step time (Eq. 5a, Eq. 2) for total torque T and brake b
// from speed v.  Returns false if infeasible.  next_light: the arrival node
// holds a light (the vehicle may then stop at the line).
__device__ __forceinline__ bool speed_step(const DevParams &P, float v, float F_road, float T, int b, bool next_light,
                                           float &v1, float &dt)
{
    float F_tr = __fsub_rn(__fmul_rn(T, P.ratio), b ? P.brake_force : 0.f);
    float a = __fdiv_rn(__fsub_rn(F_tr, F_road), P.mass);
    if (a < P.a_min || a > P.a_max)
        return false;
    float R = __fadd_rn(__fmul_rn(v, v), __fmul_rn(__fmul_rn(2.f, P.ds), a));
    if (R < 0.f) {
        if (!(next_light && v > 0.f))
            return false;
        v1 = 0.f;
        dt = __fdiv_rn(__fmul_rn(2.f, P.ds), v);
        return true;
    }
    v1 = __fsqrt_rn(R);
    float vs = __fadd_rn(v, v1);
    if (!(vs > 0.f))
        return false;
    dt = __fdiv_rn(__fmul_rn(2.f, P.ds), vs);
    return true;
}

// The literal standstill step of Eq. 5c (light_model 2): from v = 0 at a
// light node, a total torque T and brake b without forward acceleration (the
// acceleration within the comfort limits and v'^2 = 2 ds a <= 0, the same
// arithmetic as speed_step at v = 0) make the distance step at zero speed.
__device__ __forceinline__ bool standstill_class(const DevParams &P, float F_road, float T, int b)
{
    float F_tr = __fsub_rn(__fmul_rn(T, P.ratio), b ? P.brake_force : 0.f);
    float a = __fdiv_rn(__fsub_rn(F_tr, F_road), P.mass);
    if (a < P.a_min || a > P.a_max)
        return false;
    return !(__fadd_rn(0.f, __fmul_rn(__fmul_rn(2.f, P.ds), a)) > 0.f);
}

// Fuel rate (g/s) of the engine at speed w (rad/s) and torque Te (Nm).
__device__ __forceinline__ float fuel_rate(const DevParams &P, float w, float Te)
{
    if (!(Te > 0.f))
        return 0.f;
    float s = P.fc[0];
    s = __fadd_rn(s, __fmul_rn(P.fc[1], w));
    s = __fadd_rn(s, __fmul_rn(P.fc[2], Te));
    s = __fadd_rn(s, __fmul_rn(__fmul_rn(P.fc[3], w), Te));
    s = __fadd_rn(s, __fmul_rn(__fmul_rn(P.fc[4], w), w));
    s = __fadd_rn(s, __fmul_rn(__fmul_rn(P.fc[5], Te), Te));
    return __fmul_rn(P.fuel_scale, s);
}

// Battery current (A) for BSG torque Tm at crank speed w (Eq. 5b): zeroth-
// order circuit, written as 2P / (Voc + sqrt(Voc^2 - 4 R0 P)), the cancellation
// free form of the smaller root.  Returns false if the power exceeds what the
// circuit can deliver.
__device__ __forceinline__ bool battery_current(const DevParams &P, float w, float Tm, float &I)
{
    float Pm = __fmul_rn(Tm, w);
    float Pb = Pm > 0.f ? __fdiv_rn(Pm, P.eta) : __fmul_rn(Pm, P.eta);
    float disc = __fsub_rn(__fmul_rn(P.voc, P.voc), __fmul_rn(__fmul_rn(4.f, P.r0), Pb));
    if (disc < 0.f)
        return false;
    I = __fdiv_rn(__fmul_rn(2.f, Pb), __fadd_rn(P.voc, __fsqrt_rn(disc)));
    return true;
}

__device__ __forceinline__ float terminal_cost(const DevParams &P, float v, float xi)
{
    float sh = fmaxf(__fsub_rn(P.soc_ref, xi), 0.f);
    float dv = __fsub_rn(v, P.v_ref);
    return __fadd_rn(__fmul_rn(P.w_soc, sh), __fmul_rn(P.w_v, __fmul_rn(dv, dv)));
}

// ---- launchers (host) -------------------------------------------------------

// The support of the adjoint weights lam_k as explicit lists, so that a stage
// touches only the states that carry weight: idx[k & 1] lists the states of
// lam_k (each once: bits[k & 1] marks membership), cnt[k % 3] its length;
// stage k reads list k, appends to list k + 1 and clears cnt[(k + 2) % 3].
struct AdjFrontier {
    int *idx;        // [2][n states]
    unsigned *bits;  // [2][words(n)]
    int *cnt;        // [3]
    size_t words;    // 32-bit words of one membership bitmap
};

struct StageTables {
    const float *grade;        // [N]
    const int *light_of_node;  // [N+1], -1 = none
    const float *cycle, *red, *offset;
};

// Tables of the precompute kernel, one slot per stage k (slot k holds stage
// k; a one-stage caller uses slot 0 with its tables re-indexed as stage 0).
struct StageScratch {
    ClassRec *cls;    // [slots][n_v][n_cls]
    ClassEntry *ent;  // [slots][n_v][n_cls]
    int *row_cnt;     // [slots][n_v][2] feasible classes, splits
    SplitRec *spl;    // [slots][n_v][n_u]
    // [8] running totals (may be NULL): feasible (v, u) pairs, feasible
    // (v, class) pairs, states whose minimum ties across classes, states
    // whose argmin was recovered, (v, u) pairs kept in the tables (envelopes);
    // of the states skipped as infeasible (below): (state, class) pairs,
    // (state, line) pairs, states
    unsigned long long *stats;
    // [n_v][n_soc][n_t] packed per-state minima of the class-split Bellman
    // launch (all ones between stages); NULL: never split
    unsigned long long *part;
    // [N + 1] per stage of a sweep: the last time column of J_k holding a
    // feasible state (-1: none; all -1 before the sweep, J_N's is n_t - 1
    // without an entry).  NULL: the launch neither reads nor writes it.
    int *lmax;
    // 1: a sweep that runs alone; its tiles fill every resident CTA slot
    // (the spare ones take class slices).  0: solves that share the GPU keep
    // one tile per 128 lanes.
    int fill_slots;
};

// One instance of a batch (device-resident descriptor).
struct BatchInst {
    StageTables tb;
    StageScratch sc;
    float *V;              // [N+1] padded stages
    int16_t *pi;           // [N] stages
    size_t stage_elems, pi_elems;
    int N, chunks, tiles;  // lane chunks per speed row; tiles per stage (the completion target of a stage)
    int pad;
    int *done;             // [N] completed tiles of each stage (stage k at done[k])
    long long row_off;     // first block of this instance in the batched precompute grid
};

// Limits of the tiled path (validated at create): controls per problem and
// torque classes (per-control and per-class tables live in shared memory).
constexpr int MAX_CONTROLS = 8192;
constexpr int MAX_CLASSES = 4095;

cudaError_t launch_fill(float *p, size_t n, float val, cudaStream_t s);
cudaError_t launch_terminal(const DevParams *dP, const DevParams &hP, float *VN, cudaStream_t s);
// Tables of stages k_first .. k_first + n_k - 1 (one CTA per speed row and stage).
cudaError_t launch_precompute(const DevParams *dP, const DevParams &hP, StageTables tb, int k_first, int n_k,
                              StageScratch sc, cudaStream_t s);
// Corner quads of J for the tiled sweep: quad (iv, j, c) = {V(iv, j, c),
// V(iv, j, c + 1), V(iv + 1, j, c), V(iv + 1, j, c + 1)}, the two time columns
// of a cell at speed rows iv and iv + 1 in one 16-byte record, with V = V_BIG
// outside the grid (j < 0 or j >= n_soc, c >= n_t, iv >= n_v).  Layout
// [n_v][quad_rows][quad_ld], SoC row j at quad row j + 2: every window row a
// tile of 6 or 8 SoC rows per lane reads (SoC rows jb - 2 .. jb + R + 1) lies
// inside, so a window row is a compile-time offset from one address (no
// clamping), and quad_ld, a row stride the kernel is compiled for, is the
// smallest of 64, 128, 256 that holds n_t + 2 columns (0: no quads, the
// plain layout is read).
constexpr int QUAD_PAD = 2;  // quad rows below SoC row 0
__host__ __device__ inline int quad_rows(int n_xi)
{
    const int r6 = (n_xi + 5) / 6 * 6, r8 = (n_xi + 7) / 8 * 8;
    return (r6 > r8 ? r6 : r8) + 2 * QUAD_PAD;
}
__host__ __device__ inline int quad_ld(int n_t)
{
    return n_t + 2 <= 64 ? 64 : (n_t + 2 <= 128 ? 128 : (n_t + 2 <= 256 ? 256 : 0));
}
// Quads of a padded value array (J_N of a sweep).
cudaError_t launch_quad_from_pad(const DevParams &hP, const float *V, float4 *Q, cudaStream_t s);
// One Bellman stage.  With Qn and Qk (corner quads of J_{k+1} and J_k, the
// latter written by the launch) the unsplit tiled kernel reads its windows
// from Qn; every other path ignores them, so a sweep must pass them at every
// stage or at none.
cudaError_t launch_bellman(const DevParams *dP, const DevParams &hP, StageTables tb, int k, StageScratch sc,
                           const float *Vnext, float *Vk, int16_t *pik, int variant, cudaStream_t s,
                           const float4 *Qn = nullptr, float4 *Qk = nullptr);
cudaError_t launch_pad_from_dense(const DevParams &hP, const float *dense, float *padded, cudaStream_t s);
cudaError_t launch_dense_from_pad(const DevParams &hP, const float *padded, float *dense, cudaStream_t s);
// Where J_k lives for the stages a launch reads: base + (k - k_base)
// stage_elems, except stage k_tail, which is at `tail` (a checkpoint after a
// recomputed segment).
struct StageView {
    const float *base;
    const float *tail;
    int k_base, k_tail;
    size_t stage_elems;
    __host__ __device__ const float *at(int k) const
    {
        return k == k_tail ? tail : base + (ptrdiff_t)(k - k_base) * (ptrdiff_t)stage_elems;
    }
    __host__ __device__ static StageView all(const float *V, size_t stage_elems)
    {
        return StageView{V, nullptr, 0, -1, stage_elems};
    }
};

// Forward rollout over stages [k_begin, k_end) (a later segment continues from
// the state left in `out`; see rollout_body).
cudaError_t launch_rollout(const DevParams *dP, const DevParams &hP, StageTables tb, const StageView &view,
                           int k_begin, int k_end, double v0, double xi0, double t0, double *out, int *out_u,
                           cudaStream_t s);

// ---- batched instances (device descriptors in params[b], inst[b]) ----------

// Work list of the persistent Bellman launch (device arrays).
struct BatchSched {
    const int *order;        // [B] instances by decreasing horizon (ties: index)
    const long long *pref;   // [B + 1] prefix sums over `order` of tiles per stage
    const long long *start;  // [max_n + 1] first item of each wavefront step
    const int *m;            // [max_n] instances taking part in each step
    int max_n;
    long long n_items;
    unsigned long long *queue;  // next item (zero before the launch)
    int *error;                 // set to 1 when a dependency wait times out
    unsigned long long wait_limit_ns;  // bound of one dependency wait
};

cudaError_t launch_terminal_batched(const DevParams *params, const BatchInst *inst, int n_inst, cudaStream_t s);
// Tables of every stage of every instance: n_rows = sum over b of N_b n_v_b.
cudaError_t launch_precompute_batched(const DevParams *params, const BatchInst *inst, int n_inst, long long n_rows,
                                      int max_n_u, cudaStream_t s);
// The persistent Bellman launch; rows_per_lane in {4, 8}; ctas_per_sm <= 0:
// as many as fit.
cudaError_t launch_persistent(const DevParams *params, const BatchInst *inst, const BatchSched &S, int rows_per_lane,
                              int max_n_cls, int max_n_u, int ctas_per_sm, cudaStream_t s);
size_t persistent_smem_bytes(int rows_per_lane, int max_n_cls, int max_n_u);
int persistent_chunks_per_row(int rows_per_lane, int n_xi, int n_t);
int persistent_max_ctas_per_sm(int rows_per_lane, int max_n_cls, int max_n_u);
// One CTA per instance; instance b writes [3(N+1) + 3N + 4] doubles at
// out + out_off[b] and N ints at out_u + u_off[b] (layout of launch_rollout).
cudaError_t launch_rollout_batched(const DevParams *params, const BatchInst *inst, int n_inst, const double *x0,
                                   const long long *out_off, const long long *u_off, double *out, int *out_u,
                                   cudaStream_t s);

}  // namespace ecodp
