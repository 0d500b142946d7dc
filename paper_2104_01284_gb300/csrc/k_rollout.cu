// Forward rollout (trajectory extraction, the simulation step of Sec. V).
//
// A cluster of CTAs (one CTA per instance in the batched form) walks the N
// stages from x0.  At every stage each thread evaluates a strided subset of
// the controls at the continuous state: the one-step model (Eq. 2, 5a-5c), the
// constraints (Eq. 7, 8) and the trilinear interpolation of J_{k+1} at the
// continuous successor; an argmin over the CTA, then over the cluster through
// distributed shared memory (lowest control index on ties), selects the
// control, which every CTA applies to its copy of the state.  Cumulative time,
// fuel and cost are summed in FP64.
#include <climits>

#include <cooperative_groups.h>

#include "ecodp_internal.cuh"

#undef ECODP_FILE_TAG
#define ECODP_FILE_TAG 3

namespace ecodp {

ECODP_CHECK_ACCESSOR(check_word_rollout)

namespace {

__device__ __forceinline__ bool locate_cont(float x, float lo, float h, int n, int &i, float &f)
{
    float q = __fdiv_rn(__fsub_rn(x, lo), h);
    float top = (float)(n - 1);
    if (q < -SNAP || q > top + SNAP)
        return false;
    q = fminf(fmaxf(q, 0.f), top);
    snap_split(q, i, f);
    if (i >= n - 1) {
        i = n - 2;
        f = 1.f;
    }
    return true;
}

// Trilinear interpolation of the padded value array at a continuous point.
__device__ float interp_cont(const DevParams &P, const float *__restrict__ Vn, float v, float xi, float t)
{
    int iv, ix, it;
    float fv, fx, ft;
    if (!locate_cont(v, P.v_lo, P.h_v, P.n_v, iv, fv) || !locate_cont(xi, P.xi_lo, P.h_xi, P.n_xi, ix, fx) ||
        !locate_cont(t, P.t_lo, P.h_t, P.n_t, it, ft))
        return V_BIG;
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        float wa = a ? fv : __fsub_rn(1.f, fv);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            float wb = b ? fx : __fsub_rn(1.f, fx);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                float wc = c ? ft : __fsub_rn(1.f, ft);
                const size_t o = ((size_t)(iv + a) * P.xi_rows + (ix + b + 1)) * P.ld_t + (it + c);
                float val = DP_IN(o, (size_t)P.n_v * P.xi_rows * P.ld_t) ? Vn[o] : V_BIG;
                acc = __fmaf_rn(__fmul_rn(__fmul_rn(wa, wb), wc), val, acc);
            }
        }
    }
    return acc;
}

struct Step {
    float v1, xi1, dt, wait, mf, cost;
};

// One model step from a continuous state; false if infeasible.
__device__ bool model_step(const DevParams &P, const StageTables &tb, int k, float v, float xi, float t, int u,
                           Step &s)
{
    int ie, im, b;
    decode_u(P, u, ie, im, b);
    const float Te = node_val(P.te_lo, P.te_span, ie, P.n_te);
    const float Tm = node_val(P.tm_lo, P.tm_span, im, P.n_tm);
    const float p = tb.grade[k];
    const float sq = __fsqrt_rn(__fadd_rn(1.f, __fmul_rn(p, p)));
    const float F_road = road_load(P, v, __fdiv_rn(p, sq), __fdiv_rn(1.f, sq));
    int nl = tb.light_of_node[k + 1];
    int lk = tb.light_of_node[k];
    if (!DP_IN(nl + 1, P.n_lights + 1))
        nl = -1;
    if (!DP_IN(lk + 1, P.n_lights + 1))
        lk = -1;
    const float one_m_gamma = __fsub_rn(1.f, P.gamma);
    if (P.light_model == 2 && lk >= 0 && v == 0.f) {
        // literal Eq. 5c at the line: the zero-speed step (engine off) jumps to
        // the end of red; a departure needs green
        const float ph = phase_pos(t, tb.offset[lk], tb.cycle[lk]);
        const float wait = ph < tb.red[lk] ? __fsub_rn(tb.red[lk], ph) : 0.f;
        if (standstill_class(P, F_road, __fadd_rn(Te, Tm), b)) {
            if (Te != 0.f || !torque_allowed(P, 0.f, Te, Tm))
                return false;
            s.v1 = 0.f;
            s.xi1 = xi;
            s.dt = 0.f;
            s.wait = wait;
            s.mf = 0.f;
            s.cost = __fmul_rn(one_m_gamma, wait);
            return true;
        }
        if (wait > 0.f)
            return false;
    }
    float v1, dt;
    if (!speed_step(P, v, F_road, __fadd_rn(Te, Tm), b, nl >= 0, v1, dt))
        return false;
    float wait = 0.f;
    if (P.light_model != 2 && lk >= 0 && v == 0.f) {
        float ph = phase_pos(t, tb.offset[lk], tb.cycle[lk]);
        if (ph < tb.red[lk])
            wait = __fsub_rn(tb.red[lk], ph);
    }
    const float t1 = __fadd_rn(__fadd_rn(t, wait), dt);
    // with the sampled indicator the value function carries the light constraint
    if (P.light_model != 1 && nl >= 0 && v1 > 0.f && phase_pos(t1, tb.offset[nl], tb.cycle[nl]) < tb.red[nl])
        return false;
    const float w = __fmul_rn(v, P.ratio);
    if (!torque_allowed(P, w, Te, Tm))
        return false;
    float I;
    if (!battery_current(P, w, Tm, I))
        return false;
    const float mf = fuel_rate(P, w, Te);
    s.v1 = v1;
    s.xi1 = __fsub_rn(xi, __fdiv_rn(__fmul_rn(dt, I), P.cap));
    s.dt = dt;
    s.wait = wait;
    s.mf = mf;
    s.cost = __fadd_rn(__fmul_rn(__fadd_rn(__fmul_rn(P.gamma, mf), one_m_gamma), dt), __fmul_rn(one_m_gamma, wait));
    return true;
}

// Threads of a rollout CTA: the cluster's 8 CTAs share one stage's controls
// (~240 each at the paper-scale size), so 256 threads give every thread one
// control with the cheapest block reduction (1024 threads: 0.59 vs 0.47 ms
// per paper-scale rollout); a batched rollout's single CTA per instance takes
// every control itself and keeps 1024.
constexpr int ROLL_THREADS = 256;
constexpr int ROLL_THREADS_BATCHED = 1024;
constexpr int ROLL_CLUSTER = 8;  // CTAs (SMs) of the single-problem rollout

// A CTA's best control of a stage.
struct Cand {
    float F;
    int u;
    Step s;
};

// The rollout of one problem by a cluster of CS CTAs over stages
// [k_begin, k_end).  A later segment continues from the state, fuel, cost and
// fail stage the previous one left in `out`; the terminal cost is added by
// the segment that ends at stage N.  CTA rank 0 writes the outputs.
// Words of the stage tables a rollout stages in shared memory (grade[N],
// light_of_node[N + 1], cycle / red / offset of each light).
__host__ __device__ inline int staged_table_words(int N, int n_lights) { return 2 * N + 1 + 3 * n_lights; }

template <int CS>
__device__ void rollout_body(const DevParams *__restrict__ dP, const StageTables &tb_in, const StageView &view,
                             int k_begin, int k_end, double v0, double xi0, double t0, double *__restrict__ out,
                             int *__restrict__ out_u, bool stage_tables = false)
{
    // the stage tables in shared memory when the launch provides room: each
    // stage's model step reads them on the critical path of the walk
    extern __shared__ __align__(16) unsigned char roll_smem[];
    __shared__ DevParams P;
    __shared__ float s_v, s_xi;
    __shared__ double s_t, s_fuel, s_J;
    __shared__ float red_F[ROLL_THREADS_BATCHED / 32];
    __shared__ int red_u[ROLL_THREADS_BATCHED / 32];
    __shared__ int s_fail;
    // this CTA's candidate, double-buffered by stage parity: the cluster's
    // CTAs read it after the stage's cluster barrier, and a CTA can only
    // rewrite a buffer after the next barrier, when every CTA has read it
    __shared__ Cand s_cand[2];
    unsigned rank = 0;
    if constexpr (CS > 1)
        rank = cooperative_groups::this_cluster().block_rank();
    if (threadIdx.x == 0)
        P = *dP;
    __syncthreads();
    const int N = P.N;
    StageTables tb = tb_in;
    if (stage_tables) {
        float *sg = reinterpret_cast<float *>(roll_smem);
        int *sl = reinterpret_cast<int *>(sg + N);
        float *sc = reinterpret_cast<float *>(sl + N + 1);
        float *sr = sc + P.n_lights, *so = sr + P.n_lights;
        for (int q = threadIdx.x; q < N; q += blockDim.x)
            sg[q] = tb_in.grade[q];
        for (int q = threadIdx.x; q <= N; q += blockDim.x)
            sl[q] = tb_in.light_of_node[q];
        for (int q = threadIdx.x; q < P.n_lights; q += blockDim.x) {
            sc[q] = tb_in.cycle[q];
            sr[q] = tb_in.red[q];
            so[q] = tb_in.offset[q];
        }
        tb.grade = sg;
        tb.light_of_node = sl;
        tb.cycle = sc;
        tb.red = sr;
        tb.offset = so;
        __syncthreads();
    }
    double *traj = out;
    double *o_dt = out + 3 * (N + 1);
    double *o_wait = o_dt + N;
    double *o_fuel = o_wait + N;
    double *o_tot = o_fuel + N;
    if (threadIdx.x == 0) {
        if (k_begin == 0) {
            s_v = (float)v0;
            s_xi = (float)xi0;
            s_t = t0;
            s_fuel = 0.0;
            s_J = 0.0;
            s_fail = -1;
            traj[0] = s_v;
            traj[1] = s_xi;
            traj[2] = s_t;
        } else {
            s_v = (float)traj[3 * k_begin];
            s_xi = (float)traj[3 * k_begin + 1];
            s_t = traj[3 * k_begin + 2];
            s_fuel = o_tot[0];
            s_J = o_tot[2];
            s_fail = (int)o_tot[3];
        }
    }
    __syncthreads();
    if (s_fail >= 0)
        return;  // an earlier segment found no feasible control
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = k_begin; k < k_end; ++k) {
        const float v = s_v, xi = s_xi, t = (float)s_t;
        const float *Vn = view.at(k + 1);
        float bF = __int_as_float(0x7f800000);
        int bu = INT_MAX;
        Step bs = {};
        // CTA r of the cluster takes the controls u = r (mod CS), two per
        // thread and pass, so their loads of J_{k+1} overlap
        for (int i0 = threadIdx.x;; i0 += 2 * (int)blockDim.x) {
            const int u0 = i0 * CS + (int)rank, u1 = (i0 + (int)blockDim.x) * CS + (int)rank;
            if (u0 >= P.n_u)
                break;
            Step s0, s1;
            const bool ok0 = model_step(P, tb, k, v, xi, t, u0, s0);
            const bool ok1 = u1 < P.n_u && model_step(P, tb, k, v, xi, t, u1, s1);
            const float F0 =
                ok0 ? __fadd_rn(s0.cost, interp_cont(P, Vn, s0.v1, s0.xi1, __fadd_rn(__fadd_rn(t, s0.wait), s0.dt)))
                    : V_BIG;
            const float F1 =
                ok1 ? __fadd_rn(s1.cost, interp_cont(P, Vn, s1.v1, s1.xi1, __fadd_rn(__fadd_rn(t, s1.wait), s1.dt)))
                    : V_BIG;
            if (ok0 && F0 < V_FEAS_MAX && (F0 < bF || (F0 == bF && u0 < bu))) {
                bF = F0;
                bu = u0;
                bs = s0;
            }
            if (ok1 && F1 < V_FEAS_MAX && (F1 < bF || (F1 == bF && u1 < bu))) {
                bF = F1;
                bu = u1;
                bs = s1;
            }
        }
        const int my_u = bu;
        // block argmin on (F, u): within each warp, then every warp reduces
        // the warps' results itself, so all threads know the winner
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float oF = __shfl_down_sync(0xffffffffu, bF, off);
            const int ou = __shfl_down_sync(0xffffffffu, bu, off);
            if (oF < bF || (oF == bF && ou < bu)) {
                bF = oF;
                bu = ou;
            }
        }
        if (lane == 0) {
            red_F[warp] = bF;
            red_u[warp] = bu;
        }
        __syncthreads();
        const int n_warps = (int)(blockDim.x >> 5);
        bF = lane < n_warps ? red_F[lane] : __int_as_float(0x7f800000);
        bu = lane < n_warps ? red_u[lane] : INT_MAX;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float oF = __shfl_xor_sync(0xffffffffu, bF, off);
            const int ou = __shfl_xor_sync(0xffffffffu, bu, off);
            if (oF < bF || (oF == bF && ou < bu)) {
                bF = oF;
                bu = ou;
            }
        }
        // the CTA's winner publishes its candidate (thread 0 an empty one)
        Cand *mine = &s_cand[k & 1];
        if (bu == INT_MAX) {
            if (threadIdx.x == 0) {
                mine->F = __int_as_float(0x7f800000);
                mine->u = INT_MAX;
            }
        } else if (my_u == bu) {
            mine->F = bF;
            mine->u = bu;
            mine->s = bs;
        }
        if constexpr (CS > 1)
            cooperative_groups::this_cluster().sync();
        else
            __syncthreads();
        if (threadIdx.x == 0) {
            // the cluster's winner, lowest control index on ties
            Cand w = *mine;
            if constexpr (CS > 1) {
                cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
#pragma unroll
                for (int r = 0; r < CS; ++r) {
                    if (!DP_IN(r, (int)cl.num_blocks()))
                        break;
                    const Cand c = *cl.map_shared_rank(mine, (unsigned)r);
                    if (c.F < w.F || (c.F == w.F && c.u < w.u))
                        w = c;
                }
            }
            if (w.u == INT_MAX) {
                s_fail = k;
            } else {
                const Step s = w.s;
                const double fk = (double)s.mf * (double)s.dt;
                s_fuel += fk;
                s_J += (double)s.cost;
                s_t += (double)s.wait + (double)s.dt;
                s_v = s.v1;
                s_xi = s.xi1;
                if (rank == 0 && DP_IN(k, N)) {
                    out_u[k] = w.u;
                    o_dt[k] = s.dt;
                    o_wait[k] = s.wait;
                    o_fuel[k] = fk;
                    traj[3 * (k + 1) + 0] = s.v1;
                    traj[3 * (k + 1) + 1] = s.xi1;
                    traj[3 * (k + 1) + 2] = s_t;
                }
            }
        }
        __syncthreads();
        if (s_fail >= 0)
            break;
    }
    if (threadIdx.x == 0 && rank == 0) {
        o_tot[0] = s_fuel;
        o_tot[1] = s_t - traj[2];
        o_tot[3] = (double)s_fail;
        if (s_fail >= 0)
            o_tot[2] = __longlong_as_double(0x7ff0000000000000LL);
        else
            o_tot[2] = k_end == N ? s_J + (double)terminal_cost(P, s_v, s_xi) : s_J;
    }
    // no CTA leaves while another may still read its candidates
    if constexpr (CS > 1)
        cooperative_groups::this_cluster().sync();
}

__global__ void __cluster_dims__(ROLL_CLUSTER, 1, 1) __launch_bounds__(ROLL_THREADS)
    rollout_kernel(const DevParams *__restrict__ dP, StageTables tb, StageView view, int k_begin, int k_end,
                   double v0, double xi0, double t0, double *__restrict__ out, int *__restrict__ out_u,
                   bool stage_tables)
{
    rollout_body<ROLL_CLUSTER>(dP, tb, view, k_begin, k_end, v0, xi0, t0, out, out_u, stage_tables);
}

// Batched: one CTA per instance; instance b writes its output block at
// out + out_off[b] (doubles) and out_u + u_off[b].
__global__ void __launch_bounds__(ROLL_THREADS_BATCHED)
    rollout_batched_kernel(const DevParams *__restrict__ params, const BatchInst *__restrict__ inst,
                           const double *__restrict__ x0, const long long *__restrict__ out_off,
                           const long long *__restrict__ u_off, double *__restrict__ out, int *__restrict__ out_u)
{
    const int b = blockIdx.x;
    const BatchInst &I = inst[b];
    const StageView view = StageView::all(I.V, I.stage_elems);
    rollout_body<1>(params + b, I.tb, view, 0, I.N, x0[3 * b], x0[3 * b + 1], x0[3 * b + 2], out + out_off[b],
                 out_u + u_off[b]);
}

}  // namespace

cudaError_t launch_rollout(const DevParams *dP, const DevParams &hP, StageTables tb, const StageView &view,
                           int k_begin, int k_end, double v0, double xi0, double t0, double *out, int *out_u,
                           cudaStream_t s)
{
    // stage the tables when they fit in the default 48 KB of shared memory
    const size_t bytes = (size_t)staged_table_words(hP.N, hP.n_lights) * 4;
    const bool stage = bytes <= 32 * 1024;
    rollout_kernel<<<ROLL_CLUSTER, ROLL_THREADS, stage ? bytes : 0, s>>>(dP, tb, view, k_begin, k_end, v0, xi0, t0,
                                                                         out, out_u, stage);
    return cudaGetLastError();
}

cudaError_t launch_rollout_batched(const DevParams *params, const BatchInst *inst, int n_inst, const double *x0,
                                   const long long *out_off, const long long *u_off, double *out, int *out_u,
                                   cudaStream_t s)
{
    rollout_batched_kernel<<<n_inst, ROLL_THREADS_BATCHED, 0, s>>>(params, inst, x0, out_off, u_off, out, out_u);
    return cudaGetLastError();
}

}  // namespace ecodp
