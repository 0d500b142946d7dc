// Bellman stage kernels: J_k(v_i, xi_j, t_l) = min_u [c + J_{k+1}(f(x, u))]
// and the argmin pi_k (Eq. 9b-9d), on the per-stage tables of the precompute
// kernel.
//
// For control u in torque class C (same T_eng + T_bsg and brake flag) the
// successor is (v'_C, xi_j - dxi_u, t_l + dt_C): the speed and time axes of
// the trilinear interpolation are shared by the whole class and only the SoC
// axis depends on u (Eq. 5a-5c).  With uniform grids the SoC shift is the
// same for every j and the time shift the same for every l, so
//   J_{k+1}(f(x, u)) = w0_u G_C(j + d_u) + w1_u G_C(j + d_u + 1)
// where G_C(j') blends the two speed rows and two time columns of J_{k+1} at
// SoC row j'.  The class-level part G_C is computed once per class and
// thread; the per-control work is two FMAs and one min.
//
// Exceptions to the shared time shift: at a light stage the arrival check
// (Eq. 5c, 7c, 8) depends on the arrival time t_l + dt_C (per thread and
// class), and on the standstill row v = 0 at a light node the departure
// waits for green, which shifts the time landing per l.
//
// Two variants compute bit-identical results:
//   * bellman_direct: one thread per state, every control evaluated with its
//     own G reads (reference layout of the paper's second kernel, Sec. IV);
//   * bellman_tiled: one thread per (RJ SoC rows, one time node); per class a
//     register window of RJ + 4 blended values G, the controls of the class
//     grouped by SoC shift d in {-2, -1, 0, 1} so the window offsets are
//     compile-time constants; the class tables of the speed row staged in
//     shared memory.  It tracks only the minimum value per class; the argmin
//     is recovered after the sweep by re-evaluating the winning class, whose
//     values are reproduced bit for bit.
#include <cfloat>
#include <climits>

#include "ecodp_internal.cuh"

namespace ecodp {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// Per-thread interpolation context of one class.
struct TCtx {
    const float *r0, *r1;  // speed rows iv, iv+1 of J_{k+1}, at padded SoC row 0
    int ta, tb;            // time columns (clamped to the padding column n_t)
    float wv0, wv1, wt0, wt1;
    bool red;              // arrival during red: every value of the class is infeasible
};

struct StageInfo {
    bool wait_row;   // v_i == 0 at a light node: wait for green before departing
    int next_light;  // light index at node k+1, or -1
    float cyc1, red1, off1;
};

__device__ __forceinline__ TCtx class_ctx(const DevParams &P, const float *__restrict__ Vn, const ClassRec &C, int l,
                                          float tl, float wait, const StageInfo &si)
{
    TCtx x;
    int t0;
    float ft;
    if (!si.wait_row) {
        t0 = l + C.st;
        ft = C.ft;
    } else {
        int st;
        snap_split(__fdiv_rn(__fadd_rn(wait, C.dt), P.h_t), st, ft);
        t0 = l + st;
    }
    x.ta = min(t0, P.n_t);
    x.tb = min(t0 + 1, P.n_t);
    x.wt1 = ft;
    x.wt0 = __fsub_rn(1.f, ft);
    x.wv1 = C.fv;
    x.wv0 = __fsub_rn(1.f, C.fv);
    const size_t vrow = (size_t)P.xi_rows * P.ld_t;
    x.r0 = Vn + (size_t)C.iv * vrow;
    x.r1 = x.r0 + vrow;
    x.red = false;
    if (si.next_light >= 0 && C.v1 > 0.f) {
        float tarr = __fadd_rn(__fadd_rn(tl, wait), C.dt);
        x.red = phase_pos(tarr, si.off1, si.cyc1) < si.red1;
    }
    return x;
}

// Blended value G at SoC row j (any integer; rows outside the grid read padding).
__device__ __forceinline__ float g_at(const DevParams &P, const TCtx &x, int j)
{
    if (x.red)
        return V_BIG;
    int jp = min(max(j, -1), P.n_xi) + 1;
    size_t o = (size_t)jp * P.ld_t;
    return g_blend(x.r0 + o, x.r1 + o, x.ta, x.tb, x.wv0, x.wv1, x.wt0, x.wt1);
}

__device__ __forceinline__ float split_value(const float4 &S, float g0, float g1)
{
    return __fmaf_rn(S.z, g1, __fmaf_rn(S.y, g0, S.x));
}

__device__ __forceinline__ int split_u(const float4 &S) { return (int)(__float_as_uint(S.w) & 0xffffu); }
__device__ __forceinline__ int split_d(const float4 &S) { return (int)(short)(__float_as_uint(S.w) >> 16); }

__device__ __forceinline__ StageInfo stage_info(const DevParams &P, const StageTables &tb, int k, float v)
{
    StageInfo si;
    int lk = tb.light_of_node[k];
    si.wait_row = (lk >= 0) && (v == 0.f);
    si.next_light = tb.light_of_node[k + 1];
    si.cyc1 = si.red1 = si.off1 = 0.f;
    if (si.next_light >= 0) {
        si.cyc1 = tb.cycle[si.next_light];
        si.red1 = tb.red[si.next_light];
        si.off1 = tb.offset[si.next_light];
    }
    return si;
}

// Standstill time at a red light before departing from (v = 0, t) at node k.
__device__ __forceinline__ float wait_time(const StageTables &tb, int k, float tl, bool wait_row)
{
    if (!wait_row)
        return 0.f;
    int lk = tb.light_of_node[k];
    float ph = phase_pos(tl, tb.offset[lk], tb.cycle[lk]);
    float r = tb.red[lk];
    return ph < r ? __fsub_rn(r, ph) : 0.f;
}

// ---------------------------------------------------------------------------
// direct variant: one thread per state

__global__ void __launch_bounds__(256) bellman_direct(const DevParams *__restrict__ dP, StageTables tb, int k,
                                                      StageScratch sc, const float *__restrict__ Vn,
                                                      float *__restrict__ Vk, int16_t *__restrict__ pik)
{
    __shared__ DevParams P;
    if (threadIdx.x == 0)
        P = *dP;
    __syncthreads();
    const int i = blockIdx.y;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= P.n_xi * P.n_t)
        return;
    const int j = s / P.n_t, l = s % P.n_t;
    const float v = node_val(P.v_lo, P.v_span, i, P.n_v);
    const float tl = node_val(P.t_lo, P.t_span, l, P.n_t);
    const StageInfo si = stage_info(P, tb, k, v);
    const float wait = wait_time(tb, k, tl, si.wait_row);
    const int n_ent = sc.row_cnt[2 * i];
    const ClassRec *cls = sc.cls + (size_t)i * P.n_cls;
    const ClassEntry *ent = sc.ent + (size_t)i * P.n_cls;
    const float4 *spl = sc.spl + (size_t)i * P.n_u;

    float best = __int_as_float(0x7f800000);
    int bu = INT_MAX;
    for (int e = 0; e < n_ent; ++e) {
        const ClassEntry E = ent[e];
        const TCtx x = class_ctx(P, Vn, cls[E.cls], l, tl, wait, si);
        for (int q = E.off; q < E.off + E.n_total; ++q) {
            const float4 S = spl[q];
            const int d = split_d(S), u = split_u(S);
            const float F = split_value(S, g_at(P, x, j + d), g_at(P, x, j + d + 1));
            if (F < best || (F == best && u < bu)) {
                best = F;
                bu = u;
            }
        }
    }
    const size_t o = ((size_t)i * P.xi_rows + (j + 1)) * P.ld_t + l;
    const size_t op = ((size_t)i * P.n_xi + j) * P.n_t + l;
    if (!(best < V_FEAS_MAX)) {
        Vk[o] = V_BIG;
        pik[op] = -1;
    } else {
        Vk[o] = __fadd_rn(best, __fmul_rn(__fsub_rn(1.f, P.gamma), wait));
        pik[op] = (int16_t)bu;
    }
}

// ---------------------------------------------------------------------------
// tiled variant

struct RowSmem {
    const ClassRec *cls;
    const ClassEntry *ent;
    const float4 *spl;
};

// Minimum over the controls of class E for the thread's RJ rows.
__device__ __forceinline__ void class_min(const DevParams &P, const TCtx &x, const ClassEntry &E,
                                          const float4 *__restrict__ spl, int jb, float (&cm)[RJ])
{
    float G[RJ + 4];
#pragma unroll
    for (int w = 0; w < RJ + 4; ++w)
        G[w] = g_at(P, x, jb - 2 + w);
#pragma unroll
    for (int r = 0; r < RJ; ++r)
        cm[r] = __int_as_float(0x7f800000);
    int q = E.off;
#define ECODP_BUCKET(NB, D)                                                                   \
    for (int n = 0; n < (NB); ++n, ++q) {                                                    \
        const float4 S = spl[q];                                                             \
        _Pragma("unroll") for (int r = 0; r < RJ; ++r) cm[r] =                                \
            fminf(cm[r], split_value(S, G[r + (D) + 2], G[r + (D) + 3]));                      \
    }
    ECODP_BUCKET(E.nb[0], -2)
    ECODP_BUCKET(E.nb[1], -1)
    ECODP_BUCKET(E.nb[2], 0)
    ECODP_BUCKET(E.nb[3], 1)
#undef ECODP_BUCKET
    for (int n = 0; n < E.n_other; ++n, ++q) {
        const float4 S = spl[q];
        const int d = split_d(S);
#pragma unroll
        for (int r = 0; r < RJ; ++r)
            cm[r] = fminf(cm[r], split_value(S, g_at(P, x, jb + r + d), g_at(P, x, jb + r + d + 1)));
    }
}

// Lowest control index of class E whose value equals best[r], for rows in mask.
__device__ __forceinline__ void class_find(const DevParams &P, const TCtx &x, const ClassEntry &E,
                                           const float4 *__restrict__ spl, int jb, unsigned rows,
                                           const float (&best)[RJ], int (&ub)[RJ])
{
    for (int q = E.off; q < E.off + E.n_total; ++q) {
        const float4 S = spl[q];
        const int d = split_d(S), u = split_u(S);
#pragma unroll
        for (int r = 0; r < RJ; ++r) {
            if ((rows >> r) & 1u) {
                const float F = split_value(S, g_at(P, x, jb + r + d), g_at(P, x, jb + r + d + 1));
                if (F == best[r] && u < ub[r])
                    ub[r] = u;
            }
        }
    }
}

template <bool SMEM_SPLITS>
__global__ void __launch_bounds__(256) bellman_tiled(const DevParams *__restrict__ dP, StageTables tb, int k,
                                                     StageScratch sc, const float *__restrict__ Vn,
                                                     float *__restrict__ Vk, int16_t *__restrict__ pik)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ DevParams P;
    if (threadIdx.x == 0 && threadIdx.y == 0)
        P = *dP;
    __syncthreads();

    const int i = blockIdx.y;
    const int n_ent = sc.row_cnt[2 * i];
    const int n_spl = sc.row_cnt[2 * i + 1];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;

    // stage the row's tables: ClassRec[n_cls], ClassEntry[n_ent], float4[n_spl]
    ClassRec *s_cls = reinterpret_cast<ClassRec *>(smem_raw);
    ClassEntry *s_ent = reinterpret_cast<ClassEntry *>(s_cls + P.n_cls);
    float4 *s_spl = reinterpret_cast<float4 *>(s_ent + n_ent);
    {
        const int4 *src = reinterpret_cast<const int4 *>(sc.cls + (size_t)i * P.n_cls);
        int4 *dst = reinterpret_cast<int4 *>(s_cls);
        for (int q = tid; q < P.n_cls * 2; q += nthr)
            dst[q] = src[q];
        const int4 *src2 = reinterpret_cast<const int4 *>(sc.ent + (size_t)i * P.n_cls);
        int4 *dst2 = reinterpret_cast<int4 *>(s_ent);
        for (int q = tid; q < n_ent * 2; q += nthr)
            dst2[q] = src2[q];
        if (SMEM_SPLITS) {
            const float4 *src3 = sc.spl + (size_t)i * P.n_u;
            for (int q = tid; q < n_spl; q += nthr)
                s_spl[q] = src3[q];
        }
    }
    __syncthreads();
    const float4 *spl = SMEM_SPLITS ? s_spl : sc.spl + (size_t)i * P.n_u;

    const float v = node_val(P.v_lo, P.v_span, i, P.n_v);
    const StageInfo si = stage_info(P, tb, k, v);
    const int jb = (blockIdx.x * blockDim.y + threadIdx.y) * RJ;
    const float one_m_gamma = __fsub_rn(1.f, P.gamma);

    for (int l0 = 0; l0 < P.n_t; l0 += blockDim.x) {
        const int l_raw = l0 + threadIdx.x;
        const bool l_ok = l_raw < P.n_t;
        const int l = l_ok ? l_raw : P.n_t - 1;
        const float tl = node_val(P.t_lo, P.t_span, l, P.n_t);
        const float wait = wait_time(tb, k, tl, si.wait_row);

        float best[RJ];
        int bcls[RJ];
        unsigned tie = 0;
#pragma unroll
        for (int r = 0; r < RJ; ++r) {
            best[r] = __int_as_float(0x7f800000);
            bcls[r] = -1;
        }
        for (int e = 0; e < n_ent; ++e) {
            const ClassEntry E = s_ent[e];
            const TCtx x = class_ctx(P, Vn, s_cls[E.cls], l, tl, wait, si);
            float cm[RJ];
            class_min(P, x, E, spl, jb, cm);
#pragma unroll
            for (int r = 0; r < RJ; ++r) {
                if (cm[r] < best[r]) {
                    best[r] = cm[r];
                    bcls[r] = e;
                } else if (cm[r] == best[r] && cm[r] < V_FEAS_MAX) {
                    tie |= 1u << r;
                }
            }
        }

        // argmin recovery: lowest control index reproducing the minimum
        unsigned todo = 0;
#pragma unroll
        for (int r = 0; r < RJ; ++r)
            if (l_ok && jb + r < P.n_xi && best[r] < V_FEAS_MAX)
                todo |= 1u << r;
        tie &= todo;
        int ub[RJ];
#pragma unroll
        for (int r = 0; r < RJ; ++r)
            ub[r] = INT_MAX;
        if (__any_sync(FULL, tie != 0u)) {
            for (int e = 0; e < n_ent; ++e) {
                unsigned rows = 0;
#pragma unroll
                for (int r = 0; r < RJ; ++r)
                    if (((todo >> r) & 1u) && (((tie >> r) & 1u) || bcls[r] == e))
                        rows |= 1u << r;
                if (__any_sync(FULL, rows != 0u)) {
                    const ClassEntry E = s_ent[e];
                    const TCtx x = class_ctx(P, Vn, s_cls[E.cls], l, tl, wait, si);
                    class_find(P, x, E, spl, jb, rows, best, ub);
                }
            }
        } else {
            unsigned left = todo;
            while (__any_sync(FULL, left != 0u)) {
                int mine = INT_MAX;
#pragma unroll
                for (int r = 0; r < RJ; ++r)
                    if ((left >> r) & 1u)
                        mine = min(mine, bcls[r]);
                const int e = __reduce_min_sync(FULL, mine);
                unsigned rows = 0;
#pragma unroll
                for (int r = 0; r < RJ; ++r)
                    if (((left >> r) & 1u) && bcls[r] == e)
                        rows |= 1u << r;
                const ClassEntry E = s_ent[e];
                const TCtx x = class_ctx(P, Vn, s_cls[E.cls], l, tl, wait, si);
                class_find(P, x, E, spl, jb, rows, best, ub);
                left &= ~rows;
            }
        }

        if (l_ok) {
#pragma unroll
            for (int r = 0; r < RJ; ++r) {
                const int j = jb + r;
                if (j >= P.n_xi)
                    continue;
                const size_t o = ((size_t)i * P.xi_rows + (j + 1)) * P.ld_t + l;
                const size_t op = ((size_t)i * P.n_xi + j) * P.n_t + l;
                if ((todo >> r) & 1u) {
                    Vk[o] = __fadd_rn(best[r], __fmul_rn(one_m_gamma, wait));
                    pik[op] = (int16_t)ub[r];
                } else {
                    Vk[o] = V_BIG;
                    pik[op] = -1;
                }
            }
        }
    }
}

}  // namespace

size_t bellman_smem_bytes(const DevParams &hP, bool smem_splits)
{
    size_t b = (size_t)hP.n_cls * (sizeof(ClassRec) + sizeof(ClassEntry));
    if (smem_splits)
        b += (size_t)hP.n_u * sizeof(float4);
    return b;
}

cudaError_t launch_bellman(const DevParams *dP, const DevParams &hP, StageTables tb, int k, StageScratch sc,
                           const float *Vnext, float *Vk, int16_t *pik, int variant, cudaStream_t s)
{
    if (variant == 0) {
        dim3 grid((hP.n_xi * hP.n_t + 255) / 256, hP.n_v);
        bellman_direct<<<grid, 256, 0, s>>>(dP, tb, k, sc, Vnext, Vk, pik);
        return cudaGetLastError();
    }
    const int tx = min(256, round_up(hP.n_t, 32));
    const int ty = tx <= 128 ? 2 : 1;
    const int n_groups = (hP.n_xi + RJ - 1) / RJ;
    dim3 block(tx, ty);
    dim3 grid((n_groups + ty - 1) / ty, hP.n_v);
    const bool smem_splits = bellman_smem_bytes(hP, true) <= 160 * 1024;
    const size_t smem = bellman_smem_bytes(hP, smem_splits);
    cudaError_t err;
    if (smem_splits) {
        err = cudaFuncSetAttribute(bellman_tiled<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess)
            return err;
        bellman_tiled<true><<<grid, block, smem, s>>>(dP, tb, k, sc, Vnext, Vk, pik);
    } else {
        err = cudaFuncSetAttribute(bellman_tiled<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess)
            return err;
        bellman_tiled<false><<<grid, block, smem, s>>>(dP, tb, k, sc, Vnext, Vk, pik);
    }
    return cudaGetLastError();
}

}  // namespace ecodp
