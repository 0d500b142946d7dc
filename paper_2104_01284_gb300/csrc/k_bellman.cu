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
//     own G reads (the layout of the paper's second kernel, Sec. IV);
//   * bellman_tiled: one CTA per (speed row, 128 lanes); each lane owns one
//     (SoC group of RJ rows, time node) pair, the pairs of a row laid out back
//     to back so no lane idles on a ragged time axis.  The row's class and
//     control tables are staged in shared memory.  Per class a lane holds a
//     register window of RJ + 4 blended values G; the controls of the class
//     are grouped by SoC shift d in {-2, -1, 0, 1} so window offsets are
//     compile-time constants; two rows go through one packed FP32 FMA
//     (__ffma2_rn) and two controls through one three-input min.  Only the
//     per-class minimum is kept in the sweep; afterwards each warp buckets
//     its states by winning class in shared memory and re-evaluates each
//     state's winning class (bit for bit the same arithmetic) to recover the
//     lowest control index that reaches the minimum.
//
// Argmin order: (value, torque class, control index).  Among controls with
// exactly equal FP32 values the first class in class order (total torque
// ascending, brake flag fastest) wins, then the lowest control index inside
// it.  Exact FP32 ties are rounding coincidences of near-equal costs (the
// FP64 recursion has none on the seeded instances); resolving them toward the
// lowest global control index would re-evaluate every tied class.
#include <cfloat>
#include <climits>

#include "ecodp_internal.cuh"

namespace ecodp {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int TW = 4;  // warps per CTA of the tiled kernel
constexpr int TLANES = TW * 32;

// Per-lane interpolation context of one class.
struct TCtx {
    const float *p0, *p1;  // speed rows iv, iv+1 of J_{k+1} at padded SoC row 0, lower time column
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
    // a lower corner past the grid reads the padding column n_t; the upper
    // corner is the next column, still inside the row (ld_t >= n_t + 2)
    const int ta = min(t0, P.n_t);
    x.wt1 = ft;
    x.wt0 = __fsub_rn(1.f, ft);
    x.wv1 = C.fv;
    x.wv0 = __fsub_rn(1.f, C.fv);
    const size_t vrow = (size_t)P.xi_rows * P.ld_t;
    x.p0 = Vn + (size_t)C.iv * vrow + ta;
    x.p1 = x.p0 + vrow;
    x.red = false;
    if (si.next_light >= 0 && C.v1 > 0.f) {
        float tarr = __fadd_rn(__fadd_rn(tl, wait), C.dt);
        x.red = phase_pos(tarr, si.off1, si.cyc1) < si.red1;
    }
    return x;
}

__device__ __forceinline__ int row_offset(const DevParams &P, int j)
{
    return (min(max(j, -1), P.n_xi) + 1) * P.ld_t;
}

// Blended value G at SoC row j (any integer; rows outside the grid read padding).
__device__ __forceinline__ float g_at(const DevParams &P, const TCtx &x, int j)
{
    const int o = row_offset(P, j);
    const float g = g_blend2(x.p0 + o, x.p1 + o, x.wv0, x.wv1, x.wt0, x.wt1);
    return x.red ? V_BIG : g;
}

// c + w0 g0 + w1 g1, in this order (the packed path rounds identically).
__device__ __forceinline__ float split_value(const SplitRec &S, float g0, float g1)
{
    return __fmaf_rn(S.w1, g1, __fmaf_rn(S.w0, g0, S.c));
}

__device__ __forceinline__ int split_u(const SplitRec &S) { return (int)(S.bits & 0xffffu); }
__device__ __forceinline__ int split_d(const SplitRec &S) { return (int)(short)(S.bits >> 16); }

__device__ __forceinline__ float min3(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ StageInfo stage_info(const StageTables &tb, int k, float v)
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
    const StageInfo si = stage_info(tb, k, v);
    const float wait = wait_time(tb, k, tl, si.wait_row);
    const size_t row = (size_t)k * P.n_v + i;
    const int n_ent = sc.row_cnt[2 * row];
    const ClassRec *cls = sc.cls + row * P.n_cls;
    const ClassEntry *ent = sc.ent + row * P.n_cls;
    const SplitRec *spl = sc.spl + row * P.n_u;

    // minimum in the order (value, class, control index)
    float best = __int_as_float(0x7f800000);
    int bu = INT_MAX, be = -1;
    for (int e = 0; e < n_ent; ++e) {
        const ClassEntry E = ent[e];
        const TCtx x = class_ctx(P, Vn, cls[E.cls], l, tl, wait, si);
        for (int q = E.off; q < E.off + E.n_total; ++q) {
            const SplitRec S = spl[q];
            const int d = split_d(S), u = split_u(S);
            const float F = split_value(S, g_at(P, x, j + d), g_at(P, x, j + d + 1));
            if (F < best || (F == best && e == be && u < bu)) {
                best = F;
                bu = u;
                be = e;
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

// Minimum over the controls of one SoC-shift bucket: row r uses window values
// G[r + D + 2] and G[r + D + 3].  EV holds the even-aligned pairs
// {G[2p], G[2p+1]}, OD the odd-aligned pairs {G[2p+1], G[2p+2]}.
template <int D>
__device__ __forceinline__ void bucket_min(const SplitRec *__restrict__ spl, int q, int n,
                                           const float2 (&EV)[RJ / 2 + 2], const float2 (&OD)[RJ / 2 + 1],
                                           float (&cm)[RJ])
{
    const int end = q + n;
    for (; q + 1 < end; q += 2) {
        const SplitRec s1 = spl[q], s2 = spl[q + 1];
        const float2 c1 = make_float2(s1.c, s1.c), w01 = make_float2(s1.w0, s1.w0), w11 = make_float2(s1.w1, s1.w1);
        const float2 c2 = make_float2(s2.c, s2.c), w02 = make_float2(s2.w0, s2.w0), w12 = make_float2(s2.w1, s2.w1);
#pragma unroll
        for (int p = 0; p < RJ / 2; ++p) {
            const float2 LO = ((D & 1) == 0) ? EV[p + (D + 2) / 2] : OD[p + (D + 1) / 2];
            const float2 HI = ((D & 1) == 0) ? OD[p + (D + 2) / 2] : EV[p + (D + 3) / 2];
            const float2 F1 = __ffma2_rn(w11, HI, __ffma2_rn(w01, LO, c1));
            const float2 F2 = __ffma2_rn(w12, HI, __ffma2_rn(w02, LO, c2));
            cm[2 * p] = min3(cm[2 * p], F1.x, F2.x);
            cm[2 * p + 1] = min3(cm[2 * p + 1], F1.y, F2.y);
        }
    }
    if (q < end) {
        const SplitRec s1 = spl[q];
        const float2 c1 = make_float2(s1.c, s1.c), w01 = make_float2(s1.w0, s1.w0), w11 = make_float2(s1.w1, s1.w1);
#pragma unroll
        for (int p = 0; p < RJ / 2; ++p) {
            const float2 LO = ((D & 1) == 0) ? EV[p + (D + 2) / 2] : OD[p + (D + 1) / 2];
            const float2 HI = ((D & 1) == 0) ? OD[p + (D + 2) / 2] : EV[p + (D + 3) / 2];
            const float2 F1 = __ffma2_rn(w11, HI, __ffma2_rn(w01, LO, c1));
            cm[2 * p] = fminf(cm[2 * p], F1.x);
            cm[2 * p + 1] = fminf(cm[2 * p + 1], F1.y);
        }
    }
}

// Lowest control index of class E whose value at SoC row j equals bv (INT_MAX
// if none), re-evaluated with exactly the arithmetic of the sweep.
__device__ __forceinline__ int class_lowest_u(const DevParams &P, const TCtx &x, const ClassEntry &E,
                                              const SplitRec *__restrict__ spl, int j, float bv)
{
    float g5[5];  // SoC rows j - 2 .. j + 2
#pragma unroll
    for (int w = 0; w < 5; ++w)
        g5[w] = g_at(P, x, j - 2 + w);
    int ub = INT_MAX;
    int q = E.off;
#pragma unroll
    for (int b = 0; b < 4; ++b) {  // bucket b holds the shift d = b - 2
        for (int n = 0; n < E.nb[b]; ++n, ++q) {
            const SplitRec S = spl[q];
            const int u = split_u(S);
            if (split_value(S, g5[b], g5[b + 1]) == bv && u < ub)
                ub = u;
        }
    }
    for (int n = 0; n < E.n_other; ++n, ++q) {
        const SplitRec S = spl[q];
        const int d = split_d(S), u = split_u(S);
        if (split_value(S, g_at(P, x, j + d), g_at(P, x, j + d + 1)) == bv && u < ub)
            ub = u;
    }
    return ub;
}

constexpr int WSTATES = 32 * RJ;  // states of one warp

// Shared memory of the tiled kernel: the row's tables, then per warp the
// argmin-recovery buffers: counters [n_cls + 1], entry list [WSTATES], best
// value per state [WSTATES].
struct TiledLayout {
    size_t ent, spl, warp, warp_bytes, total;
    size_t w_list, w_best;  // offsets inside a warp's block
};

__host__ __device__ inline TiledLayout tiled_layout(int n_cls, int n_u)
{
    TiledLayout L;
    size_t o = (size_t)n_cls * sizeof(ClassRec);
    L.ent = o;
    o += (size_t)n_cls * sizeof(ClassEntry);
    L.spl = o;
    o += (size_t)n_u * sizeof(SplitRec);
    L.warp = o;
    size_t w = ((size_t)(n_cls + 1) * sizeof(int) + 15) / 16 * 16;
    L.w_list = w;
    w += (size_t)WSTATES * sizeof(unsigned);
    L.w_best = w;
    w += (size_t)WSTATES * sizeof(float);
    L.warp_bytes = w;
    L.total = o + TW * L.warp_bytes;
    return L;
}

__global__ void __launch_bounds__(TLANES, 4) bellman_tiled(const DevParams *__restrict__ dP, StageTables tb, int k,
                                                          StageScratch sc, const float *__restrict__ Vn,
                                                          float *__restrict__ Vk, int16_t *__restrict__ pik)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ DevParams P;
    const int tid = threadIdx.x;
    if (tid == 0)
        P = *dP;
    __syncthreads();

    const int i = blockIdx.y;
    const size_t row = (size_t)k * P.n_v + i;
    const int n_ent = sc.row_cnt[2 * row];
    const int n_spl = sc.row_cnt[2 * row + 1];
    const TiledLayout L = tiled_layout(P.n_cls, P.n_u);
    ClassRec *s_cls = reinterpret_cast<ClassRec *>(smem_raw);
    ClassEntry *s_ent = reinterpret_cast<ClassEntry *>(smem_raw + L.ent);
    SplitRec *s_spl = reinterpret_cast<SplitRec *>(smem_raw + L.spl);
    {
        const int4 *src = reinterpret_cast<const int4 *>(sc.cls + row * P.n_cls);
        int4 *dst = reinterpret_cast<int4 *>(s_cls);
        for (int q = tid; q < P.n_cls * 2; q += TLANES)
            dst[q] = src[q];
        const int4 *src2 = reinterpret_cast<const int4 *>(sc.ent + row * P.n_cls);
        int4 *dst2 = reinterpret_cast<int4 *>(s_ent);
        for (int q = tid; q < n_ent * 2; q += TLANES)
            dst2[q] = src2[q];
        const int4 *src3 = reinterpret_cast<const int4 *>(sc.spl + row * P.n_u);
        int4 *dst3 = reinterpret_cast<int4 *>(s_spl);
        for (int q = tid; q < n_spl; q += TLANES)
            dst3[q] = src3[q];
    }
    const int warp = tid >> 5, lane = tid & 31;
    unsigned char *wbase = smem_raw + L.warp + warp * L.warp_bytes;
    int *w_cnt = reinterpret_cast<int *>(wbase);
    unsigned *w_list = reinterpret_cast<unsigned *>(wbase + L.w_list);
    float *w_best = reinterpret_cast<float *>(wbase + L.w_best);
    __syncthreads();

    const int n_jg = (P.n_xi + RJ - 1) / RJ;
    const int n_flat = n_jg * P.n_t;
    const int chunk0 = blockIdx.x * TLANES + warp * 32;  // first flat index of this warp
    const int f_raw = chunk0 + lane;
    const bool f_ok = f_raw < n_flat;
    const int f = f_ok ? f_raw : n_flat - 1;
    const int jg = f / P.n_t;
    const int l = f - jg * P.n_t;
    const int jb = jg * RJ;
    const float one_m_gamma = __fsub_rn(1.f, P.gamma);
    const float v = node_val(P.v_lo, P.v_span, i, P.n_v);
    const StageInfo si = stage_info(tb, k, v);
    const float tl = node_val(P.t_lo, P.t_span, l, P.n_t);
    const float wait = wait_time(tb, k, tl, si.wait_row);

    int roff[RJ + 4];
#pragma unroll
    for (int w = 0; w < RJ + 4; ++w)
        roff[w] = row_offset(P, jb - 2 + w);

    // per row: the running minimum and the first class (in class order)
    // reaching it; `tie` marks rows whose minimum a later class matches
    // exactly (counted only: the order (value, class, control) decides)
    float best[RJ];
    int bcls[RJ];
    unsigned tie = 0;
#pragma unroll
    for (int r = 0; r < RJ; ++r) {
        best[r] = __int_as_float(0x7f800000);
        bcls[r] = 0;
    }
    for (int e = 0; e < n_ent; ++e) {
        const ClassEntry E = s_ent[e];
        const TCtx x = class_ctx(P, Vn, s_cls[E.cls], l, tl, wait, si);
        float G[RJ + 4];
#pragma unroll
        for (int w = 0; w < RJ + 4; ++w) {
            const float g = g_blend2(x.p0 + roff[w], x.p1 + roff[w], x.wv0, x.wv1, x.wt0, x.wt1);
            G[w] = x.red ? V_BIG : g;
        }
        float2 EV[RJ / 2 + 2], OD[RJ / 2 + 1];
#pragma unroll
        for (int p = 0; p < RJ / 2 + 2; ++p)
            EV[p] = make_float2(G[2 * p], G[2 * p + 1]);
#pragma unroll
        for (int p = 0; p < RJ / 2 + 1; ++p)
            OD[p] = make_float2(G[2 * p + 1], G[2 * p + 2]);
        float cm[RJ];
#pragma unroll
        for (int r = 0; r < RJ; ++r)
            cm[r] = __int_as_float(0x7f800000);
        int q = E.off;
        bucket_min<-2>(s_spl, q, E.nb[0], EV, OD, cm);
        q += E.nb[0];
        bucket_min<-1>(s_spl, q, E.nb[1], EV, OD, cm);
        q += E.nb[1];
        bucket_min<0>(s_spl, q, E.nb[2], EV, OD, cm);
        q += E.nb[2];
        bucket_min<1>(s_spl, q, E.nb[3], EV, OD, cm);
        q += E.nb[3];
        for (int n = 0; n < E.n_other; ++n, ++q) {
            const SplitRec S = s_spl[q];
            const int d = split_d(S);
#pragma unroll
            for (int r = 0; r < RJ; ++r)
                cm[r] = fminf(cm[r], split_value(S, g_at(P, x, jb + r + d), g_at(P, x, jb + r + d + 1)));
        }
#pragma unroll
        for (int r = 0; r < RJ; ++r) {
            if (cm[r] < best[r]) {
                best[r] = cm[r];
                bcls[r] = e;
                tie &= ~(1u << r);
            } else if (cm[r] == best[r]) {
                tie |= 1u << r;
            }
        }
    }

    // values now; argmin recovery below
    unsigned todo = 0;
#pragma unroll
    for (int r = 0; r < RJ; ++r) {
        const int j = jb + r;
        const bool valid = f_ok && j < P.n_xi;
        const bool feas = valid && best[r] < V_FEAS_MAX;
        if (feas)
            todo |= 1u << r;
        if (valid) {
            Vk[((size_t)i * P.xi_rows + (j + 1)) * P.ld_t + l] =
                feas ? __fadd_rn(best[r], __fmul_rn(one_m_gamma, wait)) : V_BIG;
            if (!feas)
                pik[((size_t)i * P.n_xi + j) * P.n_t + l] = -1;
        }
    }
    tie &= todo;
    if (sc.stats) {
        const unsigned n_tie = __reduce_add_sync(FULL, (unsigned)__popc(tie));
        const unsigned n_find = __reduce_add_sync(FULL, (unsigned)__popc(todo));
        if (lane == 0) {
            atomicAdd(sc.stats + 2, (unsigned long long)n_tie);
            atomicAdd(sc.stats + 3, (unsigned long long)n_find);
        }
    }

    // bucket the feasible states by their first winning class and recover the
    // lowest winning control of that class, warp-wide class by class
    for (int q = lane; q < n_ent; q += 32)
        w_cnt[q] = 0;
    __syncwarp();
#pragma unroll
    for (int r = 0; r < RJ; ++r) {
        if ((todo >> r) & 1u) {
            atomicAdd(&w_cnt[bcls[r]], 1);
            w_best[lane * RJ + r] = best[r];
        }
    }
    __syncwarp();
    int total = 0;  // exclusive scan of the counters, in place
    for (int b0 = 0; b0 < n_ent; b0 += 32) {
        const int q = b0 + lane;
        const int x = q < n_ent ? w_cnt[q] : 0;
        int incl = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, d);
            if (lane >= d)
                incl += y;
        }
        if (q < n_ent)
            w_cnt[q] = total + incl - x;
        total += __shfl_sync(FULL, incl, 31);
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < RJ; ++r) {
        if ((todo >> r) & 1u) {
            const int key = bcls[r];
            const int pos = atomicAdd(&w_cnt[key], 1);
            w_list[pos] = ((unsigned)key << 16) | (unsigned)(lane * RJ + r);
        }
    }
    __syncwarp();
    for (int q = lane; q < total; q += 32) {
        const unsigned en = w_list[q];
        const int e = (int)(en >> 16);
        const int s = (int)(en & 0xffffu);
        const int ln = s / RJ, r = s - ln * RJ;
        const int fq = chunk0 + ln;
        const int jgq = fq / P.n_t;
        const int lq = fq - jgq * P.n_t;
        const float tlq = node_val(P.t_lo, P.t_span, lq, P.n_t);
        const float wq = wait_time(tb, k, tlq, si.wait_row);
        const ClassEntry E = s_ent[e];
        const TCtx x = class_ctx(P, Vn, s_cls[E.cls], lq, tlq, wq, si);
        const int j = jgq * RJ + r;
        pik[((size_t)i * P.n_xi + j) * P.n_t + lq] = (int16_t)class_lowest_u(P, x, E, s_spl, j, w_best[s]);
    }
}

}  // namespace

size_t bellman_smem_bytes(const DevParams &hP) { return tiled_layout(hP.n_cls, hP.n_u).total; }

cudaError_t launch_bellman(const DevParams *dP, const DevParams &hP, StageTables tb, int k, StageScratch sc,
                           const float *Vnext, float *Vk, int16_t *pik, int variant, cudaStream_t s)
{
    if (variant == 0) {
        dim3 grid((hP.n_xi * hP.n_t + 255) / 256, hP.n_v);
        bellman_direct<<<grid, 256, 0, s>>>(dP, tb, k, sc, Vnext, Vk, pik);
        return cudaGetLastError();
    }
    const size_t smem = bellman_smem_bytes(hP);
    cudaError_t err = cudaFuncSetAttribute(bellman_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess)
        return err;
    const int n_jg = (hP.n_xi + RJ - 1) / RJ;
    const int chunks = (n_jg * hP.n_t + TLANES - 1) / TLANES;
    bellman_tiled<<<dim3(chunks, hP.n_v), TLANES, smem, s>>>(dP, tb, k, sc, Vnext, Vk, pik);
    return cudaGetLastError();
}

}  // namespace ecodp
