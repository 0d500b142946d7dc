// Device code of one Bellman tile, shared by the single-problem kernel
// (k_bellman.cu) and the batched persistent kernel (k_batch.cu).
//
// J_k(v_i, xi_j, t_l) = min_u [c + J_{k+1}(f(x, u))] and its argmin
// (Eq. 9b-9d).  For control u in torque class C (same T_eng + T_bsg and brake
// flag) the successor is (v'_C, xi_j - dxi_u, t_l + dt_C): the speed and time
// axes of the trilinear interpolation are shared by the class and only the
// SoC axis depends on u (Eq. 5a-5c).  With uniform grids the SoC shift is the
// same for every j and the time shift the same for every l, so
//   J_{k+1}(f(x, u)) = G_C(j + d_u) + f_u (G_C(j + d_u + 1) - G_C(j + d_u))
// where G_C(j') blends two speed rows and two time columns of J_{k+1} at SoC
// row j'.  For the controls of one class and one shift d the value is
// G(j + d) + (c_u + f_u D(j + d)) with D the forward difference of G, a line
// in D: the precompute kernel keeps only each bucket's lower envelope, and
// the minimum over the bucket is G(j + d) + min over its lines of
// (c_u + f_u D), one FMA and one min per line and row.  At a light stage the
// arrival check (Eq. 5c, 7c, 8) depends on the arrival time (per lane and
// class); on the standstill row v = 0 at a light node the departure waits for
// green, which shifts the time landing per time node.
//
// A tile is one speed row and TLANES lanes; each lane owns one (SoC group of
// R rows, time node) pair, the pairs of a row laid out back to back so no lane
// idles on a ragged time axis.  The row's feasible classes (one 32-byte record
// each) and envelope lines are staged in shared memory.  Per class a lane
// keeps a register window of blended values G and differences D; the lines
// of a class are grouped by shift d in {-2, -1, 0, 1} so window offsets are
// compile-time constants.  The buckets d = -1 and d = 0 take the fast path;
// the outer buckets (which also need the window's two outer rows) and lines
// of any other shift sit behind one warp-uniform test per class.  Two rows go
// through one packed FP32 FMA (__ffma2_rn) and two lines through one
// three-input min.  Two consecutive classes with the same speed cell and time
// shift share the loads of their window.  In a single-problem sweep (QLD > 0)
// the window rows come from corner quads of J_{k+1} (launch_quad_from_pad):
// one 16-byte load per row instead of four, at compile-time offsets from one
// address per class, and the epilogue writes J_k's quads for the next stage.
// Only class minima are tracked in
// the sweep; afterwards each warp buckets its states by winning class in
// shared memory and re-evaluates that class (bit for bit the same arithmetic)
// to recover the argmin.  An arrival during red points the class's time
// corner at the padding columns, so its values come out infeasible without a
// per-row select.
//
// Argmin order: (value, torque class, control index).  Among controls with
// exactly equal FP32 values the first class in class order (brake flag
// slowest, then total torque ascending) wins, then the lowest control index
// inside it.  Exact ties between classes are structural (classes with the
// same successor window reaching the value with lines of equal cost, such as
// a stop at the line with and without the brake flag); on the paper-scale
// sweep 1.5 % of the feasible states have one, and for 99 % of those the
// first class also holds the lowest control index.  Resolving the rest
// toward the lowest global index would re-evaluate every later class of such
// a state in the argmin recovery.
#pragma once

#include <climits>

#include "ecodp_internal.cuh"

#undef ECODP_FILE_TAG
#define ECODP_FILE_TAG 6

namespace ecodp {
namespace tile {

constexpr unsigned FULL = 0xffffffffu;
constexpr int TW = 4;  // warps per tile
constexpr int TLANES = TW * 32;

// Loads of J_{k+1}: through the read-only path when J_{k+1} cannot change
// during the launch (one stage per launch), through L1/L2 otherwise (a
// persistent launch whose other CTAs wrote it, ordered by an acquire).  The
// read-only loads ask L1 to evict these lines last: consecutive classes read
// nearly the same cells of J_{k+1}, while the row's tables sit in shared
// memory.
template <bool NC>
__device__ __forceinline__ float ldv(const float *p)
{
    if (NC) {
        float v;
        asm("ld.global.nc.L1::evict_last.f32 %0, [%1];" : "=f"(v) : "l"(p));
        return v;
    }
    return __ldca(p);
}

// Bilinear blend of a cell's four corners (lo: the lower speed row's two time
// columns, hi: the upper's) with the weights (wt0 wv0, wt1 wv0) on lo and
// (wt0 wv1, wt1 wv1) on hi: one packed multiply, one packed FMA and one add
// per value.  The weight products depend on the class only, so a window's
// rows share them.
__device__ __forceinline__ float blend_raw(float2 lo, float2 hi, float wv0, float wv1, float wt0, float wt1)
{
    const float2 w0 = __fmul2_rn(make_float2(wt0, wt1), make_float2(wv0, wv0));
    const float2 w1 = __fmul2_rn(make_float2(wt0, wt1), make_float2(wv1, wv1));
    const float2 S = __ffma2_rn(w1, hi, __fmul2_rn(w0, lo));
    return __fadd_rn(S.x, S.y);
}

template <bool NC>
__device__ __forceinline__ float blend(const float *p0, const float *p1, float wv0, float wv1, float wt0, float wt1)
{
    const float2 lo = make_float2(ldv<NC>(p0), ldv<NC>(p0 + 1));
    const float2 hi = make_float2(ldv<NC>(p1), ldv<NC>(p1 + 1));
    return blend_raw(lo, hi, wv0, wv1, wt0, wt1);
}

// Per-lane interpolation context of one class.
struct TCtx {
    const float *p0, *p1;  // speed rows iv, iv+1 of J_{k+1} at padded SoC row 0, lower time column
    float wv0, wv1, wt0, wt1;
    int iv, ta;  // the speed cell and lower time column read
};

struct StageInfo {
    bool wait_row;   // v_i == 0 at a light node: wait for green before departing
    int here;        // light index at node k, or -1
    int next_light;  // light index at node k+1, or -1
    float cyc1, red1, off1;
};

// The step time dt and whether v' > 0, read only on a waiting row and before
// a light (through a callback, so a tile reads them from shared memory only
// there).
struct DtFlag {
    float dt;
    bool moving;  // v' > 0
};

template <class DtFn>
__device__ __forceinline__ TCtx class_ctx_at(const DevParams &P, const float *Vn, int iv, int st, float fv, float ft_c,
                                             DtFn dtv, int l, float tl, float wait, const StageInfo &si)
{
    TCtx x;
    int t0;
    float ft;
    if (!si.wait_row) {
        t0 = l + st;
        ft = ft_c;
    } else {
        int sw;
        snap_split(__fdiv_rn(__fadd_rn(wait, dtv().dt), P.h_t), sw, ft);
        t0 = l + sw;
    }
    // an arrival during red at the next node (Eq. 5c, 7c, 8) makes every
    // value of the class infeasible: read the padding columns, which hold
    // V_BIG in every row
    bool red = false;
    if (P.light_model != 1 && si.next_light >= 0) {
        const DtFlag d = dtv();
        if (d.moving) {
            const float tarr = __fadd_rn(__fadd_rn(tl, wait), d.dt);
            red = phase_pos(tarr, si.off1, si.cyc1) < si.red1;
        }
    }
    // literal Eq. 5c: departing from the line needs green (no folded wait);
    // the zero-speed step (v' = 0) lands at the end of red
    if (P.light_model == 2 && si.wait_row && wait > 0.f && dtv().moving)
        red = true;
    // a lower corner past the grid reads the padding column n_t; the upper
    // corner is the next column, still inside the row (ld_t >= n_t + 2)
    int ta = red ? P.n_t : min(t0, P.n_t);
    // the window reads speed rows iv, iv + 1 and time columns ta, ta + 1 of
    // every padded SoC row
    if (!DP_IN(iv, P.n_v - 1) || !DP_IN(ta, P.ld_t - 1)) {
        iv = 0;
        ta = P.n_t;
    }
    x.wt1 = ft;
    x.wt0 = __fsub_rn(1.f, ft);
    x.wv1 = fv;
    x.wv0 = __fsub_rn(1.f, fv);
    const size_t vrow = (size_t)P.xi_rows * P.ld_t;
    x.p0 = Vn + (size_t)iv * vrow + ta;
    x.p1 = x.p0 + vrow;
    x.iv = iv;
    x.ta = ta;
    return x;
}

// dt's bits with bit 31 set when v' = 0 (dt is never negative)
__device__ __forceinline__ unsigned dt_flagged(const ClassRec &C)
{
    return __float_as_uint(C.dt) | (C.v1 > 0.f ? 0u : 0x80000000u);
}

__device__ __forceinline__ TCtx class_ctx(const DevParams &P, const float *Vn, const ClassRec &C, int l, float tl,
                                          float wait, const StageInfo &si)
{
    return class_ctx_at(P, Vn, C.iv, C.st, C.fv, C.ft, [&] { return DtFlag{C.dt, C.v1 > 0.f}; }, l, tl, wait, si);
}

__device__ __forceinline__ int row_offset(const DevParams &P, int j)
{
    return (min(max(j, -1), P.n_xi) + 1) * P.ld_t;
}

// Blended value G at SoC row j (any integer; rows outside the grid read padding).
template <bool NC>
__device__ __forceinline__ float g_at(const DevParams &P, const TCtx &x, int j)
{
    const int o = row_offset(P, j);
    return blend<NC>(x.p0 + o, x.p1 + o, x.wv0, x.wv1, x.wt0, x.wt1);
}

// g0 + (c + f (g1 - g0)), in this order (the tile's bucket path rounds
// identically: it takes the minimum of c + f D before adding g0, and adding
// g0 is monotone).
__device__ __forceinline__ float split_value(float c, float f, float g0, float g1)
{
    return __fadd_rn(g0, __fmaf_rn(f, __fsub_rn(g1, g0), c));
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
    si.here = lk;
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

// Green indicator sampled on the time grid (light_model 1, Sec. III, Eq. 8):
// a state moving through the light at node k at a red time node t_l is
// infeasible.
__device__ __forceinline__ bool sampled_red(const DevParams &P, const StageTables &tb, const StageInfo &si, float v,
                                            float tl)
{
    return P.light_model == 1 && si.here >= 0 && v > 0.f &&
           phase_pos(tl, tb.offset[si.here], tb.cycle[si.here]) < tb.red[si.here];
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

// Minimum over the lines of one SoC-shift bucket: row r takes
// min_u (c_u + f_u D[r + D + 2]).  Lines are staged as {c, f}; a packed FMA
// evaluates one line at two SoC rows.  EV holds the even-aligned difference
// pairs {D[2p], D[2p+1]}, OD the odd-aligned pairs {D[2p+1], D[2p+2]}.
template <int R, int D>
__device__ __forceinline__ void bucket_min(const float2 *ln, int n, const float2 (&EV)[R / 2 + 1],
                                           const float2 (&OD)[R / 2 + 1], float (&cm)[R])
{
    {
        const float2 a = ln[0];
        const float2 c1 = make_float2(a.x, a.x), f1 = make_float2(a.y, a.y);
#pragma unroll
        for (int p = 0; p < R / 2; ++p) {
            const float2 DD = ((D & 1) == 0) ? EV[p + (D + 2) / 2] : OD[p + (D + 1) / 2];
            const float2 F1 = __ffma2_rn(f1, DD, c1);
            cm[2 * p] = F1.x;
            cm[2 * p + 1] = F1.y;
        }
    }
    int q = 1;
    for (; q + 1 < n; q += 2) {
        const float2 a = ln[q], b = ln[q + 1];
        const float2 c1 = make_float2(a.x, a.x), f1 = make_float2(a.y, a.y);
        const float2 c2 = make_float2(b.x, b.x), f2 = make_float2(b.y, b.y);
#pragma unroll
        for (int p = 0; p < R / 2; ++p) {
            const float2 DD = ((D & 1) == 0) ? EV[p + (D + 2) / 2] : OD[p + (D + 1) / 2];
            const float2 F1 = __ffma2_rn(f1, DD, c1);
            const float2 F2 = __ffma2_rn(f2, DD, c2);
            cm[2 * p] = min3(cm[2 * p], F1.x, F2.x);
            cm[2 * p + 1] = min3(cm[2 * p + 1], F1.y, F2.y);
        }
    }
    if (q < n) {
        const float2 a = ln[q];
        const float2 c1 = make_float2(a.x, a.x), f1 = make_float2(a.y, a.y);
#pragma unroll
        for (int p = 0; p < R / 2; ++p) {
            const float2 DD = ((D & 1) == 0) ? EV[p + (D + 2) / 2] : OD[p + (D + 1) / 2];
            const float2 F1 = __ffma2_rn(f1, DD, c1);
            cm[2 * p] = fminf(cm[2 * p], F1.x);
            cm[2 * p + 1] = fminf(cm[2 * p + 1], F1.y);
        }
    }
}

// One bucket's candidates G[r + D + 2] + cm[r] folded into the class minimum
// (FIRST: they start it).
template <int R, int D, bool FIRST = false>
__device__ __forceinline__ void bucket_fold(const float (&G)[R + 4], const float (&cm)[R], float (&cls)[R])
{
    float cand[R];
    if ((D & 1) == 0) {
#pragma unroll
        for (int p = 0; p < R / 2; ++p) {
            const float2 s2 = __fadd2_rn(make_float2(G[2 * p + D + 2], G[2 * p + D + 3]),
                                         make_float2(cm[2 * p], cm[2 * p + 1]));
            cand[2 * p] = s2.x;
            cand[2 * p + 1] = s2.y;
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r)
            cand[r] = __fadd_rn(G[r + D + 2], cm[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        cls[r] = FIRST ? cand[r] : fminf(cls[r], cand[r]);
}

// Lowest control index of class E whose value at SoC row j equals bv (INT_MAX
// if none), re-evaluated with exactly the arithmetic of the sweep.
template <bool NC>
__device__ __forceinline__ int class_lowest_u(const DevParams &P, const TCtx &x, const ClassEntry &E,
                                              const float2 *ln, const SplitRec *g_spl,
                                              int j, float bv)
{
    float g5[5];  // SoC rows j - 2 .. j + 2
#pragma unroll
    for (int w = 0; w < 5; ++w)
        g5[w] = g_at<NC>(P, x, j - 2 + w);
    int ub = INT_MAX;
    int q = E.off;
#pragma unroll
    for (int b = 0; b < 4; ++b) {  // bucket b holds the shift d = b - 2
        for (int n = 0; n < E.nb[b]; ++n, ++q)
            if (split_value(ln[q].x, ln[q].y, g5[b], g5[b + 1]) == bv)
                ub = min(ub, split_u(g_spl[q]));
    }
    for (int n = 0; n < E.n_other; ++n, ++q) {
        const float2 a = ln[q];
        const SplitRec S = g_spl[q];
        const int d = split_d(S);
        if (split_value(a.x, a.y, g_at<NC>(P, x, j + d), g_at<NC>(P, x, j + d + 1)) == bv)
            ub = min(ub, split_u(S));
    }
    return ub;
}

// class_lowest_u on the row's global table (the per-state join).
template <bool NC>
__device__ __forceinline__ int class_lowest_u_global(const DevParams &P, const TCtx &x, const ClassEntry &E,
                                                     const SplitRec *g_spl, int j, float bv)
{
    float g5[5];  // SoC rows j - 2 .. j + 2
#pragma unroll
    for (int w = 0; w < 5; ++w)
        g5[w] = g_at<NC>(P, x, j - 2 + w);
    int ub = INT_MAX;
    int q = E.off;
#pragma unroll
    for (int b = 0; b < 4; ++b) {  // bucket b holds the shift d = b - 2
        for (int n = 0; n < E.nb[b]; ++n, ++q) {
            const SplitRec S = g_spl[q];
            if (split_value(S.c, S.f, g5[b], g5[b + 1]) == bv)
                ub = min(ub, split_u(S));
        }
    }
    for (int n = 0; n < E.n_other; ++n, ++q) {
        const SplitRec S = g_spl[q];
        const int d = split_d(S);
        if (split_value(S.c, S.f, g_at<NC>(P, x, j + d), g_at<NC>(P, x, j + d + 1)) == bv)
            ub = min(ub, split_u(S));
    }
    return ub;
}

// One corner quad of J_{k+1} (launch_quad_from_pad): the cell's two time
// columns at speed rows iv and iv + 1, read-only with the L1 evict-last hint.
__device__ __forceinline__ float4 ldq(const float4 *p)
{
    float4 v;
    asm("ld.global.nc.L1::evict_last.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}

// Blend of one corner quad.
__device__ __forceinline__ float blend_quad(const float4 c, float wv0, float wv1, float wt0, float wt1)
{
    return blend_raw(make_float2(c.x, c.y), make_float2(c.z, c.w), wv0, wv1, wt0, wt1);
}

// class_window and pair_window on the corner quads: q0 is the quad of the
// window's row w = 0 (SoC row jb - 2), row w sits QLD quads further, a
// compile-time offset.
template <int R, int QLD>
__device__ __forceinline__ void class_window_q(const float4 *q0, const TCtx &x, float (&G)[R + 4])
{
#pragma unroll
    for (int w = 1; w < R + 3; ++w)
        G[w] = blend_quad(ldq(q0 + w * QLD), x.wv0, x.wv1, x.wt0, x.wt1);
}

template <int R, int QLD>
__device__ __forceinline__ void pair_window_q(const float4 *q0, const TCtx &x, float bv0, float bv1, float bt0,
                                              float bt1, float (&G)[R + 4], float (&H)[R + 4])
{
#pragma unroll
    for (int w = 1; w < R + 3; ++w) {
        const float4 c = ldq(q0 + w * QLD);
        G[w] = blend_quad(c, x.wv0, x.wv1, x.wt0, x.wt1);
        H[w] = blend_quad(c, bv0, bv1, bt0, bt1);
    }
}

// Inner window of one class: blended values at SoC rows jb - 1 .. jb + R
// (G[1 .. R + 2]; row offsets roff), which the buckets d = -1 and d = 0 read.
template <int R, bool NC>
__device__ __forceinline__ void class_window(const TCtx &x, const int (&roff)[R + 4], float (&G)[R + 4])
{
#pragma unroll
    for (int w = 1; w < R + 3; ++w)
        G[w] = blend<NC>(x.p0 + roff[w], x.p1 + roff[w], x.wv0, x.wv1, x.wt0, x.wt1);
}

// Inner windows of two classes that read the same corners (same pointers in
// x) with their own weights: G with x's, H with (bv0, bv1, bt0, bt1); each
// corner is loaded once.
template <int R, bool NC>
__device__ __forceinline__ void pair_window(const TCtx &x, const int (&roff)[R + 4], float bv0, float bv1, float bt0,
                                            float bt1, float (&G)[R + 4], float (&H)[R + 4])
{
#pragma unroll
    for (int w = 1; w < R + 3; ++w) {
        const float *p0 = x.p0 + roff[w], *p1 = x.p1 + roff[w];
        const float2 lo = make_float2(ldv<NC>(p0), ldv<NC>(p0 + 1));
        const float2 hi = make_float2(ldv<NC>(p1), ldv<NC>(p1 + 1));
        G[w] = blend_raw(lo, hi, x.wv0, x.wv1, x.wt0, x.wt1);
        H[w] = blend_raw(lo, hi, bv0, bv1, bt0, bt1);
    }
}

// A feasible class as a tile stages it, in entry order (32 bytes): speed
// cell iv and time shift st in one word (st clamped to 2^14, beyond any time
// grid; a pair compares the word), the weights, the first line, and the line
// counts of the buckets d = -2 .. +1 (the last word also holds the count of
// lines with any other shift in its upper half).  The step time, read only on
// waiting rows and before a light, sits in a separate array.
struct TileClass {
    unsigned ivst;  // iv | min(st, 2^14) << 16
    float fv, ft;
    int off;
    int nb0, nb1, nb2;
    unsigned nb3_other;  // nb3 | n_other << 16
};

__device__ __forceinline__ TileClass tile_class(const ClassRec &C, const ClassEntry &E)
{
    TileClass T;
    T.ivst = (unsigned)C.iv | ((unsigned)min(C.st, 1 << 14) << 16);
    T.fv = C.fv;
    T.ft = C.ft;
    T.off = E.off;
    T.nb0 = E.nb[0];
    T.nb1 = E.nb[1];
    T.nb2 = E.nb[2];
    T.nb3_other = (unsigned)E.nb[3] | ((unsigned)E.n_other << 16);
    return T;
}

__device__ __forceinline__ ClassEntry tile_entry(const TileClass &T, int e)
{
    ClassEntry E;
    E.cls = e;
    E.off = T.off;
    E.nb[0] = T.nb0;
    E.nb[1] = T.nb1;
    E.nb[2] = T.nb2;
    E.nb[3] = (int)(T.nb3_other & 0xffffu);
    E.n_other = (int)(T.nb3_other >> 16);
    E.n_total = 0;
    return E;
}

__device__ __forceinline__ TCtx tile_ctx(const DevParams &P, const float *Vn, const TileClass &T,
                                         const unsigned *s_dtv, int e, int l, float tl, float wait,
                                         const StageInfo &si)
{
    return class_ctx_at(
        P, Vn, (int)(T.ivst & 0xffffu), (int)(T.ivst >> 16), T.fv, T.ft,
        [&] {
            const unsigned b = s_dtv[e];
            return DtFlag{__uint_as_float(b & 0x7fffffffu), (b >> 31) == 0u};
        },
        l, tl, wait, si);
}

// A 32-byte table record read with the streaming (evict-first) hint: it is
// staged in shared memory once per tile and must not crowd J_{k+1} out of L1.
template <class T>
__device__ __forceinline__ T ld_stream(const T *p)
{
    static_assert(sizeof(T) == 32 && alignof(T) >= 16, "32-byte records on 16-byte boundaries");
    const int4 *q = reinterpret_cast<const int4 *>(p);
    const int4 a = __ldcs(q), b = __ldcs(q + 1);
    T t;
    int4 *d = reinterpret_cast<int4 *>(&t);
    d[0] = a;
    d[1] = b;
    return t;
}

// Shared memory of a tile: the row's feasible classes (TileClass, then the
// flagged step times) and lines as {c, f} (a line outside the four buckets
// reads its shift, and argmin recovery its control index, from the global
// table), then per warp the argmin-recovery buffers: counters [n_cls + 1],
// entry list [32 R], best value per state [32 R].  Kept small: the rest of
// the SM's 256 KB of L1 and shared memory caches the J_{k+1} windows.
struct Layout {
    size_t dtv, line, warp, warp_bytes, total;
    size_t w_list, w_best;  // offsets inside a warp's block
};

template <int R>
__host__ __device__ inline Layout layout(int n_cls, int n_u)
{
    Layout L;
    size_t o = (size_t)n_cls * sizeof(TileClass);
    L.dtv = o;
    o += ((size_t)n_cls * sizeof(float) + 15) / 16 * 16;
    L.line = o;
    o += ((size_t)n_u * sizeof(float2) + 15) / 16 * 16;
    L.warp = o;
    size_t w = ((size_t)(n_cls + 1) * sizeof(int) + 15) / 16 * 16;
    L.w_list = w;
    w += (size_t)32 * R * sizeof(unsigned);
    L.w_best = w;
    w += (size_t)32 * R * sizeof(float);
    L.warp_bytes = w;
    L.total = o + TW * L.warp_bytes;
    return L;
}

// Flattened (SoC group, time) lanes of one speed row.
template <int R>
__host__ __device__ inline int chunks_per_row(int n_xi, int n_t)
{
    return ((n_xi + R - 1) / R * n_t + TLANES - 1) / TLANES;
}

// One tile: speed row i, lane chunk `chunk` of stage k.  The row's tables
// are (cls, ent, spl) with n_ent feasible classes and n_spl controls.  All
// TLANES threads of the CTA call it; it starts with a barrier so the shared
// memory can be reused by the next tile.
// Tile modes: the whole class list (TILE_FULL), or a slice [e_begin, e_end)
// of it whose per-state minimum, packed as (value bits << 32 | class), is
// merged into `part` with atomicMin (TILE_SLICE: values are non-negative, so
// their bit patterns order like the floats, and equal values keep the lower
// class, the tie order below); a per-state join then writes J_k and recovers
// the argmin from `part`.
constexpr int TILE_FULL = 0, TILE_SLICE = 1;

// Relative cost of one class in the tile's loop: the window and bookkeeping
// (weighted as 12 line evaluations, the best of 12, 24 and 40 measured for
// the slice bounds and the row plan) plus its lines.
__device__ __forceinline__ int class_cost(const TileClass &T)
{
    return 12 + T.nb0 + T.nb1 + T.nb2 + (int)(T.nb3_other & 0xffffu) + (int)(T.nb3_other >> 16);
}

// Slice s of S of the classes [0, n): contiguous, of about equal cost (slice
// t starts at the first class whose inclusive cost prefix exceeds t/S of the
// total).  Called by a whole warp; every lane gets the same bounds.
__device__ __forceinline__ void slice_bounds(const TileClass *s_tc, int n, int S, int s, int lane, int &lo, int &hi)
{
    int tot = 0;
    for (int b = 0; b < n; b += 32)
        tot += __reduce_add_sync(FULL, b + lane < n ? class_cost(s_tc[b + lane]) : 0);
    auto boundary = [&](int t) -> int {
        if (t <= 0)
            return 0;
        if (t >= S)
            return n;
        const long long target = (long long)tot * t / S;
        long long run = 0;
        for (int b = 0; b < n; b += 32) {
            const int e = b + lane;
            const int c = e < n ? class_cost(s_tc[e]) : 0;
            int incl = c;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(FULL, incl, d);
                if (lane >= d)
                    incl += y;
            }
            const unsigned m = __ballot_sync(FULL, e < n && run + incl > target);
            if (m)
                return b + __ffs((int)m) - 1;
            run += __shfl_sync(FULL, incl, 31);
        }
        return n;
    };
    lo = boundary(s);
    hi = boundary(s + 1);
}

__device__ __forceinline__ unsigned long long pack_min(float v, int e)
{
    const float z = __fadd_rn(v, 0.f);  // -0 -> +0
    return ((unsigned long long)__float_as_uint(z) << 32) | (unsigned)e;
}

template <int R, bool NC, int MODE = TILE_FULL, int QLD = 0>
__device__ void bellman_tile(const DevParams &P, const StageTables &tb, int k, const ClassRec *g_cls,
                             const ClassEntry *g_ent, const SplitRec *g_spl, int n_ent, int n_spl, const float *Vn,
                             float *__restrict__ Vk, int16_t *__restrict__ pik, int i, int chunk,
                             unsigned char *smem_raw, unsigned long long *stats, int e_begin = 0, int e_end = 0,
                             unsigned long long *__restrict__ part = nullptr, const float4 *__restrict__ Qn = nullptr,
                             float4 *__restrict__ Qk = nullptr, int lmax_next = INT_MAX, int *lmax_out = nullptr,
                             int n_chunks = 0)
{
    const int tid = threadIdx.x;
    const Layout L = layout<R>(P.n_cls, P.n_u);
    TileClass *s_tc = reinterpret_cast<TileClass *>(smem_raw);
    unsigned *s_dtv = reinterpret_cast<unsigned *>(smem_raw + L.dtv);
    float2 *s_line = reinterpret_cast<float2 *>(smem_raw + L.line);
    const int warp = tid >> 5, lane = tid & 31;
    const int n_jg = (P.n_xi + R - 1) / R;
    // Every successor time is at least the state's own (time shifts and
    // waits are non-negative), so past J_{k+1}'s last feasible time column
    // (lmax_next, with n_chunks the row's tiles in this launch; single-problem
    // sweeps only) every corner a state reads is infeasible, and so is the
    // state: the lanes cover only the n_tc time columns up to it, and the
    // states past them are written infeasible without evaluation.
    int n_tc = P.n_t;
    if constexpr (MODE == TILE_FULL && NC) {
        if (n_chunks > 0 && lmax_next < P.n_t - 1)
            n_tc = max(lmax_next + 1, 0);
    }
    const int n_act = n_jg * n_tc;  // lanes (SoC group, time column) of the row
    // Where the row's n_chunks tiles (the launch fills every resident CTA
    // slot) hold more lanes than the row needs, the classes of a lane group
    // are split over S warps (contiguous class slices, merged in class order
    // after the loop): a warp's class loop is a chain of dependent
    // instructions, and S warps finish it sooner.
    int S = 1;
    if constexpr (MODE == TILE_FULL && NC) {
        if (n_chunks > 0) {
            if ((4 * n_act + TLANES - 1) / TLANES <= n_chunks)
                S = 4;
            else if ((2 * n_act + TLANES - 1) / TLANES <= n_chunks)
                S = 2;
        }
    }
    const int grp = warp / S, slice = warp - grp * S;   // lane group (32 lanes), class slice
    const int chunk0 = chunk * (TLANES / S) + grp * 32;  // first lane of this warp's group
    const int f_raw = chunk0 + lane;
    const bool f_ok = f_raw < n_act;
    const int f = f_ok ? f_raw : max(n_act - 1, 0);
    const int jg = n_tc > 0 ? f / n_tc : 0;
    const int l = f - jg * n_tc;
    const int jb = jg * R;
    const bool tile_active = chunk * (TLANES / S) < n_act;  // uniform over the CTA
    const int qrows = quad_rows(P.n_xi);
    const size_t vrowq = (size_t)qrows * QLD;
    // J_k's value val at state (j, lj) of row i, -1 as policy where
    // infeasible, and the value in the corner quads that hold it: (i, j,
    // lj).x, (i, j, lj - 1).y, (i - 1, j, lj).z, (i - 1, j, lj - 1).w
    auto store = [&](int j, int lj, float val, bool feas) {
        const size_t ov = ((size_t)i * P.xi_rows + (j + 1)) * P.ld_t + lj;
        const size_t op = ((size_t)i * P.n_xi + j) * P.n_t + lj;
        if (!DP_IN(ov, (size_t)P.n_v * P.xi_rows * P.ld_t) || !DP_IN(op, (size_t)P.n_v * P.n_xi * P.n_t))
            return;
        Vk[ov] = val;
        if (!feas)
            pik[op] = -1;
        if (QLD > 0) {
            float *qf = reinterpret_cast<float *>(Qk);
            const size_t oq = ((size_t)i * qrows + (j + QUAD_PAD)) * QLD + lj;
            if (DP_IN(oq, (size_t)P.n_v * vrowq)) {
                qf[4 * oq] = val;
                if (lj > 0)
                    qf[4 * (oq - 1) + 1] = val;
                if (i > 0) {
                    qf[4 * (oq - vrowq) + 2] = val;
                    if (lj > 0)
                        qf[4 * (oq - vrowq - 1) + 3] = val;
                }
            }
        }
    };
    __syncthreads();  // the previous tile may still read the tables
    if (MODE == TILE_FULL && NC && n_tc < P.n_t) {
        // the row's states past the last time column that can be feasible,
        // shared out over the row's tiles
        const int w_t = P.n_t - n_tc, n_fill = P.n_xi * w_t;
        unsigned n_filled = 0;
        for (int q = chunk * TLANES + tid; q < n_fill; q += n_chunks * TLANES) {
            const int j = q / w_t;
            store(j, n_tc + (q - j * w_t), V_BIG, false);
            ++n_filled;
        }
        if (stats) {
            // the (state, class) and (state, line) pairs the tables would
            // have cost these states
            const unsigned n = __reduce_add_sync(FULL, n_filled);
            if (lane == 0 && n > 0) {
                atomicAdd(stats + 5, (unsigned long long)n * (unsigned long long)max(n_ent, 0));
                atomicAdd(stats + 6, (unsigned long long)n * (unsigned long long)max(n_spl, 0));
                atomicAdd(stats + 7, (unsigned long long)n);
            }
        }
    }
    if (tile_active) {
        // a slice stages only its own classes and their lines (same indices)
        int c_lo = 0, c_hi = n_ent, q_lo = 0, q_hi = n_spl;
        if (MODE == TILE_SLICE) {
            c_lo = e_begin;
            c_hi = min(e_end, n_ent);
            q_lo = q_hi = 0;
            if (c_lo < c_hi) {
                q_lo = g_ent[c_lo].off;
                q_hi = g_ent[c_hi - 1].off + g_ent[c_hi - 1].n_total;
            }
        }
        for (int q = c_lo + tid; q < c_hi; q += TLANES) {
            if (!DP_IN(q, P.n_cls))
                break;
            const ClassEntry E = ld_stream(g_ent + q);
            if (!DP_IN(E.cls, P.n_cls) || !DP_IN(E.off, P.n_u + 1) || !DP_IN((long long)E.off + E.n_total, P.n_u + 1))
                continue;
            const ClassRec C = ld_stream(g_cls + E.cls);
            s_tc[q] = tile_class(C, E);
            s_dtv[q] = dt_flagged(C);
        }
        for (int q = q_lo + tid; q < q_hi; q += TLANES)
            if (DP_IN(q, P.n_u))
                s_line[q] = __ldcs(reinterpret_cast<const float2 *>(g_spl + q));
    }
    unsigned char *wbase = smem_raw + L.warp + warp * L.warp_bytes;
    int *w_cnt = reinterpret_cast<int *>(wbase);
    unsigned *w_list = reinterpret_cast<unsigned *>(wbase + L.w_list);
    float *w_best = reinterpret_cast<float *>(wbase + L.w_best);
    __syncthreads();
    const bool warp_idle = !__any_sync(FULL, f_ok);

    const float one_m_gamma = __fsub_rn(1.f, P.gamma);
    const float v = node_val(P.v_lo, P.v_span, i, P.n_v);
    const StageInfo si = stage_info(tb, k, v);
    const float tl = node_val(P.t_lo, P.t_span, l, P.n_t);
    const float wait = wait_time(tb, k, tl, si.wait_row);

    int roff[R + 4];
#pragma unroll
    for (int w = 0; w < R + 4; ++w)
        roff[w] = row_offset(P, jb - 2 + w);
    // corner quads (QLD > 0): the lane's window row w = 0 (SoC row jb - 2) is
    // quad row jb - 2 + QUAD_PAD of every speed row
    const float4 *qlane = QLD > 0 ? Qn + (size_t)(jb - 2 + QUAD_PAD) * QLD : nullptr;

    // per row: the running minimum and the first class (in class order)
    // reaching it (the order (value, class, control) decides exact ties)
    float best[R];
    int bcls[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        best[r] = __int_as_float(0x7f800000);
        bcls[r] = 0;
    }
    int e_lo = MODE == TILE_SLICE ? e_begin : 0;
    int e_hi = MODE == TILE_SLICE ? min(e_end, n_ent) : n_ent;
    if (MODE == TILE_FULL && NC && S > 1)
        slice_bounds(s_tc, min(n_ent, P.n_cls), S, slice, lane, e_lo, e_hi);
    // Consecutive classes with the same speed cell and time shift read the
    // same four corners of J_{k+1} and differ only in their weights.  Where
    // the corners depend neither on the class nor on the lane (no red check
    // at the next node, no waiting row), such a pair loads its window once:
    // H keeps the second class's values for the next iteration.
    const bool can_pair = !si.wait_row && !(P.light_model != 1 && si.next_light >= 0);
    float H[R + 4];
    bool have_h = false;
    for (int e = warp_idle ? e_hi : e_lo; e < e_hi; ++e) {
        if (!DP_IN(e, P.n_cls))
            break;
        const TileClass T = s_tc[e];
        const ClassEntry E = tile_entry(T, e);
        if (!DP_IN(E.off, P.n_u + 1) ||
            !DP_IN((long long)E.off + E.nb[0] + E.nb[1] + E.nb[2] + E.nb[3] + E.n_other, P.n_u + 1))
            continue;
        // inner window rows jb - 1 .. jb + R (G[1 .. R + 2]); the outer rows
        // G[0], G[R + 3] only for the rare buckets d = -2, +1 below.  The
        // second class of a pair needs its interpolation context only there.
        float G[R + 4];
        if (have_h) {
#pragma unroll
            for (int w = 1; w < R + 3; ++w)
                G[w] = H[w];
            have_h = false;
        } else {
            const TCtx x = tile_ctx(P, Vn, T, s_dtv, e, l, tl, wait, si);
            TileClass T2;
            if (can_pair && e + 1 < e_hi) {
                T2 = s_tc[e + 1];
                have_h = T2.ivst == T.ivst;
            }
            if (QLD > 0) {
                const float4 *q0 = qlane + (size_t)x.iv * vrowq + x.ta;
                if (have_h)
                    pair_window_q<R, QLD>(q0, x, __fsub_rn(1.f, T2.fv), T2.fv, __fsub_rn(1.f, T2.ft), T2.ft, G, H);
                else
                    class_window_q<R, QLD>(q0, x, G);
            } else if (have_h) {
                pair_window<R, NC>(x, roff, __fsub_rn(1.f, T2.fv), T2.fv, __fsub_rn(1.f, T2.ft), T2.ft, G, H);
            } else {
                class_window<R, NC>(x, roff, G);
            }
        }
        // SoC differences Dg[w] = G[w + 1] - G[w] as even-aligned pairs EV[p]
        // = {Dg[2p], Dg[2p + 1]} and odd-aligned pairs OD[p] = {Dg[2p + 1],
        // Dg[2p + 2]}; the inner buckets read EV[1 .. R/2] and OD[0 .. R/2 - 1]
        float Dg[R + 3];
#pragma unroll
        for (int w = 1; w < R + 2; ++w)
            Dg[w] = __fsub_rn(G[w + 1], G[w]);
        float2 EV[R / 2 + 1], OD[R / 2 + 1];
#pragma unroll
        for (int p = 0; p < R / 2; ++p) {
            EV[p + 1] = make_float2(Dg[2 * p + 2], Dg[2 * p + 3]);
            OD[p] = make_float2(Dg[2 * p + 1], Dg[2 * p + 2]);
        }
        float cls_min[R];
        float cm[R];
        const int q1 = E.off + E.nb[0], q2 = q1 + E.nb[1];
        if (E.nb[1] > 0) {
            bucket_min<R, -1>(s_line + q1, E.nb[1], EV, OD, cm);
            bucket_fold<R, -1, true>(G, cm, cls_min);
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r)
                cls_min[r] = __int_as_float(0x7f800000);
        }
        if (E.nb[2] > 0) {
            bucket_min<R, 0>(s_line + q2, E.nb[2], EV, OD, cm);
            bucket_fold<R, 0>(G, cm, cls_min);
        }
        // rare (warp-uniform): the outer buckets d = -2, +1 and the lines of
        // any other shift
        if ((T.nb0 | (int)T.nb3_other) != 0) {  // nb[0], nb[3] or n_other
            const TCtx x = tile_ctx(P, Vn, T, s_dtv, e, l, tl, wait, si);
            if (QLD > 0) {
                const float4 *q0 = qlane + (size_t)x.iv * vrowq + x.ta;
                G[0] = blend_quad(ldq(q0), x.wv0, x.wv1, x.wt0, x.wt1);
                G[R + 3] = blend_quad(ldq(q0 + (R + 3) * QLD), x.wv0, x.wv1, x.wt0, x.wt1);
            } else {
                G[0] = blend<NC>(x.p0 + roff[0], x.p1 + roff[0], x.wv0, x.wv1, x.wt0, x.wt1);
                G[R + 3] = blend<NC>(x.p0 + roff[R + 3], x.p1 + roff[R + 3], x.wv0, x.wv1, x.wt0, x.wt1);
            }
            Dg[0] = __fsub_rn(G[1], G[0]);
            Dg[R + 2] = __fsub_rn(G[R + 3], G[R + 2]);
            EV[0] = make_float2(Dg[0], Dg[1]);
            OD[R / 2] = make_float2(Dg[R + 1], Dg[R + 2]);
            if (E.nb[0] > 0) {
                bucket_min<R, -2>(s_line + E.off, E.nb[0], EV, OD, cm);
                bucket_fold<R, -2>(G, cm, cls_min);
            }
            const int q3 = q2 + E.nb[2];
            if (E.nb[3] > 0) {
                bucket_min<R, 1>(s_line + q3, E.nb[3], EV, OD, cm);
                bucket_fold<R, 1>(G, cm, cls_min);
            }
            int q = q3 + E.nb[3];
            for (int n = 0; n < E.n_other; ++n, ++q) {
                const float2 a = s_line[q];
                const int d = split_d(g_spl[q]);
                const float c = a.x, f = a.y;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    cls_min[r] = fminf(cls_min[r], split_value(c, f, g_at<NC>(P, x, jb + r + d),
                                                               g_at<NC>(P, x, jb + r + d + 1)));
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (cls_min[r] < best[r]) {
                best[r] = cls_min[r];
                bcls[r] = e;
            }
        }
    }

    if (MODE == TILE_FULL && NC && S > 1) {
        // slices s > 0 hand their minima to slice 0 through their own
        // argmin-recovery buffers; a later slice's classes come later in
        // class order, so a strict < keeps the first class on exact ties
        if (slice > 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                w_best[lane * R + r] = best[r];
                w_list[lane * R + r] = (unsigned)bcls[r];
            }
        }
        __syncthreads();
        if (slice > 0)
            return;
        for (int s2 = 1; s2 < S; ++s2) {
            const unsigned char *ob = smem_raw + L.warp + (warp + s2) * L.warp_bytes;
            const float *o_best = reinterpret_cast<const float *>(ob + L.w_best);
            const unsigned *o_cls = reinterpret_cast<const unsigned *>(ob + L.w_list);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float vb = o_best[lane * R + r];
                if (vb < best[r]) {
                    best[r] = vb;
                    bcls[r] = (int)o_cls[lane * R + r];
                }
            }
        }
    }
    if (MODE == TILE_SLICE) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = jb + r;
            const size_t o = ((size_t)i * P.n_xi + j) * P.n_t + l;
            if (f_ok && j < P.n_xi && best[r] < __int_as_float(0x7f800000) &&
                DP_IN(o, (size_t)P.n_v * P.n_xi * P.n_t))
                atomicMin(part + o, pack_min(best[r], bcls[r]));
        }
        return;
    }
    // values now; argmin recovery below
    const bool masked = sampled_red(P, tb, si, v, tl);
    unsigned todo = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = jb + r;
        const bool valid = f_ok && j < P.n_xi;
        const bool feas = valid && !masked && best[r] < V_FEAS_MAX;
        if (feas)
            todo |= 1u << r;
        if (valid)
            store(j, l, feas ? __fadd_rn(best[r], __fmul_rn(one_m_gamma, wait)) : V_BIG, feas);
    }
    if (stats) {
        const unsigned n_find = __reduce_add_sync(FULL, (unsigned)__popc(todo));
        if (lane == 0)
            atomicAdd(stats + 3, (unsigned long long)n_find);
    }
    if (lmax_out) {
        // J_k's last feasible time column, for the next stage's skip
        const int lm = __reduce_max_sync(FULL, todo ? l : -1);
        if (lane == 0 && lm >= 0)
            atomicMax(lmax_out, lm);
    }

    // bucket the feasible states by their first winning class and recover the
    // lowest winning control of that class, warp-wide class by class
    for (int q = lane; q < n_ent; q += 32)
        if (DP_IN(q, P.n_cls + 1))
            w_cnt[q] = 0;
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (((todo >> r) & 1u) && DP_IN(bcls[r], n_ent)) {
            atomicAdd(&w_cnt[bcls[r]], 1);
            w_best[lane * R + r] = best[r];
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
    for (int r = 0; r < R; ++r) {
        if (((todo >> r) & 1u) && DP_IN(bcls[r], n_ent)) {
            const int key = bcls[r];
            const int pos = atomicAdd(&w_cnt[key], 1);
            if (DP_IN(pos, 32 * R))
                w_list[pos] = ((unsigned)key << 16) | (unsigned)(lane * R + r);
        }
    }
    __syncwarp();
    for (int q = lane; q < total; q += 32) {
        if (!DP_IN(q, 32 * R))
            break;
        const unsigned en = w_list[q];
        const int e = (int)(en >> 16);
        const int s = (int)(en & 0xffffu);
        if (!DP_IN(e, n_ent) || !DP_IN(s, 32 * R))
            continue;
        const int ln = s / R, r = s - ln * R;
        const int fq = chunk0 + ln;
        const int jgq = fq / n_tc;
        const int lq = fq - jgq * n_tc;
        const float tlq = node_val(P.t_lo, P.t_span, lq, P.n_t);
        const float wq = wait_time(tb, k, tlq, si.wait_row);
        const TileClass T = s_tc[e];
        const ClassEntry E = tile_entry(T, e);
        const TCtx x = tile_ctx(P, Vn, T, s_dtv, e, lq, tlq, wq, si);
        const int j = jgq * R + r;
        const size_t op = ((size_t)i * P.n_xi + j) * P.n_t + lq;
        if (DP_IN(op, (size_t)P.n_v * P.n_xi * P.n_t))
            pik[op] = (int16_t)class_lowest_u<NC>(P, x, E, s_line, g_spl, j, w_best[s]);
    }
}

}  // namespace tile
}  // namespace ecodp
