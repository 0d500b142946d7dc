// Per-stage precompute (the paper's first kernel, Sec. IV), terminal values
// and layout conversions.
//
// The paper's first kernel evaluates, per (v, T_eng, T_bsg), the speed change,
// the step time, the battery power and the stage cost.  Here one CTA handles
// one speed row v_i of one stage k (all stages of a sweep in one launch) and
// writes into the stage's table slot
//   * one ClassRec per torque class (speed update Eq. 5a, step time Eq. 2,
//     acceleration limits Eq. 7d, stop-at-line rule, speed-grid band Eq. 7a)
//     with the speed-axis and time-axis interpolation already resolved;
//   * the compact list of feasible classes (ClassEntry) in class order;
//   * per feasible control one SplitRec: the stage cost of Eq. (1)/(6), and
//     the SoC-axis shift d and weights (1-f, f) of xi' = xi - dt I / C_nom
//     (Eq. 5b), grouped inside each class by d.
// The per-control arithmetic runs one thread per control; the grouping then
// only reads those results back from shared memory.
#include <algorithm>

#include "ecodp_internal.cuh"

#undef ECODP_FILE_TAG
#define ECODP_FILE_TAG 1

namespace ecodp {

ECODP_CHECK_ACCESSOR(check_word_precompute)

namespace {

__global__ void fill_kernel(float *p, size_t n, float val)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = val;
}

__global__ void terminal_kernel(const DevParams *__restrict__ dP, float *__restrict__ VN)
{
    const DevParams &P = *dP;
    int total = P.n_v * P.n_xi * P.n_t;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < total; s += gridDim.x * blockDim.x) {
        int l = s % P.n_t;
        int j = (s / P.n_t) % P.n_xi;
        int i = s / (P.n_t * P.n_xi);
        float v = node_val(P.v_lo, P.v_span, i, P.n_v);
        float xi = node_val(P.xi_lo, P.xi_span, j, P.n_xi);
        const size_t o = ((size_t)i * P.xi_rows + (j + 1)) * P.ld_t + l;
        if (DP_IN(o, (size_t)P.n_v * P.xi_rows * P.ld_t))
            VN[o] = terminal_cost(P, v, xi);
    }
}

__global__ void pad_from_dense_kernel(const DevParams P, const float *__restrict__ dense, float *__restrict__ padded)
{
    int total = P.n_v * P.n_xi * P.n_t;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < total; s += gridDim.x * blockDim.x) {
        int l = s % P.n_t;
        int j = (s / P.n_t) % P.n_xi;
        int i = s / (P.n_t * P.n_xi);
        float x = dense[s];
        const size_t o = ((size_t)i * P.xi_rows + (j + 1)) * P.ld_t + l;
        if (DP_IN(o, (size_t)P.n_v * P.xi_rows * P.ld_t))
            padded[o] = (x < V_FEAS_MAX) ? x : V_BIG;
    }
}

__global__ void dense_from_pad_kernel(const DevParams P, const float *__restrict__ padded, float *__restrict__ dense)
{
    int total = P.n_v * P.n_xi * P.n_t;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < total; s += gridDim.x * blockDim.x) {
        int l = s % P.n_t;
        int j = (s / P.n_t) % P.n_xi;
        int i = s / (P.n_t * P.n_xi);
        const size_t o = ((size_t)i * P.xi_rows + (j + 1)) * P.ld_t + l;
        float x = DP_IN(o, (size_t)P.n_v * P.xi_rows * P.ld_t) ? padded[o] : V_BIG;
        dense[s] = (x < V_FEAS_MAX) ? x : __int_as_float(0x7f800000);
    }
}

// J(iv, j, c) of a padded value array, V_BIG outside the grid.
__device__ __forceinline__ float grid_value(const DevParams &P, const float *V, int iv, int j, int c)
{
    if (iv < 0 || iv >= P.n_v || j < 0 || j >= P.n_xi || c < 0 || c >= P.n_t)
        return V_BIG;
    const size_t o = ((size_t)iv * P.xi_rows + (j + 1)) * P.ld_t + c;
    return DP_IN(o, (size_t)P.n_v * P.xi_rows * P.ld_t) ? V[o] : V_BIG;
}

// Corner quads of a padded value array (launch_quad_from_pad).
__global__ void quad_from_pad_kernel(const DevParams P, const float *__restrict__ V, float4 *__restrict__ Q)
{
    const int rows = quad_rows(P.n_xi), ld = quad_ld(P.n_t);
    const size_t vrow = (size_t)rows * ld;
    const size_t total = (size_t)P.n_v * vrow;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int iv = (int)(q / vrow);
        const int rem = (int)(q - (size_t)iv * vrow);
        const int j = rem / ld - QUAD_PAD, c = rem % ld;
        float4 r;
        r.x = grid_value(P, V, iv, j, c);
        r.y = grid_value(P, V, iv, j, c + 1);
        r.z = grid_value(P, V, iv + 1, j, c);
        r.w = grid_value(P, V, iv + 1, j, c + 1);
        Q[q] = r;
    }
}

// Class numbering: c = b n_sum + s, where s indexes the total torque (the sum
// i_e + i_m, or the pair (i_e, i_m) when classes are single controls) and b
// the brake flag.  Classes of one brake flag are thus consecutive in
// ascending torque, so consecutive classes land on neighbouring successor
// speeds and mostly read the same cells of J_{k+1} (L1 reuse in the tile).
// Members (i_e, i_m) of class c in increasing i_e order (increasing u).
struct Members {
    int ie_lo, ie_hi, s;  // class_sum: i_m = s - i_e; otherwise one member
    int im_single;
};

__device__ __forceinline__ Members class_members(const DevParams &P, int c)
{
    Members m;
    int s = c % (P.n_cls / P.n_b);
    if (P.class_sum) {
        m.ie_lo = max(0, s - (P.n_tm - 1));
        m.ie_hi = min(s, P.n_te - 1);
        m.s = s;
        m.im_single = -1;
    } else {
        m.ie_lo = m.ie_hi = s / P.n_tm;
        m.im_single = s % P.n_tm;
        m.s = -1;
    }
    return m;
}

__device__ __forceinline__ int member_im(const Members &m, int ie) { return m.im_single >= 0 ? m.im_single : m.s - ie; }

__device__ __forceinline__ int class_of(const DevParams &P, int ie, int im, int b)
{
    return b * (P.n_cls / P.n_b) + (P.class_sum ? (ie + im) : (ie * P.n_tm + im));
}

// Block-wide exclusive scan of three ints per thread (warp shuffles, then
// the warps' totals through buf, which holds 3 ints per warp); returns the
// prefixes and writes the block totals.  Every thread of the block calls it.
__device__ int3 block_exclusive_scan3(int3 x, int *buf, int3 &total)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = (blockDim.x + 31) >> 5;
    int3 inc = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int a = __shfl_up_sync(full, inc.x, off), b = __shfl_up_sync(full, inc.y, off),
                  c = __shfl_up_sync(full, inc.z, off);
        if (lane >= off) {
            inc.x += a;
            inc.y += b;
            inc.z += c;
        }
    }
    if (lane == 31) {
        buf[3 * warp] = inc.x;
        buf[3 * warp + 1] = inc.y;
        buf[3 * warp + 2] = inc.z;
    }
    __syncthreads();
    int3 base = make_int3(0, 0, 0);
    total = make_int3(0, 0, 0);
    for (int w = 0; w < n_warps; ++w) {
        const int3 t = make_int3(buf[3 * w], buf[3 * w + 1], buf[3 * w + 2]);
        if (w < warp) {
            base.x += t.x;
            base.y += t.y;
            base.z += t.z;
        }
        total.x += t.x;
        total.y += t.y;
        total.z += t.z;
    }
    __syncthreads();  // buf is reused by the next call
    return make_int3(base.x + inc.x - x.x, base.y + inc.y - x.y, base.z + inc.z - x.z);
}

// Shared per-control result.  next and below link the members of one (class,
// shift bucket) into the sorted order and the envelope stack of
// class_envelopes (-1 ends a list): each control belongs to one bucket, and
// one thread builds that bucket's lists.
struct CtrlRec {
    float cost, f;
    short d;     // SoC shift, clamped to the 16-bit range (any |d| > 2 is a rare "other" shift)
    short ok;    // 1 feasible, 2 feasible and on its bucket's lower envelope
    short next;  // sorted order
    short below; // envelope stack
};
static_assert(sizeof(CtrlRec) == 16, "16-byte per-control records");

// Lower envelope of the lines y_u(x) = cost_u + f_u x over all real x, for
// the feasible members of class c with SoC shift d (bucket d + 2): marks the
// members on the envelope with ok = 2 and returns their count.  For one
// state, all controls of the bucket read the same two blended values G_lo,
// G_hi of J_{k+1} (Eq. 9b), and the interpolated value is
// G_lo + (cost_u + f_u (G_hi - G_lo)); its minimum over the bucket is
// G_lo + envelope(G_hi - G_lo).  Lines sorted by slope f descending (ties:
// lower cost, then lower u, first); a line between two others is dropped only
// when it lies on or above their lower envelope everywhere by a clear margin,
// so FP32 rounding never drops a line that is lowest over a real interval.
// (f desc, cost asc, u asc): o (control ou) comes before r (control u)
__device__ __forceinline__ bool line_before(const CtrlRec &o, int ou, const CtrlRec &r, int u)
{
    return o.f > r.f || (o.f == r.f && (o.cost < r.cost || (o.cost == r.cost && ou < u)));
}

// 16-bit field q of a packed word (signed: -1 ends a list)
__device__ __forceinline__ int field16(unsigned long long w, int q) { return (int)(short)((w >> (16 * q)) & 0xffffu); }

__device__ __forceinline__ unsigned long long with_field16(unsigned long long w, int q, int v)
{
    const int sh = 16 * q;
    return (w & ~(0xffffull << sh)) | ((unsigned long long)(v & 0xffff) << sh);
}

// The lower envelope of one bucket's sorted list (head, m members), the
// stack linked through below; marks its lines with ok = 2.
__device__ int bucket_hull(const DevParams &P, int head, int m, CtrlRec *s_ctrl)
{
    int top = -1, n = 0;
    int u = head;
    for (int g = 0; g < m && DP_IN(u, P.n_u); ++g, u = s_ctrl[u].next) {
        const CtrlRec C = s_ctrl[u];
        if (n > 0 && s_ctrl[top].f == C.f)
            continue;  // same slope, not lower: never strictly below the kept line
        while (n >= 2) {
            const int bu = top, au = s_ctrl[top].below;
            if (!DP_IN(au, P.n_u))
                break;
            const CtrlRec A = s_ctrl[au], B = s_ctrl[bu];
            // B is redundant iff x(A, C) <= x(A, B):
            // (c_C - c_A)(f_A - f_B) <= (c_B - c_A)(f_A - f_C), denominators > 0
            const float lhs = __fmul_rn(__fsub_rn(C.cost, A.cost), __fsub_rn(A.f, B.f));
            const float rhs = __fmul_rn(__fsub_rn(B.cost, A.cost), __fsub_rn(A.f, C.f));
            const float tol = __fmul_rn(1e-5f, __fadd_rn(fabsf(lhs), fabsf(rhs)));
            if (lhs < __fsub_rn(rhs, tol)) {
                top = au;
                --n;
            } else {
                break;
            }
        }
        s_ctrl[u].below = (short)top;
        top = u;
        ++n;
    }
    for (int g = 0, q = top; g < n && DP_IN(q, P.n_u); ++g, q = s_ctrl[q].below)
        s_ctrl[q].ok = 2;
    return n;
}

// The lower envelopes of the four shift buckets d = -2 .. 1 of one torque
// class (brake flag b): one pass over the members sorts each bucket's
// feasible members by (f desc, cost asc, u asc) into a list linked through
// next (heads, tails and counts packed per bucket), then each bucket's hull.
// Members arrive in decreasing engine torque: within a class and shift
// bucket the SoC fraction f falls with the motor share, so most append at
// their list's tail (O(1) each); the others walk from the head.
__device__ void class_envelopes(const DevParams &P, const Members &mem, int b, CtrlRec *s_ctrl)
{
    unsigned long long heads = ~0ull, tails = ~0ull;  // every list empty (-1)
    unsigned counts = 0u;  // 8 bits per bucket: a class has at most min(n_te, n_tm) <= 90 members (8192 controls)
    for (int ie = mem.ie_hi; ie >= mem.ie_lo; --ie) {
        const int u = (ie * P.n_tm + member_im(mem, ie)) * P.n_b + b;
        if (!DP_IN(u, P.n_u))
            continue;
        const CtrlRec r = s_ctrl[u];
        if (!r.ok || r.d < -2 || r.d > 1)
            continue;
        const int q = r.d + 2;
        const int m = (int)((counts >> (8 * q)) & 0xffu) + 1;
        counts += 1u << (8 * q);
        const int tail = field16(tails, q);
        if (tail < 0 || line_before(s_ctrl[tail], tail, r, u)) {
            s_ctrl[u].next = -1;
            if (tail < 0)
                heads = with_field16(heads, q, u);
            else
                s_ctrl[tail].next = (short)u;
            tails = with_field16(tails, q, u);
            continue;
        }
        int prev = -1, cur = field16(heads, q);
        for (int g = 0; g < m && DP_IN(cur, P.n_u) && line_before(s_ctrl[cur], cur, r, u); ++g) {
            prev = cur;
            cur = s_ctrl[cur].next;
        }
        s_ctrl[u].next = (short)cur;
        if (prev < 0)
            heads = with_field16(heads, q, u);
        else
            s_ctrl[prev].next = (short)u;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int m = (int)((counts >> (8 * q)) & 0xffu);
        if (m > 0)
            bucket_hull(P, field16(heads, q), m, s_ctrl);
    }
}

// Tables of speed row i of stage k (one CTA; P in shared memory).
__device__ void precompute_row(const DevParams &P, const StageTables &tb, int k, int i, const StageScratch &sc,
                               CtrlRec *s_ctrl, int *scan_buf)
{
    const float v = node_val(P.v_lo, P.v_span, i, P.n_v);
    const float p = tb.grade[k];
    const float sq = __fsqrt_rn(__fadd_rn(1.f, __fmul_rn(p, p)));
    const float sin_th = __fdiv_rn(p, sq), cos_th = __fdiv_rn(1.f, sq);
    const float F_road = road_load(P, v, sin_th, cos_th);
    const bool next_light = tb.light_of_node[k + 1] >= 0;
    const float w = __fmul_rn(v, P.ratio);
    const float one_m_gamma = __fsub_rn(1.f, P.gamma);

    // standing at a light node under the literal Eq. 5c (light_model 2)
    const bool stand = P.light_model == 2 && v == 0.f && tb.light_of_node[k] >= 0;
    const size_t row = (size_t)k * P.n_v + i;
    if (!DP_IN(row, (size_t)P.N * P.n_v))
        return;
    ClassRec *cls_row = sc.cls + row * P.n_cls;
    ClassEntry *ent_row = sc.ent + row * P.n_cls;
    SplitRec *spl_row = sc.spl + row * P.n_u;

    // 1. classes: speed update, step time, speed-axis band and interpolation
    for (int c = threadIdx.x; c < P.n_cls; c += blockDim.x) {
        const int b = c / (P.n_cls / P.n_b);
        const Members mem = class_members(P, c);
        const int ie0 = mem.ie_lo, im0 = member_im(mem, ie0);
        const float T =
            __fadd_rn(node_val(P.te_lo, P.te_span, ie0, P.n_te), node_val(P.tm_lo, P.tm_span, im0, P.n_tm));
        ClassRec rec = {};
        float v1 = 0.f, dt = 0.f;
        if (stand && standstill_class(P, F_road, T, b)) {
            // zero-speed step: v' = 0 (speed row 0), no driving time; the
            // time jump to the end of red is taken per time node by the tile
            rec.ok = 1;
            cls_row[c] = rec;
            continue;
        }
        bool ok = speed_step(P, v, F_road, T, b, next_light, v1, dt);
        if (ok) {
            float qv = __fdiv_rn(__fsub_rn(v1, P.v_lo), P.h_v);
            float top = (float)(P.n_v - 1);
            if (qv < -SNAP || qv > top + SNAP)
                ok = false;
            qv = fminf(fmaxf(qv, 0.f), top);
            int iv;
            float fv;
            snap_split(qv, iv, fv);
            if (iv >= P.n_v - 1) {
                iv = P.n_v - 2;
                fv = 1.f;
            }
            int st;
            float ft;
            snap_split(__fdiv_rn(dt, P.h_t), st, ft);
            rec.iv = iv;
            rec.fv = fv;
            rec.v1 = v1;
            rec.dt = dt;
            rec.st = st;
            rec.ft = ft;
        }
        rec.ok = ok;
        cls_row[c] = rec;
    }
    __syncthreads();

    // 2. controls: battery (Eq. 5b), SoC shift, stage cost (Eq. 1/6)
    for (int u = threadIdx.x; u < P.n_u; u += blockDim.x) {
        int ie, im, b;
        decode_u(P, u, ie, im, b);
        const int cu = class_of(P, ie, im, b);
        const ClassRec C = DP_IN(cu, P.n_cls) ? cls_row[cu] : ClassRec{};
        CtrlRec r = {0.f, 0.f, 0, 0, -1, -1};
        float I;
        const float Tm = node_val(P.tm_lo, P.tm_span, im, P.n_tm);
        const float Te = node_val(P.te_lo, P.te_span, ie, P.n_te);
        // the zero-speed step has the engine off (start-stop)
        const bool engine_ok = !(stand && C.v1 == 0.f && C.dt == 0.f) || Te == 0.f;
        if (C.ok && engine_ok && torque_allowed(P, w, Te, Tm) && battery_current(P, w, Tm, I)) {
            const float dxi = __fdiv_rn(__fmul_rn(C.dt, I), P.cap);
            int d;
            snap_split(__fdiv_rn(-dxi, P.h_xi), d, r.f);
            r.d = (short)min(max(d, -32768), 32767);
            const float mf = fuel_rate(P, w, Te);
            r.cost = __fmul_rn(__fadd_rn(__fmul_rn(P.gamma, mf), one_m_gamma), C.dt);
            r.ok = 1;
        }
        s_ctrl[u] = r;
    }
    __syncthreads();

    // 3. the lower envelopes of every class's SoC-shift buckets d in {-2, -1,
    // 0, 1}, one class per task (members are disjoint).  Tasks are ranked by
    // decreasing class size (the total torques nearest the middle of their
    // range first) and dealt out in a snake, so a thread's heavy task of one
    // round pairs with a light one of the next.
    const int n_sum = P.n_cls / P.n_b;
    for (int k = 0;; ++k) {
        const int task = k * blockDim.x + ((k & 1) ? blockDim.x - 1 - threadIdx.x : threadIdx.x);
        if (k * blockDim.x >= P.n_cls)
            break;
        if (task >= P.n_cls)
            continue;
        const int b = task % P.n_b, q = task / P.n_b, mid = (n_sum - 1) / 2;
        const int c = b * n_sum + mid + ((q & 1) ? (q + 1) / 2 : -(q / 2));
        const Members mem = class_members(P, c);
        if (!P.all_lines) {
            class_envelopes(P, mem, b, s_ctrl);
            continue;
        }
        // the cross-check setting: every feasible member of a bucket is a line
        for (int ie = mem.ie_lo; ie <= mem.ie_hi; ++ie) {
            const int u = (ie * P.n_tm + member_im(mem, ie)) * P.n_b + b;
            if (DP_IN(u, P.n_u) && s_ctrl[u].ok && s_ctrl[u].d >= -2 && s_ctrl[u].d <= 1)
                s_ctrl[u].ok = 2;
        }
    }
    __syncthreads();

    // 4. compact the feasible classes: the envelope lines of each bucket, then
    // every control of any other shift (rare: one SoC step is far larger than
    // a step's charge change)
    // Member buckets: 0..3 the envelope lines of shift d = bucket - 2, 4 any
    // other shift, -1 none (infeasible, or in a bucket but off its envelope).
    // Per class one pass counts the buckets (one byte each of a 64-bit word;
    // a class has fewer than 256 members) and a second writes the lines.
    auto member_bucket = [](const CtrlRec &r) -> int {
        if (!r.ok)
            return -1;
        if (r.d >= -2 && r.d <= 1)
            return r.ok == 2 ? r.d + 2 : -1;
        return 4;
    };
    int ent_carry = 0, spl_carry = 0, feas_carry = 0;
    for (int c0 = 0; c0 < P.n_cls; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        Members mem = {};
        int nfeas = 0;
        unsigned long long cnt = 0;  // byte q: lines of bucket q
        if (c < P.n_cls) {
            mem = class_members(P, c);
            const int b = c / (P.n_cls / P.n_b);
            for (int ie = mem.ie_lo; ie <= mem.ie_hi; ++ie) {
                const int u = (ie * P.n_tm + member_im(mem, ie)) * P.n_b + b;
                const CtrlRec r = DP_IN(u, P.n_u) ? s_ctrl[u] : CtrlRec{0.f, 0.f, 0, 0, -1, -1};
                nfeas += r.ok ? 1 : 0;
                const int q = member_bucket(r);
                if (q >= 0)
                    cnt += 1ull << (8 * q);
            }
        }
        // bytes 0..4 of `first`: the first line of each bucket, relative to the
        // class (exclusive prefix sums of the counts; no byte carries, the sums
        // stay below 256); byte 5: all lines of the class
        const unsigned long long first = (cnt * 0x0101010101ull) << 8;
        const int nspl = (int)((first >> 40) & 0xff);
        const int feas = nfeas > 0 ? 1 : 0;
        int3 tot;
        const int3 pre = block_exclusive_scan3(make_int3(feas, nspl, nfeas), scan_buf, tot);
        const int ent_idx = pre.x + ent_carry, spl_off = pre.y + spl_carry;
        const int ent_tot = tot.x, spl_tot = tot.y, feas_tot = tot.z;
        if (feas) {
            const int b = c / (P.n_cls / P.n_b);
            ClassEntry E;
            E.cls = c;
            E.off = spl_off;
            E.n_total = nspl;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                E.nb[q] = (int)((cnt >> (8 * q)) & 0xff);
            E.n_other = (int)((cnt >> 32) & 0xff);
            unsigned long long next = first;  // byte q: next line of bucket q
            for (int ie = mem.ie_lo; ie <= mem.ie_hi; ++ie) {
                const int u = (ie * P.n_tm + member_im(mem, ie)) * P.n_b + b;
                const CtrlRec r = DP_IN(u, P.n_u) ? s_ctrl[u] : CtrlRec{0.f, 0.f, 0, 0, -1, -1};
                const int q = member_bucket(r);
                if (q < 0)
                    continue;
                const int pos = spl_off + (int)((next >> (8 * q)) & 0xff);
                next += 1ull << (8 * q);
                const unsigned bits = (unsigned)(u & 0xffff) | ((unsigned)(r.d & 0xffff) << 16);
                if (DP_IN(pos, P.n_u))
                    spl_row[pos] = SplitRec{r.cost, r.f, bits, 0u};
            }
            if (DP_IN(ent_idx, P.n_cls))
                ent_row[ent_idx] = E;
        }
        ent_carry += ent_tot;
        spl_carry += spl_tot;
        feas_carry += feas_tot;
    }
    if (threadIdx.x == 0) {
        sc.row_cnt[2 * row] = ent_carry;
        sc.row_cnt[2 * row + 1] = spl_carry;
        if (sc.stats) {
            atomicAdd(sc.stats, (unsigned long long)feas_carry);
            atomicAdd(sc.stats + 1, (unsigned long long)ent_carry);
            atomicAdd(sc.stats + 4, (unsigned long long)spl_carry);
        }
    }
}

// 128 threads (the per-class phases keep ~1 class per thread busy at the
// paper-scale 122 classes) and 7 CTAs per SM: each holds the row's control
// table (16 bytes per control, 31 KB at 1922 controls) in shared memory
__global__ void __launch_bounds__(128, 7) precompute_kernel(const DevParams *__restrict__ dP, StageTables tb,
                                                         int k_first, StageScratch sc)
{
    extern __shared__ __align__(16) unsigned char pre_smem[];
    __shared__ DevParams P;
    __shared__ int scan_buf[256];
    if (threadIdx.x == 0)
        P = *dP;
    __syncthreads();
    precompute_row(P, tb, k_first + blockIdx.y, blockIdx.x, sc, reinterpret_cast<CtrlRec *>(pre_smem), scan_buf);
}

// Batched: one CTA per (instance, stage, speed row); blocks of instance b
// start at inst[b].row_off (rows of all its stages, stage-major).
__global__ void __launch_bounds__(256, 5) precompute_batched_kernel(const DevParams *__restrict__ params,
                                                                 const BatchInst *__restrict__ inst, int n_inst)
{
    extern __shared__ __align__(16) unsigned char pre_smem[];
    __shared__ DevParams P;
    __shared__ int scan_buf[256];
    __shared__ int s_b;
    const long long blk = blockIdx.x;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_inst - 1;  // last instance with row_off <= blk
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (inst[mid].row_off <= blk)
                lo = mid;
            else
                hi = mid - 1;
        }
        s_b = lo;
        P = params[lo];
    }
    __syncthreads();
    const BatchInst &I = inst[s_b];
    const long long r = blk - I.row_off;
    if (!DP_IN(r, (long long)P.N * P.n_v))
        return;
    precompute_row(P, I.tb, (int)(r / P.n_v), (int)(r % P.n_v), I.sc, reinterpret_cast<CtrlRec *>(pre_smem),
                   scan_buf);
}

// Batched terminal values J_N = c_T for every instance (grid-stride over instances' states).
__global__ void terminal_batched_kernel(const DevParams *__restrict__ params, const BatchInst *__restrict__ inst,
                                        int n_inst)
{
    const int b = blockIdx.y;
    if (b >= n_inst)
        return;
    const DevParams &P = params[b];
    const BatchInst &I = inst[b];
    float *VN = I.V + (size_t)P.N * I.stage_elems;
    const int total = P.n_v * P.n_xi * P.n_t;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < total; s += gridDim.x * blockDim.x) {
        const int l = s % P.n_t;
        const int j = (s / P.n_t) % P.n_xi;
        const int i = s / (P.n_t * P.n_xi);
        const size_t o = ((size_t)i * P.xi_rows + (j + 1)) * P.ld_t + l;
        if (DP_IN(o, (size_t)P.n_v * P.xi_rows * P.ld_t))
            VN[o] = terminal_cost(P, node_val(P.v_lo, P.v_span, i, P.n_v), node_val(P.xi_lo, P.xi_span, j, P.n_xi));
    }
}

}  // namespace

cudaError_t launch_precompute_batched(const DevParams *params, const BatchInst *inst, int n_inst, long long n_rows,
                                      int max_n_u, cudaStream_t s)
{
    const size_t smem = (size_t)max_n_u * sizeof(CtrlRec);
    cudaError_t err =
        cudaFuncSetAttribute(precompute_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess)
        return err;
    precompute_batched_kernel<<<(unsigned)n_rows, 256, smem, s>>>(params, inst, n_inst);
    return cudaGetLastError();
}

cudaError_t launch_terminal_batched(const DevParams *params, const BatchInst *inst, int n_inst, cudaStream_t s)
{
    terminal_batched_kernel<<<dim3(64, n_inst), 256, 0, s>>>(params, inst, n_inst);
    return cudaGetLastError();
}

cudaError_t launch_fill(float *p, size_t n, float val, cudaStream_t s)
{
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16)
        blocks = 152 * 16;
    if (blocks < 1)
        blocks = 1;
    fill_kernel<<<blocks, 256, 0, s>>>(p, n, val);
    return cudaGetLastError();
}

cudaError_t launch_terminal(const DevParams *dP, const DevParams &hP, float *VN, cudaStream_t s)
{
    int total = hP.n_v * hP.n_xi * hP.n_t;
    int blocks = (total + 255) / 256;
    terminal_kernel<<<blocks, 256, 0, s>>>(dP, VN);
    return cudaGetLastError();
}

cudaError_t launch_precompute(const DevParams *dP, const DevParams &hP, StageTables tb, int k_first, int n_k,
                              StageScratch sc, cudaStream_t s)
{
    const size_t smem = (size_t)hP.n_u * sizeof(CtrlRec);
    cudaError_t err = cudaFuncSetAttribute(precompute_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess)
        return err;
    precompute_kernel<<<dim3(hP.n_v, n_k), 128, smem, s>>>(dP, tb, k_first, sc);
    return cudaGetLastError();
}

cudaError_t launch_pad_from_dense(const DevParams &hP, const float *dense, float *padded, cudaStream_t s)
{
    int total = hP.n_v * hP.n_xi * hP.n_t;
    pad_from_dense_kernel<<<(total + 255) / 256, 256, 0, s>>>(hP, dense, padded);
    return cudaGetLastError();
}

cudaError_t launch_quad_from_pad(const DevParams &hP, const float *V, float4 *Q, cudaStream_t s)
{
    if (quad_ld(hP.n_t) == 0)
        return cudaSuccess;  // no quads for this time grid
    const size_t total = (size_t)hP.n_v * quad_rows(hP.n_xi) * quad_ld(hP.n_t);
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
    quad_from_pad_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, s>>>(hP, V, Q);
    return cudaGetLastError();
}

cudaError_t launch_dense_from_pad(const DevParams &hP, const float *padded, float *dense, cudaStream_t s)
{
    int total = hP.n_v * hP.n_xi * hP.n_t;
    dense_from_pad_kernel<<<(total + 255) / 256, 256, 0, s>>>(hP, padded, dense);
    return cudaGetLastError();
}

}  // namespace ecodp
