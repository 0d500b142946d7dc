// Adjoint: dJ_0(x0)/dtheta for theta = (mass, CdA, Crr, R0, fuel-map scale).
//
// With the argmin pi_k fixed (envelope theorem), J_k(s) = c(s, u*) +
// I_{k+1}[J_{k+1}](f(s, u*)) where I is the trilinear interpolant, so
//   dJ_0(x0)/dtheta = sum_k sum_s lam_k(s) [dc/dtheta + grad I . df/dtheta],
//   lam_0 = interpolation weights of x0, lam_{k+1}(n) = sum_s lam_k(s) w_n(f(s, pi_k(s))).
// One launch per stage walks the states of stage k, skips those with
// lam = 0, re-evaluates the step at the stored argmin with its derivatives
// (Eq. 2, 5a, 5b, 6 differentiated through a, v', dt, I and the fuel map) in
// FP32, scatters lam to the successor's corners and accumulates the gradient
// in FP64.
#include "ecodp_internal.cuh"

#undef ECODP_FILE_TAG
#define ECODP_FILE_TAG 4

namespace ecodp {

ECODP_CHECK_ACCESSOR(check_word_adjoint)

namespace {

struct DStep {
    float v1, xi1, t1;
    float dv1[5], dxi1[5], dt1[5], dcost[5];
};

__device__ bool step_grad(const DevParams &P, const StageTables &tb, int k, float v, float xi, float t, int u,
                          DStep &o)
{
    int ie, im, b;
    decode_u(P, u, ie, im, b);
    const float Te = node_val(P.te_lo, P.te_span, ie, P.n_te);
    const float Tm = node_val(P.tm_lo, P.tm_span, im, P.n_tm);
    const float T = __fadd_rn(Te, Tm);
    const float p = tb.grade[k];
    const float sq = __fsqrt_rn(__fadd_rn(1.f, __fmul_rn(p, p)));
    const float cos_th = __fdiv_rn(1.f, sq);
    const float F_road = road_load(P, v, __fdiv_rn(p, sq), cos_th);
    const int nl = tb.light_of_node[k + 1];
    int lk = tb.light_of_node[k];
    if (!DP_IN(lk + 1, P.n_lights + 1))
        lk = -1;
    if (P.light_model == 2 && lk >= 0 && v == 0.f) {
        // literal Eq. 5c at the line: the zero-speed step has no theta
        // dependence (v' = 0, SoC kept, time jump to the end of red)
        const float ph = phase_pos(t, tb.offset[lk], tb.cycle[lk]);
        const float wait = ph < tb.red[lk] ? __fsub_rn(tb.red[lk], ph) : 0.f;
        if (standstill_class(P, F_road, T, b)) {
            if (Te != 0.f || !torque_allowed(P, 0.f, Te, Tm))
                return false;
            for (int q = 0; q < 5; ++q)
                o.dv1[q] = o.dxi1[q] = o.dt1[q] = o.dcost[q] = 0.f;
            o.v1 = 0.f;
            o.xi1 = xi;
            o.t1 = __fadd_rn(t, wait);
            return true;
        }
        if (wait > 0.f)
            return false;
    }
    float v1, dt;
    if (!speed_step(P, v, F_road, T, b, nl >= 0, v1, dt))
        return false;
    float wait = 0.f;
    if (P.light_model != 2 && lk >= 0 && v == 0.f) {
        const float ph = phase_pos(t, tb.offset[lk], tb.cycle[lk]);
        if (ph < tb.red[lk])
            wait = __fsub_rn(tb.red[lk], ph);
    }
    const float w = __fmul_rn(v, P.ratio);
    float I;
    if (!battery_current(P, w, Tm, I))
        return false;
    const float mf = fuel_rate(P, w, Te);
    // derivatives of the acceleration (Eq. 5a): a = T r / M - b g_b - g (Crr cos + sin) - rho CdA v^2 / (2 M)
    const float M = P.mass;
    float da[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    da[0] = -__fdiv_rn(__fsub_rn(__fmul_rn(T, P.ratio), __fmul_rn(P.half_rho_cda, __fmul_rn(v, v))), __fmul_rn(M, M));
    da[1] = -__fdiv_rn(__fmul_rn(P.half_rho, __fmul_rn(v, v)), M);
    da[2] = -__fmul_rn(P.g, cos_th);
    float ddt[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int q = 0; q < 5; ++q)
        o.dv1[q] = 0.f;
    if (v1 > 0.f) {
        const float vs = __fadd_rn(v, v1);
        for (int q = 0; q < 5; ++q) {
            o.dv1[q] = __fdiv_rn(__fmul_rn(P.ds, da[q]), v1);
            ddt[q] = -__fmul_rn(__fdiv_rn(dt, vs), o.dv1[q]);
        }
    }
    // battery current and its R0 derivative (Eq. 5b), with P the battery power:
    // I = 2P / (Voc + sqrt(D)), D = Voc^2 - 4 R0 P, so
    // dI/dR0 = 4 P^2 / ((Voc + sqrt(D))^2 sqrt(D)), free of cancellation
    const float Pm = __fmul_rn(Tm, w);
    const float Pb = Pm > 0.f ? __fdiv_rn(Pm, P.eta) : __fmul_rn(Pm, P.eta);
    const float sD = __fsqrt_rn(fmaxf(__fsub_rn(__fmul_rn(P.voc, P.voc), __fmul_rn(__fmul_rn(4.f, P.r0), Pb)), 0.f));
    const float den = __fadd_rn(P.voc, sD);
    const float dI_dR0 =
        sD > 0.f ? __fdiv_rn(__fmul_rn(4.f, __fmul_rn(Pb, Pb)), __fmul_rn(__fmul_rn(den, den), sD)) : 0.f;
    const float poly = (P.fuel_scale != 0.f) ? __fdiv_rn(mf, P.fuel_scale) : 0.f;
    const float gmf = __fadd_rn(__fmul_rn(P.gamma, mf), __fsub_rn(1.f, P.gamma));
    for (int q = 0; q < 5; ++q) {
        const float dI = q == 3 ? dI_dR0 : 0.f;
        const float dmf = q == 4 ? poly : 0.f;
        o.dt1[q] = ddt[q];
        o.dxi1[q] = -__fdiv_rn(__fadd_rn(__fmul_rn(ddt[q], I), __fmul_rn(dt, dI)), P.cap);
        o.dcost[q] = __fadd_rn(__fmul_rn(gmf, ddt[q]), __fmul_rn(__fmul_rn(P.gamma, dmf), dt));
    }
    o.v1 = v1;
    o.xi1 = __fsub_rn(xi, __fdiv_rn(__fmul_rn(dt, I), P.cap));
    o.t1 = __fadd_rn(__fadd_rn(t, wait), dt);
    return true;
}

struct Interp {
    size_t corner[8];  // padded offsets of the 8 corners
    float w[8];
    float grad[3];
    bool bad;          // an infeasible corner entered the value or the gradient
};

// Locate x on a uniform axis: band check, clamp, snap; `snapped` if the
// fraction was moved to a node.
__device__ __forceinline__ bool locate_axis(float x, float lo, float h, int n, int &i, float &f, bool &snapped)
{
    float q = __fdiv_rn(__fsub_rn(x, lo), h);
    const float top = (float)(n - 1);
    if (q < -SNAP || q > top + SNAP)
        return false;
    q = fminf(fmaxf(q, 0.f), top);
    const float fl = floorf(q);
    const float raw = __fsub_rn(q, fl);
    snap_split(q, i, f);
    snapped = !(i == (int)fl && f == raw);
    if (i >= n - 1) {
        i = n - 2;
        f = 1.f;
    }
    return true;
}

__device__ bool interp_grad(const DevParams &P, const float *__restrict__ V, float v, float xi, float t, Interp &r)
{
    int iv, ix, it;
    float fv, fx, ft;
    bool sv, sx, st;
    if (!locate_axis(v, P.v_lo, P.h_v, P.n_v, iv, fv, sv) || !locate_axis(xi, P.xi_lo, P.h_xi, P.n_xi, ix, fx, sx) ||
        !locate_axis(t, P.t_lo, P.h_t, P.n_t, it, ft, st))
        return false;
    const float f[3] = {fv, fx, ft};
    const float h[3] = {P.h_v, P.h_xi, P.h_t};
    const bool snap[3] = {sv, sx, st};
    float val[8];
    r.bad = false;
    for (int q = 0; q < 8; ++q) {
        const int a = (q >> 2) & 1, b = (q >> 1) & 1, c = q & 1;
        r.corner[q] = ((size_t)(iv + a) * P.xi_rows + (ix + b + 1)) * P.ld_t + (it + c);
        r.w[q] = __fmul_rn(__fmul_rn(a ? fv : __fsub_rn(1.f, fv), b ? fx : __fsub_rn(1.f, fx)),
                           c ? ft : __fsub_rn(1.f, ft));
        if (!DP_IN(r.corner[q], (size_t)P.n_v * P.xi_rows * P.ld_t)) {
            r.corner[q] = 0;
            r.w[q] = 0.f;
        }
        val[q] = V[r.corner[q]];
        if (r.w[q] != 0.f && !(val[q] < V_FEAS_MAX))
            r.bad = true;
    }
    for (int ax = 0; ax < 3; ++ax) {
        float g = 0.f;
        if (!snap[ax]) {
            const int bit = 1 << (2 - ax);
            for (int q = 0; q < 8; ++q) {
                if (!(q & bit))
                    continue;
                float wo = 1.f;
                for (int o = 0; o < 3; ++o) {
                    if (o == ax)
                        continue;
                    const int bo = (q >> (2 - o)) & 1;
                    wo = __fmul_rn(wo, bo ? f[o] : __fsub_rn(1.f, f[o]));
                }
                if (wo == 0.f)
                    continue;
                const float hi = val[q], lo = val[q & ~bit];
                if (!(hi < V_FEAS_MAX) || !(lo < V_FEAS_MAX)) {
                    r.bad = true;
                    continue;
                }
                g = __fmaf_rn(wo, __fdiv_rn(__fsub_rn(hi, lo), h[ax]), g);
            }
        }
        r.grad[ax] = g;
    }
    return true;
}

// Appends state sn to the support list of parity par unless it is listed.
__device__ __forceinline__ void frontier_add(const AdjFrontier &F, int par, int cnt_slot, size_t n, int sn)
{
    const unsigned bit = 1u << (sn & 31);
    if (!DP_IN(sn, n) || (atomicOr(F.bits + par * F.words + (sn >> 5), bit) & bit))
        return;
    const int pos = atomicAdd(F.cnt + cnt_slot, 1);
    if (DP_IN(pos, n))
        F.idx[par * n + pos] = sn;
}

// lam_0 = interpolation weights of x0 on the stage-0 grid (and its support
// list); also J_0(x0).
__global__ void adjoint_init_kernel(const DevParams *__restrict__ dP, const float *__restrict__ V0, double v0,
                                    double xi0, double t0, double *__restrict__ lam0, AdjFrontier F,
                                    double *__restrict__ out)
{
    const DevParams &P = *dP;
    const size_t n = (size_t)P.n_v * P.n_xi * P.n_t;
    F.cnt[0] = F.cnt[1] = F.cnt[2] = 0;
    Interp r;
    if (!interp_grad(P, V0, (float)v0, (float)xi0, (float)t0, r)) {
        out[6] = 1.0;  // x0 off the grid
        return;
    }
    // only the corners with non-zero weight enter J_0(x0) and lam_0 (x0 does
    // not depend on theta, so the slopes of the interpolant there are unused):
    // an infeasible neighbour that only the slopes would read is no failure
    double J = 0.0;
    bool value_bad = false;
    for (int q = 0; q < 8; ++q) {
        if (r.w[q] == 0.f)
            continue;
        if (!(V0[r.corner[q]] < V_FEAS_MAX))
            value_bad = true;
        const size_t s = (r.corner[q] / P.ld_t / P.xi_rows) * (size_t)P.n_xi * P.n_t +
                         ((r.corner[q] / P.ld_t) % P.xi_rows - 1) * (size_t)P.n_t + r.corner[q] % P.ld_t;
        if (!DP_IN(s, n))
            continue;
        lam0[s] += (double)r.w[q];
        frontier_add(F, 0, 0, n, (int)s);
        J += (double)r.w[q] * (double)V0[r.corner[q]];
    }
    out[5] = value_bad ? __longlong_as_double(0x7ff0000000000000LL) : J;
    if (value_bad)
        out[6] = 2.0;
}

// Stage k of the forward lam sweep over the support list of lam_k: each
// listed state re-evaluates its step at the stored argmin, scatters its
// weight to the successor's corners (listing new ones for stage k + 1),
// leaves its lam_k entry and list bit at zero for stage k + 2, and adds its
// gradient terms.
__global__ void __launch_bounds__(256) adjoint_stage_kernel(const DevParams *__restrict__ dP, StageTables tb, int k,
                                                            const float *__restrict__ Vn,
                                                            const int16_t *__restrict__ pik,
                                                            double *__restrict__ lam_k,
                                                            double *__restrict__ lam_k1, AdjFrontier F,
                                                            double *__restrict__ out)
{
    __shared__ DevParams P;
    if (threadIdx.x == 0)
        P = *dP;
    __syncthreads();
    const size_t n = (size_t)P.n_v * P.n_xi * P.n_t;
    const int par = k & 1, par1 = (k + 1) & 1;
    const int n_list = F.cnt[k % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0)
        F.cnt[(k + 2) % 3] = 0;  // read by stage k - 1, appended to by stage k + 1
    double contrib[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    bool any = false;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < n_list; it += gridDim.x * blockDim.x) {
        if (!DP_IN(it, n))
            break;
        const int s = F.idx[par * n + it];
        if (!DP_IN(s, n))
            continue;
        atomicAnd(F.bits + par * F.words + (s >> 5), ~(1u << (s & 31)));
        const double L = lam_k[s];
        lam_k[s] = 0.0;
        if (L == 0.0)
            continue;
        any = true;
        const int u = pik[s];
        const int l = s % P.n_t, j = (s / P.n_t) % P.n_xi, i = s / (P.n_t * P.n_xi);
        DStep st;
        Interp r;
        if (u < 0 || !step_grad(P, tb, k, node_val(P.v_lo, P.v_span, i, P.n_v), node_val(P.xi_lo, P.xi_span, j, P.n_xi),
                                node_val(P.t_lo, P.t_span, l, P.n_t), u, st) ||
            !interp_grad(P, Vn, st.v1, st.xi1, st.t1, r)) {
            out[6] = 3.0;  // the support reached an infeasible state
            continue;
        }
        if (r.bad)
            out[7] = 1.0;
        for (int q = 0; q < 5; ++q) {
            const float term = __fadd_rn(
                st.dcost[q],
                __fadd_rn(__fmul_rn(r.grad[0], st.dv1[q]),
                          __fadd_rn(__fmul_rn(r.grad[1], st.dxi1[q]), __fmul_rn(r.grad[2], st.dt1[q]))));
            contrib[q] += L * (double)term;
        }
        for (int q = 0; q < 8; ++q) {
            if (r.w[q] == 0.f)
                continue;
            const size_t c = r.corner[q];
            const size_t sn = (c / P.ld_t / P.xi_rows) * (size_t)P.n_xi * P.n_t +
                              ((c / P.ld_t) % P.xi_rows - 1) * (size_t)P.n_t + c % P.ld_t;
            if (!DP_IN(sn, n))
                continue;
            atomicAdd(lam_k1 + sn, L * (double)r.w[q]);
            frontier_add(F, par1, (k + 1) % 3, n, (int)sn);
        }
    }
    // FP64 reduction of the gradient: warp, then one atomic per warp; only
    // warps that held part of the support (FP64 arithmetic is slow here)
    if (!__any_sync(0xffffffffu, any))
        return;
    for (int q = 0; q < 5; ++q) {
        double x = contrib[q];
        for (int off = 16; off > 0; off >>= 1)
            x += __shfl_down_sync(0xffffffffu, x, off);
        if ((threadIdx.x & 31) == 0 && x != 0.0)
            atomicAdd(out + q, x);
    }
}

}  // namespace

// lam_0 from x0 and J_0(x0) (out[5]); clears the gradient, both lam halves
// and both support bitmaps.
cudaError_t launch_adjoint_init(const DevParams *dP, const DevParams &hP, const float *V0, double *lam,
                                AdjFrontier F, double x0, double xi0, double t0, double *out, cudaStream_t s)
{
    const size_t n = (size_t)hP.n_v * hP.n_xi * hP.n_t;
    cudaError_t e = cudaMemsetAsync(out, 0, 8 * sizeof(double), s);
    if (e != cudaSuccess)
        return e;
    e = cudaMemsetAsync(lam, 0, 2 * n * sizeof(double), s);
    if (e != cudaSuccess)
        return e;
    e = cudaMemsetAsync(F.bits, 0, 2 * F.words * sizeof(unsigned), s);
    if (e != cudaSuccess)
        return e;
    adjoint_init_kernel<<<1, 1, 0, s>>>(dP, V0, x0, xi0, t0, lam, F, out);
    return cudaGetLastError();
}

// One stage of the forward lam sweep: lam_{k+1} from lam_k through pi_k and
// the interpolation weights on J_{k+1} (Vn), with the stage's gradient terms.
// lam_{k+1}'s half and its bitmap are all zero on entry (cleared by the init,
// then by the stage that read them two stages earlier).  A fixed grid walks
// the support list, whose length only the device knows.
cudaError_t launch_adjoint_stage(const DevParams *dP, const DevParams &hP, StageTables tb, int k, const float *Vn,
                                 const int16_t *pik, double *lam, AdjFrontier F, double *out, cudaStream_t s)
{
    const size_t n = (size_t)hP.n_v * hP.n_xi * hP.n_t;
    double *lk = lam + (size_t)(k & 1) * n;
    double *lk1 = lam + (size_t)((k + 1) & 1) * n;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 1;
    }
    adjoint_stage_kernel<<<4 * sms, 256, 0, s>>>(dP, tb, k, Vn, pik, lk, lk1, F, out);
    return cudaGetLastError();
}

}  // namespace ecodp
