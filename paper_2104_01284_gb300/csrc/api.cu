// C ABI of the ecodp solver (declared in include/ecodp.h): problem objects,
// validation, device memory through the caller's allocator, the CUDA-graph
// captured backward sweep, result copies and the rollout.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstddef>
#include <cstring>
#include <string>
#include <vector>

#include "api_internal.h"

using namespace ecodp;
using namespace ecodp::host;

namespace ecodp {
size_t bellman_smem_bytes(const DevParams &hP);
cudaError_t launch_adjoint_init(const DevParams *dP, const DevParams &hP, const float *V0, double *lam,
                                AdjFrontier F, double x0, double xi0, double t0, double *out, cudaStream_t s);
cudaError_t launch_adjoint_stage(const DevParams *dP, const DevParams &hP, StageTables tb, int k, const float *Vn,
                                 const int16_t *pik, double *lam, AdjFrontier F, double *out, cudaStream_t s);

namespace host {

namespace {
thread_local std::string g_last_error;
}

dp_status fail(dp_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

const char *last_error() { return g_last_error.c_str(); }

}  // namespace host
}  // namespace ecodp

struct dp_problem {
    int N = 0, n_v = 0, n_xi = 0, n_t = 0, n_u = 0, n_lights = 0;
    DevParams hP{};
    dp_allocator alloc{};
    bool has_alloc = false;
    cudaStream_t create_stream = nullptr;
    std::vector<void *> blocks;
    size_t bytes_held = 0;

    DevParams *dP = nullptr;
    float *d_grade = nullptr;
    int *d_lon = nullptr;
    float *d_cyc = nullptr, *d_red = nullptr, *d_off = nullptr;
    float *d_V = nullptr;
    size_t stage_elems = 0;
    int16_t *d_pi = nullptr;
    size_t pi_elems = 0;
    ClassRec *d_cls = nullptr;
    ClassEntry *d_ent = nullptr;
    int *d_rowcnt = nullptr;
    SplitRec *d_spl = nullptr;
    float *d_pad_in = nullptr, *d_pad_out = nullptr, *d_dense = nullptr;
    // corner quads of J_k for the tiled sweep, two slots by stage parity
    // (quad_rows x quad_ld per speed row, none when quad_ld is 0); entries
    // outside the grid hold V_BIG for the object's life
    float4 *d_quad = nullptr;
    size_t quad_elems = 0;
    float4 *quad(int k) const { return d_quad ? d_quad + (size_t)(k & 1) * quad_elems : nullptr; }
    int16_t *d_pi_tmp = nullptr;
    double *d_roll = nullptr;
    int *d_roll_u = nullptr;
    unsigned long long *d_stats = nullptr;
    int *d_lmax = nullptr;  // [N + 1] last feasible time column per stage of the last sweep
    bool fill_slots = true;  // the sweep's tiles fill every resident CTA slot (a solve that runs alone)
    double *d_lam = nullptr;  // adjoint weights of two consecutive stages
    int *d_front = nullptr;   // adjoint support lists (AdjFrontier)
    unsigned *d_fbits = nullptr;
    int *d_fcnt = nullptr;
    AdjFrontier frontier() const
    {
        const size_t words = (pi_elems + 31) / 32;
        return AdjFrontier{d_front, d_fbits, d_fcnt, words};
    }
    double *d_adj = nullptr;  // adjoint output: gradient[5], J_0(x0), error code, flag

    HostTables h;  // host copies of the tables (kept until the next update)

    bool solved = false;
    int variant = 1;
    cudaStream_t cap_stream = nullptr;
    // A dp_rollout that follows the solve on its stream (no other call on the
    // problem in between) needs J_1 .. J_N only: the sweep records ev_stage1
    // once J_1 is written, the rollout runs on roll_stream from there while
    // the last Bellman stage finishes, and the caller's stream waits for it.
    cudaEvent_t ev_stage1 = nullptr, ev_rolled = nullptr;
    cudaStream_t roll_stream = nullptr;
    cudaStream_t solve_stream = nullptr;
    bool rollout_may_overlap = false;
    cudaGraphExec_t gexec = nullptr;
    bool use_graph = true;

    StageTables tables() const { return StageTables{d_grade, d_lon, d_cyc, d_red, d_off}; }
    unsigned long long *d_part = nullptr;  // per-state minima of the class-split Bellman launch
    StageScratch scratch() const { return StageScratch{d_cls, d_ent, d_rowcnt, d_spl, d_stats, d_part}; }
    // Value-function storage.  ckpt == 0: every stage k at d_V + k stage_elems.
    // ckpt = K >= 2: only stages 0, K, 2K, ... and N are kept (checkpoints,
    // in that order in d_V); the backward sweep writes the other stages to
    // two ring slots, and readers recompute a segment (cK, min((c+1)K, N))
    // from its upper checkpoint into d_seg.
    int ckpt = 0;
    float *d_ring = nullptr, *d_seg = nullptr;
    bool stored(int k) const { return ckpt == 0 || k % ckpt == 0 || k == N; }
    // J_k's slot during the backward sweep
    float *Vsweep(int k) const
    {
        if (ckpt == 0)
            return d_V + (size_t)k * stage_elems;
        if (k % ckpt == 0)
            return d_V + (size_t)(k / ckpt) * stage_elems;
        if (k == N)
            return d_V + (size_t)(N / ckpt + 1) * stage_elems;
        return d_ring + (size_t)(k & 1) * stage_elems;
    }
    int n_segments() const { return ckpt == 0 ? 1 : (N + ckpt - 1) / ckpt; }
    int seg_lo(int c) const { return ckpt == 0 ? 0 : c * ckpt; }
    int seg_hi(int c) const { return ckpt == 0 ? N : std::min((c + 1) * ckpt, N); }
    // where stages seg_lo(c) + 1 .. seg_hi(c) live once segment c is recomputed
    StageView seg_view(int c) const
    {
        if (ckpt == 0)
            return StageView::all(d_V, stage_elems);
        return StageView{d_seg, Vsweep(seg_hi(c)), seg_lo(c) + 1, seg_hi(c), stage_elems};
    }
    int16_t *pi(int k) const { return d_pi + (size_t)k * pi_elems; }
};

namespace ecodp {
namespace host {

bool finite_all(std::initializer_list<double> xs)
{
    for (double x : xs)
        if (!std::isfinite(x))
            return false;
    return true;
}

dp_status validate(const dp_problem_desc *d)
{
    if (!d)
        return fail(DP_ERR_INVALID_ARG, "desc is NULL");
    if (d->n_stages < 1 || d->n_stages > 100000)
        return fail(DP_ERR_INVALID_ARG, "n_stages must be in [1, 100000]");
    if (d->n_v < 2 || d->n_soc < 2 || d->n_t < 2)
        return fail(DP_ERR_INVALID_ARG, "state grids need at least 2 nodes");
    if (d->n_v > 4096 || d->n_soc > 4096 || d->n_t > 4096)
        return fail(DP_ERR_INVALID_ARG, "state grids are limited to 4096 nodes per axis");
    if (d->n_te < 1 || d->n_tm < 1 || (d->n_brake != 1 && d->n_brake != 2))
        return fail(DP_ERR_INVALID_ARG, "control grids need n_te, n_tm >= 1 and n_brake in {1, 2}");
    if ((long long)d->n_te * d->n_tm * d->n_brake > 32767)
        return fail(DP_ERR_INVALID_ARG, "at most 32767 controls (int16 policy)");
    if ((long long)d->n_te * d->n_tm * d->n_brake > MAX_CONTROLS)
        return fail(DP_ERR_INVALID_ARG, "at most 8192 controls (per-control tables live in shared memory)");
    if (!d->grade)
        return fail(DP_ERR_INVALID_ARG, "grade is NULL");
    if (!finite_all({d->ds, d->v_lo, d->v_hi, d->soc_lo, d->soc_hi, d->t_lo, d->t_hi, d->te_lo, d->te_hi,
                     d->tm_lo, d->tm_hi, d->brake_decel, d->a_min, d->a_max, d->mass, d->cda, d->crr, d->rho,
                     d->g, d->r_wheel, d->gear, d->eta_motor, d->voc, d->r0, d->capacity_As, d->fuel_scale,
                     d->gamma, d->soc_ref, d->w_soc, d->v_ref, d->w_v, d->fuel_coef[0], d->fuel_coef[1],
                     d->fuel_coef[2], d->fuel_coef[3], d->fuel_coef[4], d->fuel_coef[5]}))
        return fail(DP_ERR_INVALID_ARG, "non-finite parameter");
    if (!(d->ds > 0 && d->v_hi > d->v_lo && d->v_lo >= 0 && d->soc_hi > d->soc_lo && d->t_hi > d->t_lo))
        return fail(DP_ERR_INVALID_ARG, "need ds > 0, 0 <= v_lo < v_hi, soc_lo < soc_hi, t_lo < t_hi");
    if (!(d->te_hi >= d->te_lo && d->tm_hi >= d->tm_lo && d->te_lo >= 0))
        return fail(DP_ERR_INVALID_ARG, "torque grids need lo <= hi and te_lo >= 0");
    if ((d->n_te == 1 && d->te_hi != d->te_lo) || (d->n_tm == 1 && d->tm_hi != d->tm_lo))
        return fail(DP_ERR_INVALID_ARG, "a one-point torque grid needs lo == hi");
    if (!(d->mass > 0 && d->r_wheel > 0 && d->gear > 0 && d->eta_motor > 0 && d->eta_motor <= 1 && d->voc > 0 &&
          d->r0 > 0 && d->capacity_As > 0 && d->gamma >= 0 && d->gamma <= 1 && d->a_min <= d->a_max &&
          d->w_soc >= 0 && d->w_v >= 0 && d->fuel_scale >= 0 && d->g >= 0 && d->cda >= 0 && d->crr >= 0))
        return fail(DP_ERR_INVALID_ARG, "model parameter out of range");
    double vmax = std::fmax(std::fabs(d->v_hi - d->v_ref), std::fabs(d->v_lo - d->v_ref));
    if (d->w_soc * std::fabs(d->soc_ref - d->soc_lo) + d->w_v * vmax * vmax > 1e9)
        return fail(DP_ERR_INVALID_ARG, "terminal cost weights too large (costs must stay below 1e9)");
    for (int q = 0; q < d->n_stages; ++q)
        if (!std::isfinite(d->grade[q]) || std::fabs(d->grade[q]) > 1.0)
            return fail(DP_ERR_INVALID_ARG, "grade must be finite with |grade| <= 1");
    if (d->light_model < 0 || d->light_model > 2)
        return fail(DP_ERR_INVALID_ARG, "light_model must be 0, 1 or 2");
    if (d->torque_limits != 0 && d->torque_limits != 1)
        return fail(DP_ERR_INVALID_ARG, "torque_limits must be 0 or 1");
    if (d->torque_limits &&
        (!finite_all({d->te_max_coef[0], d->te_max_coef[1], d->te_max_coef[2], d->bsg_power_max}) ||
         d->bsg_power_max < 0))
        return fail(DP_ERR_INVALID_ARG, "torque limits need finite coefficients and bsg_power_max >= 0");
    if (d->n_lights < 0 || d->n_lights > d->n_stages)
        return fail(DP_ERR_INVALID_ARG, "bad n_lights");
    if (d->n_lights > 0 && (!d->light_stage || !d->cycle || !d->red || !d->offset))
        return fail(DP_ERR_INVALID_ARG, "light arrays are NULL");
    std::vector<char> seen(d->n_stages + 1, 0);
    for (int q = 0; q < d->n_lights; ++q) {
        int s = d->light_stage[q];
        if (s < 1 || s > d->n_stages - 1 || seen[s])
            return fail(DP_ERR_INVALID_ARG, "lights must sit at distinct nodes in [1, n_stages - 1]");
        seen[s] = 1;
        if (!finite_all({d->cycle[q], d->red[q], d->offset[q]}) || !(d->cycle[q] > 0) || d->red[q] < 0 ||
            d->red[q] > d->cycle[q])
            return fail(DP_ERR_INVALID_ARG, "light cycle/red/offset out of range");
    }
    return DP_OK;
}

namespace {
float f32(double x) { return (float)x; }
}  // namespace

void fill_params(const dp_problem_desc *d, DevParams &P)
{
    P.N = d->n_stages;
    P.n_v = d->n_v;
    P.n_xi = d->n_soc;
    P.n_t = d->n_t;
    P.n_te = d->n_te;
    P.n_tm = d->n_tm;
    P.n_b = d->n_brake;
    P.n_u = d->n_te * d->n_tm * d->n_brake;
    // torque classes: when both torque grids share one step, controls with
    // i_e + i_m equal have the same total torque
    double he = d->n_te > 1 ? (d->te_hi - d->te_lo) / (d->n_te - 1) : 0.0;
    double hm = d->n_tm > 1 ? (d->tm_hi - d->tm_lo) / (d->n_tm - 1) : 0.0;
    bool same_step = (d->n_te == 1 || d->n_tm == 1) ? true : (he == hm);
    P.class_sum = same_step ? 1 : 0;
    P.n_cls = (same_step ? (d->n_te + d->n_tm - 1) : (d->n_te * d->n_tm)) * d->n_brake;
    P.ld_t = round_up(d->n_t + 2, 4);
    P.xi_rows = d->n_soc + 2;
    P.n_lights = d->n_lights;
    P.v_lo = f32(d->v_lo);
    P.v_span = f32(d->v_hi - d->v_lo);
    P.xi_lo = f32(d->soc_lo);
    P.xi_span = f32(d->soc_hi - d->soc_lo);
    P.t_lo = f32(d->t_lo);
    P.t_span = f32(d->t_hi - d->t_lo);
    P.te_lo = f32(d->te_lo);
    P.te_span = f32(d->te_hi - d->te_lo);
    P.tm_lo = f32(d->tm_lo);
    P.tm_span = f32(d->tm_hi - d->tm_lo);
    P.h_v = f32((d->v_hi - d->v_lo) / (d->n_v - 1));
    P.h_xi = f32((d->soc_hi - d->soc_lo) / (d->n_soc - 1));
    P.h_t = f32((d->t_hi - d->t_lo) / (d->n_t - 1));
    P.ds = f32(d->ds);
    P.mass = f32(d->mass);
    P.g = f32(d->g);
    P.crr = f32(d->crr);
    P.half_rho_cda = f32(0.5 * d->rho * d->cda);
    P.half_rho = f32(0.5 * d->rho);
    P.ratio = f32(d->gear / d->r_wheel);
    P.brake_force = f32(d->mass * d->brake_decel);
    P.a_min = f32(d->a_min);
    P.a_max = f32(d->a_max);
    P.eta = f32(d->eta_motor);
    P.voc = f32(d->voc);
    P.r0 = f32(d->r0);
    P.cap = f32(d->capacity_As);
    for (int q = 0; q < 6; ++q)
        P.fc[q] = f32(d->fuel_coef[q]);
    P.fuel_scale = f32(d->fuel_scale);
    P.gamma = f32(d->gamma);
    P.soc_ref = f32(d->soc_ref);
    P.w_soc = f32(d->w_soc);
    P.v_ref = f32(d->v_ref);
    P.w_v = f32(d->w_v);
    P.light_model = d->light_model;
    P.torque_limits = d->torque_limits;
    for (int q = 0; q < 3; ++q)
        P.te_max_c[q] = d->torque_limits ? f32(d->te_max_coef[q]) : 0.f;
    P.bsg_pmax = d->torque_limits ? f32(d->bsg_power_max) : 0.f;
    P.all_lines = 0;
}

void fill_tables(const dp_problem_desc *d, HostTables &t)
{
    t.grade.assign(d->n_stages, 0.f);
    for (int q = 0; q < d->n_stages; ++q)
        t.grade[q] = f32(d->grade[q]);
    int nl = d->n_lights;
    t.cyc.assign(nl > 0 ? nl : 1, 1.f);
    t.red.assign(nl > 0 ? nl : 1, 0.f);
    t.off.assign(nl > 0 ? nl : 1, 0.f);
    t.lon.assign(d->n_stages + 1, -1);
    for (int q = 0; q < nl; ++q) {
        t.cyc[q] = f32(d->cycle[q]);
        t.red[q] = f32(d->red[q]);
        t.off[q] = f32(d->offset[q]);
        t.lon[d->light_stage[q]] = q;
    }
}

bool finite3(const double x[3]) { return finite_all({x[0], x[1], x[2]}); }

dp_status checks_after(dp_status st)
{
#ifdef ECODP_CHECKS
    if (st != DP_OK && st != DP_ERR_INFEASIBLE)
        return st;
    uint64_t site = 0;
    const dp_status c = dp_debug_checks(nullptr, &site);
    if (c != DP_OK)
        return c;
#endif
    return st;
}

}  // namespace host
}  // namespace ecodp

namespace {


dp_status dev_alloc(dp_problem *p, size_t bytes, void **out)
{
    void *ptr = nullptr;
    bytes = (bytes + 255) & ~(size_t)255;
    if (p->has_alloc) {
        ptr = p->alloc.alloc(bytes, (void *)p->create_stream, p->alloc.ctx);
        if (!ptr)
            return fail(DP_ERR_OOM, "allocator returned NULL for " + std::to_string(bytes) + " bytes");
    } else {
        cudaError_t e = cudaMallocAsync(&ptr, bytes, p->create_stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? DP_ERR_OOM : DP_ERR_CUDA,
                        std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        }
    }
    p->blocks.push_back(ptr);
    p->bytes_held += bytes;
    *out = ptr;
    return DP_OK;
}

template <class T>
dp_status dev_alloc_n(dp_problem *p, size_t n, T **out)
{
    void *v = nullptr;
    dp_status s = dev_alloc(p, n * sizeof(T), &v);
    *out = (T *)v;
    return s;
}

void release(dp_problem *p)
{
    if (p->gexec)
        cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
    if (p->cap_stream)
        cudaStreamDestroy(p->cap_stream);
    p->cap_stream = nullptr;
    if (p->roll_stream) {
        cudaStreamSynchronize(p->roll_stream);
        cudaStreamDestroy(p->roll_stream);
    }
    p->roll_stream = nullptr;
    if (p->ev_stage1)
        cudaEventDestroy(p->ev_stage1);
    if (p->ev_rolled)
        cudaEventDestroy(p->ev_rolled);
    p->ev_stage1 = p->ev_rolled = nullptr;
    if (!p->blocks.empty())
        cudaStreamSynchronize(p->create_stream);
    for (void *b : p->blocks) {
        if (p->has_alloc)
            p->alloc.free(b, (void *)p->create_stream, p->alloc.ctx);
        else
            cudaFree(b);
    }
    p->blocks.clear();
}

void dev_free(dp_problem *p, void *ptr, size_t bytes)
{
    if (!ptr)
        return;
    for (size_t q = 0; q < p->blocks.size(); ++q)
        if (p->blocks[q] == ptr) {
            p->blocks.erase(p->blocks.begin() + q);
            break;
        }
    if (p->has_alloc)
        p->alloc.free(ptr, (void *)p->create_stream, p->alloc.ctx);
    else
        cudaFreeAsync(ptr, p->create_stream);
    p->bytes_held -= (bytes + 255) & ~(size_t)255;
}

size_t v_slots(const dp_problem *p)
{
    return p->ckpt == 0 ? (size_t)p->N + 1 : (size_t)(p->N / p->ckpt + 1 + (p->N % p->ckpt ? 1 : 0));
}

// Value-function storage for the current checkpoint setting; every cell
// starts as V_BIG (the padding keeps it for the object's life).
dp_status alloc_value_storage(dp_problem *p)
{
    const size_t se = p->stage_elems;
    dp_status st = dev_alloc_n(p, se * v_slots(p), &p->d_V);
    if (st != DP_OK)
        return st;
    DP_CUDA(launch_fill(p->d_V, se * v_slots(p), V_BIG, p->create_stream));
    if (p->ckpt > 0) {
        st = dev_alloc_n(p, se * 2, &p->d_ring);
        if (st != DP_OK)
            return st;
        st = dev_alloc_n(p, se * (size_t)std::max(1, p->ckpt - 1), &p->d_seg);
        if (st != DP_OK)
            return st;
        DP_CUDA(launch_fill(p->d_ring, se * 2, V_BIG, p->create_stream));
        DP_CUDA(launch_fill(p->d_seg, se * (size_t)std::max(1, p->ckpt - 1), V_BIG, p->create_stream));
    }
    return DP_OK;
}

void free_value_storage(dp_problem *p)
{
    const size_t se = p->stage_elems;
    dev_free(p, p->d_V, se * v_slots(p) * sizeof(float));
    if (p->ckpt > 0) {
        dev_free(p, p->d_ring, se * 2 * sizeof(float));
        dev_free(p, p->d_seg, se * (size_t)std::max(1, p->ckpt - 1) * sizeof(float));
    }
    p->d_V = p->d_ring = p->d_seg = nullptr;
}

// Recompute J_k for the stages strictly inside segment c into d_seg, from
// the segment's upper checkpoint, with the sweep's own kernels and tables
// (bit-identical to the values the backward sweep produced).
dp_status recompute_segment(dp_problem *p, int c, cudaStream_t s)
{
    if (p->ckpt == 0)
        return DP_OK;
    const int lo = p->seg_lo(c), hi = p->seg_hi(c);
    const StageView view = p->seg_view(c);
    StageScratch sc = p->scratch();
    sc.stats = nullptr;
    for (int k = hi - 1; k > lo; --k)
        DP_CUDA(launch_bellman(p->dP, p->hP, p->tables(), k, sc, view.at(k + 1), const_cast<float *>(view.at(k)),
                               p->d_pi_tmp, p->variant, s));
    return DP_OK;
}

dp_status upload_tables(dp_problem *p, cudaStream_t s)
{
    DP_CUDA(cudaMemcpyAsync(p->dP, &p->hP, sizeof(DevParams), cudaMemcpyHostToDevice, s));
    DP_CUDA(cudaMemcpyAsync(p->d_grade, p->h.grade.data(), p->h.grade.size() * sizeof(float),
                            cudaMemcpyHostToDevice, s));
    DP_CUDA(cudaMemcpyAsync(p->d_lon, p->h.lon.data(), p->h.lon.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    DP_CUDA(cudaMemcpyAsync(p->d_cyc, p->h.cyc.data(), p->h.cyc.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    DP_CUDA(cudaMemcpyAsync(p->d_red, p->h.red.data(), p->h.red.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    DP_CUDA(cudaMemcpyAsync(p->d_off, p->h.off.data(), p->h.off.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    return DP_OK;
}

// Stage k of a full backward sweep: J_{k+1} and its corner quads in, J_k,
// pi_k and J_k's quads out (the tiled kernel keeps the quads of every stage;
// the other paths ignore them).
cudaError_t sweep_stage(dp_problem *p, int k, cudaStream_t s)
{
    StageScratch sc = p->scratch();
    sc.lmax = p->d_lmax;  // J_{k+1}'s last feasible time column in, J_k's out
    sc.fill_slots = p->fill_slots ? 1 : 0;
    return launch_bellman(p->dP, p->hP, p->tables(), k, sc, p->Vsweep(k + 1), p->Vsweep(k), p->pi(k), p->variant, s,
                          p->quad(k + 1), p->quad(k));
}

// Counters and per-stage time limits reset before a sweep (memset nodes when
// the sweep is captured).
cudaError_t sweep_reset(dp_problem *p, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(p->d_stats, 0, 8 * sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(p->d_lmax, 0xff, (size_t)(p->N + 1) * sizeof(int), s);
    return e;
}

// The backward sweep's launches: terminal values (and their corner quads),
// the precompute tables of every stage (they depend on the route, not on J),
// then the N Bellman stages in backward order.
dp_status enqueue_sweep(dp_problem *p, cudaStream_t s)
{
    DP_CUDA(sweep_reset(p, s));
    DP_CUDA(launch_terminal(p->dP, p->hP, p->Vsweep(p->N), s));
    if (p->d_quad)
        DP_CUDA(launch_quad_from_pad(p->hP, p->Vsweep(p->N), p->quad(p->N), s));
    DP_CUDA(launch_precompute(p->dP, p->hP, p->tables(), 0, p->N, p->scratch(), s));
    for (int k = p->N - 1; k >= 0; --k) {
        DP_CUDA(sweep_stage(p, k, s));
        if (k == 1)  // J_1 .. J_N complete (an event node of the graph when captured)
            DP_CUDA(cudaEventRecordWithFlags(p->ev_stage1, s, cudaEventRecordExternal));
    }
    return DP_OK;
}

}  // namespace

namespace ecodp {
namespace host {

void set_fill_slots(dp_problem *p, bool on)
{
    if (p->fill_slots != on) {
        p->fill_slots = on;
        if (p->gexec)
            cudaGraphExecDestroy(p->gexec);  // the captured launches hold the grid
        p->gexec = nullptr;
    }
}


size_t roll_doubles(int N) { return (size_t)(3 * (N + 1) + 3 * N + 4); }

dp_status rollout_async(dp_problem *p, const double x0[3], double *h_out, int *h_u, cudaStream_t s, bool overlap)
{
    if (overlap && p->rollout_may_overlap && s == p->solve_stream && p->n_segments() == 1) {
        // from J_1 on, beside the sweep's last stage (the rollout never reads J_0)
        DP_CUDA(cudaStreamWaitEvent(p->roll_stream, p->ev_stage1, 0));
        DP_CUDA(launch_rollout(p->dP, p->hP, p->tables(), p->seg_view(0), 0, p->N, x0[0], x0[1], x0[2], p->d_roll,
                               p->d_roll_u, p->roll_stream));
        DP_CUDA(cudaEventRecord(p->ev_rolled, p->roll_stream));
        DP_CUDA(cudaStreamWaitEvent(s, p->ev_rolled, 0));
        DP_CUDA(cudaMemcpyAsync(h_out, p->d_roll, roll_doubles(p->N) * sizeof(double), cudaMemcpyDeviceToHost, s));
        DP_CUDA(cudaMemcpyAsync(h_u, p->d_roll_u, (size_t)p->N * sizeof(int), cudaMemcpyDeviceToHost, s));
        return DP_OK;
    }
    for (int c = 0; c < p->n_segments(); ++c) {
        dp_status st = recompute_segment(p, c, s);
        if (st != DP_OK)
            return st;
        DP_CUDA(launch_rollout(p->dP, p->hP, p->tables(), p->seg_view(c), p->seg_lo(c), p->seg_hi(c), x0[0], x0[1],
                               x0[2], p->d_roll, p->d_roll_u, s));
    }
    DP_CUDA(cudaMemcpyAsync(h_out, p->d_roll, roll_doubles(p->N) * sizeof(double), cudaMemcpyDeviceToHost, s));
    DP_CUDA(cudaMemcpyAsync(h_u, p->d_roll_u, (size_t)p->N * sizeof(int), cudaMemcpyDeviceToHost, s));
    return DP_OK;
}

int unpack_rollout(int N, const double *h, const int *hu, dp_trajectory *traj)
{
    const double *tot = h + 3 * (N + 1) + 3 * N;
    const int fail_stage = (int)tot[3];
    const int reached = fail_stage >= 0 ? fail_stage : N;
    for (int q = 0; q <= N; ++q) {
        const bool ok = q <= reached;
        traj->v[q] = ok ? h[3 * q] : NAN;
        traj->soc[q] = ok ? h[3 * q + 1] : NAN;
        traj->t[q] = ok ? h[3 * q + 2] : NAN;
    }
    for (int q = 0; q < N; ++q) {
        const bool ok = q < reached;
        traj->u[q] = ok ? hu[q] : -1;
        traj->dt[q] = ok ? h[3 * (N + 1) + q] : NAN;
        traj->wait[q] = ok ? h[3 * (N + 1) + N + q] : NAN;
        traj->fuel[q] = ok ? h[3 * (N + 1) + 2 * N + q] : NAN;
    }
    traj->fuel_g = tot[0];
    traj->time_s = tot[1];
    traj->J = tot[2];
    traj->fail_stage = fail_stage;
    return fail_stage;
}

size_t problem_bytes(const dp_problem *p) { return p->bytes_held; }

int problem_stages(const dp_problem *p) { return p->N; }

bool problem_fits(const dp_problem *p, const dp_problem_desc *d)
{
    if (d->n_stages != p->N || d->n_v != p->n_v || d->n_soc != p->n_xi || d->n_t != p->n_t ||
        d->n_te * d->n_tm * d->n_brake != p->n_u || d->n_te != p->hP.n_te || d->n_brake != p->hP.n_b)
        return false;
    DevParams P;
    fill_params(d, P);
    return P.n_cls == p->hP.n_cls;
}

}  // namespace host
}  // namespace ecodp

extern "C" {

const char *dp_status_string(dp_status s)
{
    switch (s) {
    case DP_OK: return "DP_OK";
    case DP_ERR_INVALID_ARG: return "DP_ERR_INVALID_ARG";
    case DP_ERR_OOM: return "DP_ERR_OOM";
    case DP_ERR_CUDA: return "DP_ERR_CUDA";
    case DP_ERR_INFEASIBLE: return "DP_ERR_INFEASIBLE";
    case DP_ERR_NOT_SOLVED: return "DP_ERR_NOT_SOLVED";
    case DP_ERR_TIMEOUT: return "DP_ERR_TIMEOUT";
    case DP_ERR_INTERNAL: return "DP_ERR_INTERNAL";
    }
    return "DP_ERR_UNKNOWN";
}

const char *dp_last_error(void) { return last_error(); }

dp_status dp_problem_create(const dp_problem_desc *desc, const dp_allocator *alloc, void *stream, dp_problem_t *out)
{
    if (!out)
        return fail(DP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    dp_status st = validate(desc);
    if (st != DP_OK)
        return st;
    if (alloc && (!alloc->alloc || !alloc->free))
        return fail(DP_ERR_INVALID_ARG, "allocator needs both alloc and free");
    dp_problem *p = new (std::nothrow) dp_problem();
    if (!p)
        return fail(DP_ERR_OOM, "host allocation failed");
    p->create_stream = (cudaStream_t)stream;
    if (alloc) {
        p->alloc = *alloc;
        p->has_alloc = true;
    }
    fill_params(desc, p->hP);
    fill_tables(desc, p->h);
    p->N = desc->n_stages;
    p->n_v = desc->n_v;
    p->n_xi = desc->n_soc;
    p->n_t = desc->n_t;
    p->n_u = p->hP.n_u;
    p->n_lights = desc->n_lights;
    const DevParams &P = p->hP;
    p->stage_elems = (size_t)P.n_v * P.xi_rows * P.ld_t;
    p->pi_elems = (size_t)P.n_v * P.n_xi * P.n_t;
    if (const char *e = std::getenv("ECODP_GRAPH"))
        p->use_graph = std::atoi(e) != 0;

#define TRY(x)              \
    do {                    \
        st = (x);           \
        if (st != DP_OK) {  \
            release(p);     \
            delete p;       \
            return st;      \
        }                   \
    } while (0)
    TRY(dev_alloc_n(p, 1, &p->dP));
    TRY(dev_alloc_n(p, p->h.grade.size(), &p->d_grade));
    TRY(dev_alloc_n(p, p->h.lon.size(), &p->d_lon));
    // light tables sized for the most lights a route of N stages can hold,
    // so that dp_problem_update may change the light count
    const size_t light_cap = std::max<size_t>(p->h.cyc.size(), (size_t)p->N);
    TRY(dev_alloc_n(p, light_cap, &p->d_cyc));
    TRY(dev_alloc_n(p, light_cap, &p->d_red));
    TRY(dev_alloc_n(p, light_cap, &p->d_off));
    TRY(alloc_value_storage(p));
    TRY(dev_alloc_n(p, p->pi_elems * (size_t)p->N, &p->d_pi));
    if (P.n_cls > MAX_CLASSES) {
        release(p);
        delete p;
        return fail(DP_ERR_INVALID_ARG, "at most 4095 torque classes (unequal torque steps give one per control)");
    }
    const size_t rows = (size_t)P.N * P.n_v;  // one table slot per stage
    TRY(dev_alloc_n(p, rows * P.n_cls, &p->d_cls));
    TRY(dev_alloc_n(p, rows * P.n_cls, &p->d_ent));
    TRY(dev_alloc_n(p, rows * 2, &p->d_rowcnt));
    TRY(dev_alloc_n(p, rows * P.n_u, &p->d_spl));
    p->quad_elems = (size_t)P.n_v * quad_rows(P.n_xi) * quad_ld(P.n_t);
    if (p->quad_elems > 0)
        TRY(dev_alloc_n(p, 2 * p->quad_elems, &p->d_quad));
    TRY(dev_alloc_n(p, p->stage_elems, &p->d_pad_in));
    TRY(dev_alloc_n(p, p->stage_elems, &p->d_pad_out));
    TRY(dev_alloc_n(p, p->pi_elems, &p->d_dense));
    TRY(dev_alloc_n(p, p->pi_elems, &p->d_pi_tmp));
    TRY(dev_alloc_n(p, (size_t)(3 * (P.N + 1) + 3 * P.N + 4), &p->d_roll));
    TRY(dev_alloc_n(p, (size_t)P.N, &p->d_roll_u));
    TRY(dev_alloc_n(p, (size_t)8, &p->d_stats));
    TRY(dev_alloc_n(p, (size_t)p->N + 1, &p->d_lmax));
    TRY(dev_alloc_n(p, 2 * p->pi_elems, &p->d_lam));
    TRY(dev_alloc_n(p, 2 * p->pi_elems, &p->d_front));
    TRY(dev_alloc_n(p, 2 * ((p->pi_elems + 31) / 32), &p->d_fbits));
    TRY(dev_alloc_n(p, (size_t)3, &p->d_fcnt));
    TRY(dev_alloc_n(p, (size_t)8, &p->d_adj));
    TRY(dev_alloc_n(p, p->pi_elems, &p->d_part));
    TRY(upload_tables(p, p->create_stream));
    auto cuda_try = [&](cudaError_t e, const char *what) -> dp_status {
        if (e != cudaSuccess)
            return fail(DP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
        return DP_OK;
    };
    TRY(cuda_try(cudaMemsetAsync(p->d_part, 0xff, p->pi_elems * sizeof(unsigned long long), p->create_stream),
                 "clear split minima"));
    // every padding cell holds the infeasible sentinel for the object's life
    if (p->d_quad)
        TRY(cuda_try(launch_fill(reinterpret_cast<float *>(p->d_quad), 8 * p->quad_elems, V_BIG, p->create_stream),
                     "fill"));
    TRY(cuda_try(launch_fill(p->d_pad_in, p->stage_elems, V_BIG, p->create_stream), "fill"));
    TRY(cuda_try(launch_fill(p->d_pad_out, p->stage_elems, V_BIG, p->create_stream), "fill"));
    TRY(cuda_try(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking), "cudaStreamCreate"));
    TRY(cuda_try(cudaStreamCreateWithFlags(&p->roll_stream, cudaStreamNonBlocking), "cudaStreamCreate"));
    TRY(cuda_try(cudaEventCreateWithFlags(&p->ev_stage1, cudaEventDisableTiming), "cudaEventCreate"));
    TRY(cuda_try(cudaEventCreateWithFlags(&p->ev_rolled, cudaEventDisableTiming), "cudaEventCreate"));
    size_t smem = bellman_smem_bytes(P);
    if (smem > 227 * 1024) {
        release(p);
        delete p;
        return fail(DP_ERR_INVALID_ARG, "too many torque classes for the shared-memory tables");
    }
#undef TRY
    *out = p;
    return DP_OK;
}

dp_status dp_problem_update(dp_problem_t p, const dp_problem_desc *desc, void *stream)
{
    if (!p)
        return fail(DP_ERR_INVALID_ARG, "problem is NULL");
    dp_status st = validate(desc);
    if (st != DP_OK)
        return st;
    if (desc->n_stages != p->N || desc->n_v != p->n_v || desc->n_soc != p->n_xi || desc->n_t != p->n_t ||
        desc->n_te * desc->n_tm * desc->n_brake != p->n_u || desc->n_te != p->hP.n_te ||
        desc->n_brake != p->hP.n_b)
        return fail(DP_ERR_INVALID_ARG, "update must keep the problem's sizes");
    DevParams P;
    fill_params(desc, P);
    if (P.n_cls != p->hP.n_cls)
        return fail(DP_ERR_INVALID_ARG, "update changes the torque class structure");
    P.all_lines = p->hP.all_lines;  // a setting of the problem object, not of the descriptor
    p->hP = P;
    p->n_lights = desc->n_lights;
    fill_tables(desc, p->h);
    st = upload_tables(p, (cudaStream_t)stream);
    p->solved = false;
    p->rollout_may_overlap = false;
    return st;
}

dp_status dp_problem_destroy(dp_problem_t p)
{
    if (!p)
        return DP_OK;
    release(p);
    delete p;
    return DP_OK;
}

dp_status dp_problem_sizes(dp_problem_t p, int32_t sizes[5])
{
    if (!p || !sizes)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    sizes[0] = p->N;
    sizes[1] = p->n_v;
    sizes[2] = p->n_xi;
    sizes[3] = p->n_t;
    sizes[4] = p->n_u;
    return DP_OK;
}

dp_status dp_sweep_stats(dp_problem_t p, int64_t out[8], void *stream)
{
    if (!p || !out)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    if (!p->solved)
        return fail(DP_ERR_NOT_SOLVED, "call dp_solve_backward first");
    unsigned long long h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    cudaStream_t s = (cudaStream_t)stream;
    DP_CUDA(cudaMemcpyAsync(h, p->d_stats, sizeof h, cudaMemcpyDeviceToHost, s));
    DP_CUDA(cudaStreamSynchronize(s));
    out[0] = (int64_t)h[0] * p->n_xi * p->n_t;
    out[1] = (int64_t)h[1] * p->n_xi * p->n_t - (int64_t)h[5];
    // bytes of one dp_problem_update (tables) and one dp_rollout (trajectory)
    out[2] = (int64_t)(sizeof(DevParams) + p->h.bytes());
    out[3] = (int64_t)((3 * (p->N + 1) + 3 * p->N + 4) * sizeof(double) + p->N * sizeof(int));
    out[4] = (int64_t)h[2];
    out[5] = (int64_t)h[3];
    out[6] = (int64_t)h[4] * p->n_xi * p->n_t - (int64_t)h[6];
    out[7] = (int64_t)h[7];
    return DP_OK;
}

dp_status dp_set_checkpointing(dp_problem_t p, int32_t every)
{
    if (!p)
        return fail(DP_ERR_INVALID_ARG, "problem is NULL");
    if (every < 0 || every > p->N)
        return fail(DP_ERR_INVALID_ARG, "every must be in [0, n_stages]");
    const int K = every <= 1 ? 0 : every;
    if (K == p->ckpt)
        return DP_OK;
    // the old storage may still be read by queued work on any stream
    DP_CUDA(cudaDeviceSynchronize());
    free_value_storage(p);
    p->ckpt = K;
    p->rollout_may_overlap = false;
    if (p->gexec)
        cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
    p->solved = false;
    dp_status st = alloc_value_storage(p);
    if (st != DP_OK)
        return st;
    DP_CUDA(cudaStreamSynchronize(p->create_stream));
    return DP_OK;
}

dp_status dp_set_kernel_variant(dp_problem_t p, int32_t variant)
{
    if (!p || variant < 0 || variant > 3)
        return fail(DP_ERR_INVALID_ARG, "variant must be 0 (direct), 1 (tiled), 2 (tiled, 8 rows) or 3 (tiled, 6 rows)");
    if (variant != p->variant) {
        p->variant = variant;
        if (p->gexec)
            cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
    }
    return DP_OK;
}

dp_status dp_set_envelopes(dp_problem_t p, int32_t on)
{
    if (!p || (on != 0 && on != 1))
        return fail(DP_ERR_INVALID_ARG, "on must be 0 or 1");
    if (p->hP.all_lines != 1 - on) {
        p->hP.all_lines = 1 - on;
        DP_CUDA(cudaMemcpyAsync(p->dP, &p->hP, sizeof(DevParams), cudaMemcpyHostToDevice, p->create_stream));
        DP_CUDA(cudaStreamSynchronize(p->create_stream));
        if (p->gexec)
            cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
        p->solved = false;
        p->rollout_may_overlap = false;
    }
    return DP_OK;
}

dp_status dp_solve_backward(dp_problem_t p, void *stream)
{
    NvtxRange nvtx_("ecodp.sweep");
    if (!p)
        return fail(DP_ERR_INVALID_ARG, "problem is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    p->rollout_may_overlap = false;
    if (!p->use_graph) {
        dp_status st = enqueue_sweep(p, s);
        if (st != DP_OK)
            return st;
        p->solved = true;
        p->solve_stream = s;
        p->rollout_may_overlap = p->N >= 2 && p->ckpt == 0;
        return DP_OK;
    }
    if (!p->gexec) {
        cudaGraph_t g = nullptr;
        DP_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
        dp_status st = enqueue_sweep(p, p->cap_stream);
        cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
        if (st != DP_OK) {
            if (g)
                cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess)
            return fail(DP_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&p->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            p->gexec = nullptr;
            return fail(DP_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        }
    }
    DP_CUDA(cudaGraphLaunch(p->gexec, s));
    p->solved = true;
    p->solve_stream = s;
    p->rollout_may_overlap = p->N >= 2 && p->ckpt == 0;
    return DP_OK;
}

dp_status dp_profile_sweep(dp_problem_t p, void *stream, float ms[4])
{
    NvtxRange nvtx_("ecodp.profile_sweep");
    if (!p || !ms)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    p->rollout_may_overlap = false;
    cudaStream_t s = (cudaStream_t)stream;
    const int N = p->N;
    std::vector<cudaEvent_t> ev(N + 3, nullptr);
    for (auto &e : ev)
        DP_CUDA(cudaEventCreate(&e));
    dp_status st = DP_OK;
    auto run = [&]() -> dp_status {
        DP_CUDA(sweep_reset(p, s));
        DP_CUDA(cudaEventRecord(ev[0], s));
        DP_CUDA(launch_terminal(p->dP, p->hP, p->Vsweep(N), s));
        if (p->d_quad)
            DP_CUDA(launch_quad_from_pad(p->hP, p->Vsweep(N), p->quad(N), s));
        DP_CUDA(cudaEventRecord(ev[1], s));
        DP_CUDA(launch_precompute(p->dP, p->hP, p->tables(), 0, N, p->scratch(), s));
        DP_CUDA(cudaEventRecord(ev[2], s));
        for (int k = N - 1, q = 3; k >= 0; --k, ++q) {
            NvtxRange stage_range(("ecodp.stage " + std::to_string(k)).c_str());
            DP_CUDA(sweep_stage(p, k, s));
            DP_CUDA(cudaEventRecord(ev[q], s));
        }
        DP_CUDA(cudaEventSynchronize(ev[N + 2]));
        float t = 0.f, pre = 0.f, bell = 0.f, all = 0.f;
        DP_CUDA(cudaEventElapsedTime(&t, ev[0], ev[1]));
        DP_CUDA(cudaEventElapsedTime(&pre, ev[1], ev[2]));
        for (int q = 3; q < N + 3; ++q) {
            float b = 0.f;
            DP_CUDA(cudaEventElapsedTime(&b, ev[q - 1], ev[q]));
            bell += b;
        }
        DP_CUDA(cudaEventElapsedTime(&all, ev[0], ev[N + 2]));
        ms[0] = t;
        ms[1] = pre;
        ms[2] = bell;
        ms[3] = all;
        return DP_OK;
    };
    st = run();
    for (auto &e : ev)
        cudaEventDestroy(e);
    if (st == DP_OK)
        p->solved = true;
    return st;
}

dp_status dp_get_value(dp_problem_t p, int32_t stage, float *out, int32_t out_is_host, void *stream)
{
    if (!p || !out)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    if (stage < 0 || stage > p->N)
        return fail(DP_ERR_INVALID_ARG, "stage out of range");
    if (!p->solved)
        return fail(DP_ERR_NOT_SOLVED, "call dp_solve_backward first");
    cudaStream_t s = (cudaStream_t)stream;
    float *dst = out_is_host ? p->d_dense : out;
    const float *src = p->Vsweep(stage);
    if (!p->stored(stage)) {
        const int c = stage / p->ckpt;
        dp_status st = recompute_segment(p, c, s);
        if (st != DP_OK)
            return st;
        src = p->seg_view(c).at(stage);
    }
    DP_CUDA(launch_dense_from_pad(p->hP, src, dst, s));
    if (out_is_host) {
        DP_CUDA(cudaMemcpyAsync(out, p->d_dense, p->pi_elems * sizeof(float), cudaMemcpyDeviceToHost, s));
        DP_CUDA(cudaStreamSynchronize(s));
    }
    return DP_OK;
}

dp_status dp_get_policy(dp_problem_t p, int32_t stage, int16_t *out, int32_t out_is_host, void *stream)
{
    if (!p || !out)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    if (stage < 0 || stage >= p->N)
        return fail(DP_ERR_INVALID_ARG, "stage out of range");
    if (!p->solved)
        return fail(DP_ERR_NOT_SOLVED, "call dp_solve_backward first");
    cudaStream_t s = (cudaStream_t)stream;
    DP_CUDA(cudaMemcpyAsync(out, p->pi(stage), p->pi_elems * sizeof(int16_t),
                            out_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    if (out_is_host)
        DP_CUDA(cudaStreamSynchronize(s));
    return DP_OK;
}

dp_status dp_solve_stage(dp_problem_t p, int32_t k, const float *v_next, int32_t v_next_is_host, float *v_out,
                         int16_t *pi_out, int32_t out_is_host, void *stream)
{
    if (p)
        p->rollout_may_overlap = false;
    if (!p || !v_next)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    if (k < 0 || k >= p->N)
        return fail(DP_ERR_INVALID_ARG, "stage out of range");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = p->pi_elems;
    DP_CUDA(cudaMemcpyAsync(p->d_dense, v_next, n * sizeof(float),
                            v_next_is_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    StageScratch sc = p->scratch();
    sc.stats = nullptr;
    DP_CUDA(launch_pad_from_dense(p->hP, p->d_dense, p->d_pad_in, s));
    DP_CUDA(launch_precompute(p->dP, p->hP, p->tables(), k, 1, sc, s));
    DP_CUDA(launch_bellman(p->dP, p->hP, p->tables(), k, sc, p->d_pad_in, p->d_pad_out, p->d_pi_tmp, p->variant, s));
    if (v_out) {
        DP_CUDA(launch_dense_from_pad(p->hP, p->d_pad_out, p->d_dense, s));
        DP_CUDA(cudaMemcpyAsync(v_out, p->d_dense, n * sizeof(float),
                                out_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    }
    if (pi_out)
        DP_CUDA(cudaMemcpyAsync(pi_out, p->d_pi_tmp, n * sizeof(int16_t),
                                out_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    if (out_is_host)
        DP_CUDA(cudaStreamSynchronize(s));
    return DP_OK;
}

static dp_status adjoint_impl(dp_problem_t p, const double x0[3], double dJ_dtheta[5], double *J0, void *stream)
{
    if (p)
        p->rollout_may_overlap = false;
    if (!p || !x0 || !dJ_dtheta)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    if (!finite_all({x0[0], x0[1], x0[2]}))
        return fail(DP_ERR_INVALID_ARG, "x0 must be finite");
    if (!p->solved)
        return fail(DP_ERR_NOT_SOLVED, "call dp_solve_backward first");
    cudaStream_t s = (cudaStream_t)stream;
    DP_CUDA(launch_adjoint_init(p->dP, p->hP, p->Vsweep(0), p->d_lam, p->frontier(), x0[0], x0[1], x0[2], p->d_adj,
                                s));
    for (int c = 0; c < p->n_segments(); ++c) {
        dp_status st = recompute_segment(p, c, s);
        if (st != DP_OK)
            return st;
        const StageView view = p->seg_view(c);
        for (int k = p->seg_lo(c); k < p->seg_hi(c); ++k)
            DP_CUDA(launch_adjoint_stage(p->dP, p->hP, p->tables(), k, view.at(k + 1), p->pi(k), p->d_lam,
                                         p->frontier(), p->d_adj,
                                         s));
    }
    double h[8];
    DP_CUDA(cudaMemcpyAsync(h, p->d_adj, sizeof h, cudaMemcpyDeviceToHost, s));
    DP_CUDA(cudaStreamSynchronize(s));
    for (int q = 0; q < 5; ++q)
        dJ_dtheta[q] = h[q];
    if (J0)
        *J0 = h[5];
    if (h[6] == 1.0 || h[6] == 2.0 || !(h[5] < 1e12))
        return fail(DP_ERR_INFEASIBLE, "x0 is outside the grid or infeasible");
    if (h[6] == 3.0)
        return fail(DP_ERR_INTERNAL, "the adjoint support reached an infeasible state");
    return DP_OK;
}

static dp_status rollout_impl(dp_problem_t p, const double x0[3], dp_trajectory *traj, void *stream)
{
    if (!p || !x0 || !traj)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    if (!traj->v || !traj->soc || !traj->t || !traj->u || !traj->dt || !traj->wait || !traj->fuel)
        return fail(DP_ERR_INVALID_ARG, "trajectory arrays must all be provided");
    if (!finite_all({x0[0], x0[1], x0[2]}))
        return fail(DP_ERR_INVALID_ARG, "x0 must be finite");
    if (!p->solved)
        return fail(DP_ERR_NOT_SOLVED, "call dp_solve_backward first");
    cudaStream_t s = (cudaStream_t)stream;
    const int N = p->N;
    std::vector<double> h(roll_doubles(N));
    std::vector<int> hu(N, -1);
    dp_status st = rollout_async(p, x0, h.data(), hu.data(), s, true);
    if (st != DP_OK)
        return st;
    DP_CUDA(cudaStreamSynchronize(s));
    const int fail_stage = unpack_rollout(N, h.data(), hu.data(), traj);
    if (fail_stage >= 0)
        return fail(DP_ERR_INFEASIBLE, "no feasible control at stage " + std::to_string(fail_stage));
    return DP_OK;
}

dp_status dp_rollout(dp_problem_t p, const double x0[3], dp_trajectory *traj, void *stream)
{
    NvtxRange nvtx_("ecodp.rollout");
    return checks_after(rollout_impl(p, x0, traj, stream));
}

dp_status dp_adjoint(dp_problem_t p, const double x0[3], double dJ_dtheta[5], double *J0, void *stream)
{
    NvtxRange nvtx_("ecodp.adjoint");
    return checks_after(adjoint_impl(p, x0, dJ_dtheta, J0, stream));
}

dp_status dp_debug_checks(int32_t *enabled, uint64_t *site)
{
#ifdef ECODP_CHECKS
    if (enabled)
        *enabled = 1;
#else
    if (enabled)
        *enabled = 0;
#endif
    if (!site)
        return DP_OK;
    *site = 0;
#ifdef ECODP_CHECKS
    DP_CUDA(cudaDeviceSynchronize());
    cudaError_t (*const words[])(unsigned long long *) = {check_word_precompute, check_word_bellman,
                                                          check_word_rollout, check_word_adjoint, check_word_batch};
    for (auto fn : words) {
        unsigned long long w = 0;
        DP_CUDA(fn(&w));
        if (w && !*site)
            *site = w;
    }
    if (*site) {
        const unsigned tag_line = (unsigned)(*site >> 32);
        return fail(DP_ERR_INTERNAL, "bounds check failed in kernel source " + std::to_string(tag_line >> 16) +
                                         " at line " + std::to_string(tag_line & 0xffffu) + ", index " +
                                         std::to_string((int)(unsigned)(*site & 0xffffffffu)));
    }
#endif
    return DP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free single stage (dp_solve_stage_static).
//
// Its working memory is one file-scope device array, sized for the limits
// below and resident on every GPU that loads this library until the process
// exits.  Host code must not pass the array's name to a kernel (on the host
// it only stands in for the symbol); every call looks up the current device's
// address of the array with cudaGetSymbolAddress (a host-side lookup; after a
// device reset the module is reloaded and the address may change, so it is
// not cached).

// The stage's own route tables, re-indexed as stage 0 of a one-stage
// problem: grade, light index at the departure node (0) and at the arrival
// node (1), and those lights' timings.  (Outside the anonymous namespace: it
// appears in a kernel's signature.)
struct StaticTables {
    float grade[4];
    int lon[2];
    float cyc[2], red[2], off[2];
};

// Stores one call's parameters and stage tables into the static array.  They
// travel as kernel arguments, so no host buffer has to outlive the call and
// no host-to-device copy is issued.  (In a named namespace: nvcc's launch
// stubs cannot name a kernel of this file's second anonymous namespace.)
namespace stage_static {
__global__ void static_setup_kernel(DevParams P, StaticTables t, DevParams *dP, StaticTables *dT)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *dP = P;
        *dT = t;
    }
}
}  // namespace stage_static

namespace {

constexpr int STATIC_MAX_V = 64, STATIC_MAX_SOC = 64, STATIC_MAX_T = 255, STATIC_MAX_U = 2048,
              STATIC_MAX_CLS = 256;
constexpr size_t STATIC_LD_T = (STATIC_MAX_T + 2 + 3) / 4 * 4;  // the largest ld_t = round_up(n_t + 2, 4)
constexpr size_t STATIC_PAD_ELEMS = (size_t)STATIC_MAX_V * (STATIC_MAX_SOC + 2) * STATIC_LD_T;

constexpr size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t ST_OFF_PARAMS = 0;
constexpr size_t ST_OFF_TABLES = ST_OFF_PARAMS + a256(sizeof(DevParams));
constexpr size_t ST_TABLE_BYTES = a256(sizeof(StaticTables));
constexpr size_t ST_OFF_CLS = ST_OFF_TABLES + ST_TABLE_BYTES;
constexpr size_t ST_OFF_ENT = ST_OFF_CLS + a256((size_t)STATIC_MAX_V * STATIC_MAX_CLS * sizeof(ClassRec));
constexpr size_t ST_OFF_ROWCNT = ST_OFF_ENT + a256((size_t)STATIC_MAX_V * STATIC_MAX_CLS * sizeof(ClassEntry));
constexpr size_t ST_OFF_SPL = ST_OFF_ROWCNT + a256((size_t)STATIC_MAX_V * 2 * sizeof(int));
constexpr size_t ST_OFF_PAD_IN = ST_OFF_SPL + a256((size_t)STATIC_MAX_V * STATIC_MAX_U * sizeof(SplitRec));
constexpr size_t ST_OFF_PAD_OUT = ST_OFF_PAD_IN + a256(STATIC_PAD_ELEMS * sizeof(float));
constexpr size_t ST_BYTES = ST_OFF_PAD_OUT + a256(STATIC_PAD_ELEMS * sizeof(float));  // about 12 MB

__device__ __align__(256) unsigned char g_stage_scratch[ST_BYTES];

// Device address of g_stage_scratch on the current device.
dp_status static_scratch(unsigned char **out)
{
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_stage_scratch);
    if (e != cudaSuccess || !ptr)
        return fail(DP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = (unsigned char *)ptr;
    return DP_OK;
}

}  // namespace

extern "C" dp_status dp_solve_stage_static(const dp_problem_desc *desc, int32_t k, const float *v_next, float *v_out,
                                           int16_t *pi_out, void *stream)
{
    dp_status st = validate(desc);
    if (st != DP_OK)
        return st;
    if (!v_next || !v_out || !pi_out)
        return fail(DP_ERR_INVALID_ARG, "v_next, v_out and pi_out must be device pointers");
    if (k < 0 || k >= desc->n_stages)
        return fail(DP_ERR_INVALID_ARG, "stage out of range");
    DevParams P;
    fill_params(desc, P);
    if (P.n_v > STATIC_MAX_V || P.n_xi > STATIC_MAX_SOC || P.n_t > STATIC_MAX_T || P.n_u > STATIC_MAX_U ||
        P.n_cls > STATIC_MAX_CLS)
        return fail(DP_ERR_INVALID_ARG,
                    "dp_solve_stage_static supports at most 64 speeds, 64 SoC points, 255 times, 2048 controls and "
                    "256 torque classes; use dp_solve_stage for larger problems");
    unsigned char *base = nullptr;
    st = static_scratch(&base);
    if (st != DP_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;

    StaticTables tbl = {};
    tbl.grade[0] = (float)desc->grade[k];
    tbl.lon[0] = tbl.lon[1] = -1;
    tbl.cyc[0] = tbl.cyc[1] = 1.f;
    for (int q = 0; q < desc->n_lights; ++q) {
        for (int side = 0; side < 2; ++side) {
            if (desc->light_stage[q] == k + side) {
                tbl.lon[side] = side;
                tbl.cyc[side] = (float)desc->cycle[q];
                tbl.red[side] = (float)desc->red[q];
                tbl.off[side] = (float)desc->offset[q];
            }
        }
    }
    StaticTables *tb_dev = (StaticTables *)(base + ST_OFF_TABLES);
    DevParams *dP = (DevParams *)(base + ST_OFF_PARAMS);
    unsigned char *tb_bytes = base + ST_OFF_TABLES;
    StageTables tb{(const float *)(tb_bytes + offsetof(StaticTables, grade)),
                   (const int *)(tb_bytes + offsetof(StaticTables, lon)),
                   (const float *)(tb_bytes + offsetof(StaticTables, cyc)),
                   (const float *)(tb_bytes + offsetof(StaticTables, red)),
                   (const float *)(tb_bytes + offsetof(StaticTables, off))};
    StageScratch sc{(ClassRec *)(base + ST_OFF_CLS), (ClassEntry *)(base + ST_OFF_ENT), (int *)(base + ST_OFF_ROWCNT),
                    (SplitRec *)(base + ST_OFF_SPL), nullptr, nullptr};
    if (P.ld_t > (int)STATIC_LD_T || (size_t)P.n_v * P.xi_rows * P.ld_t > STATIC_PAD_ELEMS)
        return fail(DP_ERR_INTERNAL, "static working memory layout too small");
    float *pad_in = (float *)(base + ST_OFF_PAD_IN);
    float *pad_out = (float *)(base + ST_OFF_PAD_OUT);
    const size_t pad_elems = (size_t)P.n_v * P.xi_rows * P.ld_t;

    stage_static::static_setup_kernel<<<1, 32, 0, s>>>(P, tbl, dP, tb_dev);
    DP_CUDA(cudaGetLastError());
    // the padding of J_{k+1} must read as infeasible: refill it every call,
    // since the array keeps whatever the previous call left there
    DP_CUDA(launch_fill(pad_in, pad_elems, V_BIG, s));
    DP_CUDA(launch_pad_from_dense(P, v_next, pad_in, s));
    DP_CUDA(launch_precompute(dP, P, tb, 0, 1, sc, s));
    DP_CUDA(launch_bellman(dP, P, tb, 0, sc, pad_in, pad_out, pi_out, 1, s));
    DP_CUDA(launch_dense_from_pad(P, pad_out, v_out, s));
    return DP_OK;
}
