// C ABI of batched solves (dp_multi_*, declared in include/ecodp.h): many
// independent problems of uneven horizon and grid size, solved by one
// persistent Bellman launch (k_batch.cu) after one batched terminal launch
// and one batched precompute launch, the three captured in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "api_internal.h"

using namespace ecodp;
using namespace ecodp::host;

struct dp_multi {
    int B = 0;
    std::vector<DevParams> hP;
    std::vector<HostTables> ht;
    dp_allocator alloc{};
    bool has_alloc = false;
    cudaStream_t create_stream = nullptr;
    std::vector<void *> blocks;
    size_t bytes_held = 0;

    DevParams *d_params = nullptr;
    BatchInst *d_inst = nullptr;
    std::vector<BatchInst> h_inst;
    int *d_done = nullptr;
    size_t done_total = 0;
    // route tables of all instances, concatenated
    float *d_grade = nullptr, *d_cyc = nullptr, *d_red = nullptr, *d_off = nullptr;
    int *d_lon = nullptr;
    // work list of the persistent launch
    int *d_order = nullptr, *d_m = nullptr;
    long long *d_pref = nullptr, *d_start = nullptr;
    unsigned long long *d_queue = nullptr;
    int *d_error = nullptr;
    int max_n = 0, max_n_u = 0, max_n_cls = 0;
    long long n_rows = 0, n_items = 0;
    int rows_per_lane = 8, ctas_per_sm = 0;
    unsigned long long wait_limit_ns = 10ull * 1000 * 1000 * 1000;  // 10 s
    // rollout buffers
    double *d_x0 = nullptr, *d_out = nullptr;
    int *d_out_u = nullptr;
    long long *d_out_off = nullptr, *d_u_off = nullptr;
    std::vector<long long> out_off, u_off;
    long long out_total = 0, u_total = 0;
    float *d_dense = nullptr;

    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool solved = false;

    // Per-instance mode (n_streams > 0): each instance's sweep is the
    // single-problem sequence (terminal values, corner quads, tables, the
    // Bellman stages) captured as its own CUDA graph on the batch's buffers;
    // a solve deals the instances over n_streams internal streams forked
    // from the caller's stream and joins them back.
    int n_streams = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> ev_done;
    cudaEvent_t ev_start = nullptr;
    std::vector<cudaGraphExec_t> inst_graph;  // per instance, captured on first use
    std::vector<float4 *> quad;               // per instance: two slots, or null
    std::vector<size_t> quad_elems;
    std::vector<int *> lmax;  // [B][N + 1] last feasible time column per stage (per-instance mode)
    std::vector<int> stream_of, launch_order;
    bool quads_ready = false;

    BatchSched sched() const
    {
        return BatchSched{d_order, d_pref, d_start, d_m, max_n, n_items, d_queue, d_error, wait_limit_ns};
    }
};

namespace {

dp_status m_alloc(dp_multi *m, size_t bytes, void **out)
{
    void *ptr = nullptr;
    bytes = (bytes + 255) & ~(size_t)255;
    if (m->has_alloc) {
        ptr = m->alloc.alloc(bytes, (void *)m->create_stream, m->alloc.ctx);
        if (!ptr)
            return fail(DP_ERR_OOM, "allocator returned NULL for " + std::to_string(bytes) + " bytes");
    } else {
        cudaError_t e = cudaMallocAsync(&ptr, bytes, m->create_stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? DP_ERR_OOM : DP_ERR_CUDA,
                        std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        }
    }
    m->blocks.push_back(ptr);
    m->bytes_held += bytes;
    *out = ptr;
    return DP_OK;
}

template <class T>
dp_status m_alloc_n(dp_multi *m, size_t n, T **out)
{
    void *v = nullptr;
    dp_status s = m_alloc(m, n * sizeof(T), &v);
    *out = (T *)v;
    return s;
}

void release_streams(dp_multi *m)
{
    for (cudaStream_t q : m->streams) {
        cudaStreamSynchronize(q);
        cudaStreamDestroy(q);
    }
    m->streams.clear();
    for (cudaEvent_t e : m->ev_done)
        cudaEventDestroy(e);
    m->ev_done.clear();
    if (m->ev_start)
        cudaEventDestroy(m->ev_start);
    m->ev_start = nullptr;
}

void m_release(dp_multi *m)
{
    if (m->gexec)
        cudaGraphExecDestroy(m->gexec);
    m->gexec = nullptr;
    for (cudaGraphExec_t g : m->inst_graph)
        if (g)
            cudaGraphExecDestroy(g);
    m->inst_graph.clear();
    release_streams(m);
    if (m->cap_stream)
        cudaStreamDestroy(m->cap_stream);
    m->cap_stream = nullptr;
    if (!m->blocks.empty())
        cudaStreamSynchronize(m->create_stream);
    for (void *b : m->blocks) {
        if (m->has_alloc)
            m->alloc.free(b, (void *)m->create_stream, m->alloc.ctx);
        else
            cudaFree(b);
    }
    m->blocks.clear();
}

// Tiles per stage for the current rows_per_lane, the wavefront work list and
// the device descriptors (uploaded on stream s).
dp_status build_schedule(dp_multi *m, cudaStream_t s)
{
    const int B = m->B;
    for (int b = 0; b < B; ++b) {
        const DevParams &P = m->hP[b];
        m->h_inst[b].chunks = persistent_chunks_per_row(m->rows_per_lane, P.n_xi, P.n_t);
        m->h_inst[b].tiles = P.n_v * m->h_inst[b].chunks;
    }
    std::vector<int> order(B);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return m->hP[a].N > m->hP[b].N; });
    std::vector<long long> pref(B + 1, 0);
    for (int r = 0; r < B; ++r)
        pref[r + 1] = pref[r] + m->h_inst[order[r]].tiles;
    std::vector<long long> start(m->max_n + 1, 0);
    std::vector<int> mj(std::max(m->max_n, 1), 0);
    int cnt = B;
    for (int j = 0; j < m->max_n; ++j) {
        while (cnt > 0 && m->hP[order[cnt - 1]].N <= j)
            --cnt;
        mj[j] = cnt;
        start[j + 1] = start[j] + pref[cnt];
    }
    m->n_items = start[m->max_n];
    DP_CUDA(cudaMemcpyAsync(m->d_order, order.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    DP_CUDA(cudaMemcpyAsync(m->d_pref, pref.data(), (B + 1) * sizeof(long long), cudaMemcpyHostToDevice, s));
    DP_CUDA(cudaMemcpyAsync(m->d_start, start.data(), (m->max_n + 1) * sizeof(long long), cudaMemcpyHostToDevice,
                            s));
    DP_CUDA(cudaMemcpyAsync(m->d_m, mj.data(), mj.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    DP_CUDA(cudaMemcpyAsync(m->d_inst, m->h_inst.data(), B * sizeof(BatchInst), cudaMemcpyHostToDevice, s));
    // the host vectors die here: make the copies complete first
    DP_CUDA(cudaStreamSynchronize(s));
    return DP_OK;
}

dp_status enqueue_multi(dp_multi *m, cudaStream_t s, cudaEvent_t ev_mid)
{
    DP_CUDA(cudaMemsetAsync(m->d_done, 0, m->done_total * sizeof(int), s));
    DP_CUDA(cudaMemsetAsync(m->d_queue, 0, sizeof(unsigned long long), s));
    DP_CUDA(cudaMemsetAsync(m->d_error, 0, sizeof(int), s));
    DP_CUDA(launch_terminal_batched(m->d_params, m->d_inst, m->B, s));
    DP_CUDA(launch_precompute_batched(m->d_params, m->d_inst, m->B, m->n_rows, m->max_n_u, s));
    if (ev_mid)
        DP_CUDA(cudaEventRecord(ev_mid, s));
    DP_CUDA(launch_persistent(m->d_params, m->d_inst, m->sched(), m->rows_per_lane, m->max_n_cls, m->max_n_u,
                              m->ctas_per_sm, s));
    return DP_OK;
}

dp_status check_error_flag(dp_multi *m, cudaStream_t s)
{
    int flag = 0;
    DP_CUDA(cudaMemcpyAsync(&flag, m->d_error, sizeof(int), cudaMemcpyDeviceToHost, s));
    DP_CUDA(cudaStreamSynchronize(s));
    if (flag)
        return fail(DP_ERR_TIMEOUT, "a dependency wait of the persistent Bellman launch timed out");
    return DP_OK;
}

// One instance's sweep with the single-problem launchers on the batch's
// buffers (results identical to a dp_problem of the same descriptor).
dp_status enqueue_instance(dp_multi *m, int b, cudaStream_t s)
{
    const DevParams &P = m->hP[b];
    const BatchInst &I = m->h_inst[b];
    const DevParams *dP = m->d_params + b;
    float4 *q = m->quad[b];
    auto V = [&](int k) { return I.V + (size_t)k * I.stage_elems; };
    auto Q = [&](int k) { return q ? q + (size_t)(k & 1) * m->quad_elems[b] : nullptr; };
    // the stages' last feasible time columns, as in a single-problem sweep
    StageScratch sc = I.sc;
    sc.lmax = b < (int)m->lmax.size() ? m->lmax[b] : nullptr;
    if (sc.lmax)
        DP_CUDA(cudaMemsetAsync(sc.lmax, 0xff, (size_t)(P.N + 1) * sizeof(int), s));
    DP_CUDA(launch_terminal(dP, P, V(P.N), s));
    if (q)
        DP_CUDA(launch_quad_from_pad(P, V(P.N), Q(P.N), s));
    DP_CUDA(launch_precompute(dP, P, I.tb, 0, P.N, I.sc, s));
    for (int k = P.N - 1; k >= 0; --k)
        DP_CUDA(launch_bellman(dP, P, I.tb, k, sc, V(k + 1), V(k), I.pi + (size_t)k * I.pi_elems, 1, s, Q(k + 1),
                               Q(k)));
    return DP_OK;
}

// Switch to the per-instance mode with K streams: corner quads and per-instance
// graphs on first use, the instances dealt by decreasing work to the stream
// with the least work so far.
dp_status set_streams(dp_multi *m, int K)
{
    if (K < 1 || K > 16)
        return fail(DP_ERR_INVALID_ARG, "streams must be in [1, 16]");
    cudaStream_t cs = m->create_stream;
    if (!m->quads_ready) {
        m->quad.assign(m->B, nullptr);
        m->quad_elems.assign(m->B, 0);
        m->lmax.assign(m->B, nullptr);
        for (int b = 0; b < m->B; ++b) {
            const DevParams &P = m->hP[b];
            dp_status st_l = m_alloc_n(m, (size_t)P.N + 1, &m->lmax[b]);
            if (st_l != DP_OK)
                return st_l;
            const size_t e = (size_t)P.n_v * quad_rows(P.n_xi) * quad_ld(P.n_t);
            if (e == 0)
                continue;
            dp_status st = m_alloc_n(m, 2 * e, &m->quad[b]);
            if (st != DP_OK)
                return st;
            m->quad_elems[b] = e;
            DP_CUDA(launch_fill(reinterpret_cast<float *>(m->quad[b]), 8 * e, V_BIG, cs));
        }
        DP_CUDA(cudaStreamSynchronize(cs));
        m->quads_ready = true;
    }
    if (m->inst_graph.empty()) {
        m->inst_graph.assign(m->B, nullptr);
        for (int b = 0; b < m->B; ++b) {
            cudaGraph_t g = nullptr;
            DP_CUDA(cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
            dp_status st = enqueue_instance(m, b, m->cap_stream);
            cudaError_t e = cudaStreamEndCapture(m->cap_stream, &g);
            if (st != DP_OK) {
                if (g)
                    cudaGraphDestroy(g);
                return st;
            }
            if (e != cudaSuccess)
                return fail(DP_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
            e = cudaGraphInstantiate(&m->inst_graph[b], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                m->inst_graph[b] = nullptr;
                return fail(DP_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
            }
        }
    }
    if ((int)m->streams.size() != K) {
        release_streams(m);
        m->streams.assign(K, nullptr);
        m->ev_done.assign(K, nullptr);
        for (int q = 0; q < K; ++q) {
            DP_CUDA(cudaStreamCreateWithFlags(&m->streams[q], cudaStreamNonBlocking));
            DP_CUDA(cudaEventCreateWithFlags(&m->ev_done[q], cudaEventDisableTiming));
        }
        DP_CUDA(cudaEventCreateWithFlags(&m->ev_start, cudaEventDisableTiming));
    }
    std::vector<double> work(m->B);
    for (int b = 0; b < m->B; ++b) {
        const DevParams &P = m->hP[b];
        work[b] = (double)P.N * P.n_v * P.n_xi * P.n_t * P.n_u;
    }
    m->launch_order.resize(m->B);
    std::iota(m->launch_order.begin(), m->launch_order.end(), 0);
    std::stable_sort(m->launch_order.begin(), m->launch_order.end(), [&](int a, int b) { return work[a] > work[b]; });
    std::vector<double> load(K, 0.0);
    m->stream_of.assign(m->B, 0);
    for (int b : m->launch_order) {
        const int q = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        m->stream_of[b] = q;
        load[q] += work[b];
    }
    m->n_streams = K;
    m->solved = false;
    return DP_OK;
}

// The per-instance solve on the caller's stream s (forked and joined).
dp_status enqueue_streams(dp_multi *m, cudaStream_t s)
{
    DP_CUDA(cudaMemsetAsync(m->d_error, 0, sizeof(int), s));  // no dependency waits in this mode
    DP_CUDA(cudaEventRecord(m->ev_start, s));
    for (cudaStream_t q : m->streams)
        DP_CUDA(cudaStreamWaitEvent(q, m->ev_start, 0));
    for (int b : m->launch_order)
        DP_CUDA(cudaGraphLaunch(m->inst_graph[b], m->streams[m->stream_of[b]]));
    for (size_t q = 0; q < m->streams.size(); ++q) {
        DP_CUDA(cudaEventRecord(m->ev_done[q], m->streams[q]));
        DP_CUDA(cudaStreamWaitEvent(s, m->ev_done[q], 0));
    }
    return DP_OK;
}

dp_status set_config(dp_multi *m, int rows_per_lane, int ctas_per_sm)
{
    if (rows_per_lane != 0 && rows_per_lane != 4 && rows_per_lane != 8)
        return fail(DP_ERR_INVALID_ARG, "rows_per_lane must be 0, 4 or 8");
    const int R = rows_per_lane ? rows_per_lane : 8;
    const int fit = persistent_max_ctas_per_sm(R, m->max_n_cls, m->max_n_u);
    if (fit < 1)
        return fail(DP_ERR_INVALID_ARG, "the largest instance's tables do not fit in shared memory");
    if (ctas_per_sm < 0 || ctas_per_sm > fit)
        return fail(DP_ERR_INVALID_ARG, "ctas_per_sm must be in [0, " + std::to_string(fit) + "]");
    m->rows_per_lane = R;
    m->ctas_per_sm = ctas_per_sm;
    m->n_streams = 0;
    if (m->gexec)
        cudaGraphExecDestroy(m->gexec);
    m->gexec = nullptr;
    m->solved = false;
    return build_schedule(m, m->create_stream);
}

}  // namespace

extern "C" {

dp_status dp_multi_create(const dp_problem_desc *descs, int32_t n, const dp_multi_opts *opts,
                          const dp_allocator *alloc, void *stream, dp_multi_t *out)
{
    if (!out)
        return fail(DP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!descs || n < 1 || n > (1 << 20))
        return fail(DP_ERR_INVALID_ARG, "need 1 <= n <= 2^20 descriptors");
    if (alloc && (!alloc->alloc || !alloc->free))
        return fail(DP_ERR_INVALID_ARG, "allocator needs both alloc and free");
    for (int b = 0; b < n; ++b) {
        dp_status st = validate(&descs[b]);
        if (st != DP_OK)
            return fail(st, "instance " + std::to_string(b) + ": " + last_error());
    }
    dp_multi *m = new (std::nothrow) dp_multi();
    if (!m)
        return fail(DP_ERR_OOM, "host allocation failed");
    m->B = n;
    m->create_stream = (cudaStream_t)stream;
    if (alloc) {
        m->alloc = *alloc;
        m->has_alloc = true;
    }
    m->hP.resize(n);
    m->ht.resize(n);
    m->h_inst.resize(n);
    size_t n_grade = 0, n_lon = 0, n_light = 0;
    for (int b = 0; b < n; ++b) {
        fill_params(&descs[b], m->hP[b]);
        fill_tables(&descs[b], m->ht[b]);
        const DevParams &P = m->hP[b];
        m->max_n = std::max(m->max_n, P.N);
        m->max_n_u = std::max(m->max_n_u, P.n_u);
        m->max_n_cls = std::max(m->max_n_cls, P.n_cls);
        m->n_rows += (long long)P.N * P.n_v;
        m->done_total += P.N;
        n_grade += m->ht[b].grade.size();
        n_lon += m->ht[b].lon.size();
        n_light += m->ht[b].cyc.size();
    }
    dp_status st = DP_OK;
#define TRY(x)              \
    do {                    \
        st = (x);           \
        if (st != DP_OK) {  \
            m_release(m);   \
            delete m;       \
            return st;      \
        }                   \
    } while (0)
    if (m->max_n_cls > MAX_CLASSES)
        TRY(fail(DP_ERR_INVALID_ARG, "at most 4095 torque classes per instance"));
    TRY(m_alloc_n(m, n, &m->d_params));
    TRY(m_alloc_n(m, n, &m->d_inst));
    TRY(m_alloc_n(m, m->done_total, &m->d_done));
    TRY(m_alloc_n(m, n_grade, &m->d_grade));
    TRY(m_alloc_n(m, n_lon, &m->d_lon));
    TRY(m_alloc_n(m, n_light, &m->d_cyc));
    TRY(m_alloc_n(m, n_light, &m->d_red));
    TRY(m_alloc_n(m, n_light, &m->d_off));
    TRY(m_alloc_n(m, n, &m->d_order));
    TRY(m_alloc_n(m, (size_t)n + 1, &m->d_pref));
    TRY(m_alloc_n(m, (size_t)m->max_n + 1, &m->d_start));
    TRY(m_alloc_n(m, (size_t)m->max_n, &m->d_m));
    TRY(m_alloc_n(m, 1, &m->d_queue));
    TRY(m_alloc_n(m, 1, &m->d_error));
    size_t o_grade = 0, o_lon = 0, o_light = 0, o_done = 0, max_pi = 0;
    long long row_off = 0;
    m->out_off.resize(n);
    m->u_off.resize(n);
    std::vector<float> all_grade, all_cyc, all_red, all_off;
    std::vector<int> all_lon;
    for (int b = 0; b < n; ++b) {
        const DevParams &P = m->hP[b];
        const HostTables &T = m->ht[b];
        BatchInst &I = m->h_inst[b];
        I.tb = StageTables{m->d_grade + o_grade, m->d_lon + o_lon, m->d_cyc + o_light, m->d_red + o_light,
                           m->d_off + o_light};
        all_grade.insert(all_grade.end(), T.grade.begin(), T.grade.end());
        all_lon.insert(all_lon.end(), T.lon.begin(), T.lon.end());
        all_cyc.insert(all_cyc.end(), T.cyc.begin(), T.cyc.end());
        all_red.insert(all_red.end(), T.red.begin(), T.red.end());
        all_off.insert(all_off.end(), T.off.begin(), T.off.end());
        o_grade += T.grade.size();
        o_lon += T.lon.size();
        o_light += T.cyc.size();
        I.stage_elems = (size_t)P.n_v * P.xi_rows * P.ld_t;
        I.pi_elems = (size_t)P.n_v * P.n_xi * P.n_t;
        max_pi = std::max(max_pi, I.pi_elems);
        I.N = P.N;
        I.pad = 0;
        I.done = m->d_done + o_done;
        o_done += P.N;
        I.row_off = row_off;
        row_off += (long long)P.N * P.n_v;
        const size_t rows = (size_t)P.N * P.n_v;
        TRY(m_alloc_n(m, I.stage_elems * (size_t)(P.N + 1), &I.V));
        TRY(m_alloc_n(m, I.pi_elems * (size_t)P.N, &I.pi));
        TRY(m_alloc_n(m, rows * P.n_cls, &I.sc.cls));
        TRY(m_alloc_n(m, rows * P.n_cls, &I.sc.ent));
        TRY(m_alloc_n(m, rows * 2, &I.sc.row_cnt));
        TRY(m_alloc_n(m, rows * P.n_u, &I.sc.spl));
        I.sc.stats = nullptr;
        I.sc.part = nullptr;
        I.sc.lmax = nullptr;
        I.sc.fill_slots = 0;  // the instances share the GPU
        m->out_off[b] = m->out_total;
        m->out_total += (long long)roll_doubles(P.N);
        m->u_off[b] = m->u_total;
        m->u_total += P.N;
    }
    TRY(m_alloc_n(m, (size_t)3 * n, &m->d_x0));
    TRY(m_alloc_n(m, (size_t)m->out_total, &m->d_out));
    TRY(m_alloc_n(m, (size_t)m->u_total, &m->d_out_u));
    TRY(m_alloc_n(m, (size_t)n, &m->d_out_off));
    TRY(m_alloc_n(m, (size_t)n, &m->d_u_off));
    TRY(m_alloc_n(m, max_pi, &m->d_dense));
    cudaStream_t s = m->create_stream;
    auto cuda_try = [&](cudaError_t e, const char *what) -> dp_status {
        if (e != cudaSuccess)
            return fail(DP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
        return DP_OK;
    };
    TRY(cuda_try(cudaMemsetAsync(m->d_error, 0, sizeof(int), s), "clear error flag"));
    TRY(cuda_try(cudaMemcpyAsync(m->d_params, m->hP.data(), n * sizeof(DevParams), cudaMemcpyHostToDevice, s),
                 "copy params"));
    TRY(cuda_try(cudaMemcpyAsync(m->d_grade, all_grade.data(), all_grade.size() * sizeof(float),
                                 cudaMemcpyHostToDevice, s),
                 "copy grade"));
    TRY(cuda_try(cudaMemcpyAsync(m->d_lon, all_lon.data(), all_lon.size() * sizeof(int), cudaMemcpyHostToDevice, s),
                 "copy lights"));
    TRY(cuda_try(cudaMemcpyAsync(m->d_cyc, all_cyc.data(), all_cyc.size() * sizeof(float), cudaMemcpyHostToDevice,
                                 s),
                 "copy cycles"));
    TRY(cuda_try(cudaMemcpyAsync(m->d_red, all_red.data(), all_red.size() * sizeof(float), cudaMemcpyHostToDevice,
                                 s),
                 "copy red"));
    TRY(cuda_try(cudaMemcpyAsync(m->d_off, all_off.data(), all_off.size() * sizeof(float), cudaMemcpyHostToDevice,
                                 s),
                 "copy offsets"));
    TRY(cuda_try(cudaMemcpyAsync(m->d_out_off, m->out_off.data(), n * sizeof(long long), cudaMemcpyHostToDevice, s),
                 "copy offsets"));
    TRY(cuda_try(cudaMemcpyAsync(m->d_u_off, m->u_off.data(), n * sizeof(long long), cudaMemcpyHostToDevice, s),
                 "copy offsets"));
    // every padding cell of every V holds the infeasible sentinel for the object's life
    for (int b = 0; b < n; ++b) {
        const BatchInst &I = m->h_inst[b];
        TRY(cuda_try(launch_fill(I.V, I.stage_elems * (size_t)(I.N + 1), V_BIG, s), "fill V"));
    }
    TRY(cuda_try(cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking), "cudaStreamCreate"));
    if (opts && opts->wait_limit_ms < 0)
        TRY(fail(DP_ERR_INVALID_ARG, "wait_limit_ms must be >= 0"));
    if (opts && opts->wait_limit_ms > 0)
        m->wait_limit_ns = (unsigned long long)opts->wait_limit_ms * 1000000ull;
    // build_schedule synchronises s, so the host staging vectors above outlive their copies
    TRY(set_config(m, opts ? opts->rows_per_lane : 0, opts ? opts->ctas_per_sm : 0));
#undef TRY
    *out = m;
    return DP_OK;
}

dp_status dp_multi_destroy(dp_multi_t m)
{
    if (!m)
        return DP_OK;
    m_release(m);
    delete m;
    return DP_OK;
}

dp_status dp_multi_set_config(dp_multi_t m, int32_t rows_per_lane, int32_t ctas_per_sm)
{
    if (!m)
        return fail(DP_ERR_INVALID_ARG, "batch is NULL");
    return set_config(m, rows_per_lane, ctas_per_sm);
}

dp_status dp_multi_solve(dp_multi_t m, void *stream)
{
    NvtxRange nvtx_("ecodp.batch.solve");
    if (!m)
        return fail(DP_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (m->n_streams > 0) {
        dp_status st = enqueue_streams(m, s);
        if (st != DP_OK)
            return st;
        m->solved = true;
        return DP_OK;
    }
    if (!m->gexec) {
        cudaGraph_t g = nullptr;
        DP_CUDA(cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
        dp_status st = enqueue_multi(m, m->cap_stream, nullptr);
        cudaError_t e = cudaStreamEndCapture(m->cap_stream, &g);
        if (st != DP_OK) {
            if (g)
                cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess)
            return fail(DP_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&m->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            m->gexec = nullptr;
            return fail(DP_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        }
    }
    DP_CUDA(cudaGraphLaunch(m->gexec, s));
    m->solved = true;
    return DP_OK;
}

dp_status dp_multi_wait(dp_multi_t m, void *stream)
{
    if (!m)
        return fail(DP_ERR_INVALID_ARG, "batch is NULL");
    return checks_after(check_error_flag(m, (cudaStream_t)stream));
}

dp_status dp_multi_profile(dp_multi_t m, void *stream, float ms[3])
{
    if (!m || !ms)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    for (auto &e : ev)
        DP_CUDA(cudaEventCreate(&e));
    auto run = [&]() -> dp_status {
        DP_CUDA(cudaEventRecord(ev[0], s));
        dp_status st = DP_OK;
        if (m->n_streams > 0) {  // not separable: everything counts as Bellman time
            DP_CUDA(cudaEventRecord(ev[1], s));
            st = enqueue_streams(m, s);
        } else {
            st = enqueue_multi(m, s, ev[1]);
        }
        if (st != DP_OK)
            return st;
        DP_CUDA(cudaEventRecord(ev[2], s));
        DP_CUDA(cudaEventSynchronize(ev[2]));
        DP_CUDA(cudaEventElapsedTime(&ms[0], ev[0], ev[1]));
        DP_CUDA(cudaEventElapsedTime(&ms[1], ev[1], ev[2]));
        DP_CUDA(cudaEventElapsedTime(&ms[2], ev[0], ev[2]));
        return check_error_flag(m, s);
    };
    dp_status st = run();
    for (auto &e : ev)
        cudaEventDestroy(e);
    if (st == DP_OK)
        m->solved = true;
    return st;
}

dp_status dp_multi_set_streams(dp_multi_t m, int32_t streams)
{
    if (!m)
        return fail(DP_ERR_INVALID_ARG, "batch is NULL");
    if (streams == 0)
        return set_config(m, m->rows_per_lane, m->ctas_per_sm);
    return set_streams(m, streams);
}

dp_status dp_multi_autotune(dp_multi_t m, void *stream, int32_t repeats, int32_t best[3], float *best_ms)
{
    if (!m || !best)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    if (repeats < 1 || repeats > 100)
        return fail(DP_ERR_INVALID_ARG, "repeats must be in [1, 100]");
    float t_best = INFINITY;
    int r_best = 0, c_best = 0, k_best = 0;
    const int Rs[2] = {4, 8};
    for (int R : Rs) {
        const int fit = persistent_max_ctas_per_sm(R, m->max_n_cls, m->max_n_u);
        for (int c = 1; c <= fit; ++c) {
            dp_status st = set_config(m, R, c);
            if (st != DP_OK)
                return st;
            float t = INFINITY;
            for (int q = 0; q < repeats + 1; ++q) {  // the first run warms up
                float ms[3];
                st = dp_multi_profile(m, stream, ms);
                if (st != DP_OK)
                    return st;
                if (q > 0)
                    t = std::min(t, ms[2]);
            }
            if (t < t_best) {
                t_best = t;
                r_best = R;
                c_best = c;
            }
        }
    }
    // the per-instance mode on 2, 4 and 8 streams
    const int Ks[3] = {2, 4, 8};
    for (int K : Ks) {
        dp_status st = set_streams(m, K);
        if (st != DP_OK)
            return st;
        float t = INFINITY;
        for (int q = 0; q < repeats + 1; ++q) {
            float ms[3];
            st = dp_multi_profile(m, stream, ms);
            if (st != DP_OK)
                return st;
            if (q > 0)
                t = std::min(t, ms[2]);
        }
        if (t < t_best) {
            t_best = t;
            k_best = K;
        }
    }
    dp_status st = k_best > 0 ? set_streams(m, k_best) : set_config(m, r_best, c_best);
    if (st != DP_OK)
        return st;
    float ms[3];
    st = dp_multi_profile(m, stream, ms);  // leaves the batch solved in the chosen configuration
    if (st != DP_OK)
        return st;
    best[0] = k_best > 0 ? 0 : r_best;
    best[1] = k_best > 0 ? 0 : c_best;
    best[2] = k_best;
    if (best_ms)
        *best_ms = t_best;
    return DP_OK;
}

dp_status dp_multi_debug_stall(dp_multi_t m, int32_t b)
{
    if (!m || b < 0 || b >= m->B)
        return fail(DP_ERR_INVALID_ARG, "bad batch or instance");
    BatchInst I = m->h_inst[b];
    I.tiles += 1;  // a completion target that the instance's tiles never reach
    DP_CUDA(cudaMemcpyAsync(m->d_inst + b, &I, sizeof I, cudaMemcpyHostToDevice, m->create_stream));
    DP_CUDA(cudaStreamSynchronize(m->create_stream));
    return DP_OK;
}

dp_status dp_multi_info(dp_multi_t m, int64_t out[9])
{
    if (!m || !out)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    int dev = 0, sms = 0;
    DP_CUDA(cudaGetDevice(&dev));
    DP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int fit = persistent_max_ctas_per_sm(m->rows_per_lane, m->max_n_cls, m->max_n_u);
    const int per_sm = m->ctas_per_sm > 0 ? std::min(m->ctas_per_sm, fit) : fit;
    int64_t nominal = 0;
    for (const DevParams &P : m->hP)
        nominal += (int64_t)P.N * P.n_v * P.n_xi * P.n_t * P.n_u;
    out[0] = m->B;
    out[1] = m->n_items;
    out[2] = (int64_t)sms * per_sm;
    out[3] = m->rows_per_lane;
    out[4] = per_sm;
    out[5] = nominal;
    out[6] = (int64_t)m->bytes_held;
    out[7] = m->max_n;
    out[8] = m->n_streams;
    return DP_OK;
}

dp_status dp_multi_get_value(dp_multi_t m, int32_t b, int32_t stage, float *out, int32_t out_is_host, void *stream)
{
    if (!m || !out)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    if (b < 0 || b >= m->B)
        return fail(DP_ERR_INVALID_ARG, "instance out of range");
    const DevParams &P = m->hP[b];
    const BatchInst &I = m->h_inst[b];
    if (stage < 0 || stage > P.N)
        return fail(DP_ERR_INVALID_ARG, "stage out of range");
    if (!m->solved)
        return fail(DP_ERR_NOT_SOLVED, "call dp_multi_solve first");
    cudaStream_t s = (cudaStream_t)stream;
    float *dst = out_is_host ? m->d_dense : out;
    DP_CUDA(launch_dense_from_pad(P, I.V + (size_t)stage * I.stage_elems, dst, s));
    if (out_is_host)
        DP_CUDA(cudaMemcpyAsync(out, m->d_dense, I.pi_elems * sizeof(float), cudaMemcpyDeviceToHost, s));
    return check_error_flag(m, s);
}

dp_status dp_multi_get_policy(dp_multi_t m, int32_t b, int32_t stage, int16_t *out, int32_t out_is_host,
                              void *stream)
{
    if (!m || !out)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    if (b < 0 || b >= m->B)
        return fail(DP_ERR_INVALID_ARG, "instance out of range");
    const DevParams &P = m->hP[b];
    const BatchInst &I = m->h_inst[b];
    if (stage < 0 || stage >= P.N)
        return fail(DP_ERR_INVALID_ARG, "stage out of range");
    if (!m->solved)
        return fail(DP_ERR_NOT_SOLVED, "call dp_multi_solve first");
    cudaStream_t s = (cudaStream_t)stream;
    DP_CUDA(cudaMemcpyAsync(out, I.pi + (size_t)stage * I.pi_elems, I.pi_elems * sizeof(int16_t),
                            out_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    return check_error_flag(m, s);
}

static dp_status multi_rollout_impl(dp_multi_t m, const double *x0, dp_trajectory *traj, void *stream)
{
    if (!m || !x0 || !traj)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    for (int b = 0; b < m->B; ++b) {
        const dp_trajectory &T = traj[b];
        if (!T.v || !T.soc || !T.t || !T.u || !T.dt || !T.wait || !T.fuel)
            return fail(DP_ERR_INVALID_ARG, "trajectory " + std::to_string(b) + ": arrays must all be provided");
        if (!finite3(x0 + 3 * b))
            return fail(DP_ERR_INVALID_ARG, "x0 must be finite");
    }
    if (!m->solved)
        return fail(DP_ERR_NOT_SOLVED, "call dp_multi_solve first");
    cudaStream_t s = (cudaStream_t)stream;
    DP_CUDA(cudaMemcpyAsync(m->d_x0, x0, 3 * m->B * sizeof(double), cudaMemcpyHostToDevice, s));
    DP_CUDA(launch_rollout_batched(m->d_params, m->d_inst, m->B, m->d_x0, m->d_out_off, m->d_u_off, m->d_out,
                                   m->d_out_u, s));
    std::vector<double> h(m->out_total);
    std::vector<int> hu(m->u_total);
    DP_CUDA(cudaMemcpyAsync(h.data(), m->d_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    DP_CUDA(cudaMemcpyAsync(hu.data(), m->d_out_u, hu.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
    dp_status st = check_error_flag(m, s);  // synchronises s
    if (st != DP_OK)
        return st;
    int first_fail = -1;
    for (int b = 0; b < m->B; ++b) {
        const int fs = unpack_rollout(m->hP[b].N, h.data() + m->out_off[b], hu.data() + m->u_off[b], &traj[b]);
        if (fs >= 0 && first_fail < 0)
            first_fail = b;
    }
    if (first_fail >= 0)
        return fail(DP_ERR_INFEASIBLE, "instance " + std::to_string(first_fail) + ": no feasible control at stage " +
                                           std::to_string(traj[first_fail].fail_stage));
    return DP_OK;
}

dp_status dp_multi_rollout(dp_multi_t m, const double *x0, dp_trajectory *traj, void *stream)
{
    return checks_after(multi_rollout_impl(m, x0, traj, stream));
}

}  // extern "C"
