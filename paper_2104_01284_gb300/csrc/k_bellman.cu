// Bellman stage kernels for one problem (Eq. 9b-9d), on the per-stage tables
// of the precompute kernel.  Two variants compute bit-identical results:
//   * bellman_direct: one thread per state, every control evaluated with its
//     own reads of J_{k+1} (the layout of the paper's second kernel, Sec. IV);
//   * bellman_tiled: one CTA per tile (speed row, 128 lanes) running the
//     torque-class tile of bellman_tile.cuh; on grids whose tiles cannot fill
//     the GPU, bellman_slice + bellman_join split each tile's classes.
#include <cfloat>
#include <climits>

#include <algorithm>

#include "bellman_tile.cuh"

#undef ECODP_FILE_TAG
#define ECODP_FILE_TAG 2

namespace ecodp {

ECODP_CHECK_ACCESSOR(check_word_bellman)

namespace {

using namespace tile;

// SoC rows per lane of the single-problem kernels: 8, or 6 where it fills
// the lanes markedly better (tile_rows); CTAs per SM the register budget is
// sized for: 4 at 8 rows (128 registers), 5 at 6 rows (96 registers).
template <int R>
constexpr int tile_minb() { return R == 8 ? 4 : 5; }

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
    if (!DP_IN(row, (size_t)P.N * P.n_v))
        return;
    const int n_ent = sc.row_cnt[2 * row];
    const ClassRec *cls = sc.cls + row * P.n_cls;
    const ClassEntry *ent = sc.ent + row * P.n_cls;
    const SplitRec *spl = sc.spl + row * P.n_u;

    // minimum in the order (value, class, control index)
    float best = __int_as_float(0x7f800000);
    int bu = INT_MAX, be = -1;
    for (int e = 0; e < n_ent; ++e) {
        if (!DP_IN(e, P.n_cls))
            break;
        const ClassEntry E = ent[e];
        if (!DP_IN(E.cls, P.n_cls) || !DP_IN(E.off, P.n_u + 1) || !DP_IN((long long)E.off + E.n_total, P.n_u + 1))
            continue;
        const TCtx x = class_ctx(P, Vn, cls[E.cls], l, tl, wait, si);
        for (int q = E.off; q < E.off + E.n_total; ++q) {
            const SplitRec S = spl[q];
            const int d = split_d(S), u = split_u(S);
            const float F = split_value(S.c, S.f, g_at<true>(P, x, j + d), g_at<true>(P, x, j + d + 1));
            if (F < best || (F == best && e == be && u < bu)) {
                best = F;
                bu = u;
                be = e;
            }
        }
    }
    const size_t o = ((size_t)i * P.xi_rows + (j + 1)) * P.ld_t + l;
    const size_t op = ((size_t)i * P.n_xi + j) * P.n_t + l;
    if (!(best < V_FEAS_MAX) || sampled_red(P, tb, si, v, tl)) {
        Vk[o] = V_BIG;
        pik[op] = -1;
    } else {
        Vk[o] = __fadd_rn(best, __fmul_rn(__fsub_rn(1.f, P.gamma), wait));
        pik[op] = (int16_t)bu;
    }
}

// QLD > 0: windows read from the corner quads Qn of J_{k+1} (row stride QLD),
// J_k's quads written to Qk (a sweep whose every stage takes this kernel).
template <int R, int QLD>
__global__ void __launch_bounds__(TLANES, tile_minb<R>())
    bellman_tiled(const DevParams *__restrict__ dP, StageTables tb, int k, StageScratch sc,
                  const float *__restrict__ Vn, float *__restrict__ Vk, int16_t *__restrict__ pik,
                  const float4 *__restrict__ Qn, float4 *__restrict__ Qk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ DevParams P;
    if (threadIdx.x == 0)
        P = *dP;
    __syncthreads();
    // speed rows in descending order: the CTA scheduler places CTAs round
    // robin over the SMs, so the light low-speed rows (few feasible classes)
    // come last and fill the SMs that received a fourth CTA
    const int i = gridDim.y - 1 - blockIdx.y;
    const size_t row = (size_t)k * P.n_v + i;
    // in a sweep: J_{k+1}'s last feasible time column (J_N is finite
    // everywhere), and J_k's to record
    int lmax_next = INT_MAX;
    int *lmax_out = nullptr;
    if (sc.lmax && DP_IN(k, P.N)) {
        lmax_next = k + 1 >= P.N ? P.n_t - 1 : sc.lmax[k + 1];
        lmax_out = sc.lmax + k;
    }
    bellman_tile<R, true, TILE_FULL, QLD>(P, tb, k, sc.cls + row * P.n_cls, sc.ent + row * P.n_cls,
                                           sc.spl + row * P.n_u, sc.row_cnt[2 * row], sc.row_cnt[2 * row + 1], Vn,
                                           Vk, pik, i, blockIdx.x, smem_raw, sc.stats, 0, 0, nullptr, Qn, Qk,
                                           lmax_next, lmax_out, sc.lmax ? (int)gridDim.x : 0);
}

// Row plan of a sweep stage that runs alone (every CTA computes the same):
// speed row r's class table costs 12 per class plus its lines (class_cost in
// bellman_tile.cuh), and takes c1, c2 or c4 tiles (its lanes at 1, 2 or 4 class
// slices per lane group) for the least target cost tau such that the rows
// with cost <= tau take c1, <= 2 tau c2, the rest c4, and all tiles fit in
// the launch's G CTAs; so the rows that cost most split their classes first.
// CTA b takes the row whose tiles, in row order, hold b: out = {row, tile of
// the row, tiles of the row}, row -1 for a CTA beyond them.  Warp 0 only.
constexpr int PLAN_ROWS_PER_LANE = 8;  // up to 256 speed rows

__device__ void plan_tile(const DevParams &P, const StageScratch &sc, int k, int n_act, int b, int G, int *out)
{
    const int lane = threadIdx.x & 31;
    const int c1 = max((n_act + TLANES - 1) / TLANES, 1);
    const int c2 = max((2 * n_act + TLANES - 1) / TLANES, 1);
    const int c4 = max((4 * n_act + TLANES - 1) / TLANES, 1);
    int cost[PLAN_ROWS_PER_LANE];
    int cmax = 0;
#pragma unroll
    for (int q = 0; q < PLAN_ROWS_PER_LANE; ++q) {
        const int r = lane + 32 * q;
        cost[q] = -1;
        if (r < P.n_v) {
            const size_t row = (size_t)k * P.n_v + r;
            cost[q] = 12 * max(sc.row_cnt[2 * row], 0) + max(sc.row_cnt[2 * row + 1], 0);
            cmax = max(cmax, cost[q]);
        }
    }
    cmax = __reduce_max_sync(0xffffffffu, cmax);
    auto tiles = [&](int c, int tau) { return c < 0 ? 0 : (c <= tau ? c1 : (c <= 2 * tau ? c2 : c4)); };
    int lo = 0, hi = cmax;  // at tau = cmax every row takes c1, which fits (the host checks)
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        int n = 0;
#pragma unroll
        for (int q = 0; q < PLAN_ROWS_PER_LANE; ++q)
            n += tiles(cost[q], mid);
        if (__reduce_add_sync(0xffffffffu, n) <= G)
            hi = mid;
        else
            lo = mid + 1;
    }
    int base = 0, f_row = -1, f_tile = 0, f_n = 0;
#pragma unroll
    for (int q = 0; q < PLAN_ROWS_PER_LANE; ++q) {
        const int c = tiles(cost[q], lo);
        int incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d)
                incl += y;
        }
        const int start = base + incl - c;
        if (c > 0 && b >= start && b < start + c) {
            f_row = lane + 32 * q;
            f_tile = b - start;
            f_n = c;
        }
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
    const unsigned m = __ballot_sync(0xffffffffu, f_row >= 0);
    const int src = m ? __ffs((int)m) - 1 : 0;
    const int row = __shfl_sync(0xffffffffu, f_row, src), tile = __shfl_sync(0xffffffffu, f_tile, src),
              n = __shfl_sync(0xffffffffu, f_n, src);
    if (lane == 0) {
        out[0] = m ? row : -1;
        out[1] = tile;
        out[2] = n;
    }
}

// A sweep stage that runs alone, its tiles placed by the row plan above on a
// 1-D grid of every resident CTA slot.
template <int R, int QLD>
__global__ void __launch_bounds__(TLANES, tile_minb<R>())
    bellman_planned(const DevParams *__restrict__ dP, StageTables tb, int k, StageScratch sc,
                    const float *__restrict__ Vn, float *__restrict__ Vk, int16_t *__restrict__ pik,
                    const float4 *__restrict__ Qn, float4 *__restrict__ Qk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ DevParams P;
    __shared__ int s_plan[3];
    if (threadIdx.x == 0)
        P = *dP;
    __syncthreads();
    if (!DP_IN(k, P.N) || !sc.lmax)
        return;
    const int lmax_next = k + 1 >= P.N ? P.n_t - 1 : sc.lmax[k + 1];
    const int n_tc = lmax_next >= P.n_t - 1 ? P.n_t : max(lmax_next + 1, 0);  // as bellman_tile
    const int n_act = (P.n_xi + R - 1) / R * n_tc;
    if (threadIdx.x < 32)
        plan_tile(P, sc, k, n_act, (int)blockIdx.x, (int)gridDim.x, s_plan);
    __syncthreads();
    const int i = s_plan[0];
    if (i < 0 || i >= P.n_v || s_plan[2] < 1)
        return;  // a spare slot (uniform over the CTA)
    const size_t row = (size_t)k * P.n_v + i;
    bellman_tile<R, true, TILE_FULL, QLD>(P, tb, k, sc.cls + row * P.n_cls, sc.ent + row * P.n_cls,
                                           sc.spl + row * P.n_u, sc.row_cnt[2 * row], sc.row_cnt[2 * row + 1], Vn,
                                           Vk, pik, i, s_plan[1], smem_raw, sc.stats, 0, 0, nullptr, Qn, Qk,
                                           lmax_next, sc.lmax + k, s_plan[2]);
}

// Class-split tiles for grids whose tiles cannot fill the GPU: blockIdx.z
// picks one of gridDim.z slices of the row's class list (TILE_SLICE in
// bellman_tile.cuh); a per-state join launch then writes J_k and the argmin.
template <int R>
__global__ void __launch_bounds__(TLANES, tile_minb<R>())
    bellman_slice(const DevParams *__restrict__ dP, StageTables tb, int k, StageScratch sc,
                  const float *__restrict__ Vn)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ DevParams P;
    if (threadIdx.x == 0)
        P = *dP;
    __syncthreads();
    const int i = blockIdx.y;
    const size_t row = (size_t)k * P.n_v + i;
    const int n_ent = sc.row_cnt[2 * row];
    const int e0 = (int)((long long)n_ent * blockIdx.z / gridDim.z);
    const int e1 = (int)((long long)n_ent * (blockIdx.z + 1) / gridDim.z);
    if (e0 >= e1)
        return;  // an empty slice (uniform over the CTA)
    bellman_tile<R, true, TILE_SLICE>(P, tb, k, sc.cls + row * P.n_cls, sc.ent + row * P.n_cls,
                                      sc.spl + row * P.n_u, n_ent, sc.row_cnt[2 * row + 1], Vn, nullptr, nullptr,
                                      i, blockIdx.x, smem_raw, nullptr, e0, e1, sc.part);
}

// Join of the class-split slices, one thread per state: the packed minimum
// in `part` (value bits << 32 | class entry) gives J_k, and the lowest control
// of the winning class that reaches the value is recovered with the sweep's
// arithmetic; `part` is reset for the next stage.
__global__ void __launch_bounds__(256) bellman_join(const DevParams *__restrict__ dP, StageTables tb, int k,
                                                    StageScratch sc, const float *__restrict__ Vn,
                                                    float *__restrict__ Vk, int16_t *__restrict__ pik)
{
    __shared__ DevParams P;
    if (threadIdx.x == 0)
        P = *dP;
    __syncthreads();
    const int i = blockIdx.y;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    bool found = false;
    if (s < P.n_xi * P.n_t) {
        const int j = s / P.n_t, l = s % P.n_t;
        const float v = node_val(P.v_lo, P.v_span, i, P.n_v);
        const float tl = node_val(P.t_lo, P.t_span, l, P.n_t);
        const StageInfo si = stage_info(tb, k, v);
        const float wait = wait_time(tb, k, tl, si.wait_row);
        const size_t row = (size_t)k * P.n_v + i;
        const size_t op = ((size_t)i * P.n_xi + j) * P.n_t + l;
        const size_t o = ((size_t)i * P.xi_rows + (j + 1)) * P.ld_t + l;
        const unsigned long long w = sc.part[op];
        sc.part[op] = ~0ull;
        const float best = w != ~0ull ? __uint_as_float((unsigned)(w >> 32)) : __int_as_float(0x7f800000);
        const int we = (int)(unsigned)(w & 0xffffffffu);
        if (best < V_FEAS_MAX && !sampled_red(P, tb, si, v, tl) && DP_IN(we, sc.row_cnt[2 * row]) &&
            DP_IN(row, (size_t)P.N * P.n_v)) {
            const ClassEntry E = sc.ent[row * P.n_cls + we];
            const TCtx x = class_ctx(P, Vn, sc.cls[row * P.n_cls + E.cls], l, tl, wait, si);
            Vk[o] = __fadd_rn(best, __fmul_rn(__fsub_rn(1.f, P.gamma), wait));
            pik[op] = (int16_t)class_lowest_u_global<true>(P, x, E, sc.spl + row * P.n_u, j, best);
            found = true;
        } else {
            Vk[o] = V_BIG;
            pik[op] = -1;
        }
    }
    const unsigned n_find = __reduce_add_sync(0xffffffffu, found ? 1u : 0u);
    if (sc.stats && (threadIdx.x & 31) == 0 && n_find)
        atomicAdd(sc.stats + 3, (unsigned long long)n_find);
}

int sm_count()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 1;
    }
    return sms;
}

// Class slices per tile: as many as keep the GPU's resident CTA slots (4 per
// SM) filled, at most 8; 1 (no split) when the tiles alone fill the slots.
int class_slices(int tiles)
{
    const int s = (4 * sm_count()) / (tiles > 0 ? tiles : 1);
    return s < 1 ? 1 : (s > 8 ? 8 : s);
}

// Fraction of a launch's lanes that hold a real state with R SoC rows per
// lane: SoC groups padded to R rows, flattened (group, time) lanes padded to
// whole 128-lane tiles.
double lane_fill(int R, int n_xi, int n_t)
{
    const int groups = (n_xi + R - 1) / R;
    const long long flat = (long long)groups * n_t;
    const long long lanes = (flat + TLANES - 1) / TLANES * TLANES;
    return (double)n_xi / (groups * R) * (double)flat / (double)lanes;
}

// 6 rows per lane where they fill the lanes at least 15 % better than 8
// (measured per-state cost of 6 rows: ~5 % above 8), else 8.
int tile_rows(const DevParams &hP)
{
    return lane_fill(6, hP.n_xi, hP.n_t) > 1.15 * lane_fill(8, hP.n_xi, hP.n_t) ? 6 : 8;
}

template <int R>
cudaError_t launch_tiles(const DevParams *dP, const DevParams &hP, StageTables tb, int k, StageScratch sc,
                         const float *Vnext, float *Vk, int16_t *pik, cudaStream_t s, const float4 *Qn, float4 *Qk)
{
    const size_t smem = layout<R>(hP.n_cls, hP.n_u).total;
    const int chunks = chunks_per_row<R>(hP.n_xi, hP.n_t);
    const int slices = sc.part ? class_slices(chunks * hP.n_v) : 1;
    if (slices > 1) {
        cudaError_t err =
            cudaFuncSetAttribute(bellman_slice<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess)
            return err;
        bellman_slice<R><<<dim3(chunks, hP.n_v, slices), TLANES, smem, s>>>(dP, tb, k, sc, Vnext);
        err = cudaGetLastError();
        if (err != cudaSuccess)
            return err;
        bellman_join<<<dim3((hP.n_xi * hP.n_t + 255) / 256, hP.n_v), 256, 0, s>>>(dP, tb, k, sc, Vnext, Vk, pik);
        return cudaGetLastError();
    }
    const int qld = Qn && Qk ? quad_ld(hP.n_t) : 0;
    // a sweep that runs alone fills every resident CTA slot with tiles: by
    // the row plan where the rows fit one tile per 128 lanes, else with the
    // same number of tiles per row (tiles beyond a row's lanes take class
    // slices, bellman_tile)
    const int slots = tile_minb<R>() * sm_count();
    const bool planned = sc.lmax && sc.fill_slots && hP.n_v <= 32 * PLAN_ROWS_PER_LANE && hP.n_v * chunks <= slots;
    auto run = [&](auto kernel, auto planned_kernel) {
        if (planned) {
            cudaError_t err =
                cudaFuncSetAttribute(planned_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess)
                return err;
            planned_kernel<<<slots, TLANES, smem, s>>>(dP, tb, k, sc, Vnext, Vk, pik, Qn, Qk);
            return cudaGetLastError();
        }
        cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess)
            return err;
        const int grid_x = sc.lmax && sc.fill_slots ? std::max(chunks, slots / hP.n_v) : chunks;
        kernel<<<dim3(grid_x, hP.n_v), TLANES, smem, s>>>(dP, tb, k, sc, Vnext, Vk, pik, Qn, Qk);
        return cudaGetLastError();
    };
    switch (qld) {
    case 64:
        return run(bellman_tiled<R, 64>, bellman_planned<R, 64>);
    case 128:
        return run(bellman_tiled<R, 128>, bellman_planned<R, 128>);
    case 256:
        return run(bellman_tiled<R, 256>, bellman_planned<R, 256>);
    default:
        return run(bellman_tiled<R, 0>, bellman_planned<R, 0>);
    }
}

}  // namespace

size_t bellman_smem_bytes(const DevParams &hP)
{
    const size_t a = layout<6>(hP.n_cls, hP.n_u).total, b = layout<8>(hP.n_cls, hP.n_u).total;
    return a > b ? a : b;
}

cudaError_t launch_bellman(const DevParams *dP, const DevParams &hP, StageTables tb, int k, StageScratch sc,
                           const float *Vnext, float *Vk, int16_t *pik, int variant, cudaStream_t s,
                           const float4 *Qn, float4 *Qk)
{
    if (variant == 0) {
        dim3 grid((hP.n_xi * hP.n_t + 255) / 256, hP.n_v);
        bellman_direct<<<grid, 256, 0, s>>>(dP, tb, k, sc, Vnext, Vk, pik);
        return cudaGetLastError();
    }
    const int R = variant == 2 ? 8 : (variant == 3 ? 6 : tile_rows(hP));
    return R == 6 ? launch_tiles<6>(dP, hP, tb, k, sc, Vnext, Vk, pik, s, Qn, Qk)
                  : launch_tiles<8>(dP, hP, tb, k, sc, Vnext, Vk, pik, s, Qn, Qk);
}

}  // namespace ecodp
