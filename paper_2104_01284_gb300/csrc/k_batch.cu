// Batched backward sweeps of many uneven instances in one persistent launch.
//
// Work items are (instance b, stage k, tile) with the tiles of bellman_tile.
// They are handed out from a device counter in wavefront order: every
// instance's first backward stage (k = N_b - 1), then every instance's second,
// and so on; within a step the instances follow in order of decreasing
// horizon, so the instances taking part in step j are a prefix of that order.
// A tile of stage k needs all tiles of stage k + 1 of the same instance; it
// waits on that stage's completion counter (acquire), bounded by a time limit
// after which it records an error and goes on.  Items are only handed to
// CTAs that are running (they fetch them), and every wait is for items handed
// out earlier: the unfinished item fetched first has all its inputs, so the
// waits cannot deadlock whatever the number of resident CTAs.
#include "bellman_tile.cuh"

#undef ECODP_FILE_TAG
#define ECODP_FILE_TAG 5

namespace ecodp {

ECODP_CHECK_ACCESSOR(check_word_batch)

namespace {

using namespace tile;


__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(int *p, int v)
{
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T>
__device__ __forceinline__ int upper_bound_idx(const T *a, int n, T x)  // first index with a[idx] > x
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (a[mid] <= x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// MINB: resident CTAs per SM the register budget is sized for (4: 128
// registers per thread, 5: 96, 6: 80); the launch picks the instance for the
// requested residency.
template <int R, int MINB>
__global__ void __launch_bounds__(TLANES, MINB) bellman_persistent(const DevParams *__restrict__ params,
                                                                  const BatchInst *__restrict__ inst, BatchSched S)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ DevParams P;
    __shared__ long long s_item;
    __shared__ int s_b, s_tile, s_j;
    int cur_b = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long item = (long long)atomicAdd(S.queue, 1ull);
            s_item = item;
            if (item < S.n_items) {
                int j = upper_bound_idx(S.start, S.max_n + 1, item) - 1;
                if (!DP_IN(j, S.max_n))
                    j = 0;
                const long long r = item - S.start[j];
                int rank = upper_bound_idx(S.pref, S.m[j] + 1, r) - 1;
                if (!DP_IN(rank, S.m[j]))
                    rank = 0;
                s_j = j;
                s_b = S.order[rank];
                s_tile = (int)(r - S.pref[rank]);
            }
        }
        __syncthreads();
        if (s_item >= S.n_items)
            break;
        const int b = s_b;
        if (b != cur_b) {
            __syncthreads();  // P is still read by the previous tile until here
            if (threadIdx.x == 0)
                P = params[b];
            __syncthreads();
            cur_b = b;
        }
        const BatchInst &I = inst[b];
        const int k = I.N - 1 - s_j;
        const int i = s_tile / I.chunks;
        const int chunk = s_tile - i * I.chunks;
        if (!DP_IN(k, I.N) || !DP_IN(s_tile, I.tiles) || !DP_IN(i, P.n_v)) {
            __syncthreads();
            continue;  // uniform over the CTA (shared item); the stage's counter is left short
        }
        if (k + 1 < I.N) {  // stage k + 1 must be complete (stage N is the terminal cost)
            if (threadIdx.x == 0) {
                const unsigned long long t0 = global_ns();
                while (ld_acquire(I.done + k + 1) < I.tiles) {
                    if (global_ns() - t0 > S.wait_limit_ns) {
                        atomicExch(S.error, 1);
                        break;
                    }
                    __nanosleep(256);
                }
            }
            __syncthreads();
            (void)ld_acquire(I.done + k + 1);  // every thread orders its reads after the writers
        }
        const size_t row = (size_t)k * P.n_v + i;
        bellman_tile<R, false>(P, I.tb, k, I.sc.cls + row * P.n_cls, I.sc.ent + row * P.n_cls,
                               I.sc.spl + row * P.n_u, I.sc.row_cnt[2 * row], I.sc.row_cnt[2 * row + 1],
                               I.V + (size_t)(k + 1) * I.stage_elems, I.V + (size_t)k * I.stage_elems,
                               I.pi + (size_t)k * I.pi_elems, i, chunk, smem_raw, nullptr);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            red_release_add(I.done + k, 1);
        }
    }
}

template <int R, int MINB>
cudaError_t max_ctas_rm(size_t smem, int *per_sm)
{
    cudaError_t err =
        cudaFuncSetAttribute(bellman_persistent<R, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess)
        return err;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, bellman_persistent<R, MINB>, TLANES, smem);
    if (err != cudaSuccess)
        return err;
    if (*per_sm > MINB && MINB < 6)  // a larger budget instance is only used up to its own residency
        *per_sm = MINB;
    return *per_sm < 1 ? cudaErrorInvalidConfiguration : cudaSuccess;
}

// The most CTAs per SM any instance of rows-per-lane R reaches.
template <int R>
int max_ctas_r(size_t smem)
{
    int best = 0;
    const int budgets[3] = {4, 5, 6};
    for (int mb : budgets) {
        int n = 0;
        cudaError_t e = cudaSuccess;
        if (R == 8 && mb == 4)
            e = max_ctas_rm<8, 4>(smem, &n);
        else if (R == 8 && mb == 5)
            e = max_ctas_rm<8, 5>(smem, &n);
        else if (R == 4 && mb == 4)
            e = max_ctas_rm<4, 4>(smem, &n);
        else if (R == 4 && mb == 5)
            e = max_ctas_rm<4, 5>(smem, &n);
        else if (R == 4 && mb == 6)
            e = max_ctas_rm<4, 6>(smem, &n);
        else
            continue;
        if (e != cudaSuccess)
            cudaGetLastError();
        else
            best = n > best ? n : best;
    }
    return best;
}

template <int R, int MINB>
cudaError_t launch_rm(const DevParams *params, const BatchInst *inst, const BatchSched &S, size_t smem, int per_sm,
                      int num_sms, cudaStream_t s)
{
    int fit = 0;
    cudaError_t err = max_ctas_rm<R, MINB>(smem, &fit);
    if (err != cudaSuccess)
        return err;
    if (per_sm > fit)
        return cudaErrorInvalidConfiguration;
    bellman_persistent<R, MINB><<<num_sms * per_sm, TLANES, smem, s>>>(params, inst, S);
    return cudaGetLastError();
}

}  // namespace

size_t persistent_smem_bytes(int rows_per_lane, int max_n_cls, int max_n_u)
{
    return rows_per_lane == 4 ? layout<4>(max_n_cls, max_n_u).total : layout<8>(max_n_cls, max_n_u).total;
}

int persistent_chunks_per_row(int rows_per_lane, int n_xi, int n_t)
{
    return rows_per_lane == 4 ? chunks_per_row<4>(n_xi, n_t) : chunks_per_row<8>(n_xi, n_t);
}

int persistent_max_ctas_per_sm(int rows_per_lane, int max_n_cls, int max_n_u)
{
    const size_t smem = persistent_smem_bytes(rows_per_lane, max_n_cls, max_n_u);
    return rows_per_lane == 4 ? max_ctas_r<4>(smem) : max_ctas_r<8>(smem);
}

cudaError_t launch_persistent(const DevParams *params, const BatchInst *inst, const BatchSched &S, int rows_per_lane,
                              int max_n_cls, int max_n_u, int ctas_per_sm, cudaStream_t s)
{
    int dev = 0, num_sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess)
        return err;
    err = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess)
        return err;
    const size_t smem = persistent_smem_bytes(rows_per_lane, max_n_cls, max_n_u);
    int per_sm = ctas_per_sm;
    if (per_sm <= 0)
        per_sm = persistent_max_ctas_per_sm(rows_per_lane, max_n_cls, max_n_u);
    if (per_sm < 1)
        return cudaErrorInvalidConfiguration;
    // the smallest register budget that holds the requested residency
    if (rows_per_lane == 4) {
        if (per_sm <= 4)
            return launch_rm<4, 4>(params, inst, S, smem, per_sm, num_sms, s);
        if (per_sm == 5)
            return launch_rm<4, 5>(params, inst, S, smem, per_sm, num_sms, s);
        return launch_rm<4, 6>(params, inst, S, smem, per_sm, num_sms, s);
    }
    if (per_sm <= 4)
        return launch_rm<8, 4>(params, inst, S, smem, per_sm, num_sms, s);
    return launch_rm<8, 5>(params, inst, S, smem, per_sm, num_sms, s);
}

}  // namespace ecodp
