// FP32 FMA throughput and on-chip load bandwidth probes (measurement aids; no
// counterpart in the paper).
//
// The Bellman kernels are bound by FP32 issue, and their roofline is quoted
// against SMs x 128 FP32 lanes x 2 FLOP x SM clock.  This launch measures what
// the part actually sustains: every thread runs PEAK_CHAINS independent chains
// of packed FP32 FMAs (__ffma2_rn, two FMAs per instruction) with enough warps
// per SM to hide the FMA latency, so the FMA pipes stay busy for the whole
// launch.
#include <string>

#include "api_internal.h"

#undef ECODP_FILE_TAG
#define ECODP_FILE_TAG 8

namespace ecodp {
namespace {

constexpr int PEAK_THREADS = 256;  // 8 CTAs per SM: 64 warps
constexpr int PEAK_CTAS_PER_SM = 8;
constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_ITERS = 4096;

__global__ void __launch_bounds__(PEAK_THREADS) fp32_peak_kernel(float *out, float seed)
{
    float2 a[PEAK_CHAINS];
    const float2 m = make_float2(0.9999999f, 0.9999998f), c = make_float2(1e-7f, 2e-7f);
#pragma unroll
    for (int q = 0; q < PEAK_CHAINS; ++q)
        a[q] = make_float2(seed + 1e-6f * threadIdx.x + q, seed - q);
    for (int it = 0; it < PEAK_ITERS; ++it) {
#pragma unroll
        for (int q = 0; q < PEAK_CHAINS; ++q)
            a[q] = __ffma2_rn(a[q], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < PEAK_CHAINS; ++q)
        s += a[q].x + a[q].y;
    if (s != s)  // never true for these inputs; keeps the chains alive
        out[blockIdx.x] = s;
}

// On-chip load bandwidth probes.  Every kernel keeps 8 independent 16-byte
// loads in flight per thread and folds them with XOR, so the load path, not
// the arithmetic, limits the rate; every index is masked into its buffer.
constexpr int BW_THREADS = 256;
constexpr int BW_UNROLL = 8;
constexpr int SMEM_VEC = 2048;  // 32 KB of shared memory per CTA
constexpr int L1_VEC = 1024;    // 16 KB of global memory per CTA, re-read from L1
constexpr int BW_CTAS_PER_SM = 6;

__device__ __forceinline__ void fold(uint4 &acc, const uint4 v)
{
    acc.x ^= v.x;
    acc.y ^= v.y;
    acc.z ^= v.z;
    acc.w ^= v.w;
}

__device__ __forceinline__ void keep(const uint4 acc, unsigned *out)
{
    if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x9e3779b9u)  // an unlikely pattern; keeps the loads alive
        out[blockIdx.x] = acc.x;
}

// Shared memory: a warp reads 32 consecutive 16-byte words (no bank
// conflict); the offset moves every iteration.
__global__ void __launch_bounds__(BW_THREADS) smem_bw_kernel(unsigned *out, int iters)
{
    __shared__ uint4 sbuf[SMEM_VEC];
    for (int i = threadIdx.x; i < SMEM_VEC; i += BW_THREADS)
        sbuf[i] = make_uint4(i, 3u * i, 5u * i, 7u * i);
    __syncthreads();
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < BW_UNROLL; ++u)
            fold(acc, sbuf[(threadIdx.x + u * BW_THREADS + it * 32) & (SMEM_VEC - 1)]);
    }
    keep(acc, out);
}

// L1: each CTA re-reads its own 16 KB slice of a global buffer through L1
// (ld.global.ca); after the first pass every load hits.  A thread's 8 loads
// of an iteration sit 128 words apart, distinct modulo the slice (loads that
// coincide after the mask would be merged by the compiler).
__global__ void __launch_bounds__(BW_THREADS) l1_bw_kernel(const uint4 *buf, unsigned *out, int iters)
{
    const uint4 *mine = buf + (size_t)blockIdx.x * L1_VEC;
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < BW_UNROLL; ++u)
            fold(acc, __ldca(mine + ((threadIdx.x + u * (L1_VEC / BW_UNROLL) + it * 32) & (L1_VEC - 1))));
    }
    keep(acc, out);
}

// L2: the whole grid streams a buffer that fits in L2 (n a power of two)
// with L2-only loads (ld.global.cg); a warp reads 512 contiguous bytes.
__global__ void __launch_bounds__(BW_THREADS) l2_bw_kernel(const uint4 *buf, size_t n, int reps, unsigned *out)
{
    const size_t T = (size_t)gridDim.x * BW_THREADS, mask = n - 1;
    const size_t t = (size_t)blockIdx.x * BW_THREADS + threadIdx.x;
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
    for (int r = 0; r < reps; ++r) {
#pragma unroll
        for (int u = 0; u < BW_UNROLL; ++u)
            fold(acc, __ldcg(buf + ((t + ((size_t)r * BW_UNROLL + u) * T) & mask)));
    }
    keep(acc, out);
}

}  // namespace
}  // namespace ecodp

using namespace ecodp;
using namespace ecodp::host;

extern "C" dp_status dp_measure_fp32_peak(int32_t repeats, double *tflops, double *ms, void *stream)
{
    if (!tflops || !ms || repeats < 1)
        return fail(DP_ERR_INVALID_ARG, "tflops and ms must be provided and repeats >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    DP_CUDA(cudaGetDevice(&dev));
    DP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * PEAK_CTAS_PER_SM;
    float *out = nullptr;
    DP_CUDA(cudaMallocAsync((void **)&out, sizeof(float) * blocks, s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess)
        err = cudaEventCreate(&e1);
    float best = 0.f;
    for (int r = 0; r <= repeats && err == cudaSuccess; ++r) {  // r = 0 warms up
        err = cudaEventRecord(e0, s);
        if (err == cudaSuccess) {
            fp32_peak_kernel<<<blocks, PEAK_THREADS, 0, s>>>(out, 1.f);
            err = cudaGetLastError();
        }
        if (err == cudaSuccess)
            err = cudaEventRecord(e1, s);
        if (err == cudaSuccess)
            err = cudaEventSynchronize(e1);
        float t = 0.f;
        if (err == cudaSuccess)
            err = cudaEventElapsedTime(&t, e0, e1);
        if (err == cudaSuccess && r > 0 && (best == 0.f || t < best))
            best = t;
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    cudaFreeAsync(out, s);
    if (err != cudaSuccess)
        return fail(DP_ERR_CUDA, std::string("fp32 peak probe: ") + cudaGetErrorString(err));
    DP_CUDA(cudaStreamSynchronize(s));
    const double flop = 4.0 * PEAK_CHAINS * PEAK_ITERS * (double)PEAK_THREADS * blocks;  // 2 FMAs x 2 FLOP
    *ms = best;
    *tflops = best > 0.f ? flop / (best * 1e-3) / 1e12 : 0.0;
    return DP_OK;
}

extern "C" dp_status dp_measure_onchip_bw(int32_t kind, int32_t repeats, double *gbs, double *ms, void *stream)
{
    if (!gbs || !ms || repeats < 1 || kind < 0 || kind > 2)
        return fail(DP_ERR_INVALID_ARG, "gbs and ms must be provided, repeats >= 1 and kind in {0, 1, 2}");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    DP_CUDA(cudaGetDevice(&dev));
    DP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * BW_CTAS_PER_SM;
    constexpr size_t L2_VEC = size_t(1) << 22;  // 64 MB of uint4, inside the L2
    const int iters = 4096, l2_reps = 512;
    size_t n_vec = 0;
    if (kind == 1)
        n_vec = (size_t)blocks * L1_VEC;
    else if (kind == 2)
        n_vec = L2_VEC;
    unsigned *out = nullptr;
    uint4 *buf = nullptr;
    DP_CUDA(cudaMallocAsync((void **)&out, sizeof(unsigned) * blocks, s));
    // the most shared memory for kind 0 (6 x 32 KB per SM), the most L1 for kind 1
    cudaError_t err = cudaFuncSetAttribute(smem_bw_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(l1_bw_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    if (err == cudaSuccess && n_vec > 0) {
        err = cudaMallocAsync((void **)&buf, sizeof(uint4) * n_vec, s);
        if (err == cudaSuccess)
            err = cudaMemsetAsync(buf, 0x5a, sizeof(uint4) * n_vec, s);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (err == cudaSuccess)
        err = cudaEventCreate(&e0);
    if (err == cudaSuccess)
        err = cudaEventCreate(&e1);
    float best = 0.f;
    for (int r = 0; r <= repeats && err == cudaSuccess; ++r) {  // r = 0 warms up
        err = cudaEventRecord(e0, s);
        if (err == cudaSuccess) {
            if (kind == 0)
                smem_bw_kernel<<<blocks, BW_THREADS, 0, s>>>(out, iters);
            else if (kind == 1)
                l1_bw_kernel<<<blocks, BW_THREADS, 0, s>>>(buf, out, iters);
            else
                l2_bw_kernel<<<blocks, BW_THREADS, 0, s>>>(buf, n_vec, l2_reps, out);
            err = cudaGetLastError();
        }
        if (err == cudaSuccess)
            err = cudaEventRecord(e1, s);
        if (err == cudaSuccess)
            err = cudaEventSynchronize(e1);
        float t = 0.f;
        if (err == cudaSuccess)
            err = cudaEventElapsedTime(&t, e0, e1);
        if (err == cudaSuccess && r > 0 && (best == 0.f || t < best))
            best = t;
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (buf)
        cudaFreeAsync(buf, s);
    cudaFreeAsync(out, s);
    if (err != cudaSuccess)
        return fail(DP_ERR_CUDA, std::string("on-chip bandwidth probe: ") + cudaGetErrorString(err));
    DP_CUDA(cudaStreamSynchronize(s));
    const double loads = (double)blocks * BW_THREADS * BW_UNROLL * (kind == 2 ? l2_reps : iters);
    *ms = best;
    *gbs = best > 0.f ? loads * sizeof(uint4) / (best * 1e-3) / 1e9 : 0.0;
    return DP_OK;
}
