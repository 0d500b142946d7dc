// Host helpers shared by the translation units of the C ABI (api.cu for
// single problems, api_multi.cu for batches and the serving loop).
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "../../include/ecodp.h"
#include "ecodp_internal.cuh"

struct dp_problem;

namespace ecodp {
namespace host {

// Record msg as the calling thread's last error and return s.
dp_status fail(dp_status s, const std::string &msg);

// Range checks of a problem descriptor (the limits documented in ecodp.h).
dp_status validate(const dp_problem_desc *d);

// Sizes, grids and FP32 model constants of a descriptor.
void fill_params(const dp_problem_desc *d, DevParams &P);

// Per-stage route tables in the layout of StageTables.
struct HostTables {
    std::vector<float> grade, cyc, red, off;
    std::vector<int> lon;  // light index of each node, -1 = none
    size_t bytes() const
    {
        return grade.size() * sizeof(float) + lon.size() * sizeof(int) + 3 * cyc.size() * sizeof(float);
    }
};
void fill_tables(const dp_problem_desc *d, HostTables &t);

bool finite3(const double x[3]);

// In the bounds-checked build: after a call that synchronised with the
// device, a recorded bounds failure turns st (DP_OK or DP_ERR_INFEASIBLE)
// into DP_ERR_INTERNAL.  The production build returns st unchanged.
dp_status checks_after(dp_status st);

// An NVTX range over a scope (host timeline; a profiler projects it onto the
// GPU work launched inside).  No effect unless a tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
    ~NvtxRange() { nvtxRangePop(); }
};
const char *last_error();

// Single-problem helpers (api.cu) for the batch and serving entry points.
size_t roll_doubles(int N);  // doubles of one rollout record (launch_rollout's layout)
// Launch the rollout of a solved problem and copy its record to host memory
// (pinned for an asynchronous copy) on stream s; no synchronisation.
// overlap: may run beside the last stage of the solve just enqueued on s
// (only for a caller whose previous rollout of p has completed: the record
// buffer is rewritten from another stream)
dp_status rollout_async(dp_problem *p, const double x0[3], double *h_out, int *h_u, cudaStream_t s,
                        bool overlap = false);
// Fill a caller's trajectory from a rollout record; returns its fail stage.
int unpack_rollout(int N, const double *h, const int *hu, dp_trajectory *traj);
size_t problem_bytes(const dp_problem *p);  // device bytes the problem holds
// Whether p's sweeps fill every resident CTA slot (default: a solve that runs
// alone) or keep one tile per 128 lanes (solves that share the GPU).
void set_fill_slots(dp_problem *p, bool on);
int problem_stages(const dp_problem *p);
// Whether dp_problem_update can load d into p (same sizes and class structure).
bool problem_fits(const dp_problem *p, const dp_problem_desc *d);

}  // namespace host
}  // namespace ecodp

#define DP_CUDA(call)                                                                                           \
    do {                                                                                                        \
        cudaError_t e_ = (call);                                                                                \
        if (e_ != cudaSuccess)                                                                                  \
            return ::ecodp::host::fail(DP_ERR_CUDA, std::string(#call) + " failed: " + cudaGetErrorString(e_)); \
    } while (0)
