// C ABI of the serving loop's device side (dp_batch_*, declared in
// include/ecodp.h): continuous batching of receding-horizon re-solves.
//
// A batch object owns up to max_slots slots.  A slot is a resident problem
// (its value function, policy, per-stage tables and route tables stay on the
// device), a CUDA stream, pinned host memory for the rollout record and a
// completion event.  dp_batch_submit admits a request into a free slot --
// re-using the slot's device memory through an in-place table update when
// the sizes match, creating a slot while the device-memory budget allows --
// and enqueues the solve (graph replay), the rollout and the copy of its
// record on the slot's stream, so requests submitted while others run
// overlap on the device.  dp_batch_poll hands a finished result back and
// frees its slot for the next request.
#include <cmath>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "api_internal.h"

using namespace ecodp;
using namespace ecodp::host;

struct dp_batch {
    struct Slot {
        dp_problem_t p = nullptr;
        cudaStream_t s = nullptr;
        cudaEvent_t done = nullptr;
        double *h_roll = nullptr;  // pinned rollout record
        int *h_u = nullptr;
        int N = 0;
        size_t bytes = 0;
        bool busy = false;
        uint64_t ticket = 0;
    };
    int max_slots = 0;
    size_t budget = 0;
    dp_allocator alloc{};
    bool has_alloc = false;
    std::vector<Slot> slots;
    size_t bytes_used = 0;
    uint64_t next_ticket = 1;
    std::unordered_map<uint64_t, int> inflight;  // ticket -> slot
    int64_t submitted = 0, completed = 0, rejected = 0, created = 0, reused = 0;
    std::mutex mu;
};

namespace {

void free_slot_resources(dp_batch *b, dp_batch::Slot &S)
{
    if (S.s)
        cudaStreamSynchronize(S.s);
    if (S.p) {
        dp_problem_destroy(S.p);
        b->bytes_used -= S.bytes;
    }
    if (S.h_roll)
        cudaFreeHost(S.h_roll);
    if (S.h_u)
        cudaFreeHost(S.h_u);
    if (S.done)
        cudaEventDestroy(S.done);
    if (S.s)
        cudaStreamDestroy(S.s);
    S = dp_batch::Slot{};
}

// Create the problem of a (new or emptied) slot for desc within the budget.
dp_status fill_slot(dp_batch *b, dp_batch::Slot &S, const dp_problem_desc *desc)
{
    if (!S.s)
        DP_CUDA(cudaStreamCreateWithFlags(&S.s, cudaStreamNonBlocking));
    if (!S.done)
        DP_CUDA(cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming));
    dp_status st = dp_problem_create(desc, b->has_alloc ? &b->alloc : nullptr, (void *)S.s, &S.p);
    if (st != DP_OK)
        return st;
    S.bytes = problem_bytes(S.p);
    b->bytes_used += S.bytes;
    ++b->created;
    if (b->bytes_used > b->budget) {
        cudaStreamSynchronize(S.s);
        dp_problem_destroy(S.p);
        S.p = nullptr;
        b->bytes_used -= S.bytes;
        S.bytes = 0;
        return fail(DP_ERR_OOM, "a slot for this request does not fit in the device-memory budget");
    }
    S.N = desc->n_stages;
    DP_CUDA(cudaHostAlloc((void **)&S.h_roll, roll_doubles(S.N) * sizeof(double), cudaHostAllocDefault));
    DP_CUDA(cudaHostAlloc((void **)&S.h_u, (size_t)S.N * sizeof(int), cudaHostAllocDefault));
    return DP_OK;
}

}  // namespace

extern "C" {

dp_status dp_batch_create(int32_t max_slots, size_t mem_budget, const dp_allocator *alloc, dp_batch_t *out)
{
    if (!out)
        return fail(DP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 4096)
        return fail(DP_ERR_INVALID_ARG, "max_slots must be in [1, 4096]");
    if (mem_budget == 0)
        return fail(DP_ERR_INVALID_ARG, "mem_budget must be positive");
    if (alloc && (!alloc->alloc || !alloc->free))
        return fail(DP_ERR_INVALID_ARG, "allocator needs both alloc and free");
    dp_batch *b = new (std::nothrow) dp_batch();
    if (!b)
        return fail(DP_ERR_OOM, "host allocation failed");
    b->max_slots = max_slots;
    b->budget = mem_budget;
    if (alloc) {
        b->alloc = *alloc;
        b->has_alloc = true;
    }
    b->slots.reserve(max_slots);
    *out = b;
    return DP_OK;
}

dp_status dp_batch_destroy(dp_batch_t b)
{
    if (!b)
        return DP_OK;
    for (auto &S : b->slots)
        free_slot_resources(b, S);
    delete b;
    return DP_OK;
}

dp_status dp_batch_submit(dp_batch_t b, const dp_problem_desc *desc, const double x0[3], uint64_t *ticket)
{
    NvtxRange nvtx_("ecodp.serve.admit");
    if (!b || !desc || !x0 || !ticket)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    dp_status st = validate(desc);
    if (st != DP_OK)
        return st;
    if (!finite3(x0))
        return fail(DP_ERR_INVALID_ARG, "x0 must be finite");
    std::lock_guard<std::mutex> lock(b->mu);
    // 1. a free slot whose memory fits the request: update its tables in place
    int pick = -1;
    for (int i = 0; i < (int)b->slots.size(); ++i) {
        dp_batch::Slot &S = b->slots[i];
        if (!S.busy && S.p && problem_fits(S.p, desc)) {
            pick = i;
            break;
        }
    }
    if (pick >= 0) {
        dp_batch::Slot &S = b->slots[pick];
        st = dp_problem_update(S.p, desc, (void *)S.s);
        if (st != DP_OK)
            return st;
        ++b->reused;
    } else {
        // 2. a new slot, or 3. a free slot of other sizes emptied and refilled
        int victim = -1;
        if ((int)b->slots.size() < b->max_slots) {
            b->slots.emplace_back();
            victim = (int)b->slots.size() - 1;
        } else {
            for (int i = 0; i < (int)b->slots.size(); ++i)
                if (!b->slots[i].busy) {
                    victim = i;
                    break;
                }
        }
        if (victim < 0) {
            ++b->rejected;
            return fail(DP_ERR_OOM, "every slot is busy: poll finished requests and submit again");
        }
        dp_batch::Slot &S = b->slots[victim];
        if (S.p) {
            cudaStreamSynchronize(S.s);
            dp_problem_destroy(S.p);
            b->bytes_used -= S.bytes;
            S.p = nullptr;
            S.bytes = 0;
            cudaFreeHost(S.h_roll);
            cudaFreeHost(S.h_u);
            S.h_roll = nullptr;
            S.h_u = nullptr;
        }
        st = fill_slot(b, S, desc);
        if (st != DP_OK) {
            if (!S.p && victim == (int)b->slots.size() - 1) {
                free_slot_resources(b, S);
                b->slots.pop_back();
            }
            if (st == DP_ERR_OOM)
                ++b->rejected;
            return st;
        }
        pick = victim;
    }
    dp_batch::Slot &S = b->slots[pick];
    set_fill_slots(S.p, b->max_slots == 1);  // several slots share the GPU
    st = dp_solve_backward(S.p, (void *)S.s);
    if (st != DP_OK)
        return st;
    // beside the sweep's last stage: the slot's previous rollout was collected
    st = rollout_async(S.p, x0, S.h_roll, S.h_u, S.s, true);
    if (st != DP_OK)
        return st;
    DP_CUDA(cudaEventRecord(S.done, S.s));
    S.busy = true;
    S.ticket = b->next_ticket++;
    b->inflight[S.ticket] = pick;
    ++b->submitted;
    *ticket = S.ticket;
    return DP_OK;
}

dp_status dp_batch_poll(dp_batch_t b, uint64_t ticket, dp_trajectory *traj)
{
    if (!b || !traj)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    if (!traj->v || !traj->soc || !traj->t || !traj->u || !traj->dt || !traj->wait || !traj->fuel)
        return fail(DP_ERR_INVALID_ARG, "trajectory arrays must all be provided");
    std::lock_guard<std::mutex> lock(b->mu);
    auto it = b->inflight.find(ticket);
    if (it == b->inflight.end())
        return fail(DP_ERR_INVALID_ARG, "unknown or already collected ticket");
    dp_batch::Slot &S = b->slots[it->second];
    const cudaError_t e = cudaEventQuery(S.done);
    if (e == cudaErrorNotReady)
        return DP_ERR_NOT_SOLVED;
    if (e != cudaSuccess)
        return fail(DP_ERR_CUDA, std::string("cudaEventQuery: ") + cudaGetErrorString(e));
    const int fail_stage = unpack_rollout(S.N, S.h_roll, S.h_u, traj);
    S.busy = false;
    b->inflight.erase(it);
    ++b->completed;
    if (fail_stage >= 0)
        return checks_after(fail(DP_ERR_INFEASIBLE, "no feasible control at stage " + std::to_string(fail_stage)));
    return checks_after(DP_OK);
}

dp_status dp_batch_stats(dp_batch_t b, int64_t out[8])
{
    if (!b || !out)
        return fail(DP_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(b->mu);
    int64_t busy = 0;
    for (const auto &S : b->slots)
        busy += S.busy ? 1 : 0;
    out[0] = (int64_t)b->slots.size();
    out[1] = busy;
    out[2] = (int64_t)b->bytes_used;
    out[3] = b->submitted;
    out[4] = b->completed;
    out[5] = b->rejected;
    out[6] = b->created;
    out[7] = b->reused;
    return DP_OK;
}

}  // extern "C"
