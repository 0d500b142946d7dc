"""ctypes binding of libecodp.so (the C ABI declared in include/ecodp.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Importing this module fails loudly when the library has not
been built (``python -c "import __graft_entry__ as g; g.build()"``); there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# ECODP_LIBRARY=checked loads the bounds-checked build (a debugging aid)
CHECKED = os.environ.get("ECODP_LIBRARY", "") == "checked"
LIB_PATH = os.path.join(HERE, "libecodp_checked.so" if CHECKED else "libecodp.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2104_01284_gb300.build.build() "
                      "(nvcc, sm_103a); the solver has no CPU fallback")

lib = C.CDLL(LIB_PATH)

DP_OK, DP_ERR_INVALID_ARG, DP_ERR_OOM, DP_ERR_CUDA, DP_ERR_INFEASIBLE, DP_ERR_NOT_SOLVED, \
    DP_ERR_TIMEOUT, DP_ERR_INTERNAL = range(8)

vp = C.c_void_p
dbl_p = C.POINTER(C.c_double)

ALLOC_FN = C.CFUNCTYPE(vp, C.c_size_t, vp, vp)
FREE_FN = C.CFUNCTYPE(None, vp, vp, vp)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", vp)]


class ProblemDesc(C.Structure):
    _fields_ = [
        ("n_stages", C.c_int32), ("ds", C.c_double), ("grade", dbl_p),
        ("v_lo", C.c_double), ("v_hi", C.c_double), ("n_v", C.c_int32),
        ("soc_lo", C.c_double), ("soc_hi", C.c_double), ("n_soc", C.c_int32),
        ("t_lo", C.c_double), ("t_hi", C.c_double), ("n_t", C.c_int32),
        ("te_lo", C.c_double), ("te_hi", C.c_double), ("n_te", C.c_int32),
        ("tm_lo", C.c_double), ("tm_hi", C.c_double), ("n_tm", C.c_int32),
        ("n_brake", C.c_int32), ("brake_decel", C.c_double),
        ("a_min", C.c_double), ("a_max", C.c_double),
        ("mass", C.c_double), ("cda", C.c_double), ("crr", C.c_double), ("rho", C.c_double), ("g", C.c_double),
        ("r_wheel", C.c_double), ("gear", C.c_double), ("eta_motor", C.c_double),
        ("voc", C.c_double), ("r0", C.c_double), ("capacity_As", C.c_double),
        ("fuel_coef", C.c_double * 6), ("fuel_scale", C.c_double), ("gamma", C.c_double),
        ("soc_ref", C.c_double), ("w_soc", C.c_double), ("v_ref", C.c_double), ("w_v", C.c_double),
        ("n_lights", C.c_int32), ("light_stage", C.POINTER(C.c_int32)),
        ("cycle", dbl_p), ("red", dbl_p), ("offset", dbl_p),
        ("light_model", C.c_int32), ("torque_limits", C.c_int32),
        ("te_max_coef", C.c_double * 3), ("bsg_power_max", C.c_double),
    ]


class Trajectory(C.Structure):
    _fields_ = [
        ("v", dbl_p), ("soc", dbl_p), ("t", dbl_p), ("u", C.POINTER(C.c_int32)),
        ("dt", dbl_p), ("wait", dbl_p), ("fuel", dbl_p),
        ("fuel_g", C.c_double), ("time_s", C.c_double), ("J", C.c_double), ("fail_stage", C.c_int32),
    ]


def _sig(name, *args):
    f = getattr(lib, name)
    f.argtypes = list(args)
    f.restype = C.c_int
    return f


dp_problem_create = _sig("dp_problem_create", C.POINTER(ProblemDesc), C.POINTER(Allocator), vp, C.POINTER(vp))
dp_problem_update = _sig("dp_problem_update", vp, C.POINTER(ProblemDesc), vp)
dp_problem_destroy = _sig("dp_problem_destroy", vp)
dp_problem_sizes = _sig("dp_problem_sizes", vp, C.POINTER(C.c_int32))
dp_set_kernel_variant = _sig("dp_set_kernel_variant", vp, C.c_int32)
dp_profile_sweep = _sig("dp_profile_sweep", vp, vp, C.POINTER(C.c_float))
dp_sweep_stats = _sig("dp_sweep_stats", vp, C.POINTER(C.c_int64), vp)
dp_solve_backward = _sig("dp_solve_backward", vp, vp)
dp_get_value = _sig("dp_get_value", vp, C.c_int32, vp, C.c_int32, vp)
dp_get_policy = _sig("dp_get_policy", vp, C.c_int32, vp, C.c_int32, vp)
dp_solve_stage = _sig("dp_solve_stage", vp, C.c_int32, vp, C.c_int32, vp, vp, C.c_int32, vp)
dp_rollout = _sig("dp_rollout", vp, dbl_p, C.POINTER(Trajectory), vp)
lib.dp_status_string.argtypes = [C.c_int]
lib.dp_status_string.restype = C.c_char_p
lib.dp_last_error.argtypes = []
lib.dp_last_error.restype = C.c_char_p

EXPORTED = [
    "dp_problem_create", "dp_problem_update", "dp_problem_destroy", "dp_problem_sizes",
    "dp_set_kernel_variant", "dp_profile_sweep", "dp_sweep_stats", "dp_solve_backward", "dp_get_value", "dp_get_policy", "dp_solve_stage",
    "dp_rollout", "dp_status_string", "dp_last_error",
]


class DPError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib.dp_last_error().decode(errors="replace")
        name = lib.dp_status_string(status).decode()
        super().__init__(f"{where}: {name}: {msg}")


def check(status: int, where: str):
    if status != DP_OK:
        raise DPError(status, where)

# bounds-check report of the checked build (0 / no-op in the production build)
dp_debug_checks = _sig("dp_debug_checks", C.POINTER(C.c_int32), C.POINTER(C.c_uint64))
EXPORTED.append("dp_debug_checks")
# FP32 FMA throughput probe (the measured denominator beside the derived one)
dp_measure_fp32_peak = _sig("dp_measure_fp32_peak", C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                            C.c_void_p)
EXPORTED.append("dp_measure_fp32_peak")
# lower envelopes of the stage tables on (default) or off (every line kept)
dp_set_envelopes = _sig("dp_set_envelopes", C.c_void_p, C.c_int32)
EXPORTED.append("dp_set_envelopes")
# on-chip load bandwidth probes (shared memory, L1, L2)
dp_measure_onchip_bw = _sig("dp_measure_onchip_bw", C.c_int32, C.c_int32, C.POINTER(C.c_double),
                            C.POINTER(C.c_double), C.c_void_p)
EXPORTED.append("dp_measure_onchip_bw")
ONCHIP_KINDS = {"smem": 0, "l1": 1, "l2": 2}


def debug_checks():
    """(enabled, site): whether this is the bounds-checked build, and its first
    recorded failure (0 if none; cleared by the read).  Synchronises the
    device."""
    en = C.c_int32(0)
    site = C.c_uint64(0)
    st = dp_debug_checks(C.byref(en), C.byref(site))
    if st not in (DP_OK, DP_ERR_INTERNAL):
        check(st, "dp_debug_checks")
    return bool(en.value), int(site.value)


def measure_fp32_peak(repeats: int = 10, stream=None):
    """(TFLOP/s, ms) of the fastest of `repeats` launches of the FP32 FMA
    throughput probe on the current device; synchronises the stream."""
    tf, ms = C.c_double(0.0), C.c_double(0.0)
    handle = int(stream.cuda_stream) if stream is not None else 0
    check(dp_measure_fp32_peak(int(repeats), C.byref(tf), C.byref(ms), C.c_void_p(handle)), "dp_measure_fp32_peak")
    return tf.value, ms.value


def measure_onchip_bw(kind: str, repeats: int = 10, stream=None):
    """(GB/s, ms) of the fastest of `repeats` launches of the load bandwidth
    probe `kind` ("smem", "l1" or "l2") on the current device; synchronises
    the stream."""
    gbs, ms = C.c_double(0.0), C.c_double(0.0)
    handle = int(stream.cuda_stream) if stream is not None else 0
    check(dp_measure_onchip_bw(ONCHIP_KINDS[kind], int(repeats), C.byref(gbs), C.byref(ms), C.c_void_p(handle)),
          "dp_measure_onchip_bw")
    return gbs.value, ms.value


# allocation-free single stage (static device working memory)
dp_solve_stage_static = _sig("dp_solve_stage_static", C.POINTER(ProblemDesc), C.c_int32, vp, vp, vp, vp)
EXPORTED.append("dp_solve_stage_static")

# adjoint dJ_0(x0)/dtheta, theta = (mass, CdA, Crr, R0, fuel_scale)
dp_adjoint = _sig("dp_adjoint", vp, dbl_p, dbl_p, dbl_p, vp)
EXPORTED.append("dp_adjoint")

# batches of independent problems (one persistent Bellman launch)


class MultiOpts(C.Structure):
    _fields_ = [("rows_per_lane", C.c_int32), ("ctas_per_sm", C.c_int32), ("wait_limit_ms", C.c_int32)]


dp_multi_create = _sig("dp_multi_create", C.POINTER(ProblemDesc), C.c_int32, C.POINTER(MultiOpts),
                       C.POINTER(Allocator), vp, C.POINTER(vp))
dp_multi_destroy = _sig("dp_multi_destroy", vp)
dp_multi_set_config = _sig("dp_multi_set_config", vp, C.c_int32, C.c_int32)
dp_multi_set_streams = _sig("dp_multi_set_streams", vp, C.c_int32)
dp_multi_solve = _sig("dp_multi_solve", vp, vp)
dp_multi_wait = _sig("dp_multi_wait", vp, vp)
dp_multi_profile = _sig("dp_multi_profile", vp, vp, C.POINTER(C.c_float))
dp_multi_autotune = _sig("dp_multi_autotune", vp, vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_float))
dp_multi_info = _sig("dp_multi_info", vp, C.POINTER(C.c_int64))
dp_multi_debug_stall = _sig("dp_multi_debug_stall", vp, C.c_int32)
dp_multi_get_value = _sig("dp_multi_get_value", vp, C.c_int32, C.c_int32, vp, C.c_int32, vp)
dp_multi_get_policy = _sig("dp_multi_get_policy", vp, C.c_int32, C.c_int32, vp, C.c_int32, vp)
dp_multi_rollout = _sig("dp_multi_rollout", vp, dbl_p, C.POINTER(Trajectory), vp)
EXPORTED += ["dp_multi_create", "dp_multi_destroy", "dp_multi_set_config", "dp_multi_solve", "dp_multi_wait",
             "dp_multi_profile", "dp_multi_autotune", "dp_multi_info", "dp_multi_get_value", "dp_multi_get_policy",
             "dp_multi_rollout", "dp_multi_debug_stall", "dp_multi_set_streams"]

# serving: continuous batching of receding-horizon re-solves
dp_batch_create = _sig("dp_batch_create", C.c_int32, C.c_size_t, C.POINTER(Allocator), C.POINTER(vp))
dp_batch_destroy = _sig("dp_batch_destroy", vp)
dp_batch_submit = _sig("dp_batch_submit", vp, C.POINTER(ProblemDesc), dbl_p, C.POINTER(C.c_uint64))
dp_batch_poll = _sig("dp_batch_poll", vp, C.c_uint64, C.POINTER(Trajectory))
dp_batch_stats = _sig("dp_batch_stats", vp, C.POINTER(C.c_int64))
EXPORTED += ["dp_batch_create", "dp_batch_destroy", "dp_batch_submit", "dp_batch_poll", "dp_batch_stats"]

# value-function checkpointing (every K stages; 0 = keep every stage)
dp_set_checkpointing = _sig("dp_set_checkpointing", vp, C.c_int32)
EXPORTED.append("dp_set_checkpointing")
