"""PyTorch-facing wrapper of the ecodp C ABI.

PyTorch provides device memory (the caching allocator, through the C ABI's
allocator callbacks) and streams; all computation happens in libecodp.so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import native as N

_INF = float("inf")


def make_desc(p):
    """Marshal a problems.Problem into a dp_problem_desc.  Returns (desc,
    keepalive) -- keep the second object alive while the desc is in use."""
    keep = []

    def arr(x, dtype, ctype):
        a = np.ascontiguousarray(x, dtype=dtype)
        if a.size == 0:
            a = np.zeros(1, dtype=dtype)
        keep.append(a)
        return a.ctypes.data_as(C.POINTER(ctype))

    d = N.ProblemDesc()
    d.n_stages = int(p.n_stages)
    d.ds = float(p.ds)
    d.grade = arr(p.grade, np.float64, C.c_double)
    for f in ("v_lo", "v_hi", "soc_lo", "soc_hi", "t_lo", "t_hi", "te_lo", "te_hi", "tm_lo", "tm_hi",
              "brake_decel", "a_min", "a_max", "mass", "cda", "crr", "rho", "g", "r_wheel", "gear",
              "eta_motor", "voc", "r0", "capacity_As", "fuel_scale", "gamma", "soc_ref", "w_soc", "v_ref",
              "w_v"):
        setattr(d, f, float(getattr(p, f)))
    for f in ("n_v", "n_soc", "n_t", "n_te", "n_tm", "n_brake"):
        setattr(d, f, int(getattr(p, f)))
    for q in range(6):
        d.fuel_coef[q] = float(p.fuel_coef[q])
    d.n_lights = int(len(p.light_stage))
    d.light_stage = arr(p.light_stage, np.int32, C.c_int32)
    d.cycle = arr(p.cycle, np.float64, C.c_double)
    d.red = arr(p.red, np.float64, C.c_double)
    d.offset = arr(p.offset, np.float64, C.c_double)
    d.light_model = int(getattr(p, "light_model", 0))
    d.torque_limits = int(getattr(p, "torque_limits", 0))
    coef = getattr(p, "te_max_coef", (0.0, 0.0, 0.0))
    for q in range(3):
        d.te_max_coef[q] = float(coef[q])
    d.bsg_power_max = float(getattr(p, "bsg_power_max", 0.0))
    return d, keep


class TorchAllocator:
    """dp_allocator backed by PyTorch's CUDA caching allocator."""

    def __init__(self, device: torch.device):
        self.device = device.index if device.index is not None else torch.cuda.current_device()

        def _alloc(nbytes, stream, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0)
            except Exception:  # reported to the library as NULL -> DP_ERR_OOM
                return None

        def _free(ptr, stream, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self._alloc = N.ALLOC_FN(_alloc)
        self._free = N.FREE_FN(_free)
        self.struct = N.Allocator(self._alloc, self._free, None)


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class EcoDP:
    """One receding-horizon DP problem resident on a GPU.

    >>> dp = EcoDP(problems.config1())
    >>> dp.solve()                # backward sweep (Eq. 9), asynchronous
    >>> traj = dp.rollout()       # optimal trajectory from p.x0
    """

    def __init__(self, p, device=None, stream=None, use_torch_allocator: bool = True):
        if not torch.cuda.is_available():
            raise RuntimeError("EcoDP needs a CUDA device; the solver has no CPU fallback")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.p = p
        self._alloc = TorchAllocator(self.device) if use_torch_allocator else None
        desc, keep = make_desc(p)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            s = _stream_handle(stream)
            N.check(N.dp_problem_create(C.byref(desc), C.byref(self._alloc.struct) if self._alloc else None,
                                        s, C.byref(h)), "dp_problem_create")
        del keep
        self.h = h
        sz = (C.c_int32 * 5)()
        N.check(N.dp_problem_sizes(self.h, sz), "dp_problem_sizes")
        self.n_stages, self.n_v, self.n_soc, self.n_t, self.n_controls = list(sz)
        self.shape = (self.n_v, self.n_soc, self.n_t)

    # -- lifecycle ----------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            with torch.cuda.device(self.device):
                N.check(N.dp_problem_destroy(self.h), "dp_problem_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def update(self, p, stream=None):
        """Replace grade, lights and model constants (same sizes)."""
        desc, keep = make_desc(p)
        N.check(N.dp_problem_update(self.h, C.byref(desc), _stream_handle(stream)), "dp_problem_update")
        del keep
        self.p = p

    def set_checkpointing(self, every: int):
        """Keep J_k only every `every` stages (0: all stages); rollout,
        adjoint and value() recompute the stages in between."""
        with torch.cuda.device(self.device):
            N.check(N.dp_set_checkpointing(self.h, int(every)), "dp_set_checkpointing")
        self.checkpoint_every = int(every)

    def set_variant(self, variant: str):
        N.check(N.dp_set_kernel_variant(self.h, {"direct": 0, "tiled": 1, "tiled8": 2, "tiled6": 3}[variant]),
                "dp_set_kernel_variant")

    def set_envelopes(self, on: bool = True):
        """Keep only each (torque class, SoC-shift bucket)'s lower envelope
        of lines in the stage tables (default), or every feasible control
        (a cross-check with the same results)."""
        with torch.cuda.device(self.device):
            N.check(N.dp_set_envelopes(self.h, 1 if on else 0), "dp_set_envelopes")

    # -- compute ------------------------------------------------------------
    def solve(self, stream=None):
        with torch.cuda.device(self.device):
            N.check(N.dp_solve_backward(self.h, _stream_handle(stream)), "dp_solve_backward")

    def profile_sweep(self, stream=None):
        """One backward sweep with per-kernel CUDA events (direct launches);
        returns milliseconds {terminal, precompute, bellman, sweep}."""
        ms = (C.c_float * 4)()
        with torch.cuda.device(self.device):
            N.check(N.dp_profile_sweep(self.h, _stream_handle(stream), ms), "dp_profile_sweep")
        return dict(terminal=ms[0], precompute=ms[1], bellman=ms[2], sweep=ms[3])

    def sweep_stats(self, stream=None):
        """Counters of the last sweep: effective state x control evaluations,
        state x class pairs, and the bytes of one update / one rollout copy."""
        out = (C.c_int64 * 8)()
        N.check(N.dp_sweep_stats(self.h, out, _stream_handle(stream)), "dp_sweep_stats")
        return dict(effective_evals=out[0], class_evals=out[1], h2d_update_bytes=out[2], d2h_rollout_bytes=out[3],
                    argmin_states=out[5], envelope_evals=out[6], skipped_states=out[7])

    def value(self, k: int, stream=None) -> torch.Tensor:
        out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        N.check(N.dp_get_value(self.h, int(k), out.data_ptr(), 0, _stream_handle(stream)), "dp_get_value")
        return out

    def policy(self, k: int, stream=None) -> torch.Tensor:
        out = torch.empty(self.shape, dtype=torch.int16, device=self.device)
        N.check(N.dp_get_policy(self.h, int(k), out.data_ptr(), 0, _stream_handle(stream)), "dp_get_policy")
        return out

    def solve_stage(self, k: int, v_next, stream=None):
        """One Bellman stage from a given J_{k+1} (float32 [n_v, n_soc, n_t],
        +inf = infeasible, on the device).  Returns (J_k, pi_k) tensors."""
        vn = torch.as_tensor(v_next, dtype=torch.float32, device=self.device).contiguous()
        assert tuple(vn.shape) == self.shape
        vo = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        po = torch.empty(self.shape, dtype=torch.int16, device=self.device)
        with torch.cuda.device(self.device):
            N.check(N.dp_solve_stage(self.h, int(k), vn.data_ptr(), 0, vo.data_ptr(), po.data_ptr(), 0,
                                     _stream_handle(stream)), "dp_solve_stage")
        return vo, po

    def adjoint(self, x0=None, stream=None):
        """(J_0(x0), dJ_0(x0)/dtheta) for theta = THETA, by the envelope
        theorem on the stored solution.  Returns (float, numpy[5])."""
        x = np.array(self.p.x0 if x0 is None else x0, dtype=np.float64)
        g = np.zeros(5)
        J = C.c_double(0.0)
        with torch.cuda.device(self.device):
            N.check(N.dp_adjoint(self.h, x.ctypes.data_as(C.POINTER(C.c_double)),
                                 g.ctypes.data_as(C.POINTER(C.c_double)), C.byref(J), _stream_handle(stream)),
                    "dp_adjoint")
        return J.value, g

    def rollout(self, x0=None, stream=None, raise_infeasible: bool = True):
        """Forward rollout from x0 (default p.x0); returns numpy arrays."""
        n = self.n_stages
        x = np.array(self.p.x0 if x0 is None else x0, dtype=np.float64)
        bufs = dict(v=np.empty(n + 1), soc=np.empty(n + 1), t=np.empty(n + 1), u=np.empty(n, np.int32),
                    dt=np.empty(n), wait=np.empty(n), fuel=np.empty(n))
        tr = N.Trajectory()
        for key, a in bufs.items():
            ct = C.c_int32 if a.dtype == np.int32 else C.c_double
            setattr(tr, key, a.ctypes.data_as(C.POINTER(ct)))
        with torch.cuda.device(self.device):
            st = N.dp_rollout(self.h, x.ctypes.data_as(C.POINTER(C.c_double)), C.byref(tr), _stream_handle(stream))
        if st != N.DP_OK and (raise_infeasible or st != N.DP_ERR_INFEASIBLE):
            N.check(st, "dp_rollout")
        out = dict(bufs)
        out["traj"] = np.stack([bufs["v"], bufs["soc"], bufs["t"]], axis=1)
        out.update(fuel_g=tr.fuel_g, time_s=tr.time_s, J=tr.J, fail_stage=tr.fail_stage, status=st)
        return out


THETA = ("mass", "cda", "crr", "r0", "fuel_scale")
_SOLVERS = {}


def _solver_for(p, device, checkpoint_every=10):
    """A cached EcoDP for problems of p's sizes on device (re-used through
    dp_problem_update, so repeated evaluations do not reallocate), storing
    J_k every `checkpoint_every` stages."""
    key = (str(device), p.n_stages, p.n_v, p.n_soc, p.n_t, p.n_te, p.n_tm, p.n_brake, p.te_lo, p.te_hi, p.tm_lo,
           p.tm_hi, checkpoint_every)
    dp = _SOLVERS.get(key)
    if dp is None:
        dp = EcoDP(p, device=device)
        dp.set_checkpointing(min(checkpoint_every, p.n_stages))
        _SOLVERS[key] = dp
    else:
        dp.update(p)
    return dp


class EcoDPValue(torch.autograd.Function):
    """J_0(x0; theta), the optimal cost of problem p at x0, as a function of
    theta = (mass, CdA, Crr, R0, fuel_scale) (a float64 tensor of 5).  The
    forward pass solves the backward recursion on the GPU keeping J_k every
    `checkpoint_every` stages (10 by default); the backward pass returns the
    adjoint gradient (dp_adjoint), which recomputes the stages in between."""

    @staticmethod
    def forward(ctx, theta, p, x0=None, device=None, checkpoint_every=10):
        th = theta.detach().to("cpu", torch.float64).tolist()
        q = p.replace(**dict(zip(THETA, th)))
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        dp = _solver_for(q, dev, checkpoint_every)
        dp.solve()
        J, g = dp.adjoint(x0)
        ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
        return torch.tensor(J, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None


def _trajectory_buffers(n):
    bufs = dict(v=np.empty(n + 1), soc=np.empty(n + 1), t=np.empty(n + 1), u=np.empty(n, np.int32),
                dt=np.empty(n), wait=np.empty(n), fuel=np.empty(n))
    tr = N.Trajectory()
    for key, a in bufs.items():
        ct = C.c_int32 if a.dtype == np.int32 else C.c_double
        setattr(tr, key, a.ctypes.data_as(C.POINTER(ct)))
    return bufs, tr


class EcoDPBatch:
    """Many independent problems (any horizons, grids and controls) solved by
    one persistent Bellman launch under a CUDA graph.  Values and policies are
    bit-identical to EcoDP's on the same problem.

    >>> batch = EcoDPBatch(problems.config3_batch())
    >>> batch.autotune()          # pick rows_per_lane / CTAs per SM
    >>> batch.solve()
    >>> trajs = batch.rollout()
    """

    def __init__(self, probs, device=None, stream=None, rows_per_lane: int = 0, ctas_per_sm: int = 0,
                 use_torch_allocator: bool = True, wait_limit_ms: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("EcoDPBatch needs a CUDA device; the solver has no CPU fallback")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.probs = list(probs)
        self._alloc = TorchAllocator(self.device) if use_torch_allocator else None
        descs = (N.ProblemDesc * len(self.probs))()
        keep = []
        for b, p in enumerate(self.probs):
            d, k = make_desc(p)
            descs[b] = d
            keep.append(k)
        opts = N.MultiOpts(int(rows_per_lane), int(ctas_per_sm), int(wait_limit_ms))
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            N.check(N.dp_multi_create(descs, len(self.probs), C.byref(opts),
                                      C.byref(self._alloc.struct) if self._alloc else None, _stream_handle(stream),
                                      C.byref(h)), "dp_multi_create")
        del keep
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            with torch.cuda.device(self.device):
                N.check(N.dp_multi_destroy(self.h), "dp_multi_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __len__(self):
        return len(self.probs)

    def set_config(self, rows_per_lane: int, ctas_per_sm: int):
        """The persistent launch with this tile configuration."""
        with torch.cuda.device(self.device):
            N.check(N.dp_multi_set_config(self.h, int(rows_per_lane), int(ctas_per_sm)), "dp_multi_set_config")

    def set_streams(self, streams: int):
        """The per-instance mode on `streams` internal streams (0: back to the
        persistent launch)."""
        with torch.cuda.device(self.device):
            N.check(N.dp_multi_set_streams(self.h, int(streams)), "dp_multi_set_streams")

    def solve(self, stream=None):
        with torch.cuda.device(self.device):
            N.check(N.dp_multi_solve(self.h, _stream_handle(stream)), "dp_multi_solve")

    def wait(self, stream=None):
        with torch.cuda.device(self.device):
            N.check(N.dp_multi_wait(self.h, _stream_handle(stream)), "dp_multi_wait")

    def profile(self, stream=None):
        ms = (C.c_float * 3)()
        with torch.cuda.device(self.device):
            N.check(N.dp_multi_profile(self.h, _stream_handle(stream), ms), "dp_multi_profile")
        return dict(precompute=ms[0], bellman=ms[1], solve=ms[2])

    def autotune(self, repeats: int = 1, stream=None):
        best = (C.c_int32 * 3)()
        t = C.c_float(0.0)
        with torch.cuda.device(self.device):
            N.check(N.dp_multi_autotune(self.h, _stream_handle(stream), int(repeats), best, C.byref(t)),
                    "dp_multi_autotune")
        return dict(rows_per_lane=best[0], ctas_per_sm=best[1], streams=best[2], ms=t.value)

    def debug_stall(self, b: int):
        """Test hook: make every dependency wait on instance b run out."""
        with torch.cuda.device(self.device):
            N.check(N.dp_multi_debug_stall(self.h, int(b)), "dp_multi_debug_stall")

    def info(self):
        out = (C.c_int64 * 9)()
        with torch.cuda.device(self.device):
            N.check(N.dp_multi_info(self.h, out), "dp_multi_info")
        keys = ("instances", "work_items", "ctas", "rows_per_lane", "ctas_per_sm", "nominal_evals", "device_bytes",
                "max_horizon", "streams")
        return dict(zip(keys, list(out)))

    def _shape(self, b):
        if not 0 <= b < len(self.probs):
            return (1,)  # the library rejects the index
        p = self.probs[b]
        return (p.n_v, p.n_soc, p.n_t)

    def value(self, b: int, k: int, stream=None) -> torch.Tensor:
        out = torch.empty(self._shape(b), dtype=torch.float32, device=self.device)
        with torch.cuda.device(self.device):
            N.check(N.dp_multi_get_value(self.h, int(b), int(k), out.data_ptr(), 0, _stream_handle(stream)),
                    "dp_multi_get_value")
        return out

    def policy(self, b: int, k: int, stream=None) -> torch.Tensor:
        out = torch.empty(self._shape(b), dtype=torch.int16, device=self.device)
        with torch.cuda.device(self.device):
            N.check(N.dp_multi_get_policy(self.h, int(b), int(k), out.data_ptr(), 0, _stream_handle(stream)),
                    "dp_multi_get_policy")
        return out

    def rollout(self, x0=None, stream=None, raise_infeasible: bool = True):
        """Rollout of every instance from x0 ([n, 3]; default each problem's
        x0); returns a list of dicts like EcoDP.rollout."""
        B = len(self.probs)
        x = np.array([p.x0 for p in self.probs] if x0 is None else x0, dtype=np.float64).reshape(B, 3)
        trs = (N.Trajectory * B)()
        bufs = []
        for b, p in enumerate(self.probs):
            bb, tr = _trajectory_buffers(p.n_stages)
            trs[b] = tr
            bufs.append(bb)
        with torch.cuda.device(self.device):
            st = N.dp_multi_rollout(self.h, x.ctypes.data_as(C.POINTER(C.c_double)), trs, _stream_handle(stream))
        if st != N.DP_OK and (raise_infeasible or st != N.DP_ERR_INFEASIBLE):
            N.check(st, "dp_multi_rollout")
        outs = []
        for b in range(B):
            o = dict(bufs[b])
            o["traj"] = np.stack([o["v"], o["soc"], o["t"]], axis=1)
            o.update(fuel_g=trs[b].fuel_g, time_s=trs[b].time_s, J=trs[b].J, fail_stage=trs[b].fail_stage)
            outs.append(o)
        return outs
