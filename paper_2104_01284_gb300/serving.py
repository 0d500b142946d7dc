"""Serving loop for receding-horizon MPC re-solves (continuous batching).

EcoDPServer wraps the library's dp_batch_* entry points: requests are
admitted into device-resident slots as slots (and device memory) free up,
and each runs on its own CUDA stream, so a request submitted while others are
on the GPU overlaps with them.  run_fleet drives it with a simulated fleet:
vehicles on seeded routes (problems.config4_fleet) ask for a re-solve of the
horizon ahead of them (problems.horizon_problem) at Poisson arrival times; a
finished solve moves its vehicle one distance step along the optimal
trajectory (the receding-horizon step of the paper's controller, Sec. III).

Everything here is marshalling and host-side bookkeeping; the solves run in
libecodp.so's kernels.
"""
from __future__ import annotations

import collections
import ctypes as C
import time

import numpy as np
import torch

from . import native as N
from . import problems as P
from .solver import TorchAllocator, _trajectory_buffers, make_desc


class EcoDPServer:
    """Continuous-batching solver: up to max_slots requests in flight."""

    def __init__(self, max_slots: int = 8, mem_budget_bytes: int = 8 << 30, device=None,
                 use_torch_allocator: bool = True):
        if not torch.cuda.is_available():
            raise RuntimeError("EcoDPServer needs a CUDA device; the solver has no CPU fallback")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._alloc = TorchAllocator(self.device) if use_torch_allocator else None
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            N.check(N.dp_batch_create(int(max_slots), int(mem_budget_bytes),
                                      C.byref(self._alloc.struct) if self._alloc else None, C.byref(h)),
                    "dp_batch_create")
        self.h = h
        self._pending = {}  # ticket -> (n_stages, buffers, Trajectory)

    def close(self):
        if getattr(self, "h", None):
            with torch.cuda.device(self.device):
                N.check(N.dp_batch_destroy(self.h), "dp_batch_destroy")
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

    def submit(self, p, x0=None):
        """Admit problem p (rollout from x0, default p.x0).  Returns a ticket,
        or None when no slot is free within the memory budget."""
        desc, keep = make_desc(p)
        x = np.array(p.x0 if x0 is None else x0, dtype=np.float64)
        t = C.c_uint64(0)
        with torch.cuda.device(self.device):
            st = N.dp_batch_submit(self.h, C.byref(desc), x.ctypes.data_as(C.POINTER(C.c_double)), C.byref(t))
        del keep
        if st == N.DP_ERR_OOM:
            return None
        N.check(st, "dp_batch_submit")
        bufs, tr = _trajectory_buffers(p.n_stages)
        self._pending[t.value] = (bufs, tr)
        return t.value

    def poll(self, ticket):
        """The result of a request (dict like EcoDP.rollout), or None while
        it is still running."""
        bufs, tr = self._pending[ticket]
        with torch.cuda.device(self.device):
            st = N.dp_batch_poll(self.h, C.c_uint64(ticket), C.byref(tr))
        if st == N.DP_ERR_NOT_SOLVED:
            return None
        if st not in (N.DP_OK, N.DP_ERR_INFEASIBLE):
            N.check(st, "dp_batch_poll")
        del self._pending[ticket]
        out = dict(bufs)
        out["traj"] = np.stack([bufs["v"], bufs["soc"], bufs["t"]], axis=1)
        out.update(fuel_g=tr.fuel_g, time_s=tr.time_s, J=tr.J, fail_stage=tr.fail_stage, status=st)
        return out

    def stats(self):
        out = (C.c_int64 * 8)()
        N.check(N.dp_batch_stats(self.h, out), "dp_batch_stats")
        keys = ("slots", "busy", "device_bytes", "admitted", "collected", "rejected", "slot_creations", "reused")
        return dict(zip(keys, list(out)))


class Fleet:
    """Vehicles on seeded 5 km routes (config 4).  Each vehicle's state is
    (node, v, soc, t); a request re-solves the horizon of n_stages steps
    ahead of it with its time grid starting at its current time."""

    def __init__(self, n_vehicles: int = 1000, seed: int = 4, n_stages: int = 50, n_t: int = 101,
                 x0=(10.0, 0.55)):
        self.fuel, self.routes = P.config4_fleet(seed=seed, n_vehicles=n_vehicles)
        self.n_stages = n_stages
        self.n_t = n_t
        self.route_steps = len(self.routes[0][0])
        self.state = [[0, float(x0[0]), float(x0[1]), 0.0] for _ in range(n_vehicles)]

    def request(self, vid: int):
        node, v, soc, t = self.state[vid]
        p = P.horizon_problem(self.fuel, self.routes[vid], node, t, n_stages=self.n_stages, n_t=self.n_t,
                              name=f"c4-v{vid}-n{node}")
        return p, (v, soc, t)

    def advance(self, vid: int, result):
        """Apply the first step of a finished solve (or, if it was
        infeasible, stay put and let a second pass)."""
        st = self.state[vid]
        if result is not None and result["fail_stage"] != 0:
            st[1], st[2], st[3] = float(result["v"][1]), float(result["soc"][1]), float(result["t"][1])
        else:
            st[3] += 1.0
        st[0] = (st[0] + 1) % (self.route_steps - self.n_stages)


def run_fleet(server: EcoDPServer, fleet: Fleet, rate_rps: float, duration_s: float, seed: int = 0,
              deadline_s: float = 1.0, max_requests: int | None = None):
    """Open-loop load: Poisson arrivals at rate_rps for duration_s, each for
    a uniformly drawn vehicle.  Requests wait in a FIFO host queue until a
    slot admits them; one that has waited deadline_s without admission is
    dropped (its vehicle has moved on).  Latency = arrival to collection.
    Returns the latency percentiles, solves/s and request counts."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = max(1, int(rate_rps * duration_s * 1.2) + 16)
    arr = np.cumsum(rng.exponential(1.0 / rate_rps, size=n))
    arr = arr[arr < duration_s]
    if max_requests is not None:
        arr = arr[:max_requests]
    vid = rng.integers(0, len(fleet.state), size=arr.size)
    queue = collections.deque()
    inflight = {}
    lat = []
    dropped = infeasible = 0
    i_next = 0
    head = None  # the queue head's request, built once
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        progress = False
        while i_next < arr.size and arr[i_next] <= now:
            queue.append(i_next)
            i_next += 1
        while queue and now - arr[queue[0]] > deadline_s:
            queue.popleft()
            dropped += 1
        while queue:
            r = queue[0]
            if head is None or head[0] != r:
                head = (r,) + fleet.request(int(vid[r]))
            ticket = server.submit(head[1], head[2])
            if ticket is None:
                break
            inflight[ticket] = r
            queue.popleft()
            progress = True
        for ticket in list(inflight):
            res = server.poll(ticket)
            if res is None:
                continue
            r = inflight.pop(ticket)
            lat.append(time.perf_counter() - t0 - arr[r])
            if res["status"] != N.DP_OK:
                infeasible += 1
            fleet.advance(int(vid[r]), res)
            progress = True
        if i_next >= arr.size and not queue and not inflight:
            break
        if not progress:
            # nothing finished or admitted: wait a little (at most until the next arrival)
            wait = 5e-5 if inflight or queue else arr[i_next] - (time.perf_counter() - t0)
            time.sleep(min(max(wait, 0.0), 2e-3))
    elapsed = time.perf_counter() - t0
    lat_ms = np.array(lat) * 1e3
    return {
        "offered_rps": rate_rps, "duration_s": duration_s, "arrivals": int(arr.size), "completed": len(lat),
        "dropped": dropped, "infeasible": infeasible, "elapsed_s": elapsed,
        "solves_per_s": len(lat) / elapsed if elapsed > 0 else 0.0,
        "p50_ms": float(np.percentile(lat_ms, 50)) if lat else None,
        "p99_ms": float(np.percentile(lat_ms, 99)) if lat else None,
        "mean_ms": float(lat_ms.mean()) if lat else None,
    }
