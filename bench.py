#!/usr/bin/env python
"""Benchmark: paper-scale eco-driving DP horizon solve on GB300.

One step = one pass of the whole hot path on the paper-scale instance
(1000 m horizon of 100 steps of 10 m; 51 speeds x 51 SoC x 201 times;
31 x 31 torques x brake flag = 1922 controls; 4 lights): terminal values, per
stage the precompute and Bellman kernels (the backward recursion of Eq. 9),
then the forward rollout.  The metric is state x control evaluations per
second counted as the paper counts them (N * states * controls per solve),
with ms per horizon solve beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the reference implementation of this method is
that oracle; the paper ships no code).  With --gpus N > 1 (under torchrun)
every rank solves its own replica of the instance (independent problems, no
collective on the data path) and the value is the total over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DP state x control evals/s (ms per horizon solve)"
UNIT = "evals/s"
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM (Blackwell)
FALLBACK_SM_MHZ = 2070.0  # maximum SM clock of the part, when no clock sample exists
# dram__bytes_read.sum + dram__bytes_write.sum of one Bellman launch (stage 79
# of this workload) from an ncu capture of the current kernel version (ncu's
# counters cannot be read inside a timed run; ncu empties the caches before
# the launch, so the corner quads of J_{k+1} that the launch reads come from
# DRAM there, while in the sweep the previous launch has just written them to
# L2).  None whenever the kernel has changed since the last capture.
BELLMAN_TRAFFIC_BYTES = 10.954752e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--batch", type=int, default=256, help="instances of the batched workload (0: skip it)")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="length of each serving run (0: skip serving)")
    return ap.parse_args()


def workload(seed):
    from paper_2104_01284_gb300 import problems as P
    return P.config1(seed=seed)


def config_dict(p, n_gpus, flush):
    return {"workload": f"paper-scale horizon: {p.n_stages} stages x {p.n_v}x{p.n_soc}x{p.n_t} states x "
                        f"{p.n_controls} controls, {len(p.light_stage)} lights (seed 1)",
            "n_stages": p.n_stages, "grid": [p.n_v, p.n_soc, p.n_t], "controls": p.n_controls,
            "evals_per_solve": p.evals_per_solve, "parallelism": f"replicas x{n_gpus}", "l2": flush}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(p, target_s, seed=11, single_s=4.0):
    """Time the FP64 oracle (as it stands) on the host cores on a bounded
    sample: one Bellman stage of the same instance evaluated at a seeded
    random subset of states, every control at each; on every core, and on
    one core (the analogue of the paper's serial solver column)."""
    import numpy as np

    import oracle as O
    from paper_2104_01284_gb300 import problems as P
    op = O.make(p)
    k = p.n_stages // 2
    Vn = P.synthetic_value_field(p, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    cores = os.cpu_count()

    def timed(n_target_s, nthreads):
        probe = rng.choice(p.n_states, size=1000 if nthreads == 1 else 2000, replace=False)
        t0 = time.perf_counter()
        O.stage(op, k, Vn, idx=probe, nthreads=nthreads)
        rate = probe.size / max(1e-6, time.perf_counter() - t0)
        n = int(min(p.n_states, max(500, rate * n_target_s)))
        idx = rng.choice(p.n_states, size=n, replace=False)
        t0 = time.perf_counter()
        O.stage(op, k, Vn, idx=idx, nthreads=nthreads)
        return n, time.perf_counter() - t0

    n, dt = timed(target_s, cores)
    n1, dt1 = timed(single_s, 1)
    evals, evals1 = n * p.n_controls, n1 * p.n_controls
    # the tiny configuration (10 stages, 11 x 11 x 21 states, 11 x 11
    # torques) solved whole, the same solve the GPU times in bench_c0
    p0 = P.config0()
    op0 = O.make(p0)
    c0 = {}
    for key, nthreads in (("all_cores", cores), ("one_core", 1)):
        O.solve(op0, nthreads=nthreads)
        t0 = time.perf_counter()
        for _ in range(3):
            O.solve(op0, nthreads=nthreads)
        c0[key + "_ms_per_solve"] = 1e3 * (time.perf_counter() - t0) / 3
    return {"value": evals / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "c0_full_solve": dict(c0, evals_per_solve=p0.evals_per_solve, cores=cores),
            "sample": f"one Bellman stage (k={k}) of the bench instance at {n} random states x "
                      f"{p.n_controls} controls = {evals:.3e} evals in {dt:.1f} s, FP64, OpenMP",
            "single_core": {"value": evals1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"{n1} random states of the same stage, {evals1:.3e} evals in {dt1:.1f} s",
                            "ms_per_solve_equiv": 1e3 * p.evals_per_solve / (evals1 / dt1)}}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, device) -> float:
    """The largest of every rank's x (the job's time is its slowest rank's);
    x itself when not distributed."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: every rank processed units_per_rank in `seconds`
    (the slowest rank's time)."""
    return world * units_per_rank / seconds


def run_reference(args):
    world, rank, local = dist_setup(args)
    if rank != 0:
        return 0
    import numpy as np

    import oracle as O
    from paper_2104_01284_gb300 import problems as P
    p = workload(args.seed)
    op = O.make(p)
    k = p.n_stages // 2
    Vn = P.synthetic_value_field(p, seed=11)
    rng = np.random.Generator(np.random.PCG64(12))
    probe = rng.choice(p.n_states, size=1000, replace=False)
    t0 = time.perf_counter()
    O.stage(op, k, Vn, idx=probe)
    rate = probe.size / max(1e-6, time.perf_counter() - t0)
    # every step a bounded sample: about 120 s for the whole run
    per_step_s = max(0.5, min(5.0, 120.0 / max(1, args.steps + args.warmup)))
    n = int(min(p.n_states, max(500, rate * per_step_s)))
    for _ in range(args.warmup):
        O.stage(op, k, Vn, idx=rng.choice(p.n_states, size=n, replace=False))
    times = []
    for _ in range(args.steps):
        idx = rng.choice(p.n_states, size=n, replace=False)
        t0 = time.perf_counter()
        O.stage(op, k, Vn, idx=idx)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    evals = n * p.n_controls * args.steps
    value = evals / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "ms_per_solve_equiv": 1e3 * p.evals_per_solve / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
        "config": config_dict(p, args.gpus, "CPU run"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"per step one Bellman stage (k={k}) at {n} random states x {p.n_controls} "
                                   f"controls, FP64, OpenMP"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def bench_batched(n_inst, dev, stream, steps=2):
    """Batched uneven instances (256 seeded horizons of 20-150 stages, 31-61
    speeds, 31-51 SoC points, 101-251 times, 21x21-31x31 torques x brake,
    1-6 lights) through the batched API in the mode the autotuner picks on
    the first 32 instances (one persistent launch under a CUDA graph with its
    tile configuration, or each instance's graph on internal streams); against
    the same instances solved one at a time by the single-problem path (its
    own CUDA graph per instance, on one stream).  Inputs are far larger than
    L2 (tens of GB), so no flush is needed between steps."""
    import torch

    from paper_2104_01284_gb300 import problems as P
    from paper_2104_01284_gb300.solver import EcoDP, EcoDPBatch
    probs = P.config3_batch(seed=3, n_instances=n_inst)
    with torch.cuda.stream(stream):
        with EcoDPBatch(probs[:min(32, n_inst)], device=dev, stream=stream) as tune:
            best = tune.autotune(repeats=1, stream=stream)
        bt = EcoDPBatch(probs, device=dev, stream=stream, rows_per_lane=best["rows_per_lane"],
                        ctas_per_sm=best["ctas_per_sm"])
        if best["streams"]:
            bt.set_streams(best["streams"])
        bt.solve(stream)
        bt.wait(stream)
        times = []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bt.solve(stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        bt.wait(stream)
        prof = bt.profile(stream)
        info = bt.info()
        bt.close()
        # the same instances through the single-problem path: one at a time,
        # and spread over 4 streams (the serving loop's way of sharing the GPU)
        single_ms = streams_ms = 0.0
        side = [torch.cuda.Stream(device=dev) for _ in range(4)]
        for c0 in range(0, n_inst, 32):
            dps = [EcoDP(q, device=dev, stream=stream) for q in probs[c0:c0 + 32]]
            for d in dps:
                d.solve(stream)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for d in dps:
                d.solve(stream)
            e1.record(stream)
            e1.synchronize()
            single_ms += e0.elapsed_time(e1)
            e0.record(stream)
            for q in side:
                q.wait_event(e0)
            for b, d in enumerate(dps):
                d.solve(side[b % len(side)])
            for q in side:
                done = torch.cuda.Event()
                done.record(q)
                stream.wait_event(done)
            e1.record(stream)
            e1.synchronize()
            streams_ms += e0.elapsed_time(e1)
            for d in dps:
                d.close()
    ms = statistics.median(times)
    return {"workload": f"{n_inst} uneven instances (config-3 family, seed 3)", "instances": n_inst,
            "solves_per_s": n_inst / (ms / 1e3), "ms_per_batch": ms,
            "nominal_evals_per_s": info["nominal_evals"] / (ms / 1e3),
            "single_path_solves_per_s": n_inst / (single_ms / 1e3), "single_path_ms": single_ms,
            "speedup_vs_single_path": single_ms / ms,
            "single_path_4_streams_solves_per_s": n_inst / (streams_ms / 1e3),
            "tile_config": {"rows_per_lane": best["rows_per_lane"], "ctas_per_sm": best["ctas_per_sm"],
                            "streams": best["streams"], "autotune_ms_on_32": best["ms"]},
            "persistent_ms": prof["bellman"], "precompute_ms": prof["precompute"],
            "work_items": info["work_items"], "ctas": info["ctas"], "device_gb": info["device_bytes"] / 1e9,
            "gpu_launches_per_batch": 3 if not best["streams"] else sum(q.n_stages + 3 for q in probs),
            "steps": steps}


def bench_serving(dev, seconds):
    """Serving loop for receding-horizon MPC (config 4): 1000 vehicles on
    seeded 5 km routes with 10 lights each re-solve a 500 m horizon (50
    stages, 51 x 51 x 101 states, 1922 controls) at Poisson arrival times.
    Requests are admitted into device-resident slots (continuous batching,
    one stream per slot); a request not admitted within 1 s is dropped.
    Reported: the saturation throughput for 2, 4 and 8 slots, then at the
    best slot count p50/p99 latency and counts at 200, 500, 1000 and 2000
    requests/s and at half the saturation rate, beside the one-at-a-time
    path (one slot)."""
    from paper_2104_01284_gb300.serving import EcoDPServer, Fleet, run_fleet
    fleet = Fleet(n_vehicles=1000)
    runs = {}
    sat = {}
    with EcoDPServer(max_slots=8, device=dev) as srv:
        run_fleet(srv, fleet, rate_rps=200.0, duration_s=0.3, seed=99)  # warm-up: slots, graphs
    for slots in (2, 4, 8):
        with EcoDPServer(max_slots=slots, device=dev) as srv:
            run_fleet(srv, fleet, rate_rps=500.0, duration_s=0.2, seed=98)
            sat[slots] = run_fleet(srv, fleet, rate_rps=2000.0, duration_s=seconds, seed=1)["solves_per_s"]
    best = max(sat, key=sat.get)
    half = 0.5 * sat[best]
    with EcoDPServer(max_slots=best, device=dev) as srv:
        run_fleet(srv, fleet, rate_rps=500.0, duration_s=0.2, seed=97)
        for rate in (200.0, 500.0, 1000.0, 2000.0, half):
            key = "half_saturation" if rate == half else f"{int(rate)}_rps"
            runs[key] = run_fleet(srv, fleet, rate_rps=rate, duration_s=seconds, seed=int(rate))
        stats = srv.stats()
    single = {}
    with EcoDPServer(max_slots=1, device=dev) as srv:
        run_fleet(srv, fleet, rate_rps=500.0, duration_s=0.2, seed=96)
        single["saturation"] = run_fleet(srv, fleet, rate_rps=2000.0, duration_s=seconds, seed=1)
        single["half_saturation"] = run_fleet(srv, fleet, rate_rps=half, duration_s=seconds, seed=int(half))
    import torch
    stream = torch.cuda.Stream(dev)
    persistent = {n: bench_fleet_persistent(dev, stream, n_req=n) for n in (8, 16, 32)}
    return {"workload": "1000 vehicles, 5 km routes, 10 lights; 50-stage horizon 51x51x101 states x 1922 controls",
            "saturation_solves_per_s_by_slots": sat, "slots": best, "runs": runs,
            "one_at_a_time": single, "deadline_s": 1.0, "slot_stats": stats,
            "persistent_batch_by_requests": persistent}


def bench_fleet_persistent(dev, stream, n_req=16, steps=3):
    """The serving workload's requests through the persistent batched kernel
    instead of per-slot streams: n_req fleet horizon problems (50 stages,
    51 x 51 x 101 states, 1922 controls) solved as one batch (terminal,
    precompute and one persistent Bellman launch under a CUDA graph, tile
    configuration autotuned), then rolled out; solves/s of the whole
    (backward sweeps and rollouts), for comparison with the serving loop's
    saturation throughput."""
    import torch

    from paper_2104_01284_gb300.serving import Fleet
    from paper_2104_01284_gb300.solver import EcoDPBatch
    fleet = Fleet(n_vehicles=n_req)
    reqs = [fleet.request(v) for v in range(n_req)]
    probs = [p for p, _ in reqs]
    x0 = [x for _, x in reqs]
    with torch.cuda.stream(stream):
        bt = EcoDPBatch(probs, device=dev, stream=stream)
        best = bt.autotune(repeats=1, stream=stream)
        bt.set_config(best["rows_per_lane"], best["ctas_per_sm"])
        bt.solve(stream)
        bt.rollout(x0=x0, stream=stream, raise_infeasible=False)
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            t0 = time.perf_counter()
            bt.solve(stream)
            bt.rollout(x0=x0, stream=stream, raise_infeasible=False)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        bt.close()
    s = statistics.median(times)
    return {"requests": n_req, "solves_per_s": n_req / s, "ms_per_batch": 1e3 * s,
            "tile_config": {"rows_per_lane": best["rows_per_lane"], "ctas_per_sm": best["ctas_per_sm"]}}


def bench_c0(dev, stream, reps=20):
    """The tiny configuration (10 stages, 11 x 11 x 21 states, 11 x 11
    torques, one light = 3.1e6 nominal evaluations per solve): median and
    p99 of `reps` graph-launched solves, each followed by its rollout."""
    import torch

    from paper_2104_01284_gb300 import problems as P
    from paper_2104_01284_gb300.solver import EcoDP
    p = P.config0()
    dp = EcoDP(p, device=dev, stream=stream)
    for _ in range(3):
        dp.solve(stream)
        dp.rollout(stream=stream, raise_infeasible=False)
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dp.solve(stream)
        dp.rollout(stream=stream, raise_infeasible=False)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    dp.close()
    ms = statistics.median(times)
    return {"workload": "tiny configuration: 10 stages x 11x11x21 states x 11x11 torques, one light (seed 0)",
            "evals_per_solve": p.evals_per_solve, "ms_per_solve_median": ms,
            "ms_per_solve_p99": sorted(times)[min(len(times) - 1, int(0.99 * len(times)))]}


def bench_paper_grid(dev, stream, reps=20):
    """The grid of the paper's Table I (20 steps, 35 x 26 x 40 states, 23 x 30
    torques = 5.0e8 nominal evaluations per solve), solved by the
    single-problem path: median and p99 of `reps` graph-launched solves."""
    import torch

    from paper_2104_01284_gb300 import problems as P
    from paper_2104_01284_gb300.solver import EcoDP
    p = P.paper_table1()
    dp = EcoDP(p, device=dev, stream=stream)
    for _ in range(3):
        dp.solve(stream)
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dp.solve(stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    dp.close()
    ms = statistics.median(times)
    return {"workload": "grid of the paper's Table I: 20 stages x 35x26x40 states x 23x30 torques (seed 5)",
            "evals_per_solve": p.evals_per_solve, "ms_per_solve_median": ms,
            "ms_per_solve_p99": sorted(times)[min(len(times) - 1, int(0.99 * len(times)))],
            "nominal_evals_per_s": p.evals_per_solve / (ms / 1e3),
            "paper_context_ms": {"rtx2080_parallel_mean": 98, "cpu_serial_mean": 1600}}


ROOFLINE_KEYS = ("bound", "kernel", "achieved", "peak", "unit", "frac", "traffic", "peak_basis",
                 "peak_measured", "frac_of_measured", "onchip_peaks_gbs", "bellman_ms_per_launch", "share_of_sweep",
                 "skipped_state_fraction")


def headline(adjoint, paper_grid, batched, serving, c0=None):
    """Compact numbers of the adjoint, the paper's Table I grid, the tiny
    configuration, the 256-instance batch and the serving loop."""
    h = {"adjoint_ms_per_call": adjoint["ms_per_call"],
         "paper_grid_ms_per_solve": paper_grid["ms_per_solve_median"]}
    if c0:
        h["c0_ms_per_solve_and_rollout"] = c0["ms_per_solve_median"]
    if batched:
        h["batched"] = {"instances": batched["instances"], "solves_per_s": batched["solves_per_s"],
                        "single_path_solves_per_s": batched["single_path_solves_per_s"],
                        "speedup_vs_single_path": batched["speedup_vs_single_path"],
                        "single_path_4_streams_solves_per_s": batched["single_path_4_streams_solves_per_s"],
                        "mode": (f"{batched['tile_config']['streams']} streams of per-instance graphs"
                                 if batched["tile_config"]["streams"] else "persistent launch")}
    if serving:
        half = serving["runs"]["half_saturation"]
        one = serving["one_at_a_time"]
        h["serving"] = {"slots": serving["slots"],
                        "saturation_solves_per_s": serving["saturation_solves_per_s_by_slots"][serving["slots"]],
                        "one_at_a_time_solves_per_s": one["saturation"]["solves_per_s"],
                        "half_saturation_rps": half["offered_rps"], "p50_ms": half["p50_ms"], "p99_ms": half["p99_ms"],
                        "one_at_a_time_p50_ms": one["half_saturation"]["p50_ms"],
                        "one_at_a_time_p99_ms": one["half_saturation"]["p99_ms"],
                        "persistent_batch_solves_per_s": {n: r["solves_per_s"] for n, r in
                                                          serving["persistent_batch_by_requests"].items()}}
    return h


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2104_01284_gb300.solver import EcoDP
    world, rank, local = dist_setup(args)
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    p = workload(args.seed)
    stream = torch.cuda.Stream(dev)
    dp = EcoDP(p, device=dev, stream=stream)
    # terminal, J_N's corner quads, precompute (all stages), N x Bellman, rollout
    launches_per_step = 1 + 1 + 1 + p.n_stages + 1

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            dp.solve(stream)
            dp.rollout(stream=stream)
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    times = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)  # evict the previous step's data from L2 (outside the timed pair)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dp.solve(stream)
            traj = dp.rollout(stream=stream)
            e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(times), dev)
    value = job_rate(p.evals_per_solve * args.steps, world, total_ms / 1e3)

    # per-kernel breakdown (direct launches, CUDA events on the launching stream)
    profs = [dp.profile_sweep(stream) for _ in range(3)]
    stats = dp.sweep_stats(stream)
    bell_ms = statistics.median(x["bellman"] for x in profs)
    pre_ms = statistics.median(x["precompute"] for x in profs)
    sweep_ms = statistics.median(x["sweep"] for x in profs)
    per_launch_s = bell_ms / 1e3 / p.n_stages
    # per (state, envelope line): 1 FMA; per (state, torque class): the
    # bilinear blend of J_{k+1}'s four corners (4 multiplies, 3 adds), the
    # SoC-row difference and the add
    flops_per_launch = (2.0 * stats["envelope_evals"] + 9.0 * stats["class_evals"]) / p.n_stages
    achieved = flops_per_launch / per_launch_s / 1e12
    # FP32 FMA peak from the device's SM count and the SM clock sampled
    # during the timed region
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clocks.get("sm_mhz") or FALLBACK_SM_MHZ
    peak = n_sm * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    roofline = {"bound": "alu", "kernel": "bellman_planned", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": BELLMAN_TRAFFIC_BYTES,
                "peak_basis": f"FP32 FMA: {n_sm} SMs x {FP32_LANES_PER_SM} lanes x 2 FLOP x {mhz:.0f} MHz "
                              f"({'median sampled SM clock' if clocks.get('sm_mhz') else 'maximum SM clock'})",
                "work_basis": "2 FLOP per (state, envelope line) FMA + 9 FLOP per (state, torque class) window value (bilinear blend of 4 corners: 4 mul + 3 add, the SoC difference, the add)",
                "bellman_ms_per_launch": 1e3 * per_launch_s,
                "share_of_sweep": bell_ms / sweep_ms if sweep_ms > 0 else None,
                "precompute_ms_per_launch": pre_ms / p.n_stages,
                "effective_evals_per_s": stats["effective_evals"] / (bell_ms / 1e3),
                "envelope_evals_per_launch": stats["envelope_evals"] / p.n_stages,
                "class_evals_per_launch": stats["class_evals"] / p.n_stages,
                "envelope_fraction": stats["envelope_evals"] / max(1, stats["effective_evals"]),
                # (state, stage) pairs past the next stage's last feasible
                # time column: written infeasible without evaluation (the
                # work counters above exclude them)
                "skipped_state_fraction": stats["skipped_states"] / (p.n_stages * p.n_states),
                "argmin_states": stats["argmin_states"],
                # context: the direct trilinear form evaluates every state x
                # control with 8 FMA (16 FLOP); at this kernel's time it would
                # need this rate, which the class factorisation and the
                # envelopes avoid
                "direct_form_equivalent": {
                    "flop_per_eval": 16,
                    "tflops": 16.0 * p.evals_per_solve / p.n_stages / per_launch_s / 1e12,
                    "of_peak": 16.0 * p.evals_per_solve / p.n_stages / per_launch_s / 1e12 / peak}}
    # the FP32 FMA rate the part sustains (the library's throughput probe),
    # beside the unit-count peak the fraction is quoted against
    from paper_2104_01284_gb300 import native as N
    meas_tf, _ = N.measure_fp32_peak(10, stream)
    roofline["peak_measured"] = meas_tf
    roofline["frac_of_measured"] = achieved / meas_tf if meas_tf > 0 else None
    # the on-chip load paths' measured rates (shared memory, L1 hits, L2
    # hits), the kernel's other possible bounds
    roofline["onchip_peaks_gbs"] = {k: N.measure_onchip_bw(k, 5, stream)[0] for k in ("smem", "l1", "l2")}

    # end to end through the public API with host buffers: upload the
    # problem tables, solve, read the trajectory back, every step
    for _ in range(2):
        dp.update(p, stream)
        dp.solve(stream)
        dp.rollout(stream=stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        dp.update(p, stream)
        dp.solve(stream)
        dp.rollout(stream=stream)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    e2e = {"value": job_rate(p.evals_per_solve * args.steps, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(stats["h2d_update_bytes"]), "d2h_bytes_per_step": int(stats["d2h_rollout_bytes"]),
           "ms_per_step": 1e3 * e2e_s / args.steps}

    # adjoint dJ*/dtheta at x0 on the solved instance (host-synchronous call)
    dp.solve(stream)
    dp.adjoint(stream=stream)
    t0 = time.perf_counter()
    for _ in range(3):
        J0, grad = dp.adjoint(stream=stream)
    adjoint = {"ms_per_call": 1e3 * (time.perf_counter() - t0) / 3, "J0": J0,
               "dJ_dtheta": dict(zip(("mass", "cda", "crr", "r0", "fuel_scale"), map(float, grad)))}

    paper_grid = bench_paper_grid(dev, stream)
    c0 = bench_c0(dev, stream)
    batched = bench_batched(args.batch, dev, stream) if args.batch > 0 else None
    serving = bench_serving(dev, args.serve_seconds) if args.serve_seconds > 0 else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
        "config": config_dict(p, world, "flushed between steps (256 MB write)"),
        "effective_evals_per_s": job_rate(stats["effective_evals"] * args.steps, world, total_ms / 1e3),
        "ms_per_solve_median": statistics.median(times),
        "ms_per_solve_p99": float(sorted(times)[min(len(times) - 1, int(0.99 * len(times)))]),
        "rollout": {"fuel_g": traj["fuel_g"], "time_s": traj["time_s"], "J": traj["J"]},
        "roofline": roofline, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds)
    # the other workloads' headline numbers on the JSON line; their full
    # records (per offered load, tile configuration, ...) go to stderr first
    line["headline"] = headline(adjoint, paper_grid, batched, serving, c0)
    if rank == 0:
        print(json.dumps({"details": {"adjoint": adjoint, "paper_grid": paper_grid, "c0": c0, "batched": batched,
                                      "serving": serving, "roofline": roofline}}), file=sys.stderr, flush=True)
        line["roofline"] = {k: v for k, v in roofline.items() if k in ROOFLINE_KEYS}
        print(json.dumps(line), flush=True)
    dp.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
