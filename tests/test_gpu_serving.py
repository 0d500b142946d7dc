"""Serving (continuous batching of receding-horizon re-solves) through the
C ABI (needs a GB300): each request's result is the same alone and in the
mix, slots are re-used in place, admission respects the memory budget, and
the open-loop fleet driver runs."""
import numpy as np
import pytest

from paper_2104_01284_gb300 import problems as P

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore")]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_01284_gb300 import serving, solver
    return serving, solver


def fleet_requests(n, seed=4):
    """n horizon problems of the config-4 fleet: distinct vehicles, windows
    at different route positions and start times."""
    fuel, routes = P.config4_fleet(seed=seed, n_vehicles=n)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    out = []
    for v in range(n):
        node = int(rng.integers(0, 400))
        t0 = float(rng.uniform(0.0, 300.0))
        p = P.horizon_problem(fuel, routes[v], node, t0)
        out.append((p, (10.0, 0.55, t0)))
    return out


def same(a, b):
    for key in ("v", "soc", "t", "dt", "wait", "fuel", "u"):
        x, y = np.asarray(a[key]), np.asarray(b[key])
        assert np.array_equal(x, y, equal_nan=x.dtype.kind == "f"), key
    assert a["fail_stage"] == b["fail_stage"]
    assert a["fuel_g"] == b["fuel_g"] or (np.isnan(a["fuel_g"]) and np.isnan(b["fuel_g"]))


def test_alone_equals_mix(mods):
    serving, solver = mods
    reqs = fleet_requests(12)
    alone = []
    for p, x0 in reqs:
        dp = solver.EcoDP(p)
        dp.solve()
        alone.append(dp.rollout(x0=x0, raise_infeasible=False))
        dp.close()
    with serving.EcoDPServer(max_slots=4, mem_budget_bytes=8 << 30) as srv:
        tickets = {}
        pending = list(range(len(reqs)))
        results = {}
        while pending or tickets:
            while pending:
                t = srv.submit(*reqs[pending[0]])
                if t is None:
                    break
                tickets[t] = pending.pop(0)
            for t in list(tickets):
                r = srv.poll(t)
                if r is not None:
                    results[tickets.pop(t)] = r
        st = srv.stats()
        assert st["slots"] <= 4 and st["slot_creations"] <= 4
        assert st["reused"] >= len(reqs) - 4
        assert st["collected"] == len(reqs) and st["busy"] == 0
    for i in range(len(reqs)):
        same(results[i], alone[i])


def test_budget_and_tickets(mods):
    serving, _ = mods
    import paper_2104_01284_gb300.native as N
    reqs = fleet_requests(3, seed=5)
    with serving.EcoDPServer(max_slots=2, mem_budget_bytes=1 << 20) as srv:  # 1 MB: no slot fits
        assert srv.submit(*reqs[0]) is None
        assert srv.stats()["rejected"] == 1 and srv.stats()["slots"] == 0
    with serving.EcoDPServer(max_slots=1, mem_budget_bytes=8 << 30) as srv:
        t = srv.submit(*reqs[0])
        assert t is not None
        assert srv.submit(*reqs[1]) is None  # the only slot is busy
        while srv.poll(t) is None:
            pass
        with pytest.raises(KeyError):
            srv.poll(t)  # collected
        tr = N.Trajectory()
        assert N.dp_batch_poll(srv.h, 12345, tr) == N.DP_ERR_INVALID_ARG
        t2 = srv.submit(*reqs[1])
        assert t2 is not None
        while srv.poll(t2) is None:
            pass
        assert srv.stats()["reused"] == 1


def test_fleet_loop_runs(mods):
    serving, _ = mods
    fleet = serving.Fleet(n_vehicles=50)
    with serving.EcoDPServer(max_slots=4) as srv:
        m = serving.run_fleet(srv, fleet, rate_rps=100.0, duration_s=0.5, seed=1)
    assert m["completed"] + m["dropped"] == m["arrivals"] and m["completed"] > 0
    assert m["p99_ms"] >= m["p50_ms"] > 0
    moved = sum(1 for s in fleet.state if s[0] > 0)
    assert moved > 0
