"""Batched solves (one persistent Bellman launch over uneven instances),
through the C ABI (needs a GB300).

Every instance of a batch must reproduce, bit for bit, the values, policies
and rollout of the single-problem path on the same descriptor, for every tile
configuration; one batch is also compared end to end with the FP64 oracle
(acceptance criteria of tests/_parity.py) and a slice of the paper-scale
batch is compared with single solves at sampled stages.
"""
import numpy as np
import pytest

import oracle as O
from paper_2104_01284_gb300 import problems as P
from tests._parity import compare

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore")]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_01284_gb300 import solver
    return solver


def bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint16)


def solve_alone(solver, p):
    dp = solver.EcoDP(p)
    dp.solve()
    V = [dp.value(k).cpu().numpy() for k in range(p.n_stages + 1)]
    pi = [dp.policy(k).cpu().numpy() for k in range(p.n_stages)]
    ro = dp.rollout(raise_infeasible=False)
    dp.close()
    return V, pi, ro


@pytest.fixture(scope="module")
def small(mods):
    probs = P.config3_small(seed=33, n_instances=6)
    return probs, [solve_alone(mods, p) for p in probs]


def same_traj(a, b):
    for key in ("v", "soc", "t", "dt", "wait", "fuel"):
        x, y = np.asarray(a[key]), np.asarray(b[key])
        assert np.array_equal(np.isnan(x), np.isnan(y)), key
        assert np.array_equal(x[~np.isnan(x)], y[~np.isnan(y)]), key
    assert np.array_equal(a["u"], b["u"])
    assert a["fail_stage"] == b["fail_stage"]
    if a["fail_stage"] < 0:
        assert a["fuel_g"] == b["fuel_g"] and a["time_s"] == b["time_s"] and a["J"] == b["J"]


@pytest.mark.parametrize("R,c", [(8, 0), (4, 0), (8, 1), (4, 2), (8, 5), (4, 6)])
def test_batch_bit_identical_to_alone(mods, small, R, c):
    probs, alone = small
    with mods.EcoDPBatch(probs, rows_per_lane=R, ctas_per_sm=c) as bt:
        info = bt.info()
        assert info["rows_per_lane"] == R and info["instances"] == len(probs)
        bt.solve()
        bt.wait()
        for b, p in enumerate(probs):
            V, pi, ro = alone[b]
            for k in range(p.n_stages + 1):
                assert np.array_equal(bits(bt.value(b, k).cpu().numpy()), bits(V[k])), f"inst {b} V{k}"
            for k in range(p.n_stages):
                assert np.array_equal(bt.policy(b, k).cpu().numpy(), pi[k]), f"inst {b} pi{k}"
        for b, rb in enumerate(bt.rollout(raise_infeasible=False)):
            same_traj(rb, alone[b][2])


@pytest.mark.parametrize("streams", [1, 3])
def test_batch_per_instance_streams_bit_identical_to_alone(mods, small, streams):
    """The per-instance mode (each instance's single-problem sweep as its own
    graph, the instances dealt over internal streams) equals single solves bit
    for bit, rollouts included; switching back selects the persistent launch,
    whose results are the same."""
    probs, alone = small
    with mods.EcoDPBatch(probs) as bt:
        bt.set_streams(streams)
        assert bt.info()["streams"] == streams
        bt.solve()
        bt.wait()
        for b, p in enumerate(probs):
            V, pi, ro = alone[b]
            for k in range(p.n_stages + 1):
                assert np.array_equal(bits(bt.value(b, k).cpu().numpy()), bits(V[k])), f"inst {b} V{k}"
            for k in range(p.n_stages):
                assert np.array_equal(bt.policy(b, k).cpu().numpy(), pi[k]), f"inst {b} pi{k}"
        for b, rb in enumerate(bt.rollout(raise_infeasible=False)):
            same_traj(rb, alone[b][2])
        bt.solve()  # a second solve through the same graphs
        bt.wait()
        assert np.array_equal(bits(bt.value(0, 0).cpu().numpy()), bits(alone[0][0][0]))
        bt.set_streams(0)
        assert bt.info()["streams"] == 0
        bt.solve()
        bt.wait()
        for b in range(len(probs)):
            assert np.array_equal(bits(bt.value(b, 0).cpu().numpy()), bits(alone[b][0][0]))
        import paper_2104_01284_gb300.native as N
        with pytest.raises(N.DPError) as e:
            bt.set_streams(17)
        assert e.value.status == N.DP_ERR_INVALID_ARG


def test_batch_end_to_end_oracle_parity(mods):
    probs = P.config3_small(seed=34, n_instances=4)
    with mods.EcoDPBatch(probs) as bt:
        bt.solve()
        for b, p in enumerate(probs):
            op = O.make(p)
            Vn, pin, secn = O.solve(op, O.NOMINAL)
            Vl, _, _ = O.solve(op, O.LENIENT)
            Vh, _, _ = O.solve(op, O.STRICT)
            for k in range(p.n_stages, -1, -1):
                gV = bt.value(b, k).cpu().numpy()
                gp = bt.policy(b, k).cpu().numpy() if k < p.n_stages else None
                compare(gV, gp, Vn[k], Vl[k], Vh[k], pin[k] if k < p.n_stages else None,
                        secn[k] if k < p.n_stages else None, where=f"{p.name}/k{k}")


def test_batch_repeat_and_reconfigure(mods, small):
    probs, alone = small
    with mods.EcoDPBatch(probs) as bt:
        bt.solve()
        first = [bt.value(b, 0).clone() for b in range(len(probs))]
        bt.solve()  # graph replay
        for b in range(len(probs)):
            assert torch.equal(first[b], bt.value(b, 0))
        bt.set_config(4, 1)
        import paper_2104_01284_gb300.native as N
        with pytest.raises(N.DPError) as e:
            bt.value(0, 0)
        assert e.value.status == N.DP_ERR_NOT_SOLVED
        best = bt.autotune(repeats=1)
        assert best["streams"] in (2, 4, 8) or (best["rows_per_lane"] in (4, 8) and best["ctas_per_sm"] >= 1)
        assert bt.info()["streams"] == best["streams"]
        for b in range(len(probs)):
            assert torch.equal(first[b], bt.value(b, 0))


def test_batch_errors(mods):
    import paper_2104_01284_gb300.native as N
    probs = P.config3_small(seed=35, n_instances=3)
    bad = list(probs)
    bad[1] = bad[1].replace(n_v=1)
    with pytest.raises(N.DPError) as e:
        mods.EcoDPBatch(bad)
    assert e.value.status == N.DP_ERR_INVALID_ARG and "instance 1" in str(e.value)
    with pytest.raises(N.DPError) as e:
        mods.EcoDPBatch(probs, rows_per_lane=6)
    assert e.value.status == N.DP_ERR_INVALID_ARG
    with mods.EcoDPBatch(probs) as bt:
        with pytest.raises(N.DPError) as e:
            bt.value(3, 0)
        assert e.value.status == N.DP_ERR_INVALID_ARG


def test_paper_scale_batch_slice_matches_alone(mods):
    """Eight instances of the 256-instance paper-scale batch (horizons
    20-150 stages, up to 61 x 51 x 251 states and 1922 controls): batch
    results equal single solves bit for bit at sampled stages."""
    probs = P.config3_batch(seed=3, n_instances=8)
    with mods.EcoDPBatch(probs) as bt:
        bt.autotune(repeats=1)
        bt.solve()
        bt.wait()
        for b, p in enumerate(probs):
            dp = mods.EcoDP(p)
            dp.solve()
            for k in sorted({0, p.n_stages // 2, p.n_stages - 1, int(p.light_stage[0]) - 1}):
                assert np.array_equal(bits(bt.value(b, k).cpu().numpy()), bits(dp.value(k).cpu().numpy()))
                assert torch.equal(bt.policy(b, k), dp.policy(k))
            dp.close()


def test_dependency_wait_timeout_is_reported(mods):
    """A dependency that nothing completes (test hook): every wait on the
    stalled instance gives up after its 20 ms bound, the launch ends, the
    next synchronising call reports DP_ERR_TIMEOUT, and the batch stays
    usable (reconfiguring restores the schedule; results equal single solves)."""
    import paper_2104_01284_gb300.native as N
    probs = P.config3_small(seed=36, n_instances=3)
    with mods.EcoDPBatch(probs, wait_limit_ms=20) as bt:
        bt.debug_stall(1)
        bt.solve()
        with pytest.raises(N.DPError) as e:
            bt.wait()
        assert e.value.status == N.DP_ERR_TIMEOUT
        bt.set_config(8, 0)
        bt.solve()
        bt.wait()
        for b, p in enumerate(probs):
            dp = mods.EcoDP(p)
            dp.solve()
            assert torch.equal(bt.value(b, 0), dp.value(0))
            dp.close()


def test_batch_with_wide_soc_shifts_equals_alone(mods):
    """Instances whose SoC cell shifts span -5 .. +3 (small battery: outer
    buckets and lines of other shifts) beside ordinary ones: every instance
    of the persistent launch equals its single solve bit for bit."""
    from tests.test_gpu_parity import reduced
    probs = [reduced(seed=56).replace(capacity_As=450.0), reduced(seed=57),
             reduced(seed=58, n_soc=27).replace(capacity_As=300.0)]
    for R in (8, 4):
        with mods.EcoDPBatch(probs, rows_per_lane=R) as bt:
            bt.solve()
            for b, p in enumerate(probs):
                V, pi, _ = solve_alone(mods, p)
                for k in range(p.n_stages + 1):
                    assert np.array_equal(bits(bt.value(b, k).cpu().numpy()), bits(V[k])), (R, b, k)
                for k in range(p.n_stages):
                    assert np.array_equal(bt.policy(b, k).cpu().numpy(), pi[k]), (R, b, k)
