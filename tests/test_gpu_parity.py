"""GPU parity against the FP64 oracle, through the C ABI (needs a GB300).

Stage-local comparisons feed the same J_{k+1} (the terminal cost or a seeded
synthetic field) to the oracle and to one dp_solve_stage call, so masks and
policies are compared without accumulated error.  End-to-end comparisons run
the whole backward sweep on both sides (the oracle's lenient/strict chains
bound the FP32 sweep) and the forward rollout.
"""
import numpy as np
import pytest

import oracle as O
from paper_2104_01284_gb300 import problems as P
from tests._parity import compare

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore")]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_01284_gb300.solver import EcoDP
    return EcoDP


def reduced(seed=31, short_cycles=True, **kw):
    """Config-1 structure at a size the oracle sweeps in seconds: several
    SoC tiles and time warps with ragged tails (19 = 2*8 + 3, 45 = 32 + 13)."""
    args = dict(n_stages=12, n_v=21, n_soc=19, n_t=45, n_te=11, n_tm=11, n_lights=3)
    args.update(kw)
    p = P.config1(seed=seed, **args)
    if short_cycles:
        rng = np.random.Generator(np.random.PCG64(seed + 500))
        n = len(p.light_stage)
        cyc = rng.uniform(6.0, 14.0, n)
        p = p.replace(cycle=cyc, red=cyc * rng.uniform(0.3, 0.6, n), offset=rng.uniform(0, 1, n) * cyc)
    return p


def oracle_stage3(op, k, Vn, idx=None):
    r = {m: O.stage(op, k, Vn, mode=m, idx=idx) for m in (O.NOMINAL, O.LENIENT, O.STRICT)}
    return r[O.NOMINAL], r[O.LENIENT]["V"], r[O.STRICT]["V"]


def stage_inputs(p, op, k):
    yield "terminal", O.terminal(op)
    yield "synthetic", P.synthetic_value_field(p, seed=100 + k)


def stages_of_interest(p):
    ks = {p.n_stages - 1, 0}
    for s in p.light_stage:
        ks.add(int(s) - 1)  # arrival at a light
        ks.add(int(s))      # departure from a light (standstill row waits)
    return sorted(k for k in ks if 0 <= k < p.n_stages)


PROBLEMS = {
    "c0": lambda: P.config0(),
    "reduced": lambda: reduced(),
    "reduced_s2": lambda: reduced(seed=32, n_soc=11, n_t=33, n_te=7, n_tm=9),  # unequal torque steps
    # the grid of the paper's Table I: 690 controls, one torque class each
    "paper_grid": lambda: P.paper_table1(),
    # a small battery: SoC cell shifts -5 .. +3 per step, so the outer buckets
    # d = -2, +1 and lines of other shifts are taken (elsewhere d is -1 or 0)
    "wide_shift": lambda: reduced(seed=56).replace(capacity_As=450.0),
}


@pytest.mark.parametrize("variant", ["tiled", "direct"])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_stage_local_parity(gpu, name, variant):
    p = PROBLEMS[name]()
    op = O.make(p)
    dp = gpu(p)
    dp.set_variant(variant)
    for k in stages_of_interest(p):
        for label, Vn in stage_inputs(p, op, k):
            nom, lo, hi = oracle_stage3(op, k, Vn)
            gV, gpi = dp.solve_stage(k, torch.from_numpy(Vn.astype(np.float32)))
            st = compare(gV.cpu().numpy(), gpi.cpu().numpy(), nom["V"], lo, hi, nom["pi"], nom["second"],
                         where=f"{name}/{variant}/k{k}/{label}")
            assert st["feasible"] > 0
    dp.close()


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_tiled_and_direct_bit_identical(gpu, name):
    """The tiled kernel with 8 and with 6 SoC rows per lane (and the
    automatic choice) equals the direct kernel bit for bit."""
    p = PROBLEMS[name]()
    b = gpu(p)
    b.set_variant("direct")
    b.solve()
    for variant in ("tiled", "tiled8", "tiled6"):
        a = gpu(p)
        a.set_variant(variant)
        a.solve()
        for k in range(p.n_stages + 1):
            assert torch.equal(a.value(k), b.value(k)), (variant, k)
            if k < p.n_stages:
                assert torch.equal(a.policy(k), b.policy(k)), (variant, k)
        a.close()


@pytest.mark.parametrize("name", list(PROBLEMS) + ["paper_scale"])
def test_envelopes_keep_every_minimum(gpu, name):
    """Within a torque class and SoC-shift bucket every control's value at a
    state is a line in the SoC difference of J_{k+1} (Eq. 9b), and the stage
    tables keep only each bucket's lower envelope.  The envelope drops only
    lines that can never give a state's minimum: with every feasible control
    kept (dp_set_envelopes(0)) the sweep returns bit-identical values and
    policies at every stage, in the tiled kernel and (below paper scale) in
    the direct one."""
    p = P.config1(seed=1) if name == "paper_scale" else PROBLEMS[name]()
    for variant in ("tiled",) if name == "paper_scale" else ("tiled", "direct"):
        a = gpu(p)
        a.set_variant(variant)
        a.solve()
        b = gpu(p)
        b.set_variant(variant)
        b.set_envelopes(False)
        b.solve()
        for k in range(p.n_stages + 1):
            assert torch.equal(a.value(k), b.value(k)), (variant, k)
            if k < p.n_stages:
                assert torch.equal(a.policy(k), b.policy(k)), (variant, k)
        a.close()
        b.close()


@pytest.mark.parametrize("name", ["paper_scale", "paper_grid_12_stages"])
def test_skipped_states_are_exactly_those_past_the_last_feasible_time(gpu, name):
    """The tiled sweep (grids whose tiles fill the GPU; the class-split launch
    of smaller grids evaluates every state) writes infeasible, without
    evaluating them, the states whose time lies past the last time column of
    J_{k+1} holding a feasible value (every successor time is at least the
    state's own).  From the solved values: every such state of J_k is
    infeasible, and the sweep's counter of skipped states equals their
    number, so the work counters the roofline uses exclude exactly them."""
    p = P.config1(seed=1) if name == "paper_scale" else P.config1(seed=3, n_stages=12)
    dp = gpu(p)
    dp.solve()
    st = dp.sweep_stats()
    expected = 0
    for k in range(p.n_stages):
        cols = torch.isfinite(dp.value(k + 1)).any(dim=0).any(dim=0)
        idx = torch.nonzero(cols).flatten()
        first_skipped = int(idx.max()) + 1 if idx.numel() else 0
        if first_skipped < p.n_t:
            expected += p.n_v * p.n_soc * (p.n_t - first_skipped)
            assert not torch.isfinite(dp.value(k)[:, :, first_skipped:]).any(), k
    assert st["skipped_states"] == expected
    assert expected > (0.3 * p.n_stages * p.n_states if name == "paper_scale" else 0)  # 45.7 % at paper scale
    dp.close()


@pytest.mark.parametrize("variant,n_t", [("tiled", 201), ("tiled6", 201), ("tiled", 101), ("tiled", 45),
                                         ("tiled", 62), ("tiled", 254)])
def test_unsplit_tiled_sweep_bit_identical(gpu, variant, n_t):
    """A grid with enough tiles for the unsplit tiled kernel (more than half
    of the GPU's resident CTA slots, 4 per SM), whose sweep reads J_{k+1}
    through the corner quads the previous stage wrote (row strides 256, 128
    and 64 for 201, 101 and 45 time points; 62 and 254 fill a stride of 64 and
    256 exactly, n_t + 2 columns): every J_k and pi_k of the sweep
    equals, bit for bit, the stage hook (plain loads of J_{k+1}) run on the
    sweep's own J_{k+1}, and the direct kernel's sweep.  Two lights cover the
    unpaired window loads of light stages."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n_soc, R = 51, (8 if variant == "tiled" else 6)
    chunks = (-(-n_soc // R) * n_t + 127) // 128
    n_v = max(31, 2 * sms // chunks + 1)
    assert n_v * chunks > 2 * sms  # the class-split launch is not taken
    # 60 s for 60 m: time to wait at both lights (about half of J_0 feasible)
    p = P.config1(seed=77, n_stages=6, n_v=n_v, n_soc=n_soc, n_t=n_t, n_te=11, n_tm=11, n_lights=2, t_hi=60.0)
    a = gpu(p)
    a.set_variant(variant)
    a.solve()
    b = gpu(p)
    b.set_variant("direct")
    b.solve()
    for k in range(p.n_stages - 1, -1, -1):
        vk, pk = a.solve_stage(k, a.value(k + 1))
        assert torch.equal(a.value(k), vk), k
        assert torch.equal(a.policy(k), pk), k
        assert torch.equal(a.value(k), b.value(k)), k
        assert torch.equal(a.policy(k), b.policy(k)), k
    assert torch.isfinite(a.value(0)).float().mean() > 0.3


def feasible_start(p, V0, V0lo, V0hi):
    """p.x0 if it is a robustly feasible grid node, else the node nearest to
    it (speed, then SoC, then earliest time) whose J_0 is finite in all three
    oracle modes."""
    vg, sg, tg = p.nodes("v"), p.nodes("soc"), p.nodes("t")
    ok = np.isfinite(V0) & np.isfinite(V0lo) & np.isfinite(V0hi)
    i0 = int(np.argmin(np.abs(vg - p.x0[0])))
    j0 = int(np.argmin(np.abs(sg - p.x0[1])))
    cand = np.argwhere(ok)
    assert cand.size, "no feasible start"
    key = np.abs(cand[:, 0] - i0) * 10 ** 6 + np.abs(cand[:, 1] - j0) * 10 ** 3 + cand[:, 2]
    i, j, l = cand[int(np.argmin(key))]
    return (float(vg[i]), float(sg[j]), float(tg[l]))


@pytest.mark.parametrize("name", ["c0", "reduced", "paper_grid", "wide_shift"])
def test_end_to_end_parity_and_rollout(gpu, name):
    p = PROBLEMS[name]()
    op = O.make(p)
    Vn, pin, secn = O.solve(op, O.NOMINAL)
    Vl, _, _ = O.solve(op, O.LENIENT)
    Vh, _, _ = O.solve(op, O.STRICT)
    dp = gpu(p)
    dp.solve()
    for k in range(p.n_stages, -1, -1):
        gV = dp.value(k).cpu().numpy()
        gp = dp.policy(k).cpu().numpy() if k < p.n_stages else None
        compare(gV, gp, Vn[k], Vl[k], Vh[k], pin[k] if k < p.n_stages else None,
                secn[k] if k < p.n_stages else None, where=f"{name}/e2e/k{k}")
    x0 = feasible_start(p, Vn[0], Vl[0], Vh[0])
    ro = O.rollout(op, Vn, x0)
    rg = dp.rollout(x0=x0, raise_infeasible=False)
    assert ro["status"] == 0, "the oracle rollout from x0 must be feasible"
    assert rg["status"] == 0
    assert rg["fuel_g"] == pytest.approx(ro["fuel_g"], rel=1e-3, abs=1e-6)
    assert rg["J"] == pytest.approx(ro["J"], rel=1e-3)
    assert rg["time_s"] == pytest.approx(ro["time_s"], rel=1e-3)


def test_solve_is_deterministic_and_graph_replays(gpu):
    p = reduced(seed=33)
    dp = gpu(p)
    dp.solve()
    v1 = [dp.value(k).clone() for k in range(p.n_stages + 1)]
    dp.solve()
    for k in range(p.n_stages + 1):
        assert torch.equal(v1[k], dp.value(k))


def test_rollout_beside_the_last_stage_equals_the_sequential_rollout(gpu):
    """dp_rollout issued right after the solve, on the solve's stream, starts
    once J_1 is written, beside the sweep's last Bellman stage (it never reads
    J_0); after another call on the problem (a profiled sweep, which rewrites
    every J_k bit for bit), or on another stream, it runs after the whole
    sweep.  The trajectories are identical."""
    p = reduced(seed=36)
    dp = gpu(p)
    keys = ("v", "soc", "t", "u", "dt", "wait", "fuel")
    dp.solve()
    r1 = dp.rollout(raise_infeasible=False)
    dp.profile_sweep()
    r2 = dp.rollout(raise_infeasible=False)
    side = torch.cuda.Stream()
    dp.solve()
    torch.cuda.synchronize()
    r3 = dp.rollout(stream=side, raise_infeasible=False)
    assert r1["status"] == 0
    for r in (r2, r3):
        for key in keys:
            np.testing.assert_array_equal(r1[key], r[key], err_msg=key)
        assert (r["fuel_g"], r["time_s"], r["J"]) == (r1["fuel_g"], r1["time_s"], r1["J"])


def test_update_matches_fresh_problem(gpu):
    a = reduced(seed=34)
    b = reduced(seed=35)
    dp = gpu(a)
    dp.solve()
    dp.update(b)
    dp.solve()
    fresh = gpu(b)
    fresh.solve()
    for k in range(b.n_stages + 1):
        assert torch.equal(dp.value(k), fresh.value(k))


def test_full_size_stage_local_sampled(gpu):
    """Paper-scale instance (51 x 51 x 201 states, 1922 controls): one stage
    from a seeded J_{k+1} on the GPU, compared at sampled states (plus every
    standstill state at a light's departure stage) with the oracle."""
    p = P.config1(seed=1)
    op = O.make(p)
    dp = gpu(p)
    rng = np.random.Generator(np.random.PCG64(7))
    light = int(p.light_stage[0])
    for k in (light - 1, light, p.n_stages // 2):
        Vn = P.synthetic_value_field(p, seed=200 + k)
        idx = rng.choice(p.n_states, size=1500, replace=False)
        if k == light:  # standstill row v = 0: every 7th state
            idx = np.unique(np.concatenate([idx, np.arange(0, p.n_soc * p.n_t, 7)]))
        nom, lo, hi = oracle_stage3(op, k, Vn, idx=idx)
        gV, gpi = dp.solve_stage(k, torch.from_numpy(Vn.astype(np.float32)))
        g = gV.cpu().numpy().ravel()[idx]
        gp = gpi.cpu().numpy().ravel()[idx]
        st = compare(g, gp, nom["V"], lo, hi, nom["pi"], nom["second"], where=f"c1/k{k}")
        assert st["feasible"] > 100


def test_api_errors(gpu):
    import paper_2104_01284_gb300.native as N
    p = reduced(seed=36)
    dp = gpu(p)
    with pytest.raises(N.DPError) as e:
        dp.value(0)
    assert e.value.status == N.DP_ERR_NOT_SOLVED
    dp.solve()
    with pytest.raises(N.DPError) as e:
        dp.value(p.n_stages + 1)
    assert e.value.status == N.DP_ERR_INVALID_ARG
    r = dp.rollout(x0=(25.0, 0.30, p.t_hi), raise_infeasible=False)
    assert r["status"] == N.DP_ERR_INFEASIBLE and r["fail_stage"] == 0
    bad = p.replace(n_v=1)
    with pytest.raises(N.DPError) as e:
        gpu(bad)
    assert e.value.status == N.DP_ERR_INVALID_ARG
