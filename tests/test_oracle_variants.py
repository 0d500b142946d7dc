"""Pins of the oracle's paper variants (no GPU).

* Speed-dependent torque limits (Eq. 7e, 7f): limits too loose to bind give
  the default problem exactly; an engine cap below the first positive engine
  torque node reduces the problem to the one whose only engine torque is 0,
  and a zero BSG power cap to the one whose only BSG torque is 0; tightening
  a limit never lowers a value; and on exact-landing grids the DP equals the
  brute-force minimum over all control sequences.
* Green indicator sampled on the time grid (Sec. III, Eq. 8): without lights,
  or with a light that is never red, it gives the default problem exactly; at
  a light node every state moving at a red time node is infeasible; and on
  exact-landing grids (every arrival is a time node) the DP equals the brute
  force over control sequences and the continuous-arrival DP.
"""
import numpy as np
import pytest

import oracle as O
from paper_2104_01284_gb300 import problems as P
from tests.test_oracle_dp import brute_force, exact_grids

pytestmark = pytest.mark.filterwarnings("ignore")


def small(seed=23, **kw):
    p = P.config1(seed=seed, n_stages=5, n_v=11, n_soc=9, n_t=31, n_te=5, n_tm=5, n_lights=1, t_hi=30.0)
    return p.replace(**kw)


def solve_nominal(p, grids=None):
    op = O.make(p, grids=grids)
    Vs, pis, _ = O.solve(op, O.NOMINAL)
    return op, Vs, pis


def all_equal(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


# -- speed-dependent torque limits -----------------------------------------------

def test_loose_torque_limits_change_nothing():
    p = small()
    _, V0, pi0 = solve_nominal(p)
    _, V1, pi1 = solve_nominal(p.replace(torque_limits=1, te_max_coef=np.array([1e9, 0.0, 0.0]),
                                         bsg_power_max=1e12))
    assert all_equal(V0, V1) and all_equal(pi0, pi1)


def test_engine_cap_below_first_torque_node_leaves_engine_off():
    p = small()  # engine torques 0, 50, 100, 150, 200 Nm
    _, Vc, pic = solve_nominal(p.replace(torque_limits=1, te_max_coef=np.array([10.0, 0.0, 0.0]),
                                         bsg_power_max=1e12))
    _, Vr, pir = solve_nominal(p.replace(n_te=1, te_lo=0.0, te_hi=0.0))
    assert all_equal(Vc, Vr)
    # u = (i_e n_tm + i_m) n_b + b has the same value for i_e = 0 in both
    assert all_equal(pic, pir)


def test_zero_bsg_power_leaves_bsg_idle():
    # at standstill the crank does not turn and no BSG torque draws power, so
    # the reduction holds on speed grids that stay above 0 (no lights: a stop
    # at the line would need v = 0)
    p = small().replace(v_lo=2.0, light_stage=np.zeros(0, np.int32), cycle=np.zeros(0), red=np.zeros(0),
                        offset=np.zeros(0), x0=(10.0, 0.55, 0.0))
    _, Vc, _ = solve_nominal(p.replace(torque_limits=1, te_max_coef=np.array([1e9, 0.0, 0.0]),
                                       bsg_power_max=0.0))
    _, Vr, _ = solve_nominal(p.replace(n_tm=1, tm_lo=0.0, tm_hi=0.0))
    assert all_equal(Vc, Vr)


def test_tighter_limits_never_lower_the_value():
    p = small(seed=24)
    loose = p.replace(torque_limits=1, te_max_coef=np.array([160.0, 0.5, -0.002]), bsg_power_max=9000.0)
    tight = p.replace(torque_limits=1, te_max_coef=np.array([120.0, 0.4, -0.002]), bsg_power_max=4000.0)
    _, Vl, _ = solve_nominal(loose)
    _, Vt, _ = solve_nominal(tight)
    _, Vf, _ = solve_nominal(p)
    for a, b, c in zip(Vf, Vl, Vt):
        assert np.all(b >= a) and np.all(c >= b)  # inf >= anything holds
    assert any(np.any(np.isfinite(b) & (c > b)) for b, c in zip(Vl, Vt)), "the tighter limits never bind"


def test_model_step_applies_the_limits():
    p = small(torque_limits=1, te_max_coef=np.array([100.0, 0.5, 0.0]), bsg_power_max=5000.0)
    op = O.make(p)
    # v = 10 m/s -> w = 100 rad/s: engine cap 150 Nm, BSG cap 50 Nm
    assert O.model_step(op, 0, 10.0, 0.55, 0.0, 140.0, 0.0, 0) is not None
    assert O.model_step(op, 0, 10.0, 0.55, 0.0, 160.0, 0.0, 0) is None
    assert O.model_step(op, 0, 10.0, 0.55, 0.0, 100.0, 40.0, 0) is not None
    assert O.model_step(op, 0, 10.0, 0.55, 0.0, 100.0, -60.0, 0) is None
    # at standstill the BSG power is 0 whatever its torque
    assert O.model_step(op, 0, 0.0, 0.55, 0.0, 100.0, -100.0, 0) is not None


@pytest.mark.parametrize("seed,N", [(7, 3), (9, 2)])
def test_torque_limits_bruteforce(seed, N):
    p = P.toy_problem(seed=seed, n_stages=N, with_light=True)
    # toy torques: engine {0, 150} Nm, BSG {-60, 60} Nm; at 30-60 rad/s the
    # curve caps the engine near 130-150 Nm and 2.5 kW the BSG at 40-80 Nm
    p = p.replace(x0=(4.0, 0.55, 0.0), torque_limits=1, te_max_coef=np.array([110.0, 0.6, 0.0]),
                  bsg_power_max=2500.0)
    grids = exact_grids(p, p.x0)
    op = O.make(p, grids=grids)
    Vs, _, _ = O.solve(op)
    best, _, costs = brute_force(op, p.x0, op.n_controls, p.n_stages)
    assert np.isfinite(best)
    assert Vs[0][0, 0, 0] == pytest.approx(best, rel=1e-12, abs=0)
    # the limits removed some sequences that are feasible without them
    free = O.make(p.replace(torque_limits=0), grids=grids)
    _, _, costs_free = brute_force(free, p.x0, free.n_controls, p.n_stages)
    assert np.isfinite(costs_free).sum() > np.isfinite(costs).sum()


# -- green indicator sampled on the time grid ----------------------------------

def test_sampled_indicator_without_lights_is_the_default():
    p = small(seed=25)
    p = p.replace(light_stage=np.zeros(0, np.int32), cycle=np.zeros(0), red=np.zeros(0), offset=np.zeros(0))
    _, V0, pi0 = solve_nominal(p)
    _, V1, pi1 = solve_nominal(p.replace(light_model=1))
    assert all_equal(V0, V1) and all_equal(pi0, pi1)


def test_sampled_indicator_with_an_always_green_light_is_the_default():
    p = small(seed=26)
    p = p.replace(red=np.zeros(len(p.light_stage)))
    _, V0, pi0 = solve_nominal(p)
    _, V1, pi1 = solve_nominal(p.replace(light_model=1))
    assert all_equal(V0, V1) and all_equal(pi0, pi1)


def test_sampled_indicator_masks_red_time_nodes():
    p = small(seed=27, light_model=1)
    op, Vs, pis = solve_nominal(p)
    k = int(p.light_stage[0])
    t = p.nodes("t")
    red = np.array([O.is_red(op, 0, x) for x in t])
    assert red.any() and (~red).any()
    Vk = Vs[k]
    assert np.all(np.isinf(Vk[1:, :, red]))      # moving through the light at red nodes
    assert np.all(pis[k][1:, :, red] == -1)
    assert np.isfinite(Vk[1:, :, ~red]).any()
    assert np.isfinite(Vk[0]).any()               # standing at the line is allowed


@pytest.mark.parametrize("cfg", [dict(seed=8, N=3, x0=(6.0, 0.55, 0.0)),
                                 dict(seed=13, N=2, x0=(3.0, 0.60, 0.0), spat=(10.0, 5.0, 5.0)),
                                 dict(seed=12, N=3, x0=(3.0, 0.60, 0.0), spat=(10.0, 5.0, 5.0))])
def test_sampled_indicator_bruteforce(cfg):
    p = P.toy_problem(seed=cfg["seed"], n_stages=cfg["N"], with_light=True).replace(x0=cfg["x0"])
    if "spat" in cfg:
        c, r, o = cfg["spat"]
        p = p.replace(cycle=np.array([c]), red=np.array([r]), offset=np.array([o]))
    q = p.replace(light_model=1)
    grids = exact_grids(q, q.x0)  # arrivals during red are reachable here; the DP must mask them
    op = O.make(q, grids=grids)
    Vs, _, _ = O.solve(op)
    best, _, _ = brute_force(op, q.x0, op.n_controls, q.n_stages)
    assert np.isfinite(best)
    assert Vs[0][0, 0, 0] == pytest.approx(best, rel=1e-12, abs=0)
    # and the continuous-arrival DP on its own exact grids gives the same optimum
    g0 = exact_grids(p, p.x0)
    V0s, _, _ = O.solve(O.make(p, grids=g0))
    assert V0s[0][0, 0, 0] == pytest.approx(best, rel=1e-12, abs=0)


# -- literal standstill step of Eq. (5c) -------------------------------------------

def test_literal_standstill_step_closed_form():
    """From standstill at a light node: a control without forward
    acceleration and with the engine off makes the step at zero speed, the
    clock jumping to the end of red (t_RG = red - phase), at the time-only
    cost (1 - gamma) t_RG; during green the jump is zero; a departure needs
    green; engine torque at standstill forbids the step."""
    p = P.toy_problem(seed=7, n_stages=3, with_light=True)
    p = p.replace(cycle=np.array([20.0]), red=np.array([8.0]), offset=np.array([3.0]), light_model=2,
                  n_te=2, te_lo=0.0, te_hi=150.0, n_tm=2, tm_lo=-60.0, tm_hi=60.0)
    op = O.make(p)
    k = 1  # the light node
    # red: phase (t - 3) mod 20 = 2 s at t = 5 s -> 6 s of red left
    r = O.model_step(op, k, 0.0, 0.55, 5.0, 0.0, -60.0, 0)
    assert r is not None
    assert r["v1"] == 0.0 and r["soc1"] == 0.55 and r["t1"] == pytest.approx(11.0, abs=1e-12)
    assert r["dt"] == 0.0 and r["wait"] == pytest.approx(6.0, abs=1e-12)
    assert r["cost"] == pytest.approx((1.0 - p.gamma) * 6.0, rel=1e-12)
    assert O.model_step(op, k, 0.0, 0.55, 5.0, 150.0, 60.0, 0) is None   # departing during red
    assert O.model_step(op, k, 0.0, 0.55, 5.0, 150.0, -60.0, 1) is None  # engine torque at standstill
    # green: phase 10 s at t = 13 s -> the jump takes no time and costs nothing
    g = O.model_step(op, k, 0.0, 0.55, 13.0, 0.0, -60.0, 0)
    assert g is not None and g["t1"] == 13.0 and g["cost"] == 0.0 and g["v1"] == 0.0
    dep = O.model_step(op, k, 0.0, 0.55, 13.0, 150.0, 60.0, 0)
    assert dep is not None and dep["v1"] > 0.0 and dep["wait"] == 0.0
    # away from a light node the default stopping rule applies
    assert O.model_step(op, 0, 0.0, 0.55, 5.0, 0.0, -60.0, 0) is None


def test_literal_standstill_without_lights_is_the_default():
    p = small(seed=28)
    p = p.replace(light_stage=np.zeros(0, np.int32), cycle=np.zeros(0), red=np.zeros(0), offset=np.zeros(0))
    _, V0, pi0 = solve_nominal(p)
    _, V2, pi2 = solve_nominal(p.replace(light_model=2))
    assert all_equal(V0, V2) and all_equal(pi0, pi2)


@pytest.mark.parametrize("cfg", [dict(seed=12, N=3, x0=(3.0, 0.60, 0.0), spat=(10.0, 5.0, 5.0)),
                                 dict(seed=12, N=3, x0=(2.0, 0.60, 0.0), spat=(10.0, 5.0, 0.0)),
                                 dict(seed=13, N=3, x0=(3.0, 0.60, 0.0), spat=(10.0, 5.0, 0.0)),
                                 dict(seed=8, N=3, x0=(6.0, 0.55, 0.0))])
def test_literal_standstill_bruteforce(cfg):
    p = P.toy_problem(seed=cfg["seed"], n_stages=cfg["N"], with_light=True)
    p = p.replace(x0=cfg["x0"], light_model=2)
    if "spat" in cfg:
        c, r, o = cfg["spat"]
        p = p.replace(cycle=np.array([c]), red=np.array([r]), offset=np.array([o]))
    grids = exact_grids(p, p.x0)
    op = O.make(p, grids=grids)
    Vs, _, _ = O.solve(op)
    best, arg, _ = brute_force(op, p.x0, op.n_controls, p.n_stages)
    assert np.isfinite(best)
    assert Vs[0][0, 0, 0] == pytest.approx(best, rel=1e-12, abs=0)


def test_literal_standstill_is_used():
    """With red during [0, 5) s and a slow start the optimum stops at the line
    (at 10 s, red again) and takes the standstill step to the end of red; the
    default reading instead waits at the line and departs from it, cheaper
    because it keeps the distance step for accelerating."""
    p = P.toy_problem(seed=12, n_stages=3, with_light=True).replace(
        x0=(2.0, 0.60, 0.0), light_model=2, cycle=np.array([10.0]), red=np.array([5.0]), offset=np.array([0.0]))
    grids = exact_grids(p, p.x0)
    op = O.make(p, grids=grids)
    best, arg, _ = brute_force(op, p.x0, op.n_controls, p.n_stages)
    x = np.array(p.x0, np.float64)
    used = False
    for k, u in enumerate(arg):
        te, tm, b = op.decode(u)
        r = O.model_step(op, k, x[0], x[1], x[2], te, tm, b)
        if k == 1 and x[0] == 0.0 and r["v1"] == 0.0 and r["wait"] > 0.0:
            used = True
        x = np.array([r["v1"], r["soc1"], r["t1"]])
    assert used
    default = p.replace(light_model=0)
    op0 = O.make(default, grids=exact_grids(default, default.x0))
    best0, _, _ = brute_force(op0, default.x0, op0.n_controls, default.n_stages)
    assert best0 < best
