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
