"""Pins of the oracle's backward recursion (Eq. 9a-9d), interpolation and
rollout against brute force, closed forms and invariants.

* Brute force: on few-stage toys whose per-stage grids are exactly the sets of
  reachable coordinates, every successor is a grid node, so the DP value at
  x0 must equal the minimum over all control sequences of the exact
  trajectory cost (the DP principle, Eq. 9).
* Closed form: cruising at constant speed on a flat road with the single
  control that balances the road load.
* Invariants: time-independence, monotonicity in SoC, in t_max and in the
  fuel-map scale, a lower bound from the speed limit, and invariance under a
  common shift of the clock and the light offsets.
* Interpolation: trilinear interpolation reproduces tri-affine functions
  exactly; the snap and out-of-grid band rules.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2104_01284_gb300 import problems as P

pytestmark = pytest.mark.filterwarnings("ignore")


# ---------------------------------------------------------------------------
# brute force on exact-landing grids

def exact_grids(p, x0):
    """Per-stage node arrays holding exactly the coordinates reachable from x0
    (inside the state box), built with the model step alone."""
    op = O.make(p)
    reach = [{tuple(x0)}]
    for k in range(p.n_stages):
        nxt = set()
        for x in reach[k]:
            for u in range(op.n_controls):
                te, tm, b = op.decode(u)
                r = O.model_step(op, k, x[0], x[1], x[2], te, tm, b)
                if r is None:
                    continue
                y = (r["v1"], r["soc1"], r["t1"])
                if (p.v_lo <= y[0] <= p.v_hi and p.soc_lo <= y[1] <= p.soc_hi
                        and p.t_lo <= y[2] <= p.t_hi):
                    nxt.add(y)
        assert nxt, f"nothing reachable at stage {k + 1}"
        reach.append(nxt)
    grids = []
    for R in reach:
        arr = np.array(sorted(R))
        grids.append(tuple(np.unique(arr[:, a]) for a in range(3)))
    return grids


def brute_force(op, x0, n_u, N):
    best, arg, costs = np.inf, None, []
    for seq in itertools.product(range(n_u), repeat=N):
        J, _ = O.sequence_cost(op, x0, seq)
        costs.append(J)
        if J < best:
            best, arg = J, seq
    return best, arg, np.array(costs)


TOYS = [
    # (seed, stages, light, brake, x0): 2x2 torques (x brake) over 2-3 stages
    dict(seed=7, N=3, light=False, n_brake=1, x0=(6.0, 0.55, 0.0)),
    dict(seed=8, N=3, light=True, n_brake=1, x0=(6.0, 0.55, 0.0)),
    dict(seed=9, N=2, light=True, n_brake=2, x0=(3.0, 0.60, 0.0)),
    dict(seed=11, N=3, light=True, n_brake=2, x0=(3.0, 0.60, 0.0), n_tm=1),
    # stops at the line at 6.67 s inside the red [5, 10) s and waits for green
    dict(seed=12, N=3, light=True, n_brake=2, x0=(3.0, 0.60, 0.0), n_tm=1, spat=(10.0, 5.0, 5.0)),
    dict(seed=13, N=2, light=True, n_brake=2, x0=(3.0, 0.60, 0.0), spat=(10.0, 5.0, 5.0)),
]


@pytest.mark.parametrize("cfg", TOYS, ids=lambda c: f"s{c['seed']}N{c['N']}")
def test_bruteforce_exact_grids(cfg):
    p = P.toy_problem(seed=cfg["seed"], n_stages=cfg["N"], with_light=cfg["light"])
    p = p.replace(n_brake=cfg["n_brake"], x0=cfg["x0"])
    if cfg.get("n_tm") == 1:
        p = p.replace(n_tm=1, tm_lo=0.0, tm_hi=0.0)
    if "spat" in cfg:
        c, r, o = cfg["spat"]
        p = p.replace(cycle=np.array([c]), red=np.array([r]), offset=np.array([o]))
    grids = exact_grids(p, p.x0)
    op = O.make(p, grids=grids)
    Vs, pis, _ = O.solve(op)
    best, arg, costs = brute_force(op, p.x0, op.n_controls, p.n_stages)
    assert np.isfinite(best)
    assert Vs[0].shape == (1, 1, 1)
    assert Vs[0][0, 0, 0] == pytest.approx(best, rel=1e-12, abs=0)
    finite = np.sort(costs[np.isfinite(costs)])
    if finite.size > 1 and finite[1] - finite[0] > 1e-9 * abs(finite[0]):
        assert pis[0][0, 0, 0] == arg[0]
        r = O.rollout(op, Vs)
        assert r["status"] == 0
        assert tuple(r["u"]) == tuple(arg)
        assert r["J"] == pytest.approx(best, rel=1e-12)


def test_bruteforce_exercises_stop_and_wait():
    """The braking toy reaches a standstill at the light node and departs
    after a wait on at least one enumerated sequence."""
    p = P.toy_problem(seed=13, n_stages=2, with_light=True).replace(
        n_brake=2, x0=(3.0, 0.6, 0.0), cycle=np.array([10.0]), red=np.array([5.0]), offset=np.array([5.0]))
    op = O.make(p)
    saw_stop = saw_wait = False
    for seq in itertools.product(range(op.n_controls), repeat=2):
        x = p.x0
        for k, u in enumerate(seq):
            r = O.model_step(op, k, *x, *op.decode(u))
            if r is None:
                break
            saw_stop |= k == 0 and r["v1"] == 0.0
            saw_wait |= r["wait"] > 0
            x = (r["v1"], r["soc1"], r["t1"])
    assert saw_stop and saw_wait


# ---------------------------------------------------------------------------
# closed form: constant-speed cruise

def cruise_problem(gamma):
    v0 = 10.0
    f_road = 1600 * 9.81 * 0.01 + 0.5 * 1.2 * 0.7 * v0 ** 2  # 198.96 N on a flat road
    te = f_road * 0.3 / 3.0  # engine torque that balances it (19.896 Nm)
    return P.config0().replace(
        grade=np.zeros(10), light_stage=np.zeros(0, np.int32), cycle=np.zeros(0), red=np.zeros(0),
        offset=np.zeros(0), t_lo=0.0, t_hi=40.0, n_t=41, te_lo=te, te_hi=te, n_te=1,
        tm_lo=0.0, tm_hi=0.0, n_tm=1, n_brake=1, gamma=gamma, x0=(v0, 0.55, 0.0)), te


@pytest.mark.parametrize("gamma", [0.0, 0.5, 1.0])
def test_constant_speed_closed_form(gamma):
    p, te = cruise_problem(gamma)
    op = O.make(p)
    Vs, pis, _ = O.solve(op)
    # fuel rate at w = 100 rad/s and the balancing torque, from the fuel map
    step = O.model_step(op, 0, 10.0, 0.55, 0.0, te, 0.0, 0)
    assert step["v1"] == pytest.approx(10.0, abs=1e-12)
    mf = step["fuel_rate"]
    N, dt = 10, 1.0
    expect = N * (gamma * mf + 1 - gamma) * dt  # c_T(10, 0.55) = 0
    i, j = 5, 5  # v = 10 m/s, soc = 0.55
    for l in range(0, 30):  # t0 = 0..29 s all finish by 40 s
        assert Vs[0][i, j, l] == pytest.approx(expect, rel=1e-12)
    assert not np.isfinite(Vs[0][i, j, 31])  # 31 + 10 > 40
    r = O.rollout(op, Vs)
    assert r["status"] == 0
    assert r["fuel_g"] == pytest.approx(N * mf * dt, rel=1e-12)
    assert r["time_s"] == pytest.approx(N * dt, rel=1e-12)
    assert r["J"] == pytest.approx(expect, rel=1e-12)


# ---------------------------------------------------------------------------
# invariants

def small(seed=21, **kw):
    p = P.config1(seed=seed, n_stages=6, n_v=11, n_soc=9, n_t=31, n_te=5, n_tm=5, n_lights=1, t_hi=30.0)
    return p.replace(**kw)


def no_lights(p):
    return p.replace(light_stage=np.zeros(0, np.int32), cycle=np.zeros(0), red=np.zeros(0),
                     offset=np.zeros(0))


def test_time_independence_without_lights():
    p = no_lights(small())
    Vs, _, _ = O.solve(O.make(p))
    for k in range(p.n_stages):
        V = Vs[k]
        fin = np.isfinite(V)
        # feasibility in t is a prefix and V is non-decreasing in t
        assert np.all(fin[:, :, 1:] <= fin[:, :, :-1])
        with np.errstate(invalid="ignore"):
            d = np.diff(V, axis=2)
        assert np.all((d >= -1e-12) | ~fin[:, :, 1:])
        # the earliest starts all share the same value
        ok = fin[:, :, 3]
        assert np.allclose(V[:, :, 0][ok], V[:, :, 3][ok], rtol=1e-12)


def test_monotone_in_soc_when_only_discharging():
    p = no_lights(small(tm_lo=0.0, tm_hi=100.0))
    Vs, _, _ = O.solve(O.make(p))
    for V in Vs:
        with np.errstate(invalid="ignore"):
            d = np.diff(V, axis=1)
        both = np.isfinite(V[:, 1:, :]) & np.isfinite(V[:, :-1, :])
        assert np.all(d[both] <= 1e-12)
        # feasible at soc_j implies feasible at soc_{j+1}
        assert np.all(np.isfinite(V[:, 1:, :]) >= np.isfinite(V[:, :-1, :]))


def test_raising_tmax_never_raises_value():
    p = small()
    q = p.replace(t_hi=p.t_hi + 10.0, n_t=p.n_t + 10)  # same spacing, 10 more nodes
    Vp, _, _ = O.solve(O.make(p))
    Vq, _, _ = O.solve(O.make(q))
    for a, b in zip(Vp, Vq):
        b = b[:, :, :p.n_t]
        assert np.all(np.isfinite(b) >= np.isfinite(a))
        both = np.isfinite(a)
        assert np.all(b[both] <= a[both] * (1 + 1e-12) + 1e-12)


def test_lower_bound_from_speed_limit():
    p = small()
    Vs, _, _ = O.solve(O.make(p))
    vmax = p.v_hi
    for k, V in enumerate(Vs):
        bound = (1 - p.gamma) * (p.n_stages - k) * p.ds / vmax
        fin = np.isfinite(V)
        assert np.all(V[fin] >= bound - 1e-12)


def test_shift_of_clock_and_offsets():
    p = small(seed=22)
    h = (p.t_hi - p.t_lo) / (p.n_t - 1)
    d = 7 * h
    q = p.replace(t_lo=p.t_lo + d, t_hi=p.t_hi + d, offset=p.offset + d)
    Vp, pp, _ = O.solve(O.make(p))
    Vq, pq, _ = O.solve(O.make(q))
    for a, b in zip(Vp, Vq):
        assert np.array_equal(np.isfinite(a), np.isfinite(b))
        fin = np.isfinite(a)
        assert np.allclose(a[fin], b[fin], rtol=1e-9, atol=0)


def test_monotone_in_fuel_scale():
    p = small(seed=23)
    Va, _, _ = O.solve(O.make(p))
    Vb, _, _ = O.solve(O.make(p.replace(fuel_scale=1.3)))
    for a, b in zip(Va, Vb):
        assert np.array_equal(np.isfinite(a), np.isfinite(b))
        fin = np.isfinite(a)
        assert np.all(b[fin] >= a[fin] - 1e-12)


# ---------------------------------------------------------------------------
# interpolation

def test_trilinear_reproduces_triaffine():
    p = small()
    op = O.make(p)
    v, s, t = (g[:, None, None] for g in (p.nodes("v"),)), None, None
    vv = p.nodes("v")[:, None, None]
    ss = p.nodes("soc")[None, :, None]
    tt = p.nodes("t")[None, None, :]
    f = lambda a, b, c: 1.5 + 0.3 * a - 2.0 * b + 0.05 * c + 0.1 * a * b - 0.01 * a * c + 0.2 * b * c + 0.003 * a * b * c
    V = f(vv, ss, tt) + 0 * vv * ss * tt
    rng = np.random.default_rng(0)
    for _ in range(200):
        a = rng.uniform(p.v_lo, p.v_hi)
        b = rng.uniform(p.soc_lo, p.soc_hi)
        c = rng.uniform(p.t_lo, p.t_hi)
        assert O.interp(op, 1, V, a, b, c) == pytest.approx(f(a, b, c), rel=1e-12, abs=1e-12)
    # nodes reproduce node values exactly
    assert O.interp(op, 1, V, vv[3, 0, 0], ss[0, 4, 0], tt[0, 0, 7]) == V[3, 4, 7]


def test_snap_and_band_rules():
    p = small()
    op = O.make(p)
    V = np.ones(op.shapes[1])
    V[:, :, 10] = np.inf  # an infeasible time slice
    h = (p.t_hi - p.t_lo) / (p.n_t - 1)
    t9 = p.t_lo + 9 * h
    v, s = p.nodes("v")[2], p.nodes("soc")[3]
    assert O.interp(op, 1, V, v, s, t9) == 1.0
    assert O.interp(op, 1, V, v, s, t9 + 0.5e-5 * h) == 1.0  # snapped to node 9
    assert O.interp(op, 1, V, v, s, t9 + 2e-5 * h) == np.inf  # touches node 10
    assert O.interp(op, 1, V, v, s, t9 - 0.5 * h) == 1.0
    # the grid ends: clamp within 1e-5 of a cell, infeasible beyond
    assert O.interp(op, 1, V, p.v_hi + 0.5e-5 * 2.5, s, t9) == 1.0
    assert O.interp(op, 1, V, p.v_hi + 2e-5 * 2.5, s, t9) == np.inf
    assert O.interp(op, 1, V, v, p.soc_lo - 0.5e-5 * 0.0625, t9) == 1.0
    assert O.interp(op, 1, V, v, p.soc_lo - 2e-5 * 0.0625, t9) == np.inf


# ---------------------------------------------------------------------------
# the stage loop against a direct composition of the primitives

def test_stage_loop_matches_direct_minimisation():
    p = small(seed=24)
    op = O.make(p)
    Vn = P.synthetic_value_field(p, seed=5)
    k = int(p.light_stage[0]) - 1  # the stage whose successor holds the light
    res = O.stage(op, k, Vn)
    rng = np.random.default_rng(1)
    vg, sg, tg = p.nodes("v"), p.nodes("soc"), p.nodes("t")
    for _ in range(60):
        i, j, l = rng.integers(p.n_v), rng.integers(p.n_soc), rng.integers(p.n_t)
        best, bu = np.inf, -1
        for u in range(op.n_controls):
            r = O.model_step(op, k, vg[i], sg[j], tg[l], *op.decode(u))
            if r is None:
                continue
            F = r["cost"] + O.interp(op, k + 1, Vn, r["v1"], r["soc1"], r["t1"])
            if F < best:
                best, bu = F, u
        got = res["V"][i, j, l]
        if np.isfinite(best):
            assert got == pytest.approx(best, rel=1e-13)
            assert res["pi"][i, j, l] == bu
        else:
            assert not np.isfinite(got) and res["pi"][i, j, l] == -1
    # sampling returns the same numbers as the full sweep
    idx = rng.integers(0, p.n_states, size=50)
    sm = O.stage(op, k, Vn, idx=idx)
    assert np.array_equal(sm["V"], res["V"].ravel()[idx])
    assert np.array_equal(sm["pi"], res["pi"].ravel()[idx])


def test_modes_bracket_nominal():
    p = small(seed=25)
    op = O.make(p)
    Vn = P.synthetic_value_field(p, seed=6)
    out = {m: O.stage(op, 2, Vn, mode=m)["V"] for m in (O.NOMINAL, O.LENIENT, O.STRICT)}
    lo, nom, hi = out[O.LENIENT], out[O.NOMINAL], out[O.STRICT]
    assert np.all(np.isfinite(lo) >= np.isfinite(nom))
    assert np.all(np.isfinite(nom) >= np.isfinite(hi))
    f = np.isfinite(hi)
    assert np.all(lo[f] <= nom[f] * (1 + 1e-9)) and np.all(nom[f] <= hi[f] * (1 + 1e-9))
    # with no fragility band the three modes coincide
    op0 = O.make(p, fp_band=0.0, phase_band=0.0)
    r = [O.stage(op0, 2, Vn, mode=m)["V"] for m in (0, 1, 2)]
    assert np.array_equal(r[0], r[1]) and np.array_equal(r[0], r[2])
