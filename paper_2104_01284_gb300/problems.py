"""Seeded synthetic problem instances for the eco-driving DP.

This module only *describes* inputs: route grade, traffic-light schedules
(SPaT), grids, control sets and model constants.  It holds none of the DP's
arithmetic (no dynamics, no costs, no interpolation), so both the FP64 oracle
and the CUDA path can consume the same instances without sharing any of the
method.

Model readings fixed here (the paper leaves them open, Sec. II and Sec. III):

* Drivetrain: one fixed total ratio gear / r_wheel = 3.0 / 0.3 m^-1; the BSG sits
  on the crankshaft (P0), so engine and motor torques add (Sec. II).
* Road load: rho = 1.2 kg/m^3, g = 9.81 m/s^2, grade as a fraction per
  distance step (Eq. 5a).
* Fuel map: a seeded quadratic in engine speed and torque,
  mdot = s_f (c0 + c1 w + c2 T + c3 w T + c4 w^2 + c5 T^2) g/s for T > 0 and 0
  for T = 0 (start-stop, Sec. II).
* Motor efficiency constant 0.90; battery: zeroth-order circuit, Voc = 360 V,
  R0 = 0.1 ohm, 5 Ah (Eq. 5b).
* Terminal cost c_T = w_soc max(0, soc_ref - soc) + w_v (v - v_ref)^2 with
  soc_ref = 0.55, w_soc = 1000, v_ref = 10 m/s, w_v = 1 (Eq. 6, Eq. 9a).
* gamma = 0.5 in the stage cost (Eq. 1, Eq. 6).
* Light schedule: red iff ((t - offset) mod cycle) lies in [0, red) (Fig. 3).

Random draws use numpy ``Generator(PCG64(seed))`` in the order documented in
each factory.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem",
    "config0",
    "config1",
    "config2_seeds",
    "config3_batch",
    "config3_small",
    "config4_fleet",
    "paper_table1",
    "toy_problem",
    "uniform_nodes",
    "synthetic_value_field",
]


def uniform_nodes(lo: float, hi: float, n: int) -> np.ndarray:
    """Grid nodes lo + (hi - lo) * i / (n - 1), evaluated in that order.

    Multiplying before dividing keeps integer-valued nodes (0, 100, ...)
    exact, so a symmetric torque grid contains an exact 0.
    """
    if n == 1:
        return np.array([lo], np.float64)
    i = np.arange(n, dtype=np.float64)
    return lo + (hi - lo) * i / (n - 1)


@dataclass
class Problem:
    """One receding-horizon DP instance (all SI units; grade is a fraction)."""

    name: str = "problem"
    n_stages: int = 10
    ds: float = 10.0
    grade: np.ndarray = field(default_factory=lambda: np.zeros(10))
    # state grids (uniform, inclusive ends)
    v_lo: float = 0.0
    v_hi: float = 20.0
    n_v: int = 11
    soc_lo: float = 0.40
    soc_hi: float = 0.70
    n_soc: int = 11
    t_lo: float = 0.0
    t_hi: float = 40.0
    n_t: int = 21
    # control grids: engine torque, motor (BSG) torque, brake flag count
    te_lo: float = 0.0
    te_hi: float = 200.0
    n_te: int = 11
    tm_lo: float = -100.0
    tm_hi: float = 100.0
    n_tm: int = 11
    n_brake: int = 1
    brake_decel: float = 2.0
    # comfort acceleration limits (Eq. 7d)
    a_min: float = -3.0
    a_max: float = 2.5
    # vehicle and powertrain
    mass: float = 1600.0
    cda: float = 0.7
    crr: float = 0.01
    rho: float = 1.2
    g: float = 9.81
    r_wheel: float = 0.3
    gear: float = 3.0
    eta_motor: float = 0.90
    # battery
    voc: float = 360.0
    r0: float = 0.1
    capacity_As: float = 5.0 * 3600.0
    # fuel map and cost weights
    fuel_coef: np.ndarray = field(default_factory=lambda: np.zeros(6))
    fuel_scale: float = 1.0
    gamma: float = 0.5
    # terminal cost
    soc_ref: float = 0.55
    w_soc: float = 1000.0
    v_ref: float = 10.0
    w_v: float = 1.0
    # traffic lights: node index k (position / ds), cycle, red duration, offset
    light_stage: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    cycle: np.ndarray = field(default_factory=lambda: np.zeros(0))
    red: np.ndarray = field(default_factory=lambda: np.zeros(0))
    offset: np.ndarray = field(default_factory=lambda: np.zeros(0))
    # initial state for rollout / adjoint
    x0: tuple = (10.0, 0.55, 0.0)
    # paper variants (0 = the default readings):
    # light_model 1: green indicator sampled on the time grid (Sec. III, Eq. 8)
    light_model: int = 0
    # torque_limits 1: speed-dependent limits (Eq. 7e, 7f): engine torque
    # <= c0 + c1 w + c2 w^2 and BSG power |T_bsg| w <= bsg_power_max, with w
    # the crank speed (rad/s).  The default curve peaks near 200 Nm at
    # w = 180 rad/s; 12 kW caps the BSG above w = 120 rad/s.
    torque_limits: int = 0
    te_max_coef: np.ndarray = field(default_factory=lambda: np.array([120.0, 0.9, -0.0025]))
    bsg_power_max: float = 12000.0

    # -- derived sizes ---------------------------------------------------
    @property
    def n_controls(self) -> int:
        return self.n_te * self.n_tm * self.n_brake

    @property
    def n_states(self) -> int:
        return self.n_v * self.n_soc * self.n_t

    @property
    def evals_per_solve(self) -> int:
        """Nominal state x control evaluations of one backward sweep."""
        return self.n_stages * self.n_states * self.n_controls

    def nodes(self, axis: str) -> np.ndarray:
        lo, hi, n = {
            "v": (self.v_lo, self.v_hi, self.n_v),
            "soc": (self.soc_lo, self.soc_hi, self.n_soc),
            "t": (self.t_lo, self.t_hi, self.n_t),
            "te": (self.te_lo, self.te_hi, self.n_te),
            "tm": (self.tm_lo, self.tm_hi, self.n_tm),
        }[axis]
        return uniform_nodes(lo, hi, n)

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)

    def copy(self) -> "Problem":
        p = dataclasses.replace(self)
        for f in ("grade", "fuel_coef", "light_stage", "cycle", "red", "offset", "te_max_coef"):
            setattr(p, f, np.array(getattr(self, f), copy=True))
        return p


# -- draws ----------------------------------------------------------------

def _draw_fuel(rng: np.random.Generator) -> np.ndarray:
    """Six fuel-map coefficients, drawn in the order c0..c5."""
    lo = np.array([0.10, 0.0, 0.0, 4e-5, 0.0, 0.0])
    hi = np.array([0.20, 5e-4, 2e-3, 7e-5, 2e-6, 5e-6])
    return np.array([rng.uniform(lo[i], hi[i]) for i in range(6)])


def _draw_lights(rng: np.random.Generator, n_lights: int, node_lo: int, node_hi: int):
    """Distinct light nodes in [node_lo, node_hi], then per light (in node
    order) cycle ~ U[40, 90] s, red = cycle * U[0.3, 0.6], offset ~ U[0, cycle)."""
    nodes = np.sort(rng.choice(np.arange(node_lo, node_hi + 1), size=n_lights, replace=False))
    cyc = np.empty(n_lights)
    red = np.empty(n_lights)
    off = np.empty(n_lights)
    for j in range(n_lights):
        cyc[j] = rng.uniform(40.0, 90.0)
        red[j] = cyc[j] * rng.uniform(0.3, 0.6)
        off[j] = rng.uniform(0.0, cyc[j])
    return nodes.astype(np.int32), cyc, red, off


# -- configurations ---------------------------------------------------------

def config0(seed: int = 0) -> Problem:
    """Tiny single horizon: 100 m flat road, 10 stages, 11x11x21 states,
    11x11 torque controls (no brake flag), one light at 60 m (node 6) with a
    30 s cycle, 15 s red, offset 0.  Draws: fuel coefficients only."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return Problem(
        name=f"c0-tiny-s{seed}",
        n_stages=10,
        ds=10.0,
        grade=np.zeros(10),
        v_lo=0.0, v_hi=20.0, n_v=11,
        soc_lo=0.40, soc_hi=0.70, n_soc=11,
        t_lo=0.0, t_hi=40.0, n_t=21,
        te_lo=0.0, te_hi=200.0, n_te=11,
        tm_lo=-100.0, tm_hi=100.0, n_tm=11,
        n_brake=1,
        fuel_coef=_draw_fuel(rng),
        light_stage=np.array([6], np.int32),
        cycle=np.array([30.0]),
        red=np.array([15.0]),
        offset=np.array([0.0]),
        # (10 m/s, 0.55, 0 s) cannot reach the light at 60 m after its red
        # phase [0, 15) s without a brake; start slower, with some charge to use.
        x0=(4.0, 0.58, 0.0),
    )


def config1(seed: int = 1, n_stages: int = 100, n_v: int = 51, n_soc: int = 51,
            n_t: int = 201, n_te: int = 31, n_tm: int = 31, n_lights: int = 4,
            t_hi: float | None = None) -> Problem:
    """Paper-scale single horizon: 1000 m (100 stages of 10 m), grade i.i.d.
    U(-3 %, +3 %) per step, v 51 pts over 0-25 m/s, SoC 51 pts over 0.30-0.80,
    t 201 pts over 0-200 s, 31x31 torques x brake flag, 4 lights at distinct
    nodes in [5, 95].  Draw order: fuel coefficients, grade, lights.

    The keyword sizes let tests shrink the same instance family (fewer stages
    or grid points) while keeping its structure."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fuel = _draw_fuel(rng)
    grade = rng.uniform(-0.03, 0.03, size=n_stages)
    lo = max(1, int(round(0.05 * n_stages)))
    hi = max(lo, min(n_stages - 1, int(round(0.95 * n_stages))))
    n_l = min(n_lights, hi - lo + 1)
    nodes, cyc, red, off = _draw_lights(rng, n_l, lo, hi)
    if t_hi is None:
        t_hi = 200.0 * n_stages / 100.0
    return Problem(
        name=f"c1-paper-s{seed}" if n_stages == 100 else f"c1-N{n_stages}-s{seed}",
        n_stages=n_stages,
        ds=10.0,
        grade=grade,
        v_lo=0.0, v_hi=25.0, n_v=n_v,
        soc_lo=0.30, soc_hi=0.80, n_soc=n_soc,
        t_lo=0.0, t_hi=float(t_hi), n_t=n_t,
        te_lo=0.0, te_hi=200.0, n_te=n_te,
        tm_lo=-100.0, tm_hi=100.0, n_tm=n_tm,
        n_brake=2,
        fuel_coef=fuel,
        light_stage=nodes,
        cycle=cyc,
        red=red,
        offset=off,
    )


def config2_seeds(first: int = 100, count: int = 20) -> list[int]:
    """Seeds scanned (in order) for the adjoint study on config-1 problems."""
    return list(range(first, first + count))


def config3_batch(seed: int = 3, n_instances: int = 256) -> list[Problem]:
    """Batched uneven instances: per instance, in order, horizon U{20..150}
    stages, n_v U{31..61}, n_soc U{31..51}, n_t U{101..251}, n_te = n_tm
    U{21..31} (x2 brake), lights U{1..6}, then the fuel map, grade and
    lights.  The t range scales with the horizon (2 s per 10 m step)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(n_instances):
        n_stages = int(rng.integers(20, 151))
        n_v = int(rng.integers(31, 62))
        n_soc = int(rng.integers(31, 52))
        n_t = int(rng.integers(101, 252))
        n_u = int(rng.integers(21, 32))
        n_l = int(rng.integers(1, 7))
        fuel = _draw_fuel(rng)
        grade = rng.uniform(-0.03, 0.03, size=n_stages)
        lo, hi = 1, n_stages - 1
        nodes, cyc, red, off = _draw_lights(rng, min(n_l, hi - lo + 1), lo, hi)
        out.append(Problem(
            name=f"c3-s{seed}-{b}", n_stages=n_stages, ds=10.0, grade=grade,
            v_lo=0.0, v_hi=25.0, n_v=n_v, soc_lo=0.30, soc_hi=0.80, n_soc=n_soc,
            t_lo=0.0, t_hi=2.0 * n_stages, n_t=n_t,
            te_lo=0.0, te_hi=200.0, n_te=n_u, tm_lo=-100.0, tm_hi=100.0, n_tm=n_u,
            n_brake=2, fuel_coef=fuel, light_stage=nodes, cycle=cyc, red=red, offset=off))
    return out


def config3_small(seed: int = 33, n_instances: int = 6) -> list[Problem]:
    """Uneven instances at sizes the oracle sweeps in seconds, for batch
    parity: per instance, in order, horizon U{4..14} stages, n_v U{9..21},
    n_soc U{7..19}, n_t U{17..45}, n_te U{5..9}, n_tm U{5..9} (unequal steps
    give one torque class per control), brake flag with probability 1/2,
    lights U{1..3} with short cycles U(6, 14) s (red fraction 0.3-0.6), then
    the fuel map and grade.  t spans 2.5 s per step."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(n_instances):
        n_stages = int(rng.integers(4, 15))
        n_v = int(rng.integers(9, 22))
        n_soc = int(rng.integers(7, 20))
        n_t = int(rng.integers(17, 46))
        n_te = int(rng.integers(5, 10))
        n_tm = int(rng.integers(5, 10))
        n_brake = int(rng.integers(1, 3))
        n_l = min(int(rng.integers(1, 4)), n_stages - 1)
        fuel = _draw_fuel(rng)
        grade = rng.uniform(-0.03, 0.03, size=n_stages)
        nodes = np.sort(rng.choice(np.arange(1, n_stages), size=n_l, replace=False)).astype(np.int32)
        cyc = rng.uniform(6.0, 14.0, n_l)
        red = cyc * rng.uniform(0.3, 0.6, n_l)
        off = rng.uniform(0.0, 1.0, n_l) * cyc
        out.append(Problem(
            name=f"c3-small-s{seed}-{b}", n_stages=n_stages, ds=10.0, grade=grade,
            v_lo=0.0, v_hi=20.0, n_v=n_v, soc_lo=0.40, soc_hi=0.70, n_soc=n_soc,
            t_lo=0.0, t_hi=2.5 * n_stages, n_t=n_t,
            te_lo=0.0, te_hi=200.0, n_te=n_te, tm_lo=-100.0, tm_hi=100.0, n_tm=n_tm,
            n_brake=n_brake, fuel_coef=fuel, light_stage=nodes, cycle=cyc, red=red, offset=off,
            x0=(4.0, 0.58, 0.0)))
    return out


def config4_fleet(seed: int = 4, n_vehicles: int = 1000, route_m: float = 5000.0,
                  n_lights: int = 10):
    """Routes for the serving study: per vehicle a 5 km route (500 steps of
    10 m) with grade U(+-3 %) and 10 lights at distinct nodes, SPaT as in
    config 1.  Returns (fuel_coef, list of (grade[500], nodes, cycle, red,
    offset)).  One fuel map is shared by the fleet."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fuel = _draw_fuel(rng)
    n_steps = int(round(route_m / 10.0))
    routes = []
    for _ in range(n_vehicles):
        grade = rng.uniform(-0.03, 0.03, size=n_steps)
        nodes, cyc, red, off = _draw_lights(rng, n_lights, 1, n_steps - 1)
        routes.append((grade, nodes, cyc, red, off))
    return fuel, routes


def horizon_problem(fuel: np.ndarray, route, start_node: int, t0: float,
                    n_stages: int = 50, n_t: int = 101, name: str = "c4", n_v: int = 51, n_soc: int = 51,
                    n_te: int = 31, n_tm: int = 31) -> Problem:
    """The receding-horizon window [start_node, start_node + n_stages) of a
    route as a stand-alone problem whose time grid starts at t0 (absolute
    route time), as in config 4: grids as config 1 but 101 time points over
    the window's 2 s/step budget.  The keyword sizes shrink the grids for
    tests while keeping the structure."""
    grade, nodes, cyc, red, off = route
    g = np.asarray(grade)[start_node:start_node + n_stages]
    if g.size < n_stages:
        g = np.concatenate([g, np.zeros(n_stages - g.size)])
    rel = nodes - start_node
    keep = (rel >= 1) & (rel <= n_stages - 1)
    return Problem(
        name=name, n_stages=n_stages, ds=10.0, grade=g,
        v_lo=0.0, v_hi=25.0, n_v=n_v, soc_lo=0.30, soc_hi=0.80, n_soc=n_soc,
        t_lo=float(t0), t_hi=float(t0) + 2.0 * n_stages, n_t=n_t,
        te_lo=0.0, te_hi=200.0, n_te=n_te, tm_lo=-100.0, tm_hi=100.0, n_tm=n_tm,
        n_brake=2, fuel_coef=np.array(fuel, copy=True),
        light_stage=rel[keep].astype(np.int32), cycle=cyc[keep], red=red[keep],
        offset=off[keep])


def paper_table1(seed: int = 5) -> Problem:
    """The grid of the paper's timing study (Sec. V, Table I): a 200 m
    horizon of 20 steps of 10 m with t_f = 80 s; 35 speeds x 26 SoC points x
    40 time points; 23 engine x 30 BSG torques (no brake flag: the paper's
    controls are the two torques).  Seeded stand-in for its routes: grade
    U(+-3 %), one light in the window with the SPaT of config 1.  Draw order:
    fuel coefficients, grade, light."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fuel = _draw_fuel(rng)
    grade = rng.uniform(-0.03, 0.03, size=20)
    nodes, cyc, red, off = _draw_lights(rng, 1, 2, 18)
    return Problem(
        name=f"paper-table1-s{seed}", n_stages=20, ds=10.0, grade=grade,
        v_lo=0.0, v_hi=25.0, n_v=35, soc_lo=0.30, soc_hi=0.80, n_soc=26,
        t_lo=0.0, t_hi=80.0, n_t=40,
        te_lo=0.0, te_hi=200.0, n_te=23, tm_lo=-100.0, tm_hi=100.0, n_tm=30,
        n_brake=1, fuel_coef=fuel, light_stage=nodes, cycle=cyc, red=red, offset=off)


def toy_problem(seed: int = 7, n_stages: int = 3, with_light: bool = True) -> Problem:
    """A few-stage toy with a handful of controls (2 engine torques x 2
    motor torques x brake flag = 8) and one light at node 1 (when
    with_light) for brute-force enumeration.  Draws: fuel coefficients, grade
    U(+-2 %) per step, light cycle/red/offset."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fuel = _draw_fuel(rng)
    grade = rng.uniform(-0.02, 0.02, size=n_stages)
    cyc = rng.uniform(6.0, 12.0)
    red = cyc * rng.uniform(0.3, 0.6)
    off = rng.uniform(0.0, cyc)
    lights = dict(light_stage=np.array([1], np.int32), cycle=np.array([cyc]),
                  red=np.array([red]), offset=np.array([off])) if with_light else {}
    return Problem(
        name=f"toy-s{seed}", n_stages=n_stages, ds=10.0, grade=grade,
        v_lo=0.0, v_hi=20.0, n_v=11, soc_lo=0.40, soc_hi=0.70, n_soc=11,
        t_lo=0.0, t_hi=40.0, n_t=21,
        te_lo=0.0, te_hi=150.0, n_te=2, tm_lo=-60.0, tm_hi=60.0, n_tm=2,
        n_brake=2, fuel_coef=fuel, **lights)


def synthetic_value_field(p: Problem, seed: int, inf_frac: float = 0.15) -> np.ndarray:
    """A seeded stand-in for a next-stage cost-to-go on p's grid
    ([n_v][n_soc][n_t], float64): a smooth bowl in (v, soc) plus a ramp in t
    and small noise, with +inf on a random t-suffix per (v, soc) row (about
    inf_frac of the states).  It feeds single-stage comparisons and carries no
    DP arithmetic."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = p.nodes("v")[:, None, None]
    s = p.nodes("soc")[None, :, None]
    t = p.nodes("t")[None, None, :]
    base = (v - p.v_ref) ** 2 + 300.0 * np.maximum(0.0, p.soc_ref - s) + 0.05 * (t - p.t_lo)
    base = base + rng.uniform(0.0, 0.5, size=(p.n_v, p.n_soc, p.n_t))
    cut = rng.uniform(1.0 - 2.0 * inf_frac, 1.0 + 0.2, size=(p.n_v, p.n_soc, 1))
    lt = (np.arange(p.n_t)[None, None, :] / max(1, p.n_t - 1))
    base = np.where(lt > cut, np.inf, base)
    return np.ascontiguousarray(base)
