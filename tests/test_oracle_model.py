"""Pins of the oracle's one-step model against physics and special cases.

Each expectation below comes from a textbook law or a hand-derived special
case, not from re-typing the oracle's expressions:
  * uniform-acceleration kinematics (Eq. 5a, Eq. 2),
  * the road-load special cases (grade only, rolling only, drag only),
  * the battery circuit's power balance Voc*I - R0*I^2 = P (Eq. 5b),
  * charge conservation dSoC * C = I * dt,
  * the cost weighting extremes gamma = 0 and gamma = 1 (Eq. 1, Eq. 6),
  * the light schedule of config 0 (30 s cycle, 15 s red, offset 0; Fig. 3),
  * the stop-at-line, red-arrival and wait readings (Eq. 5c).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2104_01284_gb300 import problems as P

pytestmark = pytest.mark.filterwarnings("ignore")


def bare(**kw):
    """A flat, loss-free single-stage problem (no drag, rolling or grade)."""
    p = P.config0().replace(n_stages=2, grade=np.zeros(2), cda=0.0, crr=0.0,
                            light_stage=np.zeros(0, np.int32), cycle=np.zeros(0), red=np.zeros(0),
                            offset=np.zeros(0), a_min=-50.0, a_max=50.0)
    return p.replace(**kw)


def test_constant_acceleration_kinematics():
    # F = (Te + Tm) * gear / r_wheel = 100 Nm * 10 /m = 1000 N on 1600 kg
    p = bare()
    op = O.make(p)
    r = O.model_step(op, 0, 5.0, 0.5, 3.0, 100.0, 0.0, 0)
    a = 1000.0 / 1600.0
    # v1^2 = v^2 + 2 a d   (textbook)
    assert r["v1"] == pytest.approx(math.sqrt(25.0 + 2 * a * 10.0), rel=1e-14)
    # d = v dt + a dt^2 / 2   (textbook, independent of Eq. 2's mean-speed form)
    dt = r["dt"]
    assert 5.0 * dt + 0.5 * a * dt * dt == pytest.approx(10.0, rel=1e-12)
    assert r["t1"] == pytest.approx(3.0 + dt, rel=1e-15)
    assert r["wait"] == 0.0


def test_coasting_on_flat_loss_free_road_keeps_speed():
    op = O.make(bare())
    r = O.model_step(op, 0, 8.0, 0.5, 0.0, 0.0, 0.0, 0)
    assert r["v1"] == 8.0
    assert r["dt"] == pytest.approx(10.0 / 8.0, rel=1e-15)
    assert r["soc1"] == 0.5
    assert r["fuel_rate"] == 0.0


@pytest.mark.parametrize("grade", [0.03, -0.02])
def test_grade_only_deceleration(grade):
    # on an incline of slope tan(theta) = grade the free deceleration is g sin(theta)
    p = bare(grade=np.array([grade, 0.0]))
    op = O.make(p)
    r = O.model_step(op, 0, 10.0, 0.5, 0.0, 0.0, 0.0, 0)
    sin_th = grade / math.sqrt(1 + grade * grade)
    assert r["v1"] ** 2 == pytest.approx(100.0 - 2 * 9.81 * sin_th * 10.0, rel=1e-13)


def test_rolling_and_drag_special_cases():
    # rolling only: a = -g * Crr = -0.0981 m/s^2
    op = O.make(bare(crr=0.01))
    r = O.model_step(op, 0, 10.0, 0.5, 0.0, 0.0, 0.0, 0)
    assert r["v1"] ** 2 == pytest.approx(100.0 - 2 * 0.0981 * 10.0, rel=1e-13)
    # drag only at 10 m/s: 0.5 * 1.2 * 0.7 * 100 = 42 N -> a = -0.02625 m/s^2
    op = O.make(bare(cda=0.7))
    r = O.model_step(op, 0, 10.0, 0.5, 0.0, 0.0, 0.0, 0)
    assert r["v1"] ** 2 == pytest.approx(100.0 - 2 * 0.02625 * 10.0, rel=1e-13)


def test_brake_adds_its_deceleration():
    op = O.make(bare(brake_decel=2.0))
    r = O.model_step(op, 0, 10.0, 0.5, 0.0, 0.0, 0.0, 1)
    assert r["v1"] ** 2 == pytest.approx(100.0 - 2 * 2.0 * 10.0, rel=1e-13)


@pytest.mark.parametrize("tm", [60.0, -60.0, 5.0])
def test_battery_power_balance_and_charge(tm):
    p = bare()
    op = O.make(p)
    v = 12.0
    r = O.model_step(op, 0, v, 0.6, 0.0, 50.0, tm, 0)
    w = v * 10.0  # motor speed on the crankshaft, rad/s
    pm = tm * w
    pbat = pm / 0.9 if pm > 0 else pm * 0.9
    cur = (0.6 - r["soc1"]) * 18000.0 / r["dt"]  # charge conservation
    # terminal power of a source with internal resistance: Voc I - R0 I^2
    assert 360.0 * cur - 0.1 * cur * cur == pytest.approx(pbat, rel=1e-9)
    assert abs(cur) < 360.0 / (2 * 0.1)  # the physical (smaller) root
    assert math.copysign(1.0, cur) == math.copysign(1.0, tm)


def test_battery_limit_infeasible():
    # P > Voc^2 / (4 R0) = 324 kW cannot be drawn from the circuit
    p = bare(tm_hi=5000.0)
    op = O.make(p)
    assert O.model_step(op, 0, 20.0, 0.6, 0.0, 0.0, 2000.0, 0) is None


def test_fuel_map_points_and_engine_off():
    p = bare(fuel_coef=np.array([0.1, 1e-3, 2e-3, 3e-5, 4e-6, 5e-6]), fuel_scale=2.0)
    op = O.make(p)
    assert O.model_step(op, 0, 10.0, 0.5, 0.0, 0.0, 0.0, 0)["fuel_rate"] == 0.0
    r = O.model_step(op, 0, 10.0, 0.5, 0.0, 100.0, 0.0, 0)
    # w = 100 rad/s, T = 100 Nm: 0.1 + 0.1 + 0.2 + 0.3 + 0.04 + 0.05 = 0.79 g/s, x2 scale
    assert r["fuel_rate"] == pytest.approx(1.58, rel=1e-12)


def test_cost_weighting_extremes():
    p = bare()
    for gamma, expect in ((0.0, "dt"), (1.0, "fuel")):
        op = O.make(p.replace(gamma=gamma))
        r = O.model_step(op, 0, 10.0, 0.5, 0.0, 120.0, 0.0, 0)
        if expect == "dt":
            assert r["cost"] == pytest.approx(r["dt"], rel=1e-15)
        else:
            assert r["cost"] == pytest.approx(r["fuel_rate"] * r["dt"], rel=1e-15)


def test_acceleration_limits():
    p = bare(a_max=0.5)
    op = O.make(p)
    # 100 Nm -> 0.625 m/s^2 > 0.5
    assert O.model_step(op, 0, 5.0, 0.5, 0.0, 100.0, 0.0, 0) is None
    assert O.model_step(op, 0, 5.0, 0.5, 0.0, 70.0, 0.0, 0) is not None
    p = bare(a_min=-1.0)
    op = O.make(p)
    assert O.model_step(op, 0, 5.0, 0.5, 0.0, 0.0, 0.0, 1) is None  # -2 m/s^2 brake


def test_light_schedule_config0():
    op = O.make(P.config0())
    # red during [0, 15) and [30, 45), green during [15, 30)
    for t, red in ((0.0, True), (14.999, True), (15.0, False), (29.999, False), (30.0, True),
                   (44.0, True), (-0.001, False), (-15.0, False), (-15.001, True)):
        assert O.is_red(op, 0, t) == red, t


def light_problem():
    # one light at node 1, 20 s cycle, 8 s red, offset 3 s: red in [3, 11) + 20 m
    return bare(n_stages=3, grade=np.zeros(3), light_stage=np.array([1], np.int32),
                cycle=np.array([20.0]), red=np.array([8.0]), offset=np.array([3.0]))


def test_stop_at_line_only_before_a_light():
    op = O.make(light_problem())
    # v = 4 m/s with 2 m/s^2 braking: v^2 + 2 d a = 16 - 40 < 0
    r = O.model_step(op, 0, 4.0, 0.5, 0.0, 0.0, 0.0, 1)  # node 1 holds the light
    assert r is not None and r["v1"] == 0.0 and r["dt"] == pytest.approx(5.0)
    assert O.model_step(op, 1, 4.0, 0.5, 0.0, 0.0, 0.0, 1) is None  # node 2 has none


def test_red_arrival_is_infeasible():
    op = O.make(light_problem())
    # coasting at 10 m/s (loss-free) arrives after exactly 1 s
    assert O.model_step(op, 0, 10.0, 0.5, 1.0, 0.0, 0.0, 0) is not None  # arrives at 2 s: green
    assert O.model_step(op, 0, 10.0, 0.5, 2.5, 0.0, 0.0, 0) is None  # arrives at 3.5 s: red
    assert O.model_step(op, 0, 10.0, 0.5, 10.5, 0.0, 0.0, 0) is not None  # arrives at 11.5 s: green


def test_wait_for_green_at_standstill():
    p = light_problem().replace(gamma=0.25)
    op = O.make(p)
    # standing at node 1 at t = 5 s: red until 11 s -> wait 6 s, then drive
    r = O.model_step(op, 1, 0.0, 0.5, 5.0, 100.0, 0.0, 0)
    assert r["wait"] == pytest.approx(6.0)
    assert r["t1"] == pytest.approx(5.0 + 6.0 + r["dt"])
    # the wait costs time only: (1 - gamma) * wait on top of the driving cost
    drive = O.model_step(op, 1, 0.0, 0.5, 12.0, 100.0, 0.0, 0)  # green: no wait
    assert drive["wait"] == 0.0
    assert r["cost"] == pytest.approx(drive["cost"] + 0.75 * 6.0, rel=1e-12)
    assert r["soc1"] == drive["soc1"]


def test_terminal_cost_special_values():
    op = O.make(P.config0())
    assert O.terminal_cost(op, 10.0, 0.55) == 0.0
    assert O.terminal_cost(op, 11.0, 0.55) == pytest.approx(1.0)
    assert O.terminal_cost(op, 10.0, 0.45) == pytest.approx(100.0)
    assert O.terminal_cost(op, 10.0, 0.65) == 0.0
