"""Pins of the oracle's lenient and strict modes (the FP32-fragile decision
bookkeeping that every parity test's excuse intervals come from).

Each case builds one transition whose decision sits at a known distance from
its threshold and evaluates it in the three modes:

* inside the band (an arrival 5e-5 s from a phase boundary, Eq. 5c / 7c; an
  SoC interpolation fraction 2^-20 of a cell from the 1e-5 snap; an
  acceleration exactly at a_max, Eq. 7d): lenient must take the feasible
  side, strict the infeasible one, nominal the side the rule gives;
* outside the band (2e-4 s from the boundary, the fraction 3.5e-5 of a cell,
  the acceleration 1e-4 below the limit): lenient, nominal and strict must be
  equal, bit for bit.

A mode that never flips a fragile decision fails the first group; a band 100
times too wide (1e-2 s, 100 x 2^-18 relative) fails the second; a band 100
times too narrow misses the first group's fragile decisions and fails it too.
"""
import numpy as np
import pytest

import oracle as O
from paper_2104_01284_gb300 import problems as P

pytestmark = pytest.mark.filterwarnings("ignore")

MODES = (O.LENIENT, O.NOMINAL, O.STRICT)
# what the cases run with; test_planted_mistakes_are_caught swaps these for a
# mode mapping that never flips and for bands 100 times too wide or narrow
SETUP = dict(modes=MODES, bands={})


def mk(p, **kw):
    return O.make(p, **kw, **SETUP["bands"])


def frictionless(**kw):
    """Two 10 m stages on a flat road with no rolling or air resistance, so
    the road load is exactly 0 and the acceleration is exactly the tractive
    force over the mass."""
    base = dict(n_stages=2, grade=np.zeros(2), crr=0.0, cda=0.0, v_lo=0.0, v_hi=20.0, n_v=11,
                soc_lo=0.40, soc_hi=0.70, n_soc=11, t_lo=0.0, t_hi=40.0, n_t=41,
                te_lo=0.0, te_hi=0.0, n_te=1, tm_lo=0.0, tm_hi=0.0, n_tm=1, n_brake=1,
                fuel_coef=np.array([0.15, 2e-4, 1e-3, 5e-5, 1e-6, 2e-6]))
    base.update(kw)
    return P.Problem(**base)


def three_modes(op, k, Vn, v, soc, t, ie=0, im=0, b=0):
    out = [O.evaluate(op, k, Vn, v, soc, t, ie, im, b, m) for m in SETUP["modes"]]
    return [F for F, _ in out], out[1][1]


def light_problem(offset):
    """A light at node 1 (cycle 30 s, red 15 s); the coasting control (no
    torque) keeps v = 10 m/s, so the arrival is exactly t + 1 s."""
    return frictionless(light_stage=np.array([1], np.int32), cycle=np.array([30.0]), red=np.array([15.0]),
                        offset=np.array([offset]))


def test_coasting_step_is_exact():
    op = mk(light_problem(10.0))  # arrival phase 21 s: green
    st = O.model_step(op, 0, 10.0, 0.55, 0.0, 0.0, 0.0, 0)
    assert st["v1"] == 10.0 and st["t1"] == 1.0 and st["soc1"] == 0.55 and st["cost"] == 0.5


@pytest.mark.parametrize("delta,nominal_red", [(5e-5, True), (-5e-5, False)])
def test_arrival_inside_the_phase_band_flips(delta, nominal_red):
    """Arrival 5e-5 s after the red onset (nominal: red, infeasible) or 5e-5 s
    before it (nominal: green, feasible): lenient arrives on green, strict on
    red (Eq. 5c, 7c with the 1e-4 s band of acceptance (b))."""
    op = mk(light_problem(1.0 - delta))  # phase at arrival = delta mod 30
    Vn = np.zeros(op.shapes[1])
    (lo, nom, hi), nf = three_modes(op, 0, Vn, 10.0, 0.55, 0.0)
    assert O.is_red(op, 0, 1.0) == nominal_red
    assert nf >= 1
    assert lo == 0.5 and hi == np.inf
    assert nom == (np.inf if nominal_red else 0.5)


@pytest.mark.parametrize("delta", [2e-4, -2e-4, 15.0 + 2e-4, 15.0 - 2e-4])
def test_arrival_outside_the_phase_band_is_not_fragile(delta):
    """2e-4 s from a red onset or a green onset: every mode agrees exactly."""
    op = mk(light_problem(1.0 - delta))
    Vn = np.zeros(op.shapes[1])
    (lo, nom, hi), _ = three_modes(op, 0, Vn, 10.0, 0.55, 0.0)
    assert lo == nom == hi
    assert nom == (np.inf if (delta % 30.0) < 15.0 else 0.5)


def test_arrival_at_the_green_onset_band_flips():
    """Arrival 5e-5 s before the end of red: nominal red; lenient green."""
    op = mk(light_problem(1.0 - (15.0 - 5e-5)))
    Vn = np.zeros(op.shapes[1])
    (lo, nom, hi), nf = three_modes(op, 0, Vn, 10.0, 0.55, 0.0)
    assert nf >= 1 and lo == 0.5 and nom == np.inf and hi == np.inf


def soc_problem(frac):
    """A charging step (BSG torque -50 Nm at 10 m/s, no light) and a stage-1
    SoC grid placed so that the arrival SoC sits `frac` of a cell above node
    5; everything else lands exactly on nodes."""
    p = frictionless(tm_lo=-50.0, tm_hi=-50.0, te_lo=50.0, te_hi=50.0)
    op0 = mk(p)
    st = O.model_step(op0, 0, 10.0, 0.55, 0.0, 50.0, -50.0, 0)
    assert st is not None and st["v1"] == 10.0 and st["soc1"] > 0.55
    h = 0.03
    x1 = st["soc1"] - (5 + frac) * h + h * np.arange(11)
    v = p.nodes("v")
    t = p.nodes("t")
    grids = [(v, p.nodes("soc"), t), (v, x1, t), (v, x1, t)]
    op = mk(p, grids=grids)
    shift = (st["soc1"] - 0.55) / h
    return op, st, shift


def test_soc_band_scale_is_small():
    """The case's SoC shift is a fraction of a cell, so its FP32 band is
    2^-18 (1 + shift), about 4e-6 -- wider than 2^-20 and narrower than 2.5e-5."""
    _, _, shift = soc_problem(1e-5)
    band = 2.0 ** -18 * (1 + abs(shift))
    assert 2.0 ** -20 < band < 2.5e-5 / 4 and band * 100 > 2.5e-5


@pytest.mark.parametrize("sign", [+1, -1])
def test_soc_fraction_inside_the_snap_band_flips(sign):
    """The fraction is 1e-5 +- 2^-20 of a cell and the upper SoC corner is
    infeasible: snapping (lenient) keeps the value finite, not snapping
    (strict) makes it infinite, nominal snaps exactly when the fraction is
    below 1e-5."""
    op, st, _ = soc_problem(1e-5 + sign * 2.0 ** -20)
    Vn = np.zeros(op.shapes[1])
    Vn[:, 6, :] = np.inf  # the node above the arrival
    (lo, nom, hi), nf = three_modes(op, 0, Vn, 10.0, 0.55, 0.0)
    assert nf >= 1
    assert lo == pytest.approx(st["cost"], rel=1e-12) and hi == np.inf
    assert nom == (np.inf if sign > 0 else lo)


def test_soc_fraction_outside_the_snap_band_is_exact():
    """The fraction 3.5e-5 of a cell, beyond the band: the modes agree
    bit for bit on the interpolated value (upper corner 100 higher)."""
    frac = 3.5e-5
    op, st, _ = soc_problem(frac)
    Vn = np.zeros(op.shapes[1])
    Vn[:, 6:, :] = 100.0
    (lo, nom, hi), _ = three_modes(op, 0, Vn, 10.0, 0.55, 0.0)
    assert lo == nom == hi
    assert nom == pytest.approx(st["cost"] + 100.0 * frac, rel=1e-6)


def accel_problem(te):
    """Engine torque te on the frictionless car: a = te * 10 / 1600."""
    return frictionless(te_lo=te, te_hi=te)


def test_acceleration_at_the_limit_flips():
    """te = 400 Nm gives a = 2.5 m/s^2 = a_max exactly (Eq. 7d): nominal and
    lenient accept it, strict rejects it."""
    op = mk(accel_problem(400.0))
    Vn = np.zeros(op.shapes[1])
    (lo, nom, hi), nf = three_modes(op, 0, Vn, 10.0, 0.55, 0.0)
    assert nf >= 1
    assert np.isfinite(lo) and nom == lo and hi == np.inf


def test_acceleration_above_the_limit_within_the_band_flips():
    """a = 2.5 + 2e-6 (inside the 2^-18 relative band of the forces): nominal
    and strict reject it, lenient accepts it."""
    op = mk(accel_problem((2.5 + 2e-6) * 1600.0 / 10.0))
    Vn = np.zeros(op.shapes[1])
    (lo, nom, hi), nf = three_modes(op, 0, Vn, 10.0, 0.55, 0.0)
    assert nf >= 1 and np.isfinite(lo) and nom == np.inf and hi == np.inf


@pytest.mark.parametrize("da", [-1e-4, 1e-4])
def test_acceleration_outside_the_band_is_not_fragile(da):
    """1e-4 m/s^2 from the limit (about ten bands away): the modes agree."""
    op = mk(accel_problem((2.5 + da) * 1600.0 / 10.0))
    Vn = np.zeros(op.shapes[1])
    (lo, nom, hi), _ = three_modes(op, 0, Vn, 10.0, 0.55, 0.0)
    assert lo == nom == hi
    assert np.isfinite(nom) == (da < 0)


def test_nothing_near_a_threshold_means_no_fragile_decision():
    """A plain coasting step between two grid nodes of every axis, far from
    every threshold and with no light: no fragile decision at all."""
    p = frictionless(te_lo=20.0, te_hi=20.0, v_lo=0.5, v_hi=20.5, n_v=11)
    op = mk(p)
    Vn = np.arange(np.prod(op.shapes[1]), dtype=np.float64).reshape(op.shapes[1]) * 1e-3
    (lo, nom, hi), nf = three_modes(op, 0, Vn, 10.5, 0.55, 0.0)
    assert nf == 0 and lo == nom == hi and np.isfinite(nom)


def test_stage_modes_bracket_and_count():
    """orc_stage's three modes on the light problem's state row: lenient <=
    nominal <= strict everywhere, with the fragile arrival counted."""
    op = mk(light_problem(1.0 - 5e-5))
    Vn = np.zeros(op.shapes[1])
    r = {m: O.stage(op, 0, Vn, mode=m) for m in SETUP["modes"]}
    lo, nom, hi = (r[m]["V"] for m in SETUP["modes"])
    with np.errstate(invalid="ignore"):
        assert np.all((lo <= nom) | np.isnan(nom - lo))
        assert np.all((nom <= hi) | (hi == np.inf))
    i = 5  # v = 10 m/s
    assert lo[i, 5, 0] == 0.5 and hi[i, 5, 0] == np.inf and r[SETUP["modes"][2]]["nfrag"][i, 5, 0] >= 1


CASES = [
    lambda: test_arrival_inside_the_phase_band_flips(5e-5, True),
    lambda: test_arrival_inside_the_phase_band_flips(-5e-5, False),
    lambda: test_arrival_at_the_green_onset_band_flips(),
    lambda: [test_arrival_outside_the_phase_band_is_not_fragile(d) for d in (2e-4, -2e-4, 15 + 2e-4, 15 - 2e-4)],
    lambda: [test_soc_fraction_inside_the_snap_band_flips(s) for s in (1, -1)],
    lambda: test_soc_fraction_outside_the_snap_band_is_exact(),
    lambda: test_acceleration_at_the_limit_flips(),
    lambda: test_acceleration_above_the_limit_within_the_band_flips(),
    lambda: [test_acceleration_outside_the_band_is_not_fragile(d) for d in (-1e-4, 1e-4)],
    lambda: test_stage_modes_bracket_and_count(),
]


def _failures():
    n = 0
    for case in CASES:
        try:
            case()
        except AssertionError:
            n += 1
    return n


@pytest.mark.parametrize("mistake", ["never_flips", "band_x100", "band_div100"])
def test_planted_mistakes_are_caught(monkeypatch, mistake):
    """The cases above catch a mode that never flips (lenient and strict
    evaluated as nominal) and bands 100 times too wide or too narrow (each
    case group that should catch it fails), and all pass as written."""
    assert _failures() == 0
    if mistake == "never_flips":
        monkeypatch.setitem(SETUP, "modes", (O.NOMINAL, O.NOMINAL, O.NOMINAL))
    else:
        f = 100.0 if mistake == "band_x100" else 0.01
        monkeypatch.setitem(SETUP, "bands", dict(fp_band=O.FP_BAND * f, phase_band=O.PHASE_BAND * f))
    assert _failures() >= 3, mistake
