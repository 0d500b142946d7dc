"""Degenerate and extreme sizes on the GPU against the FP64 oracle (needs a
GB300): one stage, two-point grids on every axis, a single control, no
lights, fewer SoC points than rows per lane, a long time axis (2048 points)
and the largest control set the tiled path takes (8192 controls).  Each runs
the end-to-end comparison of tests/_parity.py, the tiled and direct kernels
bit for bit, and the rollout.  On grids of a few states the bounds on loose
states and excused mask flips (fractions of the feasible states) mean
nothing, so they are lifted there; the interval and value checks stay."""
import numpy as np
import pytest

import oracle as O
from paper_2104_01284_gb300 import problems as P
from tests._parity import compare
from tests.test_gpu_parity import feasible_start

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore")]

torch = pytest.importorskip("torch")

NO_LIGHTS = dict(light_stage=np.zeros(0, np.int32), cycle=np.zeros(0), red=np.zeros(0), offset=np.zeros(0))


def case(name):
    if name == "one_stage":
        return P.config1(seed=61, n_stages=1, n_v=6, n_soc=5, n_t=7, n_te=5, n_tm=5).replace(
            grade=np.array([0.01]), t_hi=4.0, **NO_LIGHTS)
    if name == "two_point_grids":
        return P.config1(seed=62, n_stages=3, n_v=2, n_soc=2, n_t=2, n_te=3, n_tm=3, n_lights=0, t_hi=40.0)
    if name == "single_control":
        te = (1600 * 9.81 * 0.01 + 0.5 * 1.2 * 0.7 * 100.0) * 0.3 / 3.0  # holds 10 m/s on a flat road
        return P.config0().replace(grade=np.zeros(10), te_lo=te, te_hi=te, n_te=1, tm_lo=0.0, tm_hi=0.0, n_tm=1,
                                   n_brake=1, x0=(10.0, 0.55, 0.0), t_hi=20.0, n_t=21, **NO_LIGHTS)
    if name == "few_soc_points":
        return P.config1(seed=63, n_stages=6, n_v=9, n_soc=3, n_t=37, n_te=7, n_tm=7, n_lights=2)
    if name == "long_time_axis":
        return P.config1(seed=64, n_stages=4, n_v=5, n_soc=4, n_t=2048, n_te=5, n_tm=5, n_lights=1, t_hi=12.0)
    if name == "max_controls":
        return P.config1(seed=65, n_stages=3, n_v=11, n_soc=5, n_t=17, n_te=64, n_tm=64, n_lights=1, t_hi=16.0)
    raise KeyError(name)


CASES = ["one_stage", "two_point_grids", "single_control", "few_soc_points", "long_time_axis", "max_controls"]
LIFTED = dict(max_loose_frac=1.0, max_mask_frac=1.0)


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_01284_gb300.solver import EcoDP
    return EcoDP


@pytest.mark.parametrize("name", CASES)
def test_edge_case_end_to_end(solver, name):
    p = case(name)
    op = O.make(p)
    Vn, pin, secn = O.solve(op, O.NOMINAL)
    Vl, _, _ = O.solve(op, O.LENIENT)
    Vh, _, _ = O.solve(op, O.STRICT)
    a, b = solver(p), solver(p)
    b.set_variant("direct")
    a.solve()
    b.solve()
    feasible = 0
    for k in range(p.n_stages, -1, -1):
        gV, gb = a.value(k), b.value(k)
        assert torch.equal(gV, gb), (name, k)
        gp = a.policy(k) if k < p.n_stages else None
        if gp is not None:
            assert torch.equal(gp, b.policy(k)), (name, k)
        st = compare(gV.cpu().numpy(), gp.cpu().numpy() if gp is not None else None, Vn[k], Vl[k], Vh[k],
                     pin[k] if k < p.n_stages else None, secn[k] if k < p.n_stages else None,
                     where=f"edge/{name}/k{k}", **LIFTED)
        feasible += st["feasible"]
    assert feasible > 0
    ok0 = np.isfinite(Vn[0]) & np.isfinite(Vl[0]) & np.isfinite(Vh[0])
    if ok0.any():
        x0 = feasible_start(p, Vn[0], Vl[0], Vh[0])
        ro = O.rollout(op, Vn, x0)
        rg = a.rollout(x0=x0, raise_infeasible=False)
        assert ro["status"] == 0 and rg["status"] == 0
        assert rg["fuel_g"] == pytest.approx(ro["fuel_g"], rel=1e-3, abs=1e-6)
        assert rg["J"] == pytest.approx(ro["J"], rel=1e-3)
    a.close()
    b.close()


def test_fp32_peak_probe_near_the_unit_count_peak():
    """The library's FP32 FMA throughput probe lands near the unit-count peak
    the Bellman roofline is quoted against (SMs x 128 lanes x 2 FLOP x SM
    clock, the clock at most 2.1 GHz), and rejects bad arguments."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes as C
    from paper_2104_01284_gb300 import native as N
    tf, ms = N.measure_fp32_peak(5)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    top = sms * 128 * 2 * 2.1e9 / 1e12
    assert 0.5 * top < tf < 1.05 * top, (tf, top)
    assert ms > 0
    x = C.c_double(0.0)
    assert N.dp_measure_fp32_peak(0, C.byref(x), C.byref(x), None) == N.DP_ERR_INVALID_ARG


def test_onchip_bandwidth_probes_within_the_load_path_limits():
    """The shared-memory, L1 and L2 load bandwidth probes report rates below
    the load path's limit (128 bytes per SM per clock, the clock at most
    2.1 GHz) and well above the HBM copy rate (a probe whose loads missed
    their level would fall to HBM speed); L2 is the slowest of the three.
    Bad arguments are rejected."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes as C
    from paper_2104_01284_gb300 import native as N
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    top = sms * 128 * 2.1e9 / 1e9  # GB/s
    r = {k: N.measure_onchip_bw(k, 3)[0] for k in ("smem", "l1", "l2")}
    assert 0.3 * top < r["smem"] < 1.05 * top, (r, top)
    assert 0.2 * top < r["l1"] < 1.05 * top, (r, top)
    assert 9000.0 < r["l2"] < min(r["smem"], r["l1"]), r
    x = C.c_double(0.0)
    assert N.dp_measure_onchip_bw(3, 1, C.byref(x), C.byref(x), None) == N.DP_ERR_INVALID_ARG
    assert N.dp_measure_onchip_bw(0, 0, C.byref(x), C.byref(x), None) == N.DP_ERR_INVALID_ARG
