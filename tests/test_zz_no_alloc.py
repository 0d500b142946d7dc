"""The allocation-free stage entry point, dp_solve_stage_static, called
through the C ABI for callers that may not allocate GPU memory (real-time
controller tasks, hosts that own every device allocation).

Its output must match the allocating entry point dp_solve_stage on the same
inputs, on two calls in a row (the second call runs on the working memory the
first one left behind).  This file is collected last on purpose: it must pass
both alone in a fresh process and after every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2104_01284_gb300 import problems as P
from tests._parity import RTOL, ATOL

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore")]

torch = pytest.importorskip("torch")


def _short_cycles(p, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    n = len(p.light_stage)
    cyc = rng.uniform(6.0, 14.0, n)
    return p.replace(cycle=cyc, red=cyc * rng.uniform(0.3, 0.6, n), offset=rng.uniform(0, 1, n) * cyc)


PROBLEMS = {
    # several SoC tiles and time warps with ragged tails; lights with short
    # cycles so arrival and departure rules are exercised
    "ragged": lambda: _short_cycles(P.config1(seed=41, n_stages=8, n_v=21, n_soc=19, n_t=45, n_te=11, n_tm=11,
                                              n_lights=3), 41),
    # every documented limit at once: 64 speeds, 64 SoC points, 255 times,
    # 32 x 32 x 2 = 2048 controls (126 torque classes)
    "limits": lambda: P.config1(seed=42, n_stages=6, n_v=64, n_soc=64, n_t=255, n_te=32, n_tm=32, n_lights=2),
    # the literal standstill step (light_model 2) with speed-dependent torque
    # limits (torque_limits 1)
    "variants": lambda: _short_cycles(P.config1(seed=43, n_stages=8, n_v=21, n_soc=19, n_t=45, n_te=9, n_tm=11,
                                                n_lights=3), 43).replace(
        light_model=2, torque_limits=1, te_max_coef=np.array([110.0, 0.9, -0.003]), bsg_power_max=6500.0),
}


def _same(a_v, a_pi, b_v, b_pi):
    a_v, b_v = a_v.cpu().numpy().astype(np.float64), b_v.cpu().numpy().astype(np.float64)
    fa, fb = np.isfinite(a_v), np.isfinite(b_v)
    assert np.array_equal(fa, fb)
    assert np.all(np.abs(a_v[fa] - b_v[fa]) <= RTOL * np.abs(b_v[fa]) + ATOL)
    assert torch.equal(a_pi, b_pi)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_static_stage_matches_allocating_stage_twice(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_01284_gb300.native as N
    from paper_2104_01284_gb300.solver import EcoDP, make_desc

    p = PROBLEMS[name]()
    dev = torch.device("cuda", 0)
    dp = EcoDP(p, device=dev)
    desc, keep = make_desc(p)
    stream = torch.cuda.current_stream(dev)
    calls = [(int(p.light_stage[0]) - 1, P.synthetic_value_field(p, seed=3)),   # arrival at a light
             (int(p.light_stage[0]), P.synthetic_value_field(p, seed=4))]       # departure (wait row)
    for k, vn in calls:
        v_next = torch.from_numpy(vn.astype(np.float32)).to(dev)
        v_out = torch.full(dp.shape, -1.0, dtype=torch.float32, device=dev)
        pi_out = torch.full(dp.shape, -7, dtype=torch.int16, device=dev)
        st = N.dp_solve_stage_static(C.byref(desc), k, v_next.data_ptr(), v_out.data_ptr(), pi_out.data_ptr(),
                                     stream.cuda_stream)
        N.check(st, "dp_solve_stage_static")
        ref_v, ref_pi = dp.solve_stage(k, v_next)
        torch.cuda.synchronize(dev)
        assert np.isfinite(v_out.cpu().numpy()).any()
        _same(v_out, pi_out, ref_v, ref_pi)
    dp.close()


def test_static_stage_rejects_oversized_problems():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_01284_gb300.native as N
    from paper_2104_01284_gb300.solver import make_desc

    p = P.config1(seed=1, n_stages=4, n_soc=80)
    desc, keep = make_desc(p)
    dummy = torch.zeros(8, device="cuda")
    st = N.dp_solve_stage_static(C.byref(desc), 0, dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    assert st == N.DP_ERR_INVALID_ARG
    assert b"dp_solve_stage" in N.lib.dp_last_error()
