"""Value-function checkpointing (dp_set_checkpointing): with J_k kept only
every K stages, the rollout, the adjoint and every stage's value (recomputed
segment by segment) equal those of the default full storage (needs a GB300)."""
import numpy as np
import pytest

from paper_2104_01284_gb300 import problems as P

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore")]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_01284_gb300 import solver as S
    return S


def reduced(seed=41):
    p = P.config1(seed=seed, n_stages=12, n_v=21, n_soc=19, n_t=45, n_te=11, n_tm=11, n_lights=3)
    rng = np.random.Generator(np.random.PCG64(seed + 500))
    n = len(p.light_stage)
    cyc = rng.uniform(6.0, 14.0, n)
    return p.replace(cycle=cyc, red=cyc * rng.uniform(0.3, 0.6, n), offset=rng.uniform(0, 1, n) * cyc,
                     x0=(8.0, 0.6, 0.0))


def bits(t):
    return t.cpu().numpy().view(np.uint32)


def full_reference(S, p):
    dp = S.EcoDP(p)
    dp.solve()
    ref = dict(V=[bits(dp.value(k)) for k in range(p.n_stages + 1)],
               pi=[dp.policy(k).cpu().numpy() for k in range(p.n_stages)],
               roll=dp.rollout(raise_infeasible=False), adj=dp.adjoint())
    dp.close()
    return ref


@pytest.mark.parametrize("K", [2, 3, 5, 12])
def test_checkpointed_equals_full(solver, K):
    p = reduced()
    ref = full_reference(solver, p)
    dp = solver.EcoDP(p)
    dp.set_checkpointing(K)
    dp.solve()
    r = dp.rollout(raise_infeasible=False)
    for key in ("v", "soc", "t", "u", "dt", "wait", "fuel"):
        assert np.array_equal(r[key], ref["roll"][key], equal_nan=r[key].dtype.kind == "f"), key
    assert r["fuel_g"] == ref["roll"]["fuel_g"] or (np.isnan(r["fuel_g"]) and np.isnan(ref["roll"]["fuel_g"]))
    if ref["roll"]["fail_stage"] < 0:
        J, g = dp.adjoint()
        assert J == ref["adj"][0]
        np.testing.assert_allclose(g, ref["adj"][1], rtol=1e-12, atol=0)
    for k in range(p.n_stages, -1, -1):  # every stage, stored or recomputed
        assert np.array_equal(bits(dp.value(k)), ref["V"][k]), f"K={K} stage {k}"
    for k in range(p.n_stages):
        assert np.array_equal(dp.policy(k).cpu().numpy(), ref["pi"][k])
    dp.set_checkpointing(0)  # back to full storage: unsolved until the next solve
    import paper_2104_01284_gb300.native as N
    with pytest.raises(N.DPError) as e:
        dp.value(0)
    assert e.value.status == N.DP_ERR_NOT_SOLVED
    dp.solve()
    assert np.array_equal(bits(dp.value(1)), ref["V"][1])
    dp.close()


def test_paper_scale_checkpoint_every_10(solver):
    """The adjoint configuration: the paper-scale problem with J_k kept
    every 10 stages, through the autograd function."""
    p = P.config1(seed=1)
    ref = full_reference(solver, p)
    theta = torch.tensor([getattr(p, n) for n in solver.THETA], dtype=torch.float64, requires_grad=True)
    J = solver.EcoDPValue.apply(theta, p, None, None, 10)
    J.backward()
    assert float(J) == ref["adj"][0]
    np.testing.assert_allclose(theta.grad.numpy(), ref["adj"][1], rtol=1e-10, atol=0)
    dp = solver._solver_for(p, torch.device("cuda", torch.cuda.current_device()), 10)
    assert dp.checkpoint_every == 10
    dp.solve()  # the cached solver was re-loaded (update) by the lookup
    r = dp.rollout()
    assert r["fuel_g"] == ref["roll"]["fuel_g"] and r["J"] == ref["roll"]["J"]
