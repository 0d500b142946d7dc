"""GPU parity of the paper variants with the FP64 oracle, through the C ABI
(needs a GB300): speed-dependent torque limits (Eq. 7e, 7f), the green
indicator sampled on the time grid (Sec. III, Eq. 8), alone and together, and
the literal standstill step of Eq. 5c;
stage-local and end-to-end with the acceptance criteria of tests/_parity.py,
tiled and direct kernels bit-identical, and variant instances inside a batch
equal to their single solves."""
import numpy as np
import pytest

import oracle as O
from tests._parity import compare
from tests.test_gpu_parity import feasible_start, oracle_stage3, reduced, stage_inputs, stages_of_interest

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore")]

torch = pytest.importorskip("torch")

LIMITS = dict(torque_limits=1, te_max_coef=np.array([110.0, 0.9, -0.003]), bsg_power_max=6000.0)

# The "limits" instance puts the BSG power cap exactly on a grid product
# (80 Nm x 75 rad/s = 6000 W at v = 7.5 m/s), so every decision of that speed
# row sits on its threshold: the oracle counts it as fragile, and the
# lenient/strict intervals of the states that reach the row widen backward
# through the sweep.  Its comparisons keep the interval check but lift the
# bounds on loose states and excused mask flips.
BOUNDS = {"limits": dict(max_loose_frac=1.0, max_mask_frac=0.05)}

VARIANTS = {
    "limits": lambda: reduced(seed=51).replace(**LIMITS),
    "sampled": lambda: reduced(seed=52).replace(light_model=1),
    "both": lambda: reduced(seed=53, n_te=7, n_tm=9).replace(light_model=1, **LIMITS),
    "literal": lambda: reduced(seed=55).replace(light_model=2),
}


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_01284_gb300 import solver as S
    return S


@pytest.mark.parametrize("kernel", ["tiled", "direct"])
@pytest.mark.parametrize("name", list(VARIANTS))
def test_variant_stage_local_parity(solver, name, kernel):
    p = VARIANTS[name]()
    op = O.make(p)
    dp = solver.EcoDP(p)
    dp.set_variant(kernel)
    for k in stages_of_interest(p):
        for label, Vn in stage_inputs(p, op, k):
            nom, lo, hi = oracle_stage3(op, k, Vn)
            gV, gpi = dp.solve_stage(k, torch.from_numpy(Vn.astype(np.float32)))
            st = compare(gV.cpu().numpy(), gpi.cpu().numpy(), nom["V"], lo, hi, nom["pi"], nom["second"],
                         where=f"{name}/{kernel}/k{k}/{label}", **BOUNDS.get(name, {}))
            assert st["feasible"] > 0
    dp.close()


@pytest.mark.parametrize("name", list(VARIANTS))
def test_variant_end_to_end_parity(solver, name):
    p = VARIANTS[name]()
    op = O.make(p)
    Vn, pin, secn = O.solve(op, O.NOMINAL)
    Vl, _, _ = O.solve(op, O.LENIENT)
    Vh, _, _ = O.solve(op, O.STRICT)
    a, b = solver.EcoDP(p), solver.EcoDP(p)
    b.set_variant("direct")
    a.solve()
    b.solve()
    others = []
    for variant in ("tiled8", "tiled6"):  # both row counts, whichever the default picks
        c = solver.EcoDP(p)
        c.set_variant(variant)
        c.solve()
        others.append(c)
    for k in range(p.n_stages, -1, -1):
        gV = a.value(k)
        gp = a.policy(k) if k < p.n_stages else None
        assert torch.equal(gV, b.value(k)) and all(torch.equal(gV, c.value(k)) for c in others)
        if gp is not None:
            assert torch.equal(gp, b.policy(k)) and all(torch.equal(gp, c.policy(k)) for c in others)
        compare(gV.cpu().numpy(), gp.cpu().numpy() if gp is not None else None, Vn[k], Vl[k], Vh[k],
                pin[k] if k < p.n_stages else None, secn[k] if k < p.n_stages else None, where=f"{name}/k{k}",
                **BOUNDS.get(name, {}))
    x0 = feasible_start(p, Vn[0], Vl[0], Vh[0])
    ro = O.rollout(op, Vn, x0)
    rg = a.rollout(x0=x0, raise_infeasible=False)
    assert ro["status"] == 0 and rg["status"] == 0
    assert rg["fuel_g"] == pytest.approx(ro["fuel_g"], rel=1e-3, abs=1e-6)
    assert rg["J"] == pytest.approx(ro["J"], rel=1e-3)
    a.close()
    b.close()
    for c in others:
        c.close()


def test_sampled_indicator_masks_red_nodes_on_gpu(solver):
    p = VARIANTS["sampled"]()
    op = O.make(p)
    dp = solver.EcoDP(p)
    dp.solve()
    for j, node in enumerate(p.light_stage):
        red = np.array([O.is_red(op, j, t) for t in p.nodes("t")])
        V = dp.value(int(node)).cpu().numpy()
        assert np.all(np.isinf(V[1:, :, red]))
        assert np.all(dp.policy(int(node)).cpu().numpy()[1:, :, red] == -1)
    dp.close()


def test_variants_in_a_batch_equal_alone(solver):
    probs = [VARIANTS[n]() for n in VARIANTS] + [reduced(seed=54)]
    with solver.EcoDPBatch(probs) as bt:
        bt.solve()
        for b, p in enumerate(probs):
            dp = solver.EcoDP(p)
            dp.solve()
            for k in range(p.n_stages + 1):
                assert torch.equal(bt.value(b, k), dp.value(k)), (b, k)
                if k < p.n_stages:
                    assert torch.equal(bt.policy(b, k), dp.policy(k)), (b, k)
            dp.close()
