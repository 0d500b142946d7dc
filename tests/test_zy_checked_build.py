"""The bounds-checked build (libecodp_checked.so, -DECODP_CHECKS) on the GPU:
the tiny and reduced problems, the paper's Table I grid, two paper variants,
two grids large enough for the unsplit tiled kernel with corner quads, a
checkpointed adjoint and a 4-instance batch run through it in a child
process (the binding loads one library per process), and the device's
bounds-check record stays empty after every phase.  The checks change no
arithmetic: J_0 equals the production build's bit for bit."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore")]

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_records_no_bounds_failure():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_01284_gb300 import build
    build.build(checks=True)
    env = dict(os.environ, ECODP_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_checked_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(out["phases"]) >= 20 and "batch" in out["phases"] and "adjoint" in out["phases"]
    from paper_2104_01284_gb300 import problems as P
    from paper_2104_01284_gb300.solver import EcoDP
    from tests.test_gpu_parity import PROBLEMS
    dp = EcoDP(PROBLEMS["reduced"]())
    dp.solve()
    ref = dp.value(0).cpu().numpy().astype(np.float64)
    assert np.array_equal(np.asarray(out["digest"]["reduced"]), ref)
    dp.close()
    dp = EcoDP(P.config0())
    dp.solve()
    assert np.array_equal(np.asarray(out["digest"]["c0"]), dp.value(0).cpu().numpy().astype(np.float64))
    dp.close()
    from tests._checked_run import UNSPLIT, j0_hash
    for name, p in UNSPLIT.items():
        dp = EcoDP(p)
        dp.solve()
        assert out["hashes"][name] == j0_hash(dp), name
        dp.close()
