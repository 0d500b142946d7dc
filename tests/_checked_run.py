"""Runs the solver's paths through the bounds-checked library (started by
tests/test_zy_checked_build.py with ECODP_LIBRARY=checked): after every
phase the device's bounds-check record must be empty.  Prints one JSON line
with the phases run and, per problem, a digest of J_0 for the caller to
compare with the production library."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import paper_2104_01284_gb300.native as N  # noqa: E402
from paper_2104_01284_gb300 import problems as P  # noqa: E402
from paper_2104_01284_gb300.solver import EcoDP, EcoDPBatch  # noqa: E402
from tests.test_gpu_parity import PROBLEMS  # noqa: E402
from tests.test_gpu_variants import VARIANTS  # noqa: E402


UNSPLIT = {
    "unsplit": P.config1(seed=77, n_stages=6, n_v=31, n_soc=51, n_t=201, n_te=11, n_tm=11, n_lights=2, t_hi=60.0),
    "unsplit_t101": P.config1(seed=77, n_stages=6, n_v=51, n_soc=51, n_t=101, n_te=11, n_tm=11, n_lights=2,
                              t_hi=60.0),
}


def j0_hash(dp):
    import hashlib
    return hashlib.sha1(dp.value(0).cpu().numpy().astype(np.float32).tobytes()).hexdigest()


def clean(phase, done):
    en, site = N.debug_checks()
    assert en, "the checked library is not loaded"
    assert site == 0, f"{phase}: bounds check failed: {N.lib.dp_last_error().decode()}"
    done.append(phase)


def main():
    assert N.CHECKED and N.LIB_PATH.endswith("libecodp_checked.so")
    done, digest = [], {}
    probs = {"c0": P.config0(), "reduced": PROBLEMS["reduced"](), "wide_shift": PROBLEMS["wide_shift"](),
             "paper_grid": P.paper_table1(), "literal": VARIANTS["literal"](), "both": VARIANTS["both"]()}
    # grids with enough tiles for the unsplit tiled kernel and its corner
    # quads (row strides 256 and 128); J_0 reported as a hash
    probs.update(UNSPLIT)
    hashes = {}
    for name, p in probs.items():
        for variant in ("tiled", "direct"):
            dp = EcoDP(p)
            dp.set_variant(variant)
            dp.solve()
            clean(f"{name}/{variant}/sweep", done)
            if variant == "tiled" and name in UNSPLIT:
                hashes[name] = j0_hash(dp)
            elif variant == "tiled":
                digest[name] = np.asarray(dp.value(0).cpu().numpy(), np.float64).tolist()
                dp.rollout(raise_infeasible=False)
                clean(f"{name}/rollout", done)
                vn = torch.from_numpy(P.synthetic_value_field(p, seed=5).astype(np.float32)).cuda()
                dp.solve_stage(p.n_stages - 1, vn)
                clean(f"{name}/stage", done)
            dp.close()
    # adjoint with checkpointing on a small problem
    p = P.config1(seed=101, n_stages=8, n_v=15, n_soc=13, n_t=33, n_te=7, n_tm=7, n_lights=1, t_hi=16.0)
    dp = EcoDP(p)
    dp.set_checkpointing(3)
    dp.solve()
    dp.adjoint((10.0, 0.55, 0.0))
    clean("adjoint", done)
    dp.close()
    # the allocation-free stage on the reduced problem
    import ctypes as C
    from paper_2104_01284_gb300.solver import make_desc
    p = probs["reduced"]
    desc, keep = make_desc(p)
    vn = torch.from_numpy(P.synthetic_value_field(p, seed=6).astype(np.float32)).cuda()
    v_out = torch.empty_like(vn)
    pi_out = torch.empty(vn.shape, dtype=torch.int16, device="cuda")
    N.check(N.dp_solve_stage_static(C.byref(desc), int(p.light_stage[0]), vn.data_ptr(), v_out.data_ptr(),
                                    pi_out.data_ptr(), torch.cuda.current_stream().cuda_stream),
            "dp_solve_stage_static")
    clean("static_stage", done)
    # three fleet-shaped requests through the serving loop
    from paper_2104_01284_gb300.serving import EcoDPServer
    from tests.test_gpu_serving import fleet_requests_with_lights, serve_all
    with EcoDPServer(max_slots=2) as srv:
        serve_all(srv, fleet_requests_with_lights(3))
    clean("serving", done)
    # a 4-instance uneven batch in one persistent launch, and its rollouts
    with EcoDPBatch(P.config3_small(seed=34, n_instances=4)) as bt:
        bt.solve()
        bt.wait()
        bt.rollout(raise_infeasible=False)
        clean("batch", done)
        bt.set_streams(2)  # the per-instance mode: single-problem graphs on 2 streams
        bt.solve()
        bt.wait()
        bt.rollout(raise_infeasible=False)
        clean("batch_streams", done)
    print(json.dumps({"phases": done, "digest": digest, "hashes": hashes}))


if __name__ == "__main__":
    main()
