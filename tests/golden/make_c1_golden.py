"""Write the FP64 oracle's reference results for the paper-scale instance.

Calls only the oracle and the seeded problem generator.  A full backward
sweep of the 100-stage, 51 x 51 x 201-state, 1922-control instance is about
1e11 state-control evaluations (tens of CPU-core-hours), far too slow for a
test, so its results are stored compactly in ``c1_s<seed>.npz``:

  mask_{mode}_k{k}   packed bits of isfinite(J_k) on the full grid
  idx_k{k}           sampled flat state indices (seeded)
  V_{mode}_k{k}      J_k at the sampled states
  pi_k{k}, sec_k{k}  nominal argmin and second-best value at the samples
  roll_*             the nominal forward rollout from x0

for modes nominal / lenient / strict and stages k in STAGES.

Usage: python tests/golden/make_c1_golden.py [seed] [nthreads]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2104_01284_gb300 import problems as P  # noqa: E402

STAGES = (0, 50, 99)
N_SAMPLE = 8000
MODES = {"nom": O.NOMINAL, "lo": O.LENIENT, "hi": O.STRICT}


def main(seed: int = 1, nthreads: int = 0):
    p = P.config1(seed=seed)
    op = O.make(p)
    out = dict(seed=np.int64(seed), shape=np.array(op.shapes[0]), stages=np.array(STAGES))
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    for k in STAGES:
        out[f"idx_k{k}"] = np.sort(rng.choice(p.n_states, size=N_SAMPLE, replace=False)).astype(np.int64)
    for name, mode in MODES.items():
        t0 = time.time()
        Vs, pis, secs = O.solve(op, mode, nthreads=nthreads)
        print(f"mode {name}: {time.time() - t0:.0f} s", flush=True)
        for k in STAGES:
            idx = out[f"idx_k{k}"]
            out[f"mask_{name}_k{k}"] = np.packbits(np.isfinite(Vs[k]).ravel())
            out[f"V_{name}_k{k}"] = Vs[k].ravel()[idx].copy()
            if name == "nom":
                out[f"pi_k{k}"] = pis[k].ravel()[idx].copy()
                out[f"sec_k{k}"] = secs[k].ravel()[idx].copy()
        if name == "nom":
            r = O.rollout(op, Vs)
            for key in ("traj", "u", "dt", "wait", "fuel", "cost", "gap"):
                out[f"roll_{key}"] = np.asarray(r[key])
            for key in ("fuel_g", "time_s", "J", "status", "fail_stage"):
                out[f"roll_{key}"] = np.array(r[key])
            print("rollout", r["status"], r["fuel_g"], r["time_s"], r["J"], flush=True)
        del Vs, pis, secs
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"c1_s{seed}.npz")
    np.savez_compressed(path, **out)
    print("wrote", path, os.path.getsize(path), "bytes")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 1, int(sys.argv[2]) if len(sys.argv) > 2 else 0)
