"""Write FP64 central finite differences of the optimal cost for mid-size
instances of the paper-scale family, for the adjoint acceptance test.

Calls only the oracle and the seeded problem generator.  Instances are
config-1 problems shrunk to 20 stages x 31 x 31 x 81 states x 11 x 11 x 2
controls with 2 lights; x0 = (10 m/s, 0.55, 0 s).  Seeds from 100 upward; per
seed s the oracle sweeps the problem at theta and at theta +- h for each
component (h = 1e-4 |theta|, theta = mass, CdA, Crr, R0, fuel scale) and
stores:

  fd_s<s>      (J_0(x0; theta + h) - J_0(x0; theta - h)) / (2 h) per component
  grad_s<s>    the oracle's adjoint at theta
  J0_s<s>      J_0(x0; theta)
  diag_s<s>    [status, support size, snapped, infeasible corner, min gap,
                snapped lambda mass, largest lambda mass whose argmin differs
                at theta +- h (over components), lambda mass on states with a
                gap of at most 1e-5]

A seed is stable when x0 is feasible, no infeasible corner or snapped
fraction is on the support, and both masses are at most STABLE_MASS (of 20,
one per stage): then the finite difference measures the derivative the
adjoint computes, and an FP32 solver takes the support's decisions as the
oracle does.  The scan stops after N_STABLE stable seeds or MAX_SEEDS seeds.

Usage: python tests/golden/make_adjoint_fd.py [nthreads]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2104_01284_gb300 import problems as P  # noqa: E402

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint_fd_mid.npz")
SIZE = dict(n_stages=20, n_v=31, n_soc=31, n_t=81, n_te=11, n_tm=11, n_lights=2)
X0 = (10.0, 0.55, 0.0)
STABLE_MASS = 1e-3
N_STABLE = 20
MAX_SEEDS = 120


def problem(seed):
    return P.config1(seed=seed, **SIZE)


def stable(diag) -> bool:
    status, _, snapped, corner, _, snap_mass, switch_mass, tie_mass = diag
    return (status == 0 and corner == 0 and snap_mass == 0 and switch_mass <= STABLE_MASS
            and tie_mass <= STABLE_MASS)


def main(nthreads: int = 0):
    out = dict(np.load(PATH)) if os.path.exists(PATH) else {}
    out["size"] = np.array([SIZE[k] for k in ("n_stages", "n_v", "n_soc", "n_t", "n_te", "n_tm", "n_lights")])
    n_stable = sum(stable(out[k]) for k in out if k.startswith("diag_s"))
    for seed in range(100, 100 + MAX_SEEDS):
        if n_stable >= N_STABLE:
            break
        if f"diag_s{seed}" in out:
            continue
        t0 = time.time()
        p = problem(seed)
        op = O.make(p)
        Vs, _, _ = O.solve(op, nthreads=nthreads)
        g, d, _, rc = O.adjoint(op, X0, want_lam=True)
        diag = [rc, d["support_size"], d["snapped"], d["infeasible_corner"], d["min_gap"], d["snapped_mass"]]
        fd = np.full(5, np.nan)
        switch = np.inf
        tie = np.inf
        if rc == 0 and not d["infeasible_corner"] and d["snapped_mass"] == 0:
            n = p.n_states * p.n_stages
            lam = d["lam"][:n]
            on = lam > 0
            with np.errstate(invalid="ignore", divide="ignore"):
                gap = (op._secall[:n] - op._Vall[:n]) / np.abs(op._Vall[:n])
            tie = float(lam[on & ~(gap > 1e-5)].sum())
            pi0 = op._piall[:n].copy()
            switch = 0.0
            for q, name in enumerate(O.THETA):
                th = getattr(p, name)
                h = 1e-4 * abs(th)
                vals = []
                for sgn in (+1, -1):
                    oo = O.make(p.replace(**{name: th + sgn * h}))
                    Vq, _, _ = O.solve(oo, nthreads=nthreads)
                    vals.append(O.interp(oo, 0, Vq[0], *X0))
                    switch = max(switch, float(lam[on & (oo._piall[:n] != pi0)].sum()))
                    del Vq
                fd[q] = (vals[0] - vals[1]) / (2 * h)
        diag += [switch, tie]
        out[f"diag_s{seed}"] = np.array(diag, np.float64)
        out[f"fd_s{seed}"] = fd
        out[f"grad_s{seed}"] = g
        out[f"J0_s{seed}"] = np.float64(O.interp(op, 0, Vs[0], *X0))
        ok = stable(out[f"diag_s{seed}"])
        n_stable += ok
        print(f"seed {seed}: {time.time() - t0:.0f} s, stable {ok}, diag {diag}", flush=True)
        np.savez_compressed(PATH + ".tmp.npz", **out)
        os.replace(PATH + ".tmp.npz", PATH)
    print("wrote", PATH, n_stable, "stable", flush=True)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 0)
