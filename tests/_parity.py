"""Comparison of GPU results with the FP64 oracle (acceptance criteria).

The oracle runs each stage in three modes on the same J_{k+1}: nominal (every
decision at face value), lenient and strict (every FP32-fragile decision --
an arrival within 1e-4 s of a phase boundary, an interpolation fraction or a
grid-band edge within FP32 resolution of its threshold, a model threshold
within FP32 resolution -- taken the feasible / infeasible way).  The checks:

  (a) value: |J_gpu - J_nom| <= 1e-4 |J_nom| where the three modes agree;
      elsewhere J_lo (1 - 1e-4) <= J_gpu <= J_hi (1 + 1e-4);
  (b) mask: isfinite(J_gpu) == isfinite(J_nom) except on fragile states
      (feasible in lenient mode, infeasible in strict mode), which are
      counted and returned;
  (c) policy: pi_gpu == pi_nom where the oracle's second-best value exceeds
      the best by more than 1e-4 relative and the state is not fragile.
"""
from __future__ import annotations

import numpy as np

RTOL = 1e-4
ATOL = 1e-6


def compare(gpu_V, gpu_pi, nom, lo, hi, pi_nom=None, second=None, rtol=RTOL, atol=ATOL, where=""):
    gV = np.asarray(gpu_V, np.float64)
    nom = np.asarray(nom, np.float64)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    fg, fn, fl, fh = (np.isfinite(a) for a in (gV, nom, lo, hi))
    # (b) mask: a difference from nominal must lie inside the fragile interval
    diff = fg != fn
    excused = diff & (fg <= fl) & (fg >= fh)
    bad_mask = diff & ~excused
    assert not bad_mask.any(), (
        f"{where}: {int(bad_mask.sum())} unexcused mask flips, e.g. at "
        f"{np.argwhere(bad_mask)[:5].tolist()} gpu={gV[bad_mask][:5]} nom={nom[bad_mask][:5]}")
    # (a) values
    both = fg & fn
    with np.errstate(invalid="ignore"):
        tight = both & fl & fh & np.isclose(lo, nom, rtol=1e-9, atol=0) & np.isclose(hi, nom, rtol=1e-9, atol=0)
        err = np.abs(gV - nom)
        ok_tight = err <= rtol * np.abs(nom) + atol
        bad_v = tight & ~ok_tight
        assert not bad_v.any(), (
            f"{where}: {int(bad_v.sum())} value mismatches, worst rel "
            f"{float(np.max(err[bad_v] / np.abs(nom[bad_v])))} at {np.argwhere(bad_v)[:5].tolist()} "
            f"gpu={gV[bad_v][:5]} nom={nom[bad_v][:5]}")
        loose = fg & ~tight
        lo_b = np.where(fl, lo, -np.inf)
        hi_b = np.where(fh, hi, np.inf)
        bad_i = loose & ((gV < lo_b * (1 - rtol) - atol) | (gV > hi_b * (1 + rtol) + atol))
        assert not bad_i.any(), f"{where}: {int(bad_i.sum())} values outside the fragile interval"
    stats = dict(states=int(gV.size), feasible=int(fn.sum()), mask_exceptions=int(excused.sum()),
                 fragile=int((fg & ~tight).sum()), max_rel_err=float(np.max(err[tight] / np.abs(nom[tight])))
                 if tight.any() else 0.0)
    # (c) policy
    if gpu_pi is not None and pi_nom is not None and second is not None:
        gp = np.asarray(gpu_pi).astype(np.int64)
        pn = np.asarray(pi_nom).astype(np.int64)
        sec = np.asarray(second, np.float64)
        with np.errstate(invalid="ignore", divide="ignore"):
            gap = np.where(tight, (sec - nom) / np.abs(nom), 0.0)
        decisive = tight & (gap > 1e-4)
        bad_p = decisive & (gp != pn)
        assert not bad_p.any(), (
            f"{where}: {int(bad_p.sum())} policy mismatches at decisive states, e.g. "
            f"{np.argwhere(bad_p)[:5].tolist()} gpu={gp[bad_p][:5]} nom={pn[bad_p][:5]}")
        infeas_pi = ~fg & (gp != -1)
        assert not infeas_pi.any(), f"{where}: policy must be -1 on infeasible states"
        stats["decisive"] = int(decisive.sum())
        stats["policy_equal_all"] = float(np.mean(gp[tight] == pn[tight])) if tight.any() else 1.0
    return stats
