"""Comparison of GPU results with the FP64 oracle (acceptance criteria).

The oracle runs each stage in three modes on the same J_{k+1}: nominal (every
decision at face value), lenient and strict (every FP32-fragile decision --
an arrival within 1e-4 s of a phase boundary, an interpolation fraction or a
grid-band edge within FP32 resolution of its threshold, a model threshold
within FP32 resolution -- taken the feasible / infeasible way).  Per state
the two extra modes give an interval [lo, hi] around the nominal value that
a correct FP32 solver may land anywhere in.  The checks:

  (a) value: a feasible state is "tight" when its interval is no wider than
      half the tolerance, (hi - lo) <= 0.5e-4 |nom|; there
      |J_gpu - J_nom| <= 1e-4 |nom| (acceptance (a)).  The other feasible
      states are "loose": J_lo (1 - 1e-4) <= J_gpu <= J_hi (1 + 1e-4);
  (b) mask: isfinite(J_gpu) == isfinite(J_nom) except on fragile states
      (feasible in lenient mode, infeasible in strict mode), which are
      counted and returned;
  (c) policy: pi_gpu == pi_nom wherever the oracle's second-best value
      exceeds the best by more than 1e-4 relative and by more than the
      state's interval width (a decision no fragile flip can reverse).

Every call returns its counts (feasible, mask exceptions, loose, value- and
policy-checked states) and appends them to RECORDS, which the test session
prints as one summary line at its end.  Loose states and mask exceptions are
bounded per call (max_loose_frac, max_mask_frac of the feasible states).
"""
from __future__ import annotations

import numpy as np

RTOL = 1e-4
ATOL = 1e-6
# an interval up to this fraction of the tolerance counts as tight, so a GPU
# value anywhere inside it plus FP32 rounding stays within RTOL of nominal
TIGHT_FRAC = 0.5

RECORDS: list[dict] = []


def compare(gpu_V, gpu_pi, nom, lo, hi, pi_nom=None, second=None, rtol=RTOL, atol=ATOL, where="",
            max_loose_frac=0.15, max_mask_frac=0.02):
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
        width = np.where(fn & fl & fh, hi - lo, np.inf)
        tight = both & (width <= TIGHT_FRAC * rtol * np.abs(nom))
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
        assert not bad_i.any(), (
            f"{where}: {int(bad_i.sum())} values outside the fragile interval at "
            f"{np.argwhere(bad_i)[:5].tolist()} gpu={gV[bad_i][:5]} lo={lo[bad_i][:5]} hi={hi[bad_i][:5]}")
    n_feas = int(fn.sum())
    # relative error on the checked states with a nonzero oracle value (a zero
    # value is held to the absolute tolerance)
    nz = tight & (nom != 0)
    with np.errstate(invalid="ignore", divide="ignore"):
        max_rel = float(np.max(err[nz] / np.abs(nom[nz]))) if nz.any() else 0.0
    stats = dict(where=where, states=int(gV.size), feasible=n_feas, mask_exceptions=int(excused.sum()),
                 loose=int((fn & ~tight).sum()), value_checked=int(tight.sum()), max_rel_err=max_rel)
    # (c) policy
    if gpu_pi is not None and pi_nom is not None and second is not None:
        gp = np.asarray(gpu_pi).astype(np.int64)
        pn = np.asarray(pi_nom).astype(np.int64)
        sec = np.asarray(second, np.float64)
        with np.errstate(invalid="ignore", divide="ignore"):
            gap = np.where(fn, (sec - nom) / np.abs(nom), 0.0)
            decisive_all = fn & (gap > 1e-4)
            decisive = decisive_all & fg & (gap * np.abs(nom) > width)
        bad_p = decisive & (gp != pn)
        assert not bad_p.any(), (
            f"{where}: {int(bad_p.sum())} policy mismatches at decisive states, e.g. "
            f"{np.argwhere(bad_p)[:5].tolist()} gpu={gp[bad_p][:5]} nom={pn[bad_p][:5]}")
        infeas_pi = ~fg & (gp != -1)
        assert not infeas_pi.any(), f"{where}: policy must be -1 on infeasible states"
        stats["decisive"] = int(decisive_all.sum())
        stats["policy_checked"] = int(decisive.sum())
        stats["policy_equal_all"] = float(np.mean(gp[both] == pn[both])) if both.any() else 1.0
    RECORDS.append(stats)
    if n_feas:
        assert stats["loose"] <= max_loose_frac * n_feas, (
            f"{where}: {stats['loose']} of {n_feas} feasible states have a fragile interval wider "
            f"than the tolerance")
        assert stats["mask_exceptions"] <= max_mask_frac * n_feas + 1, (
            f"{where}: {stats['mask_exceptions']} excused mask flips among {n_feas} feasible states")
    return stats


def summary(records=None) -> str:
    """One line over all comparisons: totals of feasible, value-checked,
    loose, decisive and policy-checked states and mask exceptions, and the
    worst relative value error on checked states."""
    recs = RECORDS if records is None else records
    if not recs:
        return ""
    tot = {k: sum(r.get(k, 0) for r in recs) for k in
           ("feasible", "value_checked", "loose", "mask_exceptions", "decisive", "policy_checked")}
    worst = max(r["max_rel_err"] for r in recs)
    return (f"parity: {len(recs)} comparisons, feasible {tot['feasible']}, value-checked "
            f"{tot['value_checked']} ({tot['value_checked'] / max(1, tot['feasible']):.3f}), loose "
            f"{tot['loose']}, mask exceptions {tot['mask_exceptions']}, decisive {tot['decisive']}, "
            f"policy-checked {tot['policy_checked']} ({tot['policy_checked'] / max(1, tot['decisive']):.3f}), "
            f"max rel err {worst:.2e}")
