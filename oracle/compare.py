"""Element-by-element comparison of the CUDA path's simulation outputs with the FP64
oracle's (TEST INFRASTRUCTURE ONLY: used by the GPU parity tests and by the
``cpu_baseline`` leg of ``bench.py``, which states the error of every benchmarked
result against the oracle).

Tolerances (the benchmark statement's, with one reading where it is silent):
* default steps of eq. (e:tau) bit-exact, except draws whose exponential clock lies
  within 1e-6 Lambda of the integrated intensity at a date where the two sides
  decide differently ("ties"), at most 1e-4 of all draws;
* per-path averaged targets of eq. (eq:CVA_portfolio) within 1e-4 relative, with an
  absolute floor of 1e-4 CVA_0 (a netted exposure close to zero has no relative
  accuracy in FP32; the floor ties the error to the scale of the problem);
* CVA_0 within 1e-5 relative.

Where a tie moves a draw's default step, the two sides take different, equally
valid decisions. The comparison then rebuilds the oracle's targets with the GPU's
default step on exactly those draws (the oracle's own exposures and discount
integrals at the GPU's step), so that every path and CVA_0 are still compared at
the full tolerance.
"""
from __future__ import annotations

from typing import Dict

import numpy as np

TIE_REL = 1e-6
TIE_MAX_SHARE = 1e-4
XI_RTOL = 1e-4
XI_FLOOR_CVA0 = 1e-4
CVA0_RTOL = 1e-5


def default_mismatches(idx_gpu, idx_or, Lam_or, eps, n) -> Dict[str, object]:
    """idx_* [M, N, C] default steps (n+1 = no default by t_n); Lam_or [n+1, C, M] the
    oracle's integrated intensities; eps [M, N, C] the exponential clocks. Returns
      mism       bool [M, N, C], the draws where the steps differ;
      n_mism     their number;
      n_tie      the number of draws whose clock is within the tie band of Lambda at
                 one of the oracle's two boundary dates (an upper bound of n_mism
                 when every mismatch is a tie);
      outside    the mismatches that are not ties: a step moved across a date whose
                 Lambda is not within the band of the clock (must be empty)."""
    idx_gpu = idx_gpu.astype(np.int64)
    idx_or = idx_or.astype(np.int64)
    mism = idx_gpu != idx_or
    Lam = np.transpose(Lam_or, (2, 1, 0))            # [M, C, n+1]
    outside = []
    for k, l, c in zip(*np.nonzero(mism)):
        lo, hi = sorted((int(idx_gpu[k, l, c]), int(idx_or[k, l, c])))
        e = eps[k, l, c]
        # every date the step moved across decides the comparison Lambda_j >= eps
        # differently on the two sides: each must be within the band
        crossed = range(max(lo, 1), min(hi, n + 1))
        if lo < 1 or not all(abs(Lam[k, c, j] - e) < TIE_REL * Lam[k, c, j] for j in crossed):
            outside.append((int(k), int(l), int(c), int(idx_gpu[k, l, c]), int(idx_or[k, l, c])))
    j_hi = np.minimum(idx_or, n)
    j_lo = np.maximum(idx_or - 1, 1)
    lam_hi = np.take_along_axis(Lam, np.transpose(j_hi, (0, 2, 1)), axis=2).transpose(0, 2, 1)
    lam_lo = np.take_along_axis(Lam, np.transpose(j_lo, (0, 2, 1)), axis=2).transpose(0, 2, 1)
    tie = (np.abs(lam_hi - eps) < TIE_REL * lam_hi) | (np.abs(lam_lo - eps) < TIE_REL * lam_lo)
    return {"mism": mism, "n_mism": int(mism.sum()), "n_tie": int(tie.sum()), "outside": outside,
            "draws": int(idx_or.size)}


def exposures(o: Dict[str, np.ndarray], recovery) -> np.ndarray:
    """The oracle's discounted exposure (1 - R_c) e^{-I0_j} MtM_c(t_j)^+, [n+1, C, M]."""
    return (1.0 - np.asarray(recovery, dtype=np.float64))[None, :, None] * np.exp(-o["I0"])[:, None, :] \
        * np.maximum(o["mtm"], 0.0)


def tie_corrected_targets(o: Dict[str, np.ndarray], recovery, idx_gpu, mism) -> np.ndarray:
    """The oracle's averaged targets xi_bar [n, M] with the GPU's default step on the
    mismatched draws: for each such draw (k, l, c) and date i,
      xi_bar_i^k += e^{I0_i} (1{i < j_gpu <= n} V_c(j_gpu) - 1{i < j_or <= n} V_c(j_or)) / N
    with V the oracle's exposures. Needs o["xi_bar"], o["mtm"], o["I0"], o["idx"]."""
    xi = np.array(o["xi_bar"], dtype=np.float64, copy=True)
    n, M = xi.shape
    N = o["idx"].shape[1]
    if not np.any(mism):
        return xi
    V = exposures(o, recovery)
    dates = np.arange(n)
    for k, l, c in zip(*np.nonzero(mism)):
        jg, jo = int(idx_gpu[k, l, c]), int(o["idx"][k, l, c])
        vg = V[jg, c, k] if jg <= n else 0.0
        vo = V[jo, c, k] if jo <= n else 0.0
        xi[:, k] += np.exp(o["I0"][:n, k]) * (np.where(dates < jg, vg, 0.0) - np.where(dates < jo, vo, 0.0)) / N
    return xi


def target_errors(xi_gpu, xi_ref, cva0) -> Dict[str, float]:
    """Errors of the per-path targets xi_gpu [n, M] against xi_ref [n, M]:
      worst_vs_tolerance  max |err| / (XI_RTOL |ref| + XI_FLOOR_CVA0 CVA_0)  (<= 1 passes);
      max_rel_above_floor the largest relative error among targets above the floor;
      max_abs_over_cva0   the largest absolute error in units of CVA_0."""
    a = np.asarray(xi_gpu, dtype=np.float64)
    b = np.asarray(xi_ref, dtype=np.float64)
    err = np.abs(a - b)
    bound = XI_RTOL * np.abs(b) + XI_FLOOR_CVA0 * cva0
    big = np.abs(b) > XI_FLOOR_CVA0 * cva0 / XI_RTOL
    return {"worst_vs_tolerance": float(np.max(err / np.maximum(bound, 1e-300))) if err.size else 0.0,
            "max_rel_above_floor": float(np.max(err[big] / np.abs(b[big]))) if np.any(big) else 0.0,
            "max_abs_over_cva0": float(np.max(err) / cva0) if err.size and cva0 > 0 else 0.0}
