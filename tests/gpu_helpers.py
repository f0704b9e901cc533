"""Shared comparison logic of the GPU parity tests (CPU-side numpy only)."""
import numpy as np

# Tolerances. Default-step indices: bit-exact except draws whose clock sits within
# 1e-6 * Lambda of the integrated intensity at the boundary where the two sides
# decide differently ("ties"), at most 1e-4 of all draws. Per-path targets:
# 1e-4 relative, with an absolute floor of 1e-4 CVA_0 for targets near zero (a
# netted exposure close to zero has no relative accuracy in FP32; the floor ties
# the error to the scale of the problem). CVA_0: 1e-5 relative.
TIE_REL = 1e-6
TIE_MAX_SHARE = 1e-4
XI_RTOL = 1e-4
XI_FLOOR_CVA0 = 1e-4
CVA0_RTOL = 1e-5


def compare_defaults(idx_gpu, idx_or, Lam_or, eps, n):
    """idx_* [M, N, C]; Lam_or [n+1, C, M]; eps [M, N, C]. Returns (mismatch mask over
    paths, number of mismatches, number of tie draws). Asserts every mismatch is a tie."""
    idx_gpu = idx_gpu.astype(np.int64)
    idx_or = idx_or.astype(np.int64)
    M, N, C = idx_or.shape
    mism = idx_gpu != idx_or
    Lam = np.transpose(Lam_or, (2, 1, 0))            # [M, C, n+1]
    kk, ll, cc = np.nonzero(mism)
    for k, l, c in zip(kk, ll, cc):
        j = min(idx_gpu[k, l, c], idx_or[k, l, c])
        assert 1 <= j <= n, (k, l, c, idx_gpu[k, l, c], idx_or[k, l, c])
        lam = Lam[k, c, j]
        assert abs(lam - eps[k, l, c]) < TIE_REL * lam, \
            f"default step mismatch outside the tie band at path {k} draw {l} cpty {c}"
    # all tie draws: clock within the band of Lambda at the oracle's boundary dates
    j_hi = np.minimum(idx_or, n)
    j_lo = np.maximum(idx_or - 1, 1)
    lam_hi = np.take_along_axis(Lam, np.transpose(j_hi, (0, 2, 1)), axis=2).transpose(0, 2, 1)
    lam_lo = np.take_along_axis(Lam, np.transpose(j_lo, (0, 2, 1)), axis=2).transpose(0, 2, 1)
    tie = (np.abs(lam_hi - eps) < TIE_REL * lam_hi) | (np.abs(lam_lo - eps) < TIE_REL * lam_lo)
    n_tie = int(tie.sum())
    assert int(mism.sum()) <= n_tie
    assert n_tie <= TIE_MAX_SHARE * idx_or.size + 1, (n_tie, idx_or.size)
    return mism.any(axis=(1, 2)), int(mism.sum()), n_tie


def compare_targets(xi_gpu, xi_or, skip_paths, cva0):
    """xi_* [n, M]; paths with a tie-mismatched draw are compared separately."""
    keep = ~skip_paths
    a = xi_gpu[:, keep].astype(np.float64)
    b = xi_or[:, keep]
    err = np.abs(a - b)
    bound = XI_RTOL * np.abs(b) + XI_FLOOR_CVA0 * cva0
    worst = float(np.max(err / np.maximum(bound, 1e-300))) if err.size else 0.0
    assert np.all(err <= bound), f"targets off by up to {worst:.3g} x tolerance"
    return worst
