"""Shared comparison logic of the GPU parity tests (CPU-side numpy only): asserting
wrappers around the oracle's comparison functions (oracle/compare.py), which state
the tolerances."""
import numpy as np

from oracle.compare import (CVA0_RTOL, TIE_MAX_SHARE, TIE_REL, XI_FLOOR_CVA0, XI_RTOL,  # noqa: F401
                            default_mismatches, target_errors, tie_corrected_targets)


def compare_defaults(idx_gpu, idx_or, Lam_or, eps, n):
    """idx_* [M, N, C]; Lam_or [n+1, C, M]; eps [M, N, C]. Returns (mismatch mask over
    paths, number of mismatches, number of tie draws). Asserts that every mismatch is
    a tie (the step moved only across dates whose Lambda is within the band of the
    clock) and that ties are at most 1e-4 of the draws."""
    d = default_mismatches(idx_gpu, idx_or, Lam_or, eps, n)
    assert not d["outside"], f"default step mismatches outside the tie band: {d['outside'][:5]}"
    assert d["n_mism"] <= d["n_tie"]
    assert d["n_tie"] <= TIE_MAX_SHARE * d["draws"] + 1, (d["n_tie"], d["draws"])
    return d["mism"].any(axis=(1, 2)), d["n_mism"], d["n_tie"]


def compare_targets(xi_gpu, xi_or, skip_paths, cva0):
    """xi_* [n, M]; paths flagged in skip_paths are left out (callers that cannot
    rebuild the oracle's targets at the GPU's default steps)."""
    keep = ~skip_paths
    e = target_errors(xi_gpu[:, keep], xi_or[:, keep], cva0)
    assert e["worst_vs_tolerance"] <= 1.0, f"targets off by up to {e['worst_vs_tolerance']:.3g} x tolerance"
    return e["worst_vs_tolerance"]


def compare_all_targets(xi_gpu, o, recovery, idx_gpu, Lam_or, eps, n):
    """Every path's targets and CVA_0 at full tolerance: the oracle's targets are
    rebuilt with the GPU's default step on the tie-mismatched draws (oracle/compare.py).
    Returns (tie-corrected oracle CVA_0, number of mismatched draws, number of ties)."""
    d = default_mismatches(idx_gpu, o["idx"], Lam_or, eps, n)
    assert not d["outside"], f"default step mismatches outside the tie band: {d['outside'][:5]}"
    assert d["n_mism"] <= d["n_tie"] <= TIE_MAX_SHARE * d["draws"] + 1, (d["n_mism"], d["n_tie"], d["draws"])
    ref = tie_corrected_targets(o, recovery, idx_gpu, d["mism"])
    cva0 = float(ref[0].mean())
    e = target_errors(xi_gpu, ref, cva0)
    assert e["worst_vs_tolerance"] <= 1.0, f"targets off by up to {e['worst_vs_tolerance']:.3g} x tolerance"
    return cva0, d["n_mism"], d["n_tie"]
