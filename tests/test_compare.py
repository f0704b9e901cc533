"""The comparison helpers of the parity tests (oracle/compare.py), on the CPU: the
tie-corrected targets equal the per-draw targets recomputed with the moved default
step, and a move outside the tie band is reported."""
import numpy as np

import oracle
from oracle import compare
from paper_2211_17005_gb300 import workload as W


def test_tie_corrected_targets_equal_recomputed_draws(oracle_lib):
    wl = W.make("small", M=64, N=8, n_steps=20)
    o = oracle.simulate(wl.model, wl.portfolios[0], wl.grid, 0, wl.M, wl.N, wl.seed,
                        want=("I0", "Lambda", "mtm", "idx", "xi_bar"))
    n = wl.grid.n_steps
    idx_g = o["idx"].astype(np.int64).copy()
    moved = [(3, 2, 0), (10, 5, 1), (40, 7, 0)]
    for k, l, c in moved:   # one step later, one earlier, and to "no default"
        idx_g[k, l, c] = {0: min(idx_g[k, l, c] + 1, n + 1), 1: max(idx_g[k, l, c] - 1, 1), 2: n + 1}[moved.index((k, l, c))]
    mism = idx_g != o["idx"]
    ref = compare.tie_corrected_targets(o, wl.model.recovery, idx_g, mism)
    o2 = dict(o)
    o2["idx"] = idx_g
    direct = np.stack([oracle.draw_targets(o2, np.asarray(wl.model.recovery), i).mean(axis=1) for i in range(n)])
    np.testing.assert_allclose(ref, direct, rtol=1e-12, atol=1e-15)
    untouched = np.ones(wl.M, bool)
    untouched[[k for k, _, _ in moved]] = False
    assert np.array_equal(ref[:, untouched], o["xi_bar"][:, untouched])


def test_moves_outside_the_tie_band_are_reported(oracle_lib):
    wl = W.make("small", M=32, N=4, n_steps=20)
    o = oracle.simulate(wl.model, wl.portfolios[0], wl.grid, 0, wl.M, wl.N, wl.seed, want=("Lambda", "idx"))
    eps = oracle.exp_clocks(wl.seed, 0, wl.M, wl.N, wl.model.C)
    d = compare.default_mismatches(o["idx"], o["idx"], o["Lambda"], eps, wl.grid.n_steps)
    assert d["n_mism"] == 0 and not d["outside"]
    idx_g = o["idx"].astype(np.int64).copy()
    k, l, c = np.argwhere(idx_g <= wl.grid.n_steps - 1)[0]
    idx_g[k, l, c] += 1
    d = compare.default_mismatches(idx_g, o["idx"], o["Lambda"], eps, wl.grid.n_steps)
    assert d["n_mism"] == 1 and len(d["outside"]) == 1
