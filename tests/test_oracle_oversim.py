"""Pins of the oversimulation-factor choice of Prop. 1 / Heuristic 1 (Sec. ss:choice1).

* In a frozen market (no rate volatility, constant hazards, off-market swaps) the outer
  path is deterministic, so R_i = Var(E[g | Y]) = 0 and Q_i = Var(g), which the exact
  law of the default steps (P(idx_c = j) = e^{-gamma_c t_{j-1}} - e^{-gamma_c t_j})
  gives in closed form by enumeration.
* The variance of the loss estimator under the budget M (N + kappa) = Psi is
  (R + Q / N)(N + kappa) / Psi; N = sqrt(Q kappa / R) minimises it (checked on a grid).
* The cost ratio of eq. (l:ratio) is recovered from times proportional to kappa + N.
"""
import copy

import numpy as np
import pytest

import oracle
from paper_2211_17005_gb300 import workload as W


def _frozen(M):
    wl = W.make("small", M=M, N=2)
    m = copy.deepcopy(wl.model)
    m.hw_sigma = np.zeros(1)
    wl.model = m
    pf = copy.deepcopy(wl.portfolios[0])
    pf.fixed_rate = np.full(pf.n_swaps, 0.005)
    wl.portfolios = [pf]
    return wl


def test_prop1_statistics_in_a_frozen_market(oracle_lib):
    wl = _frozen(65536)
    pf, M, n = wl.portfolios[0], wl.M, wl.grid.n_steps
    o = oracle.simulate(wl.model, pf, wl.grid, 0, M, wl.N, wl.seed, want=("idx", "mtm", "I0", "smooth"))
    rec = wl.model.recovery
    V = (1 - rec)[:, None] * np.exp(-o["I0"][:, 0])[None, :] * np.maximum(o["mtm"][:, :, 0].T, 0.0)   # [C, n+1]
    assert V.max() > 1e-3
    t = np.linspace(0.0, wl.grid.horizon, n + 1)
    for i in (5, 25):
        phi = np.full(M, 0.7 * o["smooth"][i, 0])     # any estimate computed from the (deterministic) state
        pred = np.zeros((n, M))
        pred[i] = phi
        Q, R = oracle.oversim_stats(o, rec, pred)
        # exact law: independent counterparties, deterministic exposures
        p = []
        for c in range(wl.model.C):
            surv = np.exp(-wl.model.gamma0[c] * t)
            p.append(np.concatenate([surv[:-1] - surv[1:], [surv[-1]]]))   # steps 1..n, then n+1
        j = np.arange(1, n + 2)
        contrib = [np.where((j > i) & (j <= n), V[c, np.minimum(j, n)], 0.0) for c in range(wl.model.C)]
        xi = np.exp(o["I0"][i, 0]) * (contrib[0][:, None] + contrib[1][None, :])
        w = np.outer(p[0], p[1])
        g = (xi - phi[0]) ** 2
        Eg, Eg2 = np.sum(w * g), np.sum(w * g * g)
        Q_exact = Eg2 - Eg ** 2
        # Monte Carlo errors of the two estimators, from the per-draw samples
        samp = []
        for l in range(2):
            jl = o["idx"][:, l, :].astype(np.int64)
            x = np.exp(o["I0"][i, 0]) * sum(np.where((jl[:, c] > i) & (jl[:, c] <= n),
                                                     V[c, np.minimum(jl[:, c], n)], 0.0) for c in range(2))
            samp.append((x - phi) ** 2)
        g0, g1 = samp
        se_q = np.std(0.5 * (g0 ** 2 + g1 ** 2) - g0 * g1) / np.sqrt(M)
        se_r = np.std(g0 * g1) / np.sqrt(M) + 2 * np.mean(g0) * np.std(g0) / np.sqrt(M)
        assert Q_exact > 0
        assert abs(Q[i] - Q_exact) < 5 * se_q, (i, Q[i], Q_exact, se_q)
        assert abs(R[i]) < 5 * se_r, (i, R[i], se_r)
        assert se_q < 0.05 * Q_exact          # the pin has teeth


def test_optimal_factor_minimises_the_loss_variance():
    from paper_2211_17005_gb300 import api
    Q, R, kappa, psi = np.array([2.0, 0.3, 5.0]), np.array([0.01, 0.02, 0.5]), 497.0, 1e7
    Ni, N, M = api.oversimulation_choice(Q, R, kappa, budget=psi)
    grid = np.linspace(0.5, 5000, 400001)
    for q, r, ni in zip(Q, R, Ni):
        var = (r + q / grid) * (grid + kappa) / psi
        assert abs(grid[np.argmin(var)] - ni) < 0.02 * ni
    assert N == pytest.approx(Ni.mean())
    assert M == pytest.approx(psi / (N + kappa))


def test_cost_ratio_from_two_timings():
    from paper_2211_17005_gb300 import api
    kappa, c = 123.4, 2.5e-3
    t1, t2 = c * (kappa + 8), c * (kappa + 64)
    assert api.inner_cost_ratio(t1, 8, t2, 64) == pytest.approx(kappa, rel=1e-12)
