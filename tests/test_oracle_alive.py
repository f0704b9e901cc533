"""Pins of the oracle's learner on the hierarchically simulated sample (Sec.
"Learning on Hierarchically Simulated Paths"): one row per (outer path k, inner
draw l), the features (X_i^{k,l}, Y_i^k) with X the default indicators of Sec. 4.1,
the per-draw target xi_i^{k,l} of eq. (eq:CVA_portfolio).

The closed-form pin uses a frozen market (no rate volatility, constant hazards,
off-market swaps): the exposures are deterministic and the counterparties' default
clocks independent, so E[xi_i | X_i] = sum_c (1 - X_c) a_c(i) exactly, with
a_c(i) = e^{I0_i} sum_{j>i} (1 - R_c) e^{-I0_j} MtM_c(j)^+ (e^{-(Lambda_c(j-1) - Lambda_c(i))}
- e^{-(Lambda_c(j) - Lambda_c(i))}), the loss of c given that it is alive at t_i. The
regression is then correctly specified: its intercept estimates sum_c a_c(i) and
the coefficient of X_c estimates -a_c(i)."""
import copy

import numpy as np

import oracle
from paper_2211_17005_gb300 import workload as W


def _frozen(M, N):
    wl = W.make("small", M=M, N=N)
    m = copy.deepcopy(wl.model)
    m.hw_sigma = np.zeros(1)
    wl.model = m
    pf = copy.deepcopy(wl.portfolios[0])
    pf.fixed_rate = np.full(pf.n_swaps, 0.005)
    wl.portfolios = [pf]
    return wl


def test_frozen_market_regression_recovers_the_conditional_losses(oracle_lib):
    wl = _frozen(8192, 128)
    pf, n = wl.portfolios[0], wl.grid.n_steps
    o = oracle.simulate(wl.model, pf, wl.grid, 0, wl.M, wl.N, wl.seed,
                        want=("features", "I0", "Lambda", "mtm", "idx", "xi_bar"))
    R = np.asarray(wl.model.recovery)
    C = wl.model.C
    t = np.linspace(0.0, wl.grid.horizon, n + 1)
    for i in (5, 15):
        # closed form from path 0 (every path carries the same market)
        a = np.zeros(C)
        for c in range(C):
            lam = wl.model.gamma0[c] * t
            for j in range(i + 1, n + 1):
                v = (1 - R[c]) * np.exp(-o["I0"][j, 0]) * max(o["mtm"][j, c, 0], 0.0)
                a[c] += v * (np.exp(-(lam[j - 1] - lam[i])) - np.exp(-(lam[j] - lam[i])))
            a[c] *= np.exp(o["I0"][i, 0])
        assert np.all(a > 1e-5)
        res = oracle.alive_lsq(o, R, i)
        F = o["features"].shape[1]
        assert res["dropped"] == list(range(1, 1 + F))      # the frozen state carries nothing
        w = res["w"]
        # standard errors of the correctly specified model [1, X]
        X = oracle.default_indicators(o, i).reshape(-1, C)
        D = np.concatenate([np.ones((X.shape[0], 1)), X], axis=1)
        xi = oracle.draw_targets(o, R, i).reshape(-1)
        coef = np.concatenate([[w[0]], w[1 + F:]])
        resid = xi - D @ coef
        cov = np.linalg.inv(D.T @ D) * resid.var()
        se = np.sqrt(np.diag(cov))
        want = np.concatenate([[a.sum()], -a])
        assert np.all(se < 0.1 * np.abs(want)), (se, want)  # the check below has teeth
        assert np.all(np.abs(coef - want) < 5 * se), (i, coef, want, se)
        # every counterparty alive: the fitted value is the sum of the conditional losses
        assert abs(res["alive"][0] - a.sum()) < 5 * se[0]


def test_default_indicators_follow_the_survival_curve(oracle_lib):
    """Constant hazard gamma_c: P(X_c = 1 at t_i) = 1 - e^{-gamma_c t_i} (discrete
    convention: default at the first step j with Lambda_c(t_j) >= E)."""
    wl = _frozen(2048, 64)
    pf = wl.portfolios[0]
    o = oracle.simulate(wl.model, pf, wl.grid, 0, wl.M, wl.N, wl.seed, want=("idx",))
    t = np.linspace(0.0, wl.grid.horizon, wl.grid.n_steps + 1)
    for i in (1, 10, 49):
        X = oracle.default_indicators(o, i)
        for c in range(wl.model.C):
            p = 1.0 - np.exp(-wl.model.gamma0[c] * t[i])
            se = np.sqrt(p * (1 - p) / X[..., c].size)
            assert abs(X[..., c].mean() - p) < 5 * se, (i, c)


def test_without_indicators_the_sample_regression_is_the_averaged_one(oracle_lib):
    """Reading of Sec. "Learning on Hierarchically Simulated Paths" with Y-only
    features: the M N normal equations are N times those of the averaged target,
    so the fit equals the least squares of xi_bar on Y; and the per-draw targets
    average to the oracle's own xi_bar (computed by a separate loop in C)."""
    wl = W.make("small", M=512, N=16)
    pf = wl.portfolios[0]
    o = oracle.simulate(wl.model, pf, wl.grid, 0, wl.M, wl.N, wl.seed,
                        want=("features", "I0", "Lambda", "mtm", "idx", "xi_bar"))
    R = np.asarray(wl.model.recovery)
    for i in (5, 25, 40):
        xi = oracle.draw_targets(o, R, i)
        np.testing.assert_allclose(xi.mean(axis=1), o["xi_bar"][i], rtol=1e-12, atol=1e-15)
        res = oracle.alive_lsq(o, R, i, with_defaults=False)
        _, pred = oracle.lsq(oracle.linear_features(o["features"][i]), o["xi_bar"][i])
        scale = np.abs(pred).max()
        np.testing.assert_allclose(res["alive"], pred, rtol=0, atol=1e-10 * scale)


def test_sample_regression_satisfies_its_normal_equations(oracle_lib):
    wl = W.make("small", M=512, N=16)
    pf = wl.portfolios[0]
    o = oracle.simulate(wl.model, pf, wl.grid, 0, wl.M, wl.N, wl.seed,
                        want=("features", "I0", "Lambda", "mtm", "idx", "xi_bar"))
    R = np.asarray(wl.model.recovery)
    i = 30
    res = oracle.alive_lsq(o, R, i)
    assert res["dropped"] == []
    xi = oracle.draw_targets(o, R, i)
    r = (xi - res["fitted"]).reshape(-1)
    phiY = oracle.linear_features(o["features"][i])
    X = oracle.default_indicators(o, i)
    cols = [np.repeat(phiY[:, j:j + 1], wl.N, axis=1).reshape(-1) for j in range(phiY.shape[1])]
    cols += [X[..., c].reshape(-1) for c in range(X.shape[2])]
    scale = np.abs(xi).sum()
    for col in cols:
        assert abs(float(col @ r)) < 1e-9 * scale
    # the X coefficients are not zero: the indicators matter
    assert np.all(np.abs(res["w"][-wl.model.C:]) > 1e-5)
