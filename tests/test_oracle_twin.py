"""Pins of the twin Monte Carlo validation (Sec. ss:twin, eqs. (e:val1)-(e:val2)) in
the FP64 oracle: a twin copy follows the simulation up to its branch date, and the
estimator phi^2 - (xi1 + xi2) phi + xi1 xi2 averages to the L2 error
E[(phi - E[xi | state])^2] when the copies are independent given the state.

The unbiasedness pin uses a frozen market (no rate volatility, constant hazards):
there the exposures are deterministic, so the conditional mean of the averaged
target at date i is the plain sum e^{I0_i} sum_c sum_{j>i} V_c(j) (e^{-Lambda_c(j-1)}
- e^{-Lambda_c(j)}) with Lambda_c(j) = gamma_c t_j, and an estimate phi = m + delta
has L2 error delta^2 exactly."""
import copy

import numpy as np
import pytest

import oracle
from paper_2211_17005_gb300 import workload as W


def test_twin_copy_follows_the_simulation_up_to_its_branch_date(oracle_lib):
    wl = W.make("small", M=256)
    pf = wl.portfolios[0]
    want = ("features", "I0", "Lambda", "mtm", "xi_bar")
    main = oracle.simulate(wl.model, pf, wl.grid, 0, 256, 4, wl.seed, want=want)
    for date in (0, 17, wl.grid.n_steps):
        c1 = oracle.simulate(wl.model, pf, wl.grid, 0, 256, 4, wl.seed, want=want, copy=(date, 1))
        c2 = oracle.simulate(wl.model, pf, wl.grid, 0, 256, 4, wl.seed, want=want, copy=(date, 2))
        for key in ("features", "I0", "Lambda", "mtm"):
            np.testing.assert_array_equal(c1[key][:date + 1], main[key][:date + 1])
            np.testing.assert_array_equal(c2[key][:date + 1], main[key][:date + 1])
        if date < wl.grid.n_steps:   # after the branch the copies move apart
            assert not np.array_equal(c1["features"][date + 1:], main["features"][date + 1:])
            assert not np.array_equal(c1["features"][date + 1:], c2["features"][date + 1:])
        # fresh inner clocks: the copies' targets at the branch date differ from the simulation's
        assert not np.array_equal(c1["xi_bar"][min(date, wl.grid.n_steps - 1)],
                                  main["xi_bar"][min(date, wl.grid.n_steps - 1)])


def _frozen_small():
    """The small workload with no rate volatility and off-market swaps (fixed rate
    0.5% against the 2% curve), so that the exposures are deterministic and not zero."""
    wl = W.make("small", M=16384, N=2)
    m = copy.deepcopy(wl.model)
    m.hw_sigma = np.zeros(1)
    wl.model = m
    pf = copy.deepcopy(wl.portfolios[0])
    pf.fixed_rate = np.full(pf.n_swaps, 0.005)
    wl.portfolios = [pf]
    return wl


def test_twin_estimator_is_unbiased_in_a_frozen_market(oracle_lib):
    wl = _frozen_small()
    pf, M, N, i = wl.portfolios[0], wl.M, wl.N, 10
    want = ("xi_bar", "smooth", "Lambda", "I0")
    main = oracle.simulate(wl.model, pf, wl.grid, 0, M, N, wl.seed, want=want)
    # deterministic market: the integrated hazards are gamma_c t_j on every path
    t = np.linspace(0.0, wl.grid.horizon, wl.grid.n_steps + 1)
    np.testing.assert_allclose(main["Lambda"][:, :, 0], np.outer(t, wl.model.gamma0), rtol=1e-12, atol=1e-15)
    m_i = main["smooth"][i]
    assert m_i[0] > 1e-4                          # a CVA-sized conditional mean ...
    assert np.ptp(m_i) <= 1e-12 * abs(m_i[0])   # ... the same number on every path
    x1 = oracle.simulate(wl.model, pf, wl.grid, 0, M, N, wl.seed, want=("xi_bar",), copy=(i, 1))["xi_bar"][i]
    x2 = oracle.simulate(wl.model, pf, wl.grid, 0, M, N, wl.seed, want=("xi_bar",), copy=(i, 2))["xi_bar"][i]
    sd = float(np.std(x1))
    assert sd > 0.1 * m_i[0]                      # the inner draws leave real noise in each copy
    for delta in (0.0, 0.5 * sd, -2.0 * sd):
        est, se = oracle.twin_l2(m_i + delta, x1, x2)
        assert abs(est - delta ** 2) < 4 * se + 1e-15, (delta, est, se)
    # a planted mistake: one copy used twice (not independent given the state) adds
    # Var(xi | state) to the estimate, far outside its error bars
    est_bad, se_bad = oracle.twin_l2(m_i + 0.5 * sd, x1, x1)
    assert est_bad - (0.5 * sd) ** 2 > 20 * se_bad
    # and the simulation's own targets average to the conditional mean
    xm = main["xi_bar"][i]
    assert abs(xm.mean() - m_i[0]) < 4 * xm.std() / np.sqrt(M)


def test_twin_estimate_of_a_regression_is_between_zero_and_the_target_variance(oracle_lib):
    """A least-squares regression at date i: its twin L2 error is nonnegative within
    noise and below the variance of the targets (the error of the constant mean)."""
    wl = W.make("small", M=8192, N=4)
    pf, M, N, i = wl.portfolios[0], wl.M, wl.N, 20
    main = oracle.simulate(wl.model, pf, wl.grid, 0, M, N, wl.seed, want=("features", "xi_bar"))
    _, phi = oracle.lsq(oracle.poly2_features(main["features"][i, 0]), main["xi_bar"][i])
    x1 = oracle.simulate(wl.model, pf, wl.grid, 0, M, N, wl.seed, want=("xi_bar",), copy=(i, 1))["xi_bar"][i]
    x2 = oracle.simulate(wl.model, pf, wl.grid, 0, M, N, wl.seed, want=("xi_bar",), copy=(i, 2))["xi_bar"][i]
    est, se = oracle.twin_l2(phi, x1, x2)
    const, se_c = oracle.twin_l2(np.full(M, main["xi_bar"][i].mean()), x1, x2)
    assert est > -4 * se
    assert est < const
