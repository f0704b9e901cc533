"""Pins of the oracle's forward-mode gradient (oracle/dual.py) of the smooth CVA_0
(eq. (eq:CVAint) in its exact discrete form at the first date): its value is the C
oracle's smooth CVA_0, every tangent is the C oracle's central difference along that
direction, and the recovery tangents satisfy the closed form
dCVA_0/dR_c = -CVA_0^c / (1 - R_c) (CVA_0 is linear in each loss-given-default)."""
import dataclasses

import numpy as np
import pytest

import oracle
from oracle import dual
from paper_2211_17005_gb300 import workload as W


def _case(M=48, n_steps=20, n_swaps=60):   # half-year steps: reset and mid-period dates
    wl = W.make("adjoint", M=M, n_steps=n_steps, n_swaps=n_swaps)
    pf = dataclasses.replace(wl.portfolios[0], fixed_rate=oracle.par_rates(wl.model, wl.portfolios[0]))
    return wl, pf


def _theta(model):
    """The directions of dual.smooth_cva0_grad, recoveries included."""
    return np.concatenate([model.curve, model.hw_sigma, model.fx_vol[1:], model.cir_kappa, model.cir_theta,
                           model.cir_nu, model.recovery]).astype(np.float64)


def _with(model, t):
    E, C = model.E, model.C
    o = [0]

    def take(k):
        v = np.array(t[o[0]:o[0] + k], dtype=np.float64)
        o[0] += k
        return v
    curve, sig = take(E), take(E)
    fx = np.concatenate([[model.fx_vol[0]], take(E - 1)])
    kap, the, nu, rec = take(C), take(C), take(C), take(C)
    return dataclasses.replace(model, curve=curve, hw_sigma=sig, fx_vol=fx, cir_kappa=kap, cir_theta=the,
                               cir_nu=nu, recovery=rec)


def _smooth(model, pf, grid, M, seed):
    return float(oracle.simulate(model, pf, grid, 0, M, 1, seed, want=("smooth",))["smooth"][0].mean())


def pin_value_is_the_oracle_smooth_cva0(dl):
    wl, pf = _case()
    res = dl.smooth_cva0_grad(wl.model, pf, wl.grid, wl.M, wl.seed)
    ref = _smooth(wl.model, pf, wl.grid, wl.M, wl.seed)
    assert abs(res["cva0"] - ref) <= 1e-12 * abs(ref), (res["cva0"], ref)
    assert abs(res["cva0_c"].sum() - ref) <= 1e-12 * abs(ref)


def pin_tangents_are_central_differences(dl):
    wl, pf = _case()
    res = dl.smooth_cva0_grad(wl.model, pf, wl.grid, wl.M, wl.seed)
    g = np.concatenate([res["grad"], res["grad_recovery"]])
    th = _theta(wl.model)
    assert g.size == th.size == dl.n_directions(wl.model)
    fd = np.zeros_like(g)
    for i in range(th.size):
        h = 1e-5 * max(abs(th[i]), 1e-2)
        up, dn = th.copy(), th.copy()
        up[i] += h
        dn[i] -= h
        fd[i] = (_smooth(_with(wl.model, up), pf, wl.grid, wl.M, wl.seed)
                 - _smooth(_with(wl.model, dn), pf, wl.grid, wl.M, wl.seed)) / (2 * h)
    scale = np.max(np.abs(fd))
    err = np.abs(g - fd)
    assert np.all(err <= 1e-6 * np.abs(fd) + 1e-8 * scale), [(i, g[i], fd[i]) for i in np.argsort(-err)[:5]]


def pin_recovery_closed_form(dl):
    wl, pf = _case(M=24)
    res = dl.smooth_cva0_grad(wl.model, pf, wl.grid, wl.M, wl.seed)
    cf = -res["cva0_c"] / (1.0 - wl.model.recovery)
    np.testing.assert_allclose(res["grad_recovery"], cf, rtol=1e-12, atol=0)
    assert np.all(res["cva0_c"] > 0)


PINS = [pin_value_is_the_oracle_smooth_cva0, pin_tangents_are_central_differences, pin_recovery_closed_form]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_dual_pins(pin):
    pin(dual)
