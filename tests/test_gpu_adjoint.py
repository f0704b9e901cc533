"""Adjoint sensitivities of CVA_0 (smooth form, eq. (eq:CVAint) in its exact discrete
version) against the FP64 oracle's central differences and against common-random-
number central differences of the GPU forward pass."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_17005_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2211_17005_gb300 import api as A, build
    build.build()
    oracle.build()
    return A


def _oracle_smooth(model, pf, grid, M, seed):
    o = oracle.simulate(model, pf, grid, 0, M, 1, seed, want=("smooth",))
    return float(o["smooth"][0].mean())


def _bump(theta, i, h):
    t = theta.copy()
    t[i] += h
    return t


@pytest.mark.parametrize("name", ["adjoint", "small"])
def test_smooth_forward_matches_oracle(api, name):
    wl = W.make(name, M=512, n_steps=20 if name == "adjoint" else 50)
    pf = api.frozen(wl.model, wl.portfolios[0])
    c_fwd, _ = api.grad_cva0(wl.model, pf, wl.grid, wl.M, wl.seed, forward_only=True)
    c_rev, g = api.grad_cva0(wl.model, pf, wl.grid, wl.M, wl.seed)
    ref = _oracle_smooth(wl.model, pf, wl.grid, wl.M, wl.seed)
    assert c_fwd == pytest.approx(ref, rel=1e-5)
    assert c_rev == pytest.approx(c_fwd, rel=1e-6)
    assert np.all(np.isfinite(g))


def test_adjoint_matches_oracle_central_differences(api):
    """FP64 oracle, central differences with common random numbers (same seed and
    counters) and frozen trade terms, on a 128-path sample."""
    wl = W.make("adjoint", M=128, n_steps=20)
    pf = api.frozen(wl.model, wl.portfolios[0])
    theta = api.grad_params(wl.model)
    _, g = api.grad_cva0(wl.model, pf, wl.grid, wl.M, wl.seed)
    fd = np.zeros_like(g)
    for i in range(theta.size):
        h = 1e-6 * max(abs(theta[i]), 1e-2)
        up = _oracle_smooth(api.with_params(wl.model, _bump(theta, i, h)), pf, wl.grid, wl.M, wl.seed)
        dn = _oracle_smooth(api.with_params(wl.model, _bump(theta, i, -h)), pf, wl.grid, wl.M, wl.seed)
        fd[i] = (up - dn) / (2 * h)
    scale = np.max(np.abs(fd))
    err = np.abs(g - fd)
    assert np.all(err <= 1e-4 * np.abs(fd) + 1e-5 * scale), list(zip(np.round(g, 6), np.round(fd, 6)))


@pytest.mark.parametrize("ckpt", [10, 3])
def test_adjoint_matches_oracle_forward_mode_gradient(api, ckpt):
    """The oracle's FP64 forward-mode gradient (oracle/dual.py) on the same 128 paths:
    exact derivatives of the oracle's smooth CVA_0, with no differencing error; every
    one of the 53 components within 2e-5 relative (+ 2e-6 of the largest)."""
    from oracle import dual
    wl = W.make("adjoint", M=128, n_steps=20)
    pf = api.frozen(wl.model, wl.portfolios[0])
    c0, g = api.grad_cva0(wl.model, pf, wl.grid, wl.M, wl.seed, ckpt_every=ckpt)
    ref = dual.smooth_cva0_grad(wl.model, pf, wl.grid, wl.M, wl.seed)
    assert c0 == pytest.approx(ref["cva0"], rel=1e-5)
    r = ref["grad"]
    assert g.shape == r.shape
    scale = np.max(np.abs(r))
    err = np.abs(g - r)
    worst = np.argsort(-err / (2e-5 * np.abs(r) + 2e-6 * scale))[:5]
    assert np.all(err <= 2e-5 * np.abs(r) + 2e-6 * scale), [(int(i), g[i], r[i]) for i in worst]


def test_adjoint_matches_gpu_crn_differences(api):
    """Central differences of the GPU forward pass with a 1e-4 bump and common random
    numbers, on 8192 paths."""
    wl = W.make("adjoint", M=8192, n_steps=40)
    pf = api.frozen(wl.model, wl.portfolios[0])
    theta = api.grad_params(wl.model)
    _, g = api.grad_cva0(wl.model, pf, wl.grid, wl.M, wl.seed)
    fd = np.zeros_like(g)
    h = 1e-4
    for i in range(theta.size):
        up, _ = api.grad_cva0(api.with_params(wl.model, _bump(theta, i, h)), pf, wl.grid, wl.M, wl.seed,
                              forward_only=True)
        dn, _ = api.grad_cva0(api.with_params(wl.model, _bump(theta, i, -h)), pf, wl.grid, wl.M, wl.seed,
                              forward_only=True)
        fd[i] = (up - dn) / (2 * h)
    scale = np.max(np.abs(fd))
    err = np.abs(g - fd)
    assert np.all(err <= 1e-3 * np.abs(fd) + 2e-4 * scale), list(zip(np.round(g, 5), np.round(fd, 5)))


def test_checkpoint_interval_does_not_change_the_gradient(api):
    wl = W.make("adjoint", M=1000, n_steps=30)
    pf = api.frozen(wl.model, wl.portfolios[0])
    ref_c, ref = api.grad_cva0(wl.model, pf, wl.grid, wl.M, wl.seed, ckpt_every=10)
    for K in (1, 7, 16):
        c, g = api.grad_cva0(wl.model, pf, wl.grid, wl.M, wl.seed, ckpt_every=K)
        assert c == pytest.approx(ref_c, rel=1e-7)
        np.testing.assert_allclose(g, ref, rtol=1e-5, atol=1e-7 * np.abs(ref).max())


def test_autograd_function_returns_the_adjoint(api):
    wl = W.make("adjoint", M=2048, n_steps=20)
    pf = api.frozen(wl.model, wl.portfolios[0])
    theta = torch.tensor(api.grad_params(wl.model), dtype=torch.float64, requires_grad=True)
    c0 = api.SmoothCVA0.apply(theta, wl.model, pf, wl.grid, wl.M, wl.seed)
    (2.0 * c0).backward()
    _, g = api.grad_cva0(wl.model, pf, wl.grid, wl.M, wl.seed)
    np.testing.assert_allclose(theta.grad.numpy(), 2.0 * g, rtol=1e-12)
