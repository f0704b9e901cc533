"""Parity of the least-squares regression (eq. (e:forw)) with the oracle's QR."""
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


def test_regress_same_inputs_matches_qr(api):
    """Identical FP32 inputs: FP64 normal equations + Cholesky vs Householder QR."""
    rng = np.random.default_rng(1)
    M, F = 100_003, 27
    Y = rng.normal(size=(F, M)).astype(np.float32) * 0.01 + 0.02
    xi = (0.3 + Y[:5].sum(axis=0) * 4 + 0.01 * rng.normal(size=M)).astype(np.float32)
    pred, coef = api.regress(torch.from_numpy(xi).cuda(), torch.from_numpy(Y).cuda(), basis="linear")
    phi = oracle.linear_features(Y.astype(np.float64))
    _, pred_or = oracle.lsq(phi, xi.astype(np.float64))
    scale = np.sqrt(np.mean(xi.astype(np.float64) ** 2))
    assert np.sqrt(np.mean((pred.cpu().numpy() - pred_or) ** 2)) < 1e-5 * scale
    w_raw = np.linalg.lstsq(np.vstack([np.ones(M), Y.astype(np.float64)]).T, xi.astype(np.float64), rcond=None)[0]
    np.testing.assert_allclose(coef, w_raw, rtol=1e-4, atol=1e-6 * np.abs(w_raw).max())


def test_regress_poly2_same_inputs(api):
    rng = np.random.default_rng(2)
    M = 16384
    y = (0.02 + 0.01 * rng.normal(size=M)).astype(np.float32)
    xi = (1e-3 * np.maximum(y - 0.015, 0) + 1e-5 * rng.normal(size=M)).astype(np.float32)
    pred, coef = api.regress(torch.from_numpy(xi).cuda(), torch.from_numpy(y[None]).cuda(), basis="poly2")
    _, pred_or = oracle.lsq(oracle.poly2_features(y.astype(np.float64)), xi.astype(np.float64))
    scale = np.sqrt(np.mean(xi.astype(np.float64) ** 2))
    assert np.sqrt(np.mean((pred.cpu().numpy() - pred_or) ** 2)) < 1e-5 * scale


def test_regress_all_dates_small_workload(api):
    """Every date of the small workload at full size: GPU targets/features/regression vs
    the oracle's own FP64 targets, features and QR; L2 gap <= 1e-3 CVA_0."""
    wl = W.make("small")
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, wl.N)
    sim.run(wl.seed)
    pred, coef = sim.regress_all(0, basis="poly2")
    pred = pred.cpu().numpy()
    o = oracle.simulate(wl.model, wl.portfolios[0], wl.grid, 0, wl.M, wl.N, wl.seed, want=("features", "xi_bar"))
    cva0 = float(o["xi_bar"][0].mean())
    for i in range(1, wl.grid.n_steps):
        _, p_or = oracle.lsq(oracle.poly2_features(o["features"][i, 0]), o["xi_bar"][i])
        rms = np.sqrt(np.mean((pred[i] - p_or) ** 2))
        assert rms <= 1e-3 * cva0, (i, rms, cva0)
    sim.close()


def test_regress_all_dates_paper_linear(api):
    """Paper-shaped model, linear basis [1, Y_t] (28 columns), on a 4096-path prefix."""
    wl = W.make("paper", M=4096, N=32, n_steps=20)
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, wl.N)
    sim.run(wl.seed)
    pred, coef = sim.regress_all(0, basis="linear")
    pred = pred.cpu().numpy()
    o = oracle.simulate(wl.model, wl.portfolios[0], wl.grid, 0, wl.M, wl.N, wl.seed, want=("features", "xi_bar"))
    cva0 = float(o["xi_bar"][0].mean())
    for i in range(1, wl.grid.n_steps):
        _, p_or = oracle.lsq(oracle.linear_features(o["features"][i]), o["xi_bar"][i])
        rms = np.sqrt(np.mean((pred[i] - p_or) ** 2))
        assert rms <= 1e-3 * cva0, (i, rms, cva0)
    sim.close()


def test_intercept_of_date_zero_equals_cva0(api):
    """Regressing the date-0 targets on a constant (all paths share the date-0 state)
    returns CVA_0: the poly2 fit on a degenerate factor keeps only the intercept."""
    wl = W.make("small", M=5000)
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, wl.N)
    sim.run(wl.seed)
    xi0 = sim.targets()[0, 0].contiguous()
    y = torch.zeros((1, wl.M), dtype=torch.float32, device="cuda")
    pred, _ = api.regress(xi0, y, basis="poly2", want_coef=False)
    m, _ = api.cva0(xi0)
    assert float(pred.mean()) == pytest.approx(m, rel=1e-6)
