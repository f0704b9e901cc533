"""The least-squares learner on the hierarchically simulated sample (default
indicators X_i and state Y_i over M N rows, Sec. "Learning on Hierarchically
Simulated Paths") on the GPU, against the FP64 oracle that writes the M N design
matrix out row by row and solves it by QR; at the full paper shape, against the
normal equations evaluated in FP64 on the sample itself."""
import copy

import numpy as np
import pytest
import torch

import oracle
from paper_2211_17005_gb300 import workload as W

pytestmark = pytest.mark.gpu

# RMS over paths of the difference of the fits at X = 0, and the largest difference
# of an indicator coefficient, in units of CVA_0 (the regression tolerance).
REG_TOL_CVA0 = 1e-3


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2211_17005_gb300 import api as A, build
    build.build()
    oracle.build()
    return A


def _gpu(api, wl, M, N):
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, M, N, keep_defaults=True)
    sim.run(wl.seed)
    pred, coef, dropped = sim.regress_alive(0)
    torch.cuda.synchronize()
    feats = sim.features().cpu().numpy()
    out = pred.cpu().numpy(), coef, dropped, feats
    sim.close()
    return out


def _check_against_oracle(wl, M, N, dates, pred, coef, dropped, feats):
    o = oracle.simulate(wl.model, wl.portfolios[0], wl.grid, 0, M, N, wl.seed,
                        want=("features", "I0", "Lambda", "mtm", "idx", "xi_bar"))
    R = np.asarray(wl.model.recovery)
    cva0 = float(o["xi_bar"][0].mean())
    F = o["features"].shape[1]
    for i in dates:
        ref = oracle.alive_lsq(o, R, i)
        assert int(dropped[i]) == len(ref["dropped"]), (i, dropped[i], ref["dropped"])
        err = pred[i].astype(np.float64) - ref["alive"]
        rms = float(np.sqrt(np.mean(err ** 2)))
        assert rms <= REG_TOL_CVA0 * cva0, (i, rms / cva0)
        # the indicator coefficients are the same in every affine basis of the state
        dx = np.abs(coef[i, 1 + F:] - ref["w"][1 + F:])
        assert np.all(dx <= REG_TOL_CVA0 * cva0), (i, dx / cva0)
        for j in ref["dropped"]:
            if j >= 1 + F:
                assert coef[i, j] == 0.0
        # the raw-basis coefficients reproduce the device's fit at X = 0
        raw = coef[i, 0] + feats[i].astype(np.float64).T @ coef[i, 1:1 + F]
        np.testing.assert_allclose(raw, pred[i], rtol=0, atol=1e-5 * np.abs(ref["alive"]).max())


@pytest.mark.parametrize("name,M,N,n_steps,dates", [
    ("small", 4099, 40, 50, (1, 2, 10, 25, 48, 49)),
    ("paper", 1003, 24, 20, (1, 5, 10, 18, 19)),
    ("mixed", 1531, 24, 40, (1, 7, 20, 38, 39)),   # C = 5, constant and CIR intensities interleaved
])
def test_alive_regression_matches_oracle(api, name, M, N, n_steps, dates):
    wl = W.make(name, n_steps=n_steps)
    pred, coef, dropped, feats = _gpu(api, wl, M, N)
    _check_against_oracle(wl, M, N, dates, pred, coef, dropped, feats)


def test_counterparty_that_never_defaults_is_dropped(api):
    """Zero hazard for counterparty 0: its indicator is 0 on every row, so both sides
    leave that column out at every date, and the rest of the fit still agrees."""
    wl = W.make("small", n_steps=25)
    m = copy.deepcopy(wl.model)
    m.gamma0 = np.array([0.0, 0.05])
    m.cir_theta = np.array([0.0, 0.05])
    wl.model = m
    M, N = 2048, 32
    pred, coef, dropped, feats = _gpu(api, wl, M, N)
    assert np.all(dropped[1:] == 1)
    F = feats.shape[1]
    assert np.all(coef[1:, 1 + F] == 0.0)
    _check_against_oracle(wl, M, N, (1, 12, 24), pred, coef, dropped, feats)


def test_alive_regression_is_deterministic_and_needs_the_default_steps(api):
    wl = W.make("paper", n_steps=20)
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, 4096, 32, keep_defaults=True)
    sim.run(wl.seed)
    p1, c1, _ = sim.regress_alive(0)
    p1 = p1.clone()
    p2, c2, _ = sim.regress_alive(0)
    torch.cuda.synchronize()
    assert torch.equal(p1, p2)
    np.testing.assert_array_equal(c1, c2)
    sim.close()
    bare = api.Simulation(wl.model, wl.portfolios, wl.grid, 4096, 32)
    bare.run(wl.seed)
    with pytest.raises(RuntimeError):
        bare.regress_alive(0)
    bare.close()


def test_normal_equations_hold_at_the_paper_shape(api):
    """The benchmark's shape (2^17 paths, 64 draws, 100 dates, 27 factors, 8
    counterparties: 8.4M rows per date): the residual of the device's fit is
    orthogonal to every column of the M N design, evaluated in FP64 on the sample
    (per-draw targets rebuilt from the exposures and default steps)."""
    wl = W.make("paper")
    M, N, n = wl.M, wl.N, wl.grid.n_steps
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, M, N, keep_defaults=True)
    sim.run(wl.seed)
    pred, coef, dropped = sim.regress_alive(0)
    torch.cuda.synchronize()
    assert np.all(dropped[1:] == 0)
    F, C = sim.F, sim.C
    idx = sim.defaults().to(torch.int64)                           # [M, N, C]
    expo = sim.exposures()[0].to(torch.float64)                    # [n+1, C, M]
    disc = sim.discount_integral().to(torch.float64)               # [n+1, M]
    Y = sim.features().to(torch.float64)                           # [n+1, F, M]
    E = expo.permute(2, 1, 0)                                       # [M, C, n+1]
    for i in (1, 50, n - 1):
        j = idx.clamp(max=n).permute(0, 2, 1)                       # [M, C, N]
        v = torch.gather(E, 2, j)
        live = (idx.permute(0, 2, 1) > i) & (idx.permute(0, 2, 1) <= n)
        xi = torch.exp(disc[i])[:, None] * torch.where(live, v, torch.zeros_like(v)).sum(dim=1)   # [M, N]
        X = (idx <= i).to(torch.float64)                            # [M, N, C]
        w = torch.from_numpy(coef[i]).to(xi.device)
        fit_y = w[0] + Y[i].T @ w[1:1 + F]                          # [M]
        r = xi - fit_y[:, None] - X @ w[1 + F:]                     # [M, N]
        ax = xi.abs()
        tol = 1e-4
        assert abs(float(r.sum())) <= tol * float(ax.sum())
        rk = r.sum(dim=1)
        Yc = Y[i] - Y[i][:, :1]
        for f in range(F):
            assert abs(float((Yc[f] * rk).sum())) <= tol * float((Yc[f].abs() * ax.sum(dim=1)).sum()), (i, f)
        for c in range(C):
            assert abs(float((X[..., c] * r).sum())) <= tol * float((X[..., c] * ax).sum()) + 1e-12, (i, c)
        # the device's fit at X = 0 is the raw-basis fit without the indicators
        np.testing.assert_allclose(pred[i].double().cpu().numpy(), fit_y.cpu().numpy(), rtol=0,
                                   atol=1e-5 * float(fit_y.abs().max()))
    sim.close()


def test_alive_regression_of_one_portfolio_among_several(api):
    """The 6-portfolio workload: the learner for portfolio 3 reads that portfolio's
    exposures and targets, and equals the oracle run on that portfolio alone."""
    wl = W.make("batched", n_steps=20)
    M, N, pf = 1003, 24, 3
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, M, N, keep_defaults=True)
    sim.run(wl.seed)
    pred, coef, dropped = sim.regress_alive(pf)
    torch.cuda.synchronize()
    feats = sim.features().cpu().numpy()
    pred = pred.cpu().numpy()
    sim.close()
    one = copy.copy(wl)
    one.portfolios = [wl.portfolios[pf]]
    _check_against_oracle(one, M, N, (1, 10, 19), pred, coef, dropped, feats)


def test_alive_regression_in_a_cuda_graph(api):
    """After one call (which allocates the scratch), simulate + the learner captured in
    a CUDA graph replays to the same bits as the eager calls."""
    wl = W.make("paper", n_steps=20)
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, 4096, 32, keep_defaults=True)
    pred = torch.zeros((sim.n, sim.M), dtype=torch.float32, device="cuda")
    sim.run(wl.seed)
    sim.regress_alive(0, pred=pred, want_coef=False)
    torch.cuda.synchronize()
    ref = pred.clone()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            sim.run(wl.seed, stream=s)
            sim.regress_alive(0, pred=pred, stream=s, want_coef=False)
    torch.cuda.synchronize()
    pred.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(pred, ref)
    sim.close()
