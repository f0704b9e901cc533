"""Batching: six portfolios of uneven size on one simulation, all (portfolio, date)
regressions in one grouped launch, a CUDA graph of simulate + regress, and the
autotuned tile shapes."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_17005_gb300 import workload as W
from tests.gpu_helpers import compare_all_targets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2211_17005_gb300 import api as A, build
    build.build()
    oracle.build()
    return A


@pytest.mark.parametrize("form", [1, 0, 4])
def test_six_portfolios_and_grouped_regression_match_oracle(api, form):
    """Every pricing form (constant memory, shared memory, tensor cores) against the oracle."""
    wl = W.make("batched", M=1024, N=16, n_steps=20)
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, wl.N, keep_defaults=True)
    sim.set_tiles(128, 128 if form == 0 else 256, 0, 2432, form)
    sim.run(wl.seed)
    pred, coef = sim.regress_portfolios("linear", want_coef=True)
    pred = pred.cpu().numpy()
    xi = sim.targets().cpu().numpy()
    idx = sim.defaults().cpu().numpy()
    n = wl.grid.n_steps
    for p, pf in enumerate(wl.portfolios):
        o = oracle.simulate(wl.model, pf, wl.grid, 0, wl.M, wl.N, wl.seed,
                            want=("features", "Lambda", "I0", "mtm", "idx", "xi_bar"))
        eps = oracle.exp_clocks(wl.seed, 0, wl.M, wl.N, wl.model.C)
        cva0, _, _ = compare_all_targets(xi[p], o, wl.model.recovery, idx, o["Lambda"], eps, n)
        for i in range(1, n):
            _, p_or = oracle.lsq(oracle.linear_features(o["features"][i]), o["xi_bar"][i])
            assert np.sqrt(np.mean((pred[p, i] - p_or) ** 2)) <= 1e-3 * cva0, (p, i)
    # the shared normal matrix gives each portfolio its own coefficients
    assert not np.allclose(coef[0, 5], coef[1, 5])
    sim.close()


def test_cuda_graph_replay_equals_eager(api):
    wl = W.make("batched", M=4096, N=32, n_steps=20)
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, wl.N)
    pred = torch.zeros((sim.n_pf, sim.n, sim.M), dtype=torch.float32, device="cuda")
    sim.run(wl.seed)
    sim.regress_portfolios("linear", pred=pred)       # eager: allocates the scratch
    torch.cuda.synchronize()
    ref_t = sim.targets().clone()
    ref_p = pred.clone()
    pred.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            sim.run(wl.seed, stream=s)
            sim.regress_portfolios("linear", pred=pred, stream=s)
    torch.cuda.synchronize()
    sim.targets().zero_()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(sim.targets(), ref_t)
    assert torch.equal(pred, ref_p)
    sim.close()


def test_autotune_keeps_results(api):
    wl = W.make("batched", M=8192, N=32, n_steps=20)
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, wl.N)
    sim.run(wl.seed)
    ref_t = sim.targets().clone()
    ref_p, _ = sim.regress_portfolios("linear")
    ref_p = ref_p.clone()
    choice = sim.autotune(wl.seed, "linear")
    assert choice["sim_block"] in (64, 128) and choice["price_block"] in (128, 256)
    assert choice["inner_paths_per_block"] in (2, 4, 8)
    assert choice["portfolios_per_price_block"] in (0, 1, 2, 3, 4)
    sim.run(wl.seed)
    p, _ = sim.regress_portfolios("linear")
    torch.cuda.synchronize()
    if choice["portfolios_per_price_block"] != 4:
        assert torch.equal(sim.targets(), ref_t)      # tile shapes do not change any path
    else:   # the tensor-core pricing rounds the MtM differently: targets to the parity tolerance
        from oracle.compare import target_errors
        for pf in range(sim.n_pf):
            rt = ref_t[pf].cpu().numpy().astype(np.float64)
            e = target_errors(sim.targets()[pf].cpu().numpy(), rt, float(rt[0].mean()))
            assert e["worst_vs_tolerance"] <= 1.0, (pf, e)
    scale = float(ref_p.abs().max())
    assert float((p - ref_p).abs().max()) <= 1e-4 * scale
    again = sim.autotune(wl.seed, "linear")
    assert again["cached"] is True
    sim.close()


@pytest.mark.parametrize("name,M,ppb", [("batched", 8192, 0), ("batched", 8192, 1), ("batched", 8192, 2),
                                        ("batched", 8192, 3), ("batched", 8191, 0), ("paper", 4099, 0),
                                        ("small", 1001, 0)])
def test_pricing_portfolio_groups_bit_identical(api, name, M, ppb):
    """Pricing 1, 2 or 3 portfolios per block (weights in constant memory), or every
    portfolio per thread for two paths (weights in shared memory, ppb = 0), changes no
    exposure, MtM or target bit; ragged M leaves the last thread with one path."""
    wl = W.make(name, M=M, N=32, n_steps=20 if name != "small" else 50)
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, wl.N, keep_exposures=True)
    sim.set_tiles(128, 256, 0, 2432, 1)
    sim.run(wl.seed)
    torch.cuda.synchronize()
    ref = [v.clone() for v in (sim.targets(), sim.exposures(), sim.mtm())]
    sim.set_tiles(64, 128, 4, 1216, ppb)
    for v in (sim.targets(), sim.exposures(), sim.mtm()):
        v.fill_(float("nan"))
    sim.run(wl.seed)
    torch.cuda.synchronize()
    for got, want in zip((sim.targets(), sim.exposures(), sim.mtm()), ref):
        assert torch.equal(got, want)
    with pytest.raises(RuntimeError):
        sim.set_tiles(64, 128, 4, 1216, 5)          # not one of 0, 1, 2, 3, 4
    sim.close()


@pytest.mark.parametrize("name,M", [("batched", 8192), ("batched", 8191), ("paper", 4099), ("small", 1001)])
def test_tensor_core_pricing_matches_the_fma_forms(api, name, M):
    """The tensor-core pricing form (TF32 head-and-tail products, FP32 accumulation) gives
    other rounding than the FMA forms: its MtM agrees with theirs to the parity tolerance
    against the oracle (2e-6 of the gross notional), and so do the targets (1e-4
    relative, floor 1e-4 CVA_0); ragged M leaves a partial last tile."""
    from oracle.compare import target_errors
    wl = W.make(name, M=M, N=32, n_steps=20 if name != "small" else 50)
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, wl.N, keep_exposures=True)
    sim.set_tiles(128, 256, 0, 2432, 1)
    sim.run(wl.seed)
    torch.cuda.synchronize()
    ref_t, ref_m = sim.targets().clone(), sim.mtm().clone()
    sim.set_tiles(128, 256, 0, 2432, 4)
    sim.targets().fill_(float("nan"))
    sim.mtm().fill_(float("nan"))
    sim.run(wl.seed)
    torch.cuda.synchronize()
    m, t = sim.mtm().cpu().numpy(), sim.targets().cpu().numpy()
    assert np.all(np.isfinite(m)) and np.all(np.isfinite(t))
    for p, pf in enumerate(wl.portfolios):
        gross = float(np.sum(np.abs(pf.notional)))
        np.testing.assert_allclose(m[p], ref_m[p].cpu().numpy(), rtol=0, atol=2e-6 * gross)
        rt = ref_t[p].cpu().numpy().astype(np.float64)
        e = target_errors(t[p], rt, float(rt[0].mean()))
        assert e["worst_vs_tolerance"] <= 1.0, (p, e)
    sim.close()
