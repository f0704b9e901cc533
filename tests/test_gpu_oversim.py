"""Prop. 1 statistics (Sec. ss:choice1) on the GPU against the FP64 oracle: Q_i and R_i
from the first two inner draws of every path, for the same regression predictions."""
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


@pytest.mark.parametrize("name,M,basis", [("small", 16384, "poly2"), ("paper", 384, "linear")])
def test_prop1_statistics_match_oracle(api, name, M, basis):
    wl = W.make(name, M=M)
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, M, wl.N)
    sim.run(wl.seed)
    pred, _ = sim.regress_all(0, basis=basis)
    Qg, Rg = sim.oversim_stats(pred, wl.seed)
    pred_h = pred.cpu().numpy().astype(np.float64)
    sim.close()
    o = oracle.simulate(wl.model, wl.portfolios[0], wl.grid, 0, M, wl.N, wl.seed, want=("idx", "mtm", "I0"))
    Qo, Ro = oracle.oversim_stats(o, wl.model.recovery, pred_h)
    n = wl.grid.n_steps
    assert Qg[0] == 0 and Rg[0] == 0
    live = Qo[1:n] > 0
    assert live.sum() >= (n - 1) // 2
    np.testing.assert_allclose(Qg[1:n][live], Qo[1:n][live], rtol=3e-3)
    assert np.all(np.abs(Rg[1:n] - Ro[1:n]) <= 3e-3 * np.maximum(np.abs(Ro[1:n]), 1e-2 * Qo[1:n]) + 1e-30)
