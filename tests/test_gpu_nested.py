"""Nested Monte Carlo reference (the benchmark of the paper's experiments) built from
twin copies, and the relative RMSE measure of its comparison, against plain
recomputation and against the FP64 oracle's copies."""
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


def test_nested_reference_is_the_mean_of_the_copies(api):
    wl = W.make("paper", M=4096, N=16)
    i, K = 50, 4
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, wl.N)
    ref = sim.nested_reference(wl.seed, i, K).cpu().numpy()
    copies = []
    for b in range(1, K + 1):
        sim.run_twin(wl.seed, i, b)
        copies.append(sim.targets()[0, i].cpu().numpy())
    sim.close()
    acc = copies[0].copy()
    for c in copies[1:]:
        acc = (acc + c).astype(np.float32)
    np.testing.assert_array_equal(ref, (acc * np.float32(1.0 / K)).astype(np.float32))


def test_nested_reference_matches_oracle(api):
    wl = W.make("small", M=2048)
    i, K = 20, 4
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, wl.N)
    g = sim.nested_reference(wl.seed, i, K).cpu().numpy()
    sim.close()
    o = np.mean([oracle.simulate(wl.model, wl.portfolios[0], wl.grid, 0, wl.M, wl.N, wl.seed, want=("xi_bar",),
                                 copy=(i, b))["xi_bar"][i] for b in range(1, K + 1)], axis=0)
    cva0 = float(oracle.simulate(wl.model, wl.portfolios[0], wl.grid, 0, wl.M, wl.N, wl.seed,
                                 want=("xi_bar",))["xi_bar"][0].mean())
    close = np.isclose(g, o, rtol=1e-4, atol=1e-4 * cva0)
    assert close.mean() >= 0.999, close.mean()   # the rest: draws moved one step by a tie
    assert g.mean() == pytest.approx(o.mean(), rel=1e-4)


def test_relative_rmse_matches_its_definition(api):
    rng = np.random.default_rng(9)
    M = 50_003
    ref = rng.gamma(2.0, 0.01, size=M).astype(np.float32)
    ref[rng.random(M) < 0.1] = 0.0
    phi = (ref * (1 + 0.1 * rng.normal(size=M))).astype(np.float32)
    val, cnt = api.relative_rmse(torch.from_numpy(phi).cuda(), torch.from_numpy(ref).cuda())
    nz = ref != 0
    e = (phi[nz].astype(np.float64) - ref[nz]) / ref[nz]
    assert cnt == int(nz.sum())
    assert val == pytest.approx(float(np.sqrt(np.mean(e * e))), rel=1e-12)
