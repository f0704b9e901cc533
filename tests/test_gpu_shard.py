"""Outer paths split into ranges on the GPU (paper_2211_17005_gb300.shard): two path
ranges simulated separately (their own k0), their CVA_0 partial sums and normal
matrices combined on the host, give the run of all paths at once."""
import numpy as np
import pytest
import torch

from paper_2211_17005_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2211_17005_gb300 import api as A, build
    build.build()
    return A


@pytest.mark.parametrize("name,basis,M", [("paper", "linear", 8192), ("small", "poly2", 10_001)])
def test_two_path_ranges_pool_to_the_full_run(api, name, basis, M):
    from paper_2211_17005_gb300 import _native as nat, shard
    wl = W.make(name, M=M, N=16, n_steps=20)
    full = api.Simulation(wl.model, wl.portfolios, wl.grid, M, wl.N)
    full.run(wl.seed)
    parts = []
    for r in range(2):
        k0, Mr = shard.path_range(M, r, 2)
        s = api.Simulation(wl.model, wl.portfolios, wl.grid, Mr, wl.N)
        s.run(wl.seed, k0=k0)
        parts.append(s)
    torch.cuda.synchronize()
    # the ranges are the full run's paths, bit for bit
    assert torch.equal(torch.cat([p.targets() for p in parts], dim=-1), full.targets())
    c, se = shard.combine_cva0(np.stack([shard.cva0_partial(p.targets()[0, 0]) for p in parts]))
    c_full, se_full = full.cva0(0)
    assert c == pytest.approx(c_full, rel=1e-13) and se == pytest.approx(se_full, rel=1e-9)
    b = nat.BASIS_POLY2 if basis == "poly2" else nat.BASIS_LINEAR
    nf = 1 if basis == "poly2" else wl.model.F
    scale = float(full.targets()[0].double().pow(2).mean().sqrt())
    for i in range(1, wl.grid.n_steps):
        centre = full.features()[i, :nf, 0].contiguous()          # global path 0's state, known to every range
        gram = sum(shard.regress_partial(p.targets()[0, i], p.features()[i, :nf].contiguous(), centre, basis)
                   for p in parts)
        wc, wr, nd = shard.solve(gram, nf, b, centre.cpu().numpy().astype(np.float64))
        pred = torch.cat([shard.regress_predict(p.features()[i, :nf].contiguous(), centre, wc, basis)
                          for p in parts])
        ref_pred, ref_coef = api.regress(full.targets()[0, i], full.features()[i, :nf].contiguous(), basis=basis)
        assert nd == 0
        # the same normal equations, accumulated in other chunks: FP32 runs round differently
        assert float((pred - ref_pred).double().pow(2).mean().sqrt()) <= 1e-5 * scale, i
        np.testing.assert_allclose(wr, ref_coef, rtol=1e-4, atol=1e-5 * np.abs(ref_coef).max())
    for p in parts:
        p.close()
    full.close()
