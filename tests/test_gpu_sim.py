"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs. Run on a GB300: python -m pytest tests -m gpu."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_17005_gb300 import workload as W
from tests.gpu_helpers import CVA0_RTOL, compare_all_targets, compare_defaults, compare_targets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2211_17005_gb300 import api as A, build
    build.build()
    oracle.build()
    return A


def _run_pair(api, wl, M, k0=0, n_threads=0):
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, M, wl.N, keep_defaults=True,
                         keep_exposures=True)
    sim.run(wl.seed, k0=k0)
    torch.cuda.synchronize()
    g = {"features": sim.features().cpu().numpy(), "disc": sim.discount_integral().cpu().numpy(),
         "thr": sim.thresholds().cpu().numpy(), "mtm": sim.mtm()[0].cpu().numpy(),
         "expo": sim.exposures()[0].cpu().numpy(), "idx": sim.defaults().cpu().numpy(),
         "xi": sim.targets()[0].cpu().numpy(), "cva0": sim.cva0(0)}
    o = oracle.simulate(wl.model, wl.portfolios[0], wl.grid, k0, k0 + M, wl.N, wl.seed,
                        want=("features", "I0", "Lambda", "mtm", "idx", "xi_bar"), n_threads=n_threads)
    o["eps"] = oracle.exp_clocks(wl.seed, k0, k0 + M, wl.N, wl.model.C)
    sim.close()
    return g, o


def _check_pair(g, o, wl, mtm_atol):
    n = wl.grid.n_steps
    np.testing.assert_allclose(g["features"], o["features"], rtol=0, atol=2e-6)
    np.testing.assert_allclose(g["disc"], o["I0"], rtol=0, atol=1e-6)
    np.testing.assert_allclose(g["thr"], -np.expm1(-o["Lambda"]), rtol=2e-6, atol=1e-9)
    gross = np.sum(np.abs(wl.portfolios[0].notional))
    np.testing.assert_allclose(g["mtm"], o["mtm"], rtol=0, atol=mtm_atol * gross)
    # every path and CVA_0 at full tolerance: on a tie-mismatched draw the oracle's
    # target is rebuilt at the GPU's default step (from the oracle's own exposures)
    cva0_or, n_mism, n_tie = compare_all_targets(g["xi"], o, wl.model.recovery, g["idx"], o["Lambda"], o["eps"], n)
    assert g["cva0"][0] == pytest.approx(cva0_or, rel=CVA0_RTOL)
    if n_mism == 0:
        assert cva0_or == float(o["xi_bar"][0].mean())
    return n_mism, n_tie


def test_philox_bits_equal_oracle(api):
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2 ** 32, size=(2048, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:16, 0] = np.arange(16)
    ctr[:16, 1:] = 0
    ctr[16:32] = [[k, 7, 0, (1 << 24) | 3] for k in range(16)]    # simulation layout
    seed = 0x0123456789ABCDEF
    out = api.philox4x32_10(torch.from_numpy(ctr.view(np.int32)).cuda(), seed).cpu().numpy().view(np.uint32)
    ref = np.array([oracle.philox4x32_10(c, (seed & 0xFFFFFFFF, seed >> 32)) for c in ctr], dtype=np.uint32)
    np.testing.assert_array_equal(out, ref)


def test_small_workload_full_size(api):
    """The small workload at its full size (M=16384, N=8, 50 steps)."""
    wl = W.make("small")
    g, o = _run_pair(api, wl, wl.M)
    _check_pair(g, o, wl, mtm_atol=2e-6)


def test_paper_workload_prefix(api):
    """Paper-shaped model (27 factors, 8 CIR counterparties, 500 swaps) on a path prefix."""
    wl = W.make("paper")
    g, o = _run_pair(api, wl, 384)
    _check_pair(g, o, wl, mtm_atol=2e-6)


def test_path_range_gives_the_same_paths(api):
    """Counters are keyed by the global path index: a shard [k0, k0+M) equals the oracle
    there and equals the same slice of a larger run (bit for bit)."""
    wl = W.make("paper", N=16)
    g, o = _run_pair(api, wl, 200, k0=1000)
    _check_pair(g, o, wl, mtm_atol=2e-6)
    big = api.Simulation(wl.model, wl.portfolios, wl.grid, 1300, wl.N)
    big.run(wl.seed)
    part = api.Simulation(wl.model, wl.portfolios, wl.grid, 200, wl.N)
    part.run(wl.seed, k0=1000)
    torch.cuda.synchronize()
    assert torch.equal(big.targets()[..., 1000:1200], part.targets())
    assert torch.equal(big.features()[..., 1000:1200], part.features())


@pytest.mark.parametrize("M,N,n,S", [(1, 1, 50, 1), (1000, 1, 50, 1), (333, 37, 10, 3), (130, 300, 50, 1)])
def test_edge_shapes_small_model(api, M, N, n, S):
    """Single path, N = 1 (the plain i.i.d. scheme), a ragged M, sub-steps, large N."""
    wl = W.make("small", M=M, N=N, n_steps=n, substeps=S)
    g, o = _run_pair(api, wl, M)
    _check_pair(g, o, wl, mtm_atol=2e-6)


def test_paper_full_size_sampled_paths(api):
    """At the full paper size (M=2^17, N=64, the benchmark's launch), sampled outer paths
    equal the oracle run on those paths alone."""
    wl = W.make("paper")
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, wl.N, keep_defaults=True)
    sim.run(wl.seed)
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    ks = np.sort(rng.choice(wl.M, size=24, replace=False))
    ks[-1] = wl.M - 1
    xi = sim.targets()[0][:, torch.from_numpy(ks).cuda()].cpu().numpy()
    feat = sim.features()[:, :, torch.from_numpy(ks).cuda()].cpu().numpy()
    idx = sim.defaults()[torch.from_numpy(ks).cuda()].cpu().numpy()
    for t, k in enumerate(ks):
        o = oracle.simulate(wl.model, wl.portfolios[0], wl.grid, int(k), int(k) + 1, wl.N, wl.seed,
                            want=("features", "Lambda", "idx", "xi_bar"))
        eps = oracle.exp_clocks(wl.seed, int(k), int(k) + 1, wl.N, wl.model.C)
        np.testing.assert_allclose(feat[:, :, t], o["features"][:, :, 0], rtol=0, atol=2e-6)
        o["mtm"], o["I0"] = None, None
        skip, _, _ = compare_defaults(idx[t:t + 1], o["idx"], o["Lambda"], eps, wl.grid.n_steps)
        if not skip[0]:
            compare_targets(xi[:, t:t + 1], o["xi_bar"], skip, float(o["xi_bar"][0, 0]) + 1e-12)
        else:   # a tie moved a draw: compare with the oracle's target at the GPU's default step
            o = oracle.simulate(wl.model, wl.portfolios[0], wl.grid, int(k), int(k) + 1, wl.N, wl.seed,
                                want=("Lambda", "I0", "mtm", "idx", "xi_bar"))
            compare_all_targets(xi[:, t:t + 1], o, wl.model.recovery, idx[t:t + 1], o["Lambda"], eps,
                                wl.grid.n_steps)
    sim.close()


def test_rerun_is_bitwise_deterministic(api):
    wl = W.make("paper", M=4096)
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, wl.N)
    sim.run(wl.seed)
    a = sim.targets().clone()
    sim.run(wl.seed)
    assert torch.equal(a, sim.targets())
    sim.run(wl.seed + 1)
    assert not torch.equal(a, sim.targets())


def test_cva0_reduction_matches_fp64(api):
    rng = np.random.default_rng(0)
    x = rng.lognormal(-5, 1, size=1_000_003).astype(np.float32)
    m, se = api.cva0(torch.from_numpy(x).cuda())
    x64 = x.astype(np.float64)
    assert m == pytest.approx(x64.mean(), rel=1e-13)
    assert se == pytest.approx(x64.std(ddof=1) / np.sqrt(x.size), rel=1e-9)


def test_invalid_shape_fails_loudly(api):
    from paper_2211_17005_gb300._native import CvaError
    wl = W.make("small")
    with pytest.raises(CvaError):
        api.Simulation(wl.model, wl.portfolios, W.Grid(5.0, 300, 1), 16, 2)
