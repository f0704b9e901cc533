"""The run-time-shape outer kernels (outer_generic.cu): any number of economies and
counterparties (constant and CIR intensities in any order) and up to 6 portfolios.
On a compiled shape they give the compiled kernels' bits; on a shape with no compiled
instantiation they match the FP64 oracle at the parity tolerances."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_17005_gb300 import workload as W
from tests.gpu_helpers import CVA0_RTOL, compare_all_targets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2211_17005_gb300 import api as A, build
    build.build()
    oracle.build()
    return A


def _views(sim):
    return [v.clone() for v in (sim.features(), sim.discount_integral(), sim.thresholds(), sim.exposures(),
                                sim.mtm(), sim.targets(), sim.defaults())]


@pytest.mark.parametrize("name,M", [("paper", 1000), ("small", 777), ("batched", 513)])
def test_generic_kernels_give_the_compiled_bits(api, name, M):
    from paper_2211_17005_gb300 import _native as nat
    wl = W.make(name, M=M, N=16, n_steps=20 if name != "small" else 50)
    out = []
    for generic in (False, True):
        sim = api.Simulation(wl.model, wl.portfolios, wl.grid, M, wl.N, keep_defaults=True, keep_exposures=True,
                             generic=generic)
        sim.run(wl.seed)
        torch.cuda.synchronize()
        out.append(_views(sim))
        sim.close()
    for a, b in zip(*out):
        assert torch.equal(a, b)


def test_mixed_shape_matches_the_oracle(api):
    """E = 3, C = 5 (constant, CIR, constant, CIR, CIR), four portfolios: no compiled
    instantiation exists for this shape."""
    wl = W.make("mixed", M=1531, N=24)
    n = wl.grid.n_steps
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, wl.N, keep_defaults=True, keep_exposures=True)
    assert sim.F == 8 and sim.n_pf == 4
    sim.run(wl.seed)
    torch.cuda.synchronize()
    feats, idx = sim.features().cpu().numpy(), sim.defaults().cpu().numpy()
    thr, mtm, xi = sim.thresholds().cpu().numpy(), sim.mtm().cpu().numpy(), sim.targets().cpu().numpy()
    eps = oracle.exp_clocks(wl.seed, 0, wl.M, wl.N, wl.model.C)
    for p, pf in enumerate(wl.portfolios):
        o = oracle.simulate(wl.model, pf, wl.grid, 0, wl.M, wl.N, wl.seed,
                            want=("features", "I0", "Lambda", "mtm", "idx", "xi_bar"))
        if p == 0:
            np.testing.assert_allclose(feats, o["features"], rtol=0, atol=2e-6)
            np.testing.assert_allclose(thr, -np.expm1(-o["Lambda"]), rtol=2e-6, atol=1e-9)
        gross = np.sum(np.abs(pf.notional))
        np.testing.assert_allclose(mtm[p], o["mtm"], rtol=0, atol=2e-6 * gross)
        cva0_or, _, _ = compare_all_targets(xi[p], o, wl.model.recovery, idx, o["Lambda"], eps, n)
        assert sim.cva0(p)[0] == pytest.approx(cva0_or, rel=CVA0_RTOL)
    # the least squares of every (portfolio, date) in one grouped launch
    pred, _ = sim.regress_portfolios("linear")
    assert torch.isfinite(pred[:, 1:n]).all()
    sim.close()


@pytest.mark.parametrize("ckpt", [10, 3])
def test_generic_adjoint_matches_the_oracle_gradient(api, ckpt):
    """The run-time-shape adjoint on the mixed model (E = 3; C = 5 with constant, CIR,
    constant, CIR, CIR intensities) against the oracle's FP64 forward-mode gradient
    on the same 128 paths: 3E - 1 + 3C = 23 components, those of the constant
    intensities' kappa, theta and nu exactly 0 on both sides."""
    from oracle import dual
    wl = W.make("mixed", M=128, n_steps=20)
    pf = api.frozen(wl.model, wl.portfolios[1])
    c0, g = api.grad_cva0(wl.model, pf, wl.grid, wl.M, wl.seed, ckpt_every=ckpt)
    ref = dual.smooth_cva0_grad(wl.model, pf, wl.grid, wl.M, wl.seed)
    assert c0 == pytest.approx(ref["cva0"], rel=1e-5)
    r = ref["grad"]
    assert g.shape == r.shape == (23,)
    const = [c for c in range(wl.model.C) if wl.model.cir_nu[c] == 0.0]
    E, C = wl.model.E, wl.model.C
    for c in const:
        for base in (3 * E - 1, 3 * E - 1 + C, 3 * E - 1 + 2 * C):
            assert g[base + c] == 0.0 and r[base + c] == 0.0
    scale = np.max(np.abs(r))
    err = np.abs(g - r)
    assert np.all(err <= 2e-5 * np.abs(r) + 2e-6 * scale), [(int(i), g[i], r[i]) for i in np.argsort(-err)[:5]]
    c_fwd, _ = api.grad_cva0(wl.model, pf, wl.grid, wl.M, wl.seed, forward_only=True)
    assert c_fwd == pytest.approx(c0, rel=1e-6)
