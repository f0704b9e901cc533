"""Twin Monte Carlo validation (Sec. ss:twin, eq. (e:val1)) on the GPU against the
FP64 oracle: the twin copies (simulation branched at a pricing date, fresh
increments after it and fresh inner clocks) and the FP64 estimator."""
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


def _copy_pair(api, wl, M, date, copy):
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, M, wl.N, keep_defaults=True)
    sim.run_twin(wl.seed, date, copy)
    torch.cuda.synchronize()
    g = {"features": sim.features().cpu().numpy(), "idx": sim.defaults().cpu().numpy(),
         "xi": sim.targets()[0].cpu().numpy()}
    sim.close()
    o = oracle.simulate(wl.model, wl.portfolios[0], wl.grid, 0, M, wl.N, wl.seed,
                        want=("features", "Lambda", "I0", "mtm", "idx", "xi_bar"), copy=(date, copy))
    o["eps"] = oracle.exp_clocks(wl.seed, 0, M, wl.N, wl.model.C, copy=copy)
    return g, o


@pytest.mark.parametrize("name,M,date,copy", [("small", 16384, 20, 1), ("paper", 384, 50, 2)])
def test_twin_copy_matches_oracle(api, name, M, date, copy):
    wl = W.make(name)
    g, o = _copy_pair(api, wl, M, date, copy)
    np.testing.assert_allclose(g["features"], o["features"], rtol=0, atol=2e-6)
    compare_all_targets(g["xi"], o, wl.model.recovery, g["idx"], o["Lambda"], o["eps"], wl.grid.n_steps)


def test_twin_estimator_matches_oracle_on_the_same_inputs(api):
    rng = np.random.default_rng(5)
    M = 70_001
    phi, x1, x2 = (rng.gamma(2.0, 0.01, size=M).astype(np.float32) for _ in range(3))
    est, se = api.twin_l2(*(torch.from_numpy(v).cuda() for v in (phi, x1, x2)))
    ref, ref_se = oracle.twin_l2(phi, x1, x2)
    assert est == pytest.approx(ref, rel=1e-12, abs=1e-18)
    assert se == pytest.approx(ref_se, rel=1e-6)


def test_twin_estimate_of_the_regression_matches_oracle(api):
    """End to end on the small workload: least squares at date i from the simulation,
    two twin copies, the estimator; the oracle runs the same pipeline in FP64."""
    wl = W.make("small")
    M, i = wl.M, 20
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, M, wl.N)
    sim.run(wl.seed)
    pred, _ = sim.regress_all(0, basis="poly2")
    phi = pred[i].clone()
    xs = []
    for c in (1, 2):
        sim.run_twin(wl.seed, i, c)
        xs.append(sim.targets()[0, i].clone())
    est, se = api.twin_l2(phi, xs[0], xs[1])
    sim.close()
    o = oracle.simulate(wl.model, wl.portfolios[0], wl.grid, 0, M, wl.N, wl.seed, want=("features", "xi_bar"))
    _, phi_o = oracle.lsq(oracle.poly2_features(o["features"][i, 0]), o["xi_bar"][i])
    xo = [oracle.simulate(wl.model, wl.portfolios[0], wl.grid, 0, M, wl.N, wl.seed, want=("xi_bar",),
                          copy=(i, c))["xi_bar"][i] for c in (1, 2)]
    ref, ref_se = oracle.twin_l2(phi_o, xo[0], xo[1])
    # the two implementations agree far inside the Monte Carlo error of the estimate
    assert abs(est - ref) < 0.25 * ref_se, (est, ref, ref_se)
    assert se == pytest.approx(ref_se, rel=0.05)
