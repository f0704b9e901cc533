"""Pins of the FP64 MLP oracle (NN+ of eq. (e:nnp), Algorithms 1 and 2)."""
import numpy as np
import pytest

from oracle import mlp
from paper_2211_17005_gb300 import workload as W


def _data(M=300, d=5, seed=0):
    rng = np.random.default_rng(seed)
    Z = rng.normal(size=(M, d))
    y = np.maximum(Z @ rng.normal(size=d), 0) * 0.3 + 0.05 * rng.normal(size=M) + 0.1
    return Z, y


@pytest.mark.parametrize("pos", [0, 1])
def test_backprop_matches_central_differences(pos):
    Z, y = _data()
    p = W.mlp_init(5, 8, seed=3)
    p["mu"] = np.array(0.05)
    g = mlp.grads(p, Z, y, pos)
    h = 1e-6
    for k in mlp.NAMES:
        flat = p[k].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(p, Z, y, pos)
            flat[idx] = old - h
            lm = mlp.loss(p, Z, y, pos)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert g[k].reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), (k, idx)


def test_last_layer_refit_solves_its_normal_equations():
    Z, y = _data()
    p = W.mlp_init(5, 8, seed=4)
    p["mu"] = np.array(0.02)
    mlp.refit_last_layer(p, Z, y)
    g = mlp.grads(p, Z, y, 0)
    assert np.max(np.abs(g["w3"])) < 1e-10 and abs(float(g["b3"])) < 1e-10
    # and it cannot be improved by any other (w3, b3)
    l0 = mlp.loss(p, Z, y, 0)
    rng = np.random.default_rng(1)
    for _ in range(5):
        q = {k: v.copy() for k, v in p.items()}
        q["w3"] = q["w3"] + 1e-3 * rng.normal(size=q["w3"].shape)
        assert mlp.loss(q, Z, y, 0) >= l0


def test_adam_first_step_and_bias_correction():
    p = {k: np.zeros(3) for k in mlp.NAMES}
    g = {k: np.array([2.0, -0.5, 1e-3]) for k in mlp.NAMES}
    opt = mlp.Adam(p, lr=1e-3)
    opt.step(p, g)
    # after one step the bias-corrected ratio is g / |g| (up to eps)
    np.testing.assert_allclose(p["W1"], -1e-3 * np.sign(g["W1"]), rtol=1e-4)


def test_base_alg_learns_and_keeps_the_best():
    Z, y = _data(M=1024, seed=2)
    p0 = W.mlp_init(5, 16, seed=5)
    trace = []
    best_p, best = mlp.base_alg(p0, Z, y, n_batches=8, epochs=8, lr=1e-2, trace=trace)
    assert best == pytest.approx(min(trace))
    assert best == pytest.approx(mlp.loss(best_p, Z, y, 1))
    assert best < 0.5 * mlp.loss(p0, Z, y, 1)
    assert len(trace) == 8


def test_batches_partition_the_paths():
    sl = mlp.batches(1000, 32)
    idx = np.concatenate([np.arange(1000)[s] for s in sl])
    np.testing.assert_array_equal(idx, np.arange(1000))


def test_bf16_rounding_and_rounded_gradient():
    # bfloat16 keeps 8 significand bits, ties to even
    assert mlp.bf16(1.0) == 1.0
    assert mlp.bf16(1.0 + 2 ** -8) == 1.0            # tie -> even
    assert mlp.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6
    x = np.random.default_rng(0).normal(size=1000)
    assert np.max(np.abs(mlp.bf16(x) - x) / np.abs(x)) <= 2 ** -8
    Z, y = _data()
    p = W.mlp_init(5, 8, seed=3)
    g, g16 = mlp.grads(p, Z, y, 0), mlp.grads_bf16(p, Z, y, 0)
    for k in mlp.NAMES:
        assert np.linalg.norm(g[k] - g16[k]) <= 0.05 * np.linalg.norm(g[k]) + 1e-12
