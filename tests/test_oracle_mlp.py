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


# ---- the schedule of Algorithms 1 and 2 --------------------------------------
# Each pin takes the oracle module, so that tests/test_oracle_planted.py can run
# it on copies of the module with a mistake planted in the schedule.

def pin_refit_at_half_the_epochs(m=mlp):
    """Algorithm 1 refits the output layer once, at epoch floor(E/2). With a zero
    step size Adam leaves the parameters where they are, so the full-sample loss
    after each epoch is flat except for one drop, and that drop is at epoch
    floor(E/2) (E = 8 and E = 5)."""
    Z, y = _data(M=1024, seed=6)
    for E in (8, 5):
        trace = []
        m.base_alg(W.mlp_init(5, 8, seed=5), Z, y, n_batches=4, epochs=E, lr=0.0, trace=trace)
        t = np.asarray(trace)
        drops = [e + 1 for e in range(E) if e > 0 and t[e] < t[e - 1] * (1 - 1e-9)]
        assert drops == [E // 2], (E, t)
        assert np.all(np.abs(np.diff(t[E // 2 - 1:])) <= 1e-12 * t[0]), (E, t)
        assert np.all(np.abs(np.diff(t[:E // 2 - 1])) <= 1e-12 * t[0]), (E, t)


def pin_output_relu_after_the_refit(m=mlp):
    """NN+ switches its output ReLU on after the refit (pos = 1). With every target
    equal to c < mu the refit fits y - mu exactly with zeta = c - mu < 0 at every
    sample; from then on the output is relu(zeta) + mu = mu, the ReLU blocks every
    gradient except mu's, and mu's gradient 2 (mu - c) keeps its sign, so each Adam
    step moves mu by about lr towards c and the full-sample loss (mu - c)^2 falls
    by about lr per step in its square root. Without the ReLU the refitted output
    already equals the targets and nothing is left to learn."""
    rng = np.random.default_rng(0)
    M, nb, E, lr, c = 1024, 16, 4, 1e-3, -2.0
    Z = rng.normal(size=(M, 5))
    y = np.full(M, c)
    p0 = W.mlp_init(5, 8, seed=5)
    p0["mu"] = np.array(0.0)
    trace = []
    best_p, _ = m.base_alg(p0, Z, y, n_batches=nb, epochs=E, lr=lr, trace=trace)
    s = np.sqrt(np.asarray(trace))
    moved = s[E // 2 - 1] - s[-1]
    expect = (E - E // 2) * nb * lr
    assert 0.8 * expect < moved < 1.05 * expect, (moved, expect, trace)
    _, (_, _, zeta) = m.forward(best_p, Z, 1)
    assert np.all(zeta < 0)


def _dated(seed, M=512, d=5):
    r = np.random.default_rng(seed)
    X = r.normal(size=(d, M))
    y = np.maximum(X.T @ r.normal(size=d), 0) * 0.3 + 0.1 + 0.05 * r.normal(size=M)
    return X, y


def _backward(m, replace=None):
    feats = {i: _dated(10 + i)[0] for i in (1, 2, 3)}
    targs = {i: _dated(10 + i)[1] for i in (1, 2, 3)}
    if replace is not None:
        feats[replace], targs[replace] = _dated(99)
    return m.backward_alg(W.mlp_init(5, 8, seed=7), feats, targs, dates=[1, 2, 3], n_batches=4, epochs=4, lr=1e-2)


def _same(a, b):
    return all(np.array_equal(a[0][k], b[0][k]) for k in mlp.NAMES) and np.array_equal(a[2], b[2])


def pin_backward_learning_runs_dates_downwards(m=mlp):
    """Algorithm 2 trains the last date first and moves back in time: a date's fit
    depends on its own data and the dates after it, never on earlier dates. New
    data at date 1 leaves dates 2 and 3 bit for bit unchanged."""
    base, other = _backward(m), _backward(m, replace=1)
    assert _same(base[3], other[3]) and _same(base[2], other[2])
    assert not _same(base[1], other[1])


def pin_backward_learning_warm_starts(m=mlp):
    """Algorithm 2 starts each date from the parameters learnt at the date after it:
    the few Adam steps of a date do not forget their starting point, so new data at
    date 3 changes the network learnt at date 1."""
    base, other = _backward(m), _backward(m, replace=3)
    gap = max(float(np.max(np.abs(base[1][0][k] - other[1][0][k]))) for k in mlp.NAMES)
    assert gap > 1e-3, gap


def test_refit_at_half_the_epochs():
    pin_refit_at_half_the_epochs()


def test_output_relu_after_the_refit():
    pin_output_relu_after_the_refit()


def test_backward_learning_runs_dates_downwards():
    pin_backward_learning_runs_dates_downwards()


def test_backward_learning_warm_starts():
    pin_backward_learning_warm_starts()
