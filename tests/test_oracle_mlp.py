"""Pins of the prefetcher oracle: central finite differences of the loss,
the first Adam step's known magnitude, and bf16 rounding against bit-level
definitions."""
import numpy as np

from oracle import mlp


def _net(rng, n_in=12, h=16, n_out=10):
    return dict(W1=rng.normal(0, 0.3, (n_in, h)), b1=rng.normal(0, 0.1, h), W2=rng.normal(0, 0.3, (h, h)),
                b2=rng.normal(0, 0.1, h), W3=rng.normal(0, 0.3, (h, n_out)), b3=rng.normal(0, 0.1, n_out))


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    W = _net(rng)
    x = rng.normal(size=(7, 12))
    t = (rng.random((7, 10)) < 0.3).astype(float)
    mask = (rng.random((7, 10)) < 0.8).astype(float)
    loss, g, _ = mlp.loss_and_grads(W, x, t, mask)
    eps = 1e-6
    for k in W:
        flat = W[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = mlp.bce_with_logits(mlp.forward(W, x)["logits"], t, mask)
            flat[idx] = old - eps
            lm = mlp.bce_with_logits(mlp.forward(W, x)["logits"], t, mask)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[k].reshape(-1)[idx]) < 1e-6 * max(1, abs(fd)), (k, idx)


def test_bce_matches_definition_on_extreme_logits():
    x = np.array([[-40.0, 0.0, 40.0]])
    t = np.array([[1.0, 0.5, 0.0]])
    m = np.ones_like(x)
    # -t log s(x) - (1-t) log(1 - s(x)): 40, log 2, 40 (to double precision)
    assert abs(mlp.bce_with_logits(x, t, m) - (40 + np.log(2) + 40) / 3) < 1e-12


def test_first_adam_step_moves_by_lr():
    rng = np.random.default_rng(1)
    W = _net(rng)
    g = {k: rng.normal(size=v.shape) for k, v in W.items()}
    m = {k: np.zeros_like(v) for k, v in W.items()}
    v = {k: np.zeros_like(v) for k, v in W.items()}
    W1, _, _ = mlp.adam(W, g, m, v, 1, lr=1e-3, eps=0.0)
    for k in W:
        np.testing.assert_allclose(W[k] - W1[k], 1e-3 * np.sign(g[k]), rtol=1e-9)


def test_bf16_round_bits():
    vals = np.array([1.0, 1.00390625, 1.005859375, 3.0e38, -2.5e-3], np.float32)
    r = mlp.bf16_round(vals)
    # bf16 keeps 8 significant bits: 1 + 1/128 is representable, 1 + 1/256 ties to even (1.0)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125
    assert np.all(np.abs(r - vals) <= np.abs(vals) * 2.0 ** -8)
