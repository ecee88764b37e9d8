"""Pins of the FP64 seed-network oracle (oracle.mlp) against facts that do
not come from its own code: finite differences of the loss, the closed-form
Adam step under a constant gradient, the bfloat16 conversion of PyTorch and
hand-rounded values, a network built by hand to compute x0 + x1, and the
round trip between the seed and the training target."""
import numpy as np
import pytest

from oracle import mlp
from paper_2511_11425_gb300 import inputs


def _random_weights(seed=3, scale=0.5):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, mlp.NPARAM)


def test_parameter_count_and_layout():
    assert mlp.NPARAM == 4 * 32 + 32 + 32 * 32 + 32 + 32 + 1
    w = np.arange(mlp.NPARAM, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(w)
    assert W1[0, 1] == 1 and b1[0] == 128 and W2[0, 0] == 160 and W2[1, 0] == 192
    assert b2[0] == 1184 and W3[0] == 1216 and b3 == 1248
    assert np.array_equal(mlp.pack(W1, b1, W2, b2, W3, b3), w)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(7)
    w = _random_weights()
    X = rng.normal(0.0, 1.0, (64, 4))
    y = rng.normal(0.0, 1.0, 64)
    _, g = mlp.loss_and_grad(w, X, y)
    eps = 1e-6
    idx = np.concatenate([np.arange(0, 160, 7), np.arange(160, 1216, 37), np.arange(1216, 1249)])
    for k in idx:
        wp = w.copy(); wp[k] += eps
        wm = w.copy(); wm[k] -= eps
        fd = (mlp.loss_and_grad(wp, X, y)[0] - mlp.loss_and_grad(wm, X, y)[0]) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_loss_is_the_mean_squared_error_of_forward():
    rng = np.random.default_rng(8)
    w = _random_weights(5)
    X = rng.normal(0.0, 1.0, (33, 4))
    y = rng.normal(0.0, 1.0, 33)
    loss, _ = mlp.loss_and_grad(w, X, y)
    assert abs(loss - np.mean((mlp.forward(w, X) - y) ** 2)) < 1e-12 * max(1.0, loss)


def test_adam_moves_lr_per_step_under_a_constant_gradient():
    # with a constant gradient g the bias-corrected moments are exactly g and
    # g^2, so every step is -lr g / (|g| + eps)
    g = np.array([3.0, -0.25, 1e-3, 0.0])
    w = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    lr = 0.01
    for t in range(1, 6):
        w, m, v = mlp.adam_step(w, g, m, v, t, lr)
        assert np.allclose(w, -t * lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_bf16_rounding_matches_torch_and_hand_values():
    torch = pytest.importorskip("torch")
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0                 # tie, even mantissa kept
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie, rounds up to even
    assert mlp.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert mlp.bf16(-2.5) == -2.5
    rng = np.random.default_rng(11)
    x = (rng.normal(0.0, 1.0, 100000) * np.exp(rng.normal(0.0, 5.0, 100000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)


def test_hand_built_network_computes_x0_plus_x1():
    W1 = np.zeros((32, 4)); W2 = np.zeros((32, 32)); W3 = np.zeros(32)
    W1[0, 0], W1[1, 0], W1[2, 1], W1[3, 1] = 1, -1, 1, -1
    for k in range(4):
        W2[k, k] = 1.0
    W3[:4] = [1, -1, 1, -1]
    w = mlp.pack(W1, np.zeros(32), W2, np.zeros(32), W3, 0.25)
    rng = np.random.default_rng(2)
    X = rng.normal(0.0, 3.0, (100, 4))
    assert np.allclose(mlp.forward(w, X), X[:, 0] + X[:, 1] + 0.25, rtol=0, atol=1e-12)
    # exactly representable inputs pass the bfloat16 path unchanged
    Xb = np.round(X * 4) / 4
    assert np.allclose(mlp.infer_bf16(w, Xb), Xb[:, 0] + Xb[:, 1] + 0.25, rtol=0, atol=1e-12)


def test_bf16_inference_is_within_the_rounding_bound():
    rng = np.random.default_rng(4)
    w = _random_weights(9, 0.3)
    X = rng.normal(0.0, 1.0, (500, 4))
    ref = mlp.forward(w, X)
    got = mlp.infer_bf16(w, X)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(w)
    # each of the three roundings is relative 2^-9; bound by the layer scale
    scale = np.abs(np.maximum(np.maximum(X @ W1.T + b1, 0) @ W2.T + b2, 0)) @ np.abs(W3) + 1.0
    assert np.all(np.abs(got - ref) <= 8 * 2.0 ** -9 * scale * 4)
    assert np.mean(np.abs(got - ref)) < 0.02 * np.mean(np.abs(ref))


def test_untrained_network_outputs_zero_and_seed_target_round_trip():
    w = inputs.mlp_init(5)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(w)
    assert np.all(W3 == 0) and b3 == 0 and np.abs(W1).max() <= np.sqrt(6 / 4)
    rng = np.random.default_rng(1)
    X = rng.normal(0.0, 1.0, (50, 4))
    assert np.all(mlp.forward(w, X) == 0.0)
    h = rng.uniform(0.5, 2.0, 50)
    h_new = h * np.exp(rng.normal(0.0, 0.05, 50))
    y = mlp.target(h_new, h, X)
    assert np.allclose(mlp.seed(h, X, y), h_new, rtol=1e-12)
    # the untrained network gives the continuity estimate h exp(dt divv / 3)
    divv = rng.normal(0, 3, 50)
    X = mlp.features(0.01, divv, np.full(50, 64), 64.0, h, h, 0.0)
    assert np.all(X[:, 1:] == 0.0)
    assert np.allclose(mlp.seed(h, X, np.zeros(50)), h * np.exp(0.01 * divv / 3), rtol=1e-12)
    # a particle at rest (both estimates below the tolerance) ignores the network
    Xr = np.array([[1e-5, 0.3, -2e-5, 0.1], [1e-3, 0.3, 0.0, 0.1]])
    assert np.allclose(mlp.seed(np.ones(2), Xr, np.array([5.0, 5.0]), tol=1e-6),
                       [np.exp(1e-7), np.exp(1e-5 + 0.05)], rtol=1e-14)
    # corrections inside the dead zone are dropped, larger ones kept whole
    assert np.allclose(mlp.seed(np.ones(2), Xr, np.array([5.0, 5.0]), dead=0.06),
                       [np.exp(1e-7), np.exp(1e-5)], rtol=1e-14)
    assert np.allclose(mlp.seed(np.ones(2), Xr, np.array([5.0, 5.0]), dead=0.04),
                       [np.exp(1e-7), np.exp(1e-5 + 0.05)], rtol=1e-14)


def test_training_fits_a_smooth_target():
    rng = np.random.default_rng(6)
    X = rng.uniform(-1.0, 1.0, (512, 4))
    y = 2.0 * np.sin(2.0 * X[:, 0]) + X[:, 1] * X[:, 2] - 0.5 * X[:, 3]
    w0 = inputs.mlp_init(1)
    w, losses = mlp.train(w0, X, y, 600, 3e-3)
    assert losses[-1] < 0.03 * losses[0]
