"""Pins for the oracle of the learned warm start: back-propagation against
central finite differences, the loss's sign invariance and zero set, the Adam
step's closed form on its first step, and the BF16 rounding against torch."""
import numpy as np
import pytest

from oracle import learned


def small_net(seed=0, n_in=8, h=(6, 5), n_vec=2):
    rng = np.random.default_rng(seed)
    dims = (n_in, h[0], h[1], n_vec * n_in)
    w_off, b_off, o = [], [], 0
    for l in range(3):
        w_off.append(o)
        o += dims[l] * dims[l + 1]
        b_off.append(o)
        o += dims[l + 1]
    params = rng.normal(0, 0.5, size=o)
    return dims, w_off, b_off, params


def test_gradient_matches_finite_differences():
    dims, w_off, b_off, params = small_net()
    rng = np.random.default_rng(1)
    x = rng.normal(size=(5, dims[0]))
    t = rng.normal(size=(5, dims[3]))
    # no BF16 rounding for the check: differentiate the exact function
    orig = learned.bf16_round
    learned.bf16_round = lambda a: np.asarray(a, dtype=np.float64)
    try:
        loss, g = learned.gradients(params, dims, w_off, b_off, x, t, n_vec=2)
        eps = 1e-6
        for i in rng.choice(params.size, size=40, replace=False):
            pp, pm = params.copy(), params.copy()
            pp[i] += eps
            pm[i] -= eps
            fp, _ = learned.gradients(pp, dims, w_off, b_off, x, t, n_vec=2)
            fm, _ = learned.gradients(pm, dims, w_off, b_off, x, t, n_vec=2)
            fd = (fp - fm) / (2 * eps)
            assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    finally:
        learned.bf16_round = orig


def test_loss_sign_invariant_and_zero_at_target():
    rng = np.random.default_rng(2)
    t = rng.normal(size=(3, 2 * 7))
    l0, d0 = learned.loss_and_grad(t, t, n_vec=2)
    assert l0 == pytest.approx(0.0, abs=1e-12) and np.abs(d0).max() < 1e-12
    flip = t.reshape(3, 2, 7) * np.array([1.0, -1.0])[None, :, None]
    l1, d1 = learned.loss_and_grad(flip.reshape(3, -1), t, n_vec=2)
    assert l1 == pytest.approx(0.0, abs=1e-12) and np.abs(d1).max() < 1e-12
    p = rng.normal(size=(3, 14))
    la, _ = learned.loss_and_grad(p, t, 2)
    lb, _ = learned.loss_and_grad(p, -t, 2)
    assert la == pytest.approx(lb, rel=1e-14)
    # the value is min(||p - t||^2, ||p + t||^2) averaged over samples and vectors
    P, T = p.reshape(3, 2, 7), t.reshape(3, 2, 7)
    ref = np.minimum(((P - T) ** 2).sum(-1), ((P + T) ** 2).sum(-1)).mean()
    assert la == pytest.approx(ref, rel=1e-13)


def test_adam_first_step_closed_form():
    # step 1: m_hat = g and v_hat = g^2, so the update is lr * g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    w = np.array([1.0, 2.0, 3.0, 4.0])
    w1, m, v = learned.adam_step(w, g, np.zeros(4), np.zeros(4), step=1, lr=0.01)
    np.testing.assert_allclose(w1, w - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    a = np.concatenate([rng.normal(0, 10, 1000), [0.0, -0.0, 1.0, 1.00390625, 1.0078125, 3.14159, -2.5e-3]])
    a = a.astype(np.float32)
    ref = torch.tensor(a).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(learned.bf16_round(a), ref)


def test_features_shift_invariant():
    rng = np.random.default_rng(4)
    S = np.exp(rng.normal(0, 3, size=(4, 64)))
    f1 = learned.features(S)
    f2 = learned.features(S * 123.4)                 # a constant factor drops out
    np.testing.assert_allclose(f1, f2, atol=1e-12)
    assert np.abs(f1.mean(axis=1)).max() < 1e-12     # no clamping at this spread


def test_output_weight_is_normalised_sqrt_S():
    # w = sqrt(S / sum S) recovered from the features (no clamping at this spread)
    rng = np.random.default_rng(5)
    S = np.exp(rng.normal(0, 2, size=(3, 64)))
    w = learned.out_weight(learned.features(S))
    np.testing.assert_allclose(w, np.sqrt(S / S.sum(axis=1, keepdims=True)), rtol=1e-12)


def test_forward_hand_computed():
    # 2 -> 2 -> 2 -> 2 network with small integer weights (exact in BF16), worked by hand:
    #   x = (1, 1):  h1 = relu((3, 0) + (0.5, -3)) = (3.5, 0)
    #                h2 = relu((3.5, 7) + (-1, 1)) = (2.5, 8)
    #                o  = (5 - 8, 8) + (1, -2)     = (-2, 6)
    #                w  = (1/sqrt 2, 1/sqrt 2)      (equal inputs: equal S)
    #   x = (0, 1):  h1 = (2.5, 0), h2 = (1.5, 6), o = (-2, 4),
    #                w  = sqrt((e^-8, 1) / (1 + e^-8))
    W1 = np.array([[1.0, -1.0], [2.0, 1.0]])
    b1 = np.array([0.5, -3.0])
    W2 = np.array([[1.0, 2.0], [3.0, -1.0]])
    b2 = np.array([-1.0, 1.0])
    W3 = np.array([[2.0, 0.0], [-1.0, 1.0]])
    b3 = np.array([1.0, -2.0])
    params = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])
    dims, w_off, b_off = (2, 2, 2, 2), [0, 6, 12], [4, 10, 16]
    Ws, bs = learned.unpack(params, dims, w_off, b_off)
    x = np.array([[1.0, 1.0], [0.0, 1.0]])
    h1, h2, y = learned.forward(Ws, bs, x)
    np.testing.assert_array_equal(h1, [[3.5, 0.0], [2.5, 0.0]])
    np.testing.assert_array_equal(h2, [[2.5, 8.0], [1.5, 6.0]])
    e8 = np.exp(-8.0)
    ref = np.array([[-2.0 / np.sqrt(2.0), 6.0 / np.sqrt(2.0)],
                    [-2.0 * np.sqrt(e8 / (1.0 + e8)), 4.0 * np.sqrt(1.0 / (1.0 + e8))]])
    np.testing.assert_allclose(y, ref, rtol=1e-15, atol=0)


def test_forward_rounds_activations_to_bf16():
    # identity layers: the activations are the BF16 roundings of the inputs, worked by hand:
    # 1/3 = 0x3EAAAAAB -> 0x3EAB = 0.333984375, 0.1 = 0x3DCCCCCD -> 0x3DCD = 0.10009765625
    eye = np.eye(2)
    params = np.concatenate([eye.ravel(), np.zeros(2)] * 3)
    dims, w_off, b_off = (2, 2, 2, 2), [0, 6, 12], [4, 10, 16]
    Ws, bs = learned.unpack(params, dims, w_off, b_off)
    x = np.array([[1.0 / 3.0, 0.1]])
    h1, h2, y = learned.forward(Ws, bs, x)
    np.testing.assert_array_equal(h1, [[0.333984375, 0.10009765625]])
    np.testing.assert_array_equal(h2, h1)
    np.testing.assert_allclose(y, h1 * learned.out_weight(x), rtol=1e-15)
