"""Pins of the FP64 oracle of the convolutional post-correction (CPU only).

Each pin comes from outside the oracle: SciPy's 2D correlation, central
finite differences, the closed form of Adam's first step, the definition of
bfloat16 rounding, and positive homogeneity of s N(r/s).
"""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn as K


def rand_theta(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(K.NPARAM)


def test_parameter_count():
    assert K.NPARAM == 3 * 3 * 2 * 32 + 32 + 3 * 3 * 32 * 32 + 32 + 3 * 3 * 32 * 2 + 2


def test_conv_matches_scipy_correlate2d():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((7, 9, 3))
    W = rng.standard_normal((3, 3, 3, 4))
    b = rng.standard_normal(4)
    y = K.conv3x3(x, W, b)
    for co in range(4):
        ref = b[co] + sum(correlate2d(x[:, :, ci], W[:, :, ci, co], mode="same", boundary="fill")
                          for ci in range(3))
        assert np.allclose(y[:, :, co], ref, rtol=0, atol=1e-12)


def test_conv_offset_convention():
    """A single tap W[0, 2] (dy = -1, dx = +1) reads x[i-1, j+1]."""
    x = np.zeros((5, 5, 1))
    x[1, 3, 0] = 1.0
    W = np.zeros((3, 3, 1, 1))
    W[0, 2, 0, 0] = 1.0
    y = K.conv3x3(x, W, np.zeros(1))
    assert y[2, 2, 0] == 1.0 and np.count_nonzero(y) == 1


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    theta = rand_theta(3)
    rs = [rng.standard_normal((6, 5)) + 1j * rng.standard_normal((6, 5)) for _ in range(2)]
    es = [rng.standard_normal((6, 5)) + 1j * rng.standard_normal((6, 5)) for _ in range(2)]
    L, g = K.loss_and_grad(theta, rs, es)
    idx = rng.choice(K.NPARAM, 40, replace=False)
    idx = np.concatenate([idx, [K.NPARAM - 1, K.NPARAM - 2, 3 * 3 * 2 * 32]])   # b3 and b1 entries
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (K.loss_and_grad(tp, rs, es)[0] - K.loss_and_grad(tm, rs, es)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_residual_gradient_matches_central_differences():
    """The residual loss through a complex symmetric A (a random one here)."""
    rng = np.random.default_rng(12)
    theta = rand_theta(13)
    n = 5
    M = rng.standard_normal((n * n, n * n)) + 1j * rng.standard_normal((n * n, n * n))
    M = M + M.T
    apply_A = lambda z: (M @ z.ravel()).reshape(n, n)
    xs = [rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) for _ in range(2)]
    rhos = [rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) for _ in range(2)]
    L, g = K.residual_loss_and_grad(theta, xs, rhos, apply_A)
    idx = np.concatenate([rng.choice(K.NPARAM, 30, replace=False), [K.NPARAM - 1, K.NPARAM - 2]])
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (K.residual_loss_and_grad(tp, xs, rhos, apply_A)[0] - K.residual_loss_and_grad(tm, xs, rhos, apply_A)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_adam_first_step_closed_form():
    """After one step m_hat = g and v_hat = g^2, so each parameter moves by
    lr * g / (|g| + eps): -lr sign(g) up to eps."""
    rng = np.random.default_rng(4)
    theta = rng.standard_normal(50)
    g = rng.standard_normal(50)
    opt = K.Adam(50, lr=0.01)
    t1 = opt.step(theta, g)
    assert np.allclose(t1 - theta, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=0)
    assert np.allclose(np.abs(t1 - theta), 0.01, rtol=1e-5)


def test_bf16_rounding_definition():
    one = 1.0
    assert K.to_bf16(one + 2.0 ** -8) == 1.0                     # tie -> even (1.0)
    assert K.to_bf16(one + 3 * 2.0 ** -8) == one + 2.0 ** -6      # tie -> even mantissa
    assert K.to_bf16(one + 2.0 ** -7) == one + 2.0 ** -7          # representable
    assert K.to_bf16(-3.0) == -3.0
    x = np.random.default_rng(5).standard_normal(1000)
    assert np.all(np.abs(K.to_bf16(x) - x) <= np.abs(x) * 2.0 ** -8)


def test_correction_is_positively_homogeneous():
    rng = np.random.default_rng(6)
    theta = rand_theta(7)
    r = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    c1 = K.correction(theta, r)
    c2 = K.correction(theta, 3.5 * r)
    assert np.allclose(c2, 3.5 * c1, rtol=1e-12, atol=1e-12)
    assert np.all(K.correction(theta, 0 * r) == 0)


def test_planted_transposed_tap_fails_the_scipy_pin():
    """A plausible indexing mistake (taps transposed) is caught by the pin."""
    rng = np.random.default_rng(8)
    x = rng.standard_normal((6, 6, 1))
    W = rng.standard_normal((3, 3, 1, 1))
    wrong = K.conv3x3(x, W.transpose(1, 0, 2, 3), np.zeros(1))
    ref = correlate2d(x[:, :, 0], W[:, :, 0, 0], mode="same")
    assert not np.allclose(wrong[:, :, 0], ref)


def test_planted_relu_mask_mistake_fails_the_gradient_pin():
    """Dropping the ReLU derivative in the backward pass is caught by the
    finite-difference pin (restated here with the mistake planted)."""
    rng = np.random.default_rng(9)
    theta = rand_theta(10)
    r = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
    e = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
    s = K.rms(r)
    o, c = K.forward(theta, K.image(r, s))
    do = 2.0 * (o - K.image(e, s)) / 25
    dh2, _, _ = K.conv3x3_backward(c["h2"], c["W3"], do)
    _, gW2_wrong, _ = K.conv3x3_backward(c["h1"], c["W2"], dh2)      # mask dropped
    _, g = K.loss_and_grad(theta, [r], [e])
    gW2 = K.unpack(g)["W2"]
    assert not np.allclose(gW2_wrong, gW2, rtol=1e-3, atol=1e-9)
