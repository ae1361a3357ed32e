"""Pins of the U-Net oracle (learned preconditioner) against independent
facts: a library 2-D correlation, adjoint (dot-product) identities of every
operation, central finite differences of the whole network, the first Adam
step, exact reproduction of linear functions by the bilinear resampler, and
the bfloat16 rounding rule (round to nearest, ties to even)."""
import numpy as np
import pytest

from oracle import unet as ou

signal = pytest.importorskip("scipy.signal")


def test_conv3x3_is_channel_sum_of_library_correlations():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((3, 7, 9))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    got = ou.conv3x3(X, W, b)
    for o in range(4):
        ref = b[o] + sum(signal.correlate2d(X[c], W[o, c], mode="same", boundary="fill") for c in range(3))
        assert np.allclose(got[o], ref, atol=1e-12)


def test_conv_adjoints_dot_product():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((3, 6, 10))
    W = rng.standard_normal((5, 3, 3, 3))
    Y = rng.standard_normal((5, 6, 10))
    zero = np.zeros(5)
    dX, dW, db = ou.conv3x3_backward(X, W, Y)
    lhs = np.sum(ou.conv3x3(X, W, zero) * Y)
    assert np.isclose(lhs, np.sum(X * dX), rtol=1e-12)     # adjoint in X
    assert np.isclose(lhs, np.sum(W * dW), rtol=1e-12)     # adjoint in W (linear in W)
    assert np.allclose(db, Y.sum(axis=(1, 2)))
    W1 = rng.standard_normal((5, 3, 1, 1))
    dX1, dW1, _ = ou.conv1x1_backward(X, W1, Y)
    lhs1 = np.sum(ou.conv1x1(X, W1, zero) * Y)
    assert np.isclose(lhs1, np.sum(X * dX1)) and np.isclose(lhs1, np.sum(W1 * dW1))


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((2, 8, 12))
    Yp = rng.standard_normal((2, 4, 6))
    assert np.isclose(np.sum(ou.avgpool2(X) * Yp), np.sum(X * ou.avgpool2_backward(Yp)))
    Xs = rng.standard_normal((2, 4, 6))
    Yu = rng.standard_normal((2, 8, 12))
    assert np.isclose(np.sum(ou.upsample2(Xs) * Yu), np.sum(Xs * ou.upsample2_backward(Yu)))
    assert np.allclose(ou.avgpool2(ou.upsample2(Xs)), Xs)


@pytest.mark.parametrize("levels", [2, 3])
def test_network_gradient_matches_finite_differences(levels):
    rng = np.random.default_rng(3 + levels)
    H, W = 8, 12
    params = ou.init_params(levels, 3, 5, 3, seed=10 + levels)
    params = [(Wt, rng.standard_normal(b.shape) * 0.1) for Wt, b in params]
    x = rng.standard_normal((5, H, W))
    R = rng.standard_normal((3, H, W))
    y, cache = ou.forward(params, x, levels)
    grads, dx = ou.backward(cache, R, levels)
    eps = 1e-6
    for trial in range(4):
        dP = [(rng.standard_normal(Wt.shape), rng.standard_normal(b.shape)) for Wt, b in params]
        dxd = rng.standard_normal(x.shape)
        plus = [(Wt + eps * a, b + eps * c) for (Wt, b), (a, c) in zip(params, dP)]
        minus = [(Wt - eps * a, b - eps * c) for (Wt, b), (a, c) in zip(params, dP)]
        fp = np.sum(ou.forward(plus, x + eps * dxd, levels)[0] * R)
        fm = np.sum(ou.forward(minus, x - eps * dxd, levels)[0] * R)
        fd = (fp - fm) / (2 * eps)
        an = sum(np.sum(gW * a) + np.sum(gb * c) for (gW, gb), (a, c) in zip(grads, dP)) + np.sum(dx * dxd)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (trial, fd, an)


def test_mse_gradient():
    rng = np.random.default_rng(4)
    y = rng.standard_normal((8, 4, 4))
    t = rng.standard_normal((8, 4, 4))
    L, dy = ou.mse(y, t, channels=3)
    assert np.isclose(L, np.mean((y[:3] - t[:3]) ** 2))
    assert np.all(dy[3:] == 0)
    e = np.zeros_like(y)
    e[1, 2, 3] = 1e-6
    assert np.isclose((ou.mse(y + e, t, 3)[0] - ou.mse(y - e, t, 3)[0]) / 2e-6, dy[1, 2, 3], rtol=1e-6)


def test_adam_first_step_is_lr_times_sign():
    g = np.array([3.0, -0.02, 1e-3])
    p, m, v = ou.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(p, -0.01 * np.sign(g))


def test_resample_reproduces_linear_functions_and_corners():
    sh, sw = 7, 13
    yy, xx = np.meshgrid(np.arange(sh), np.arange(sw), indexing="ij")
    src = np.stack([2.0 + 0.5 * yy - 0.25 * xx, np.full((sh, sw), 3.0)])
    out = ou.resample_bilinear(src, 16, 32)
    i, j = np.meshgrid(np.arange(16), np.arange(32), indexing="ij")
    ys, xs = i * (sh - 1) / 15, j * (sw - 1) / 31
    assert np.allclose(out[0], 2.0 + 0.5 * ys - 0.25 * xs, atol=1e-12)
    assert np.allclose(out[1], 3.0)
    assert np.allclose(ou.resample_bilinear(src, sh, sw), src)


def test_bf16_rounding_rule():
    spacing = 2.0 ** -7                           # bfloat16 spacing in [1, 2)
    vals = np.array([1.0, 1 + spacing / 2, 1 + 1.5 * spacing, 1 + 0.75 * spacing, -3.0, 0.0])
    want = np.array([1.0, 1.0, 1 + 2 * spacing, 1 + spacing, -3.0, 0.0])
    assert np.array_equal(ou.bf16(vals), want)
    x = np.random.default_rng(5).standard_normal(1000)
    assert np.max(np.abs(ou.bf16(x) - x) / np.abs(x)) <= 2.0 ** -8    # unit roundoff, 8-bit significand


def test_features_masks_are_normalised():
    x, z = np.meshgrid(np.linspace(0, 1000, 21), np.linspace(0, 500, 11))
    f = ou.features(np.full(x.shape, 2000.0), np.full(x.shape, 3000.0), np.full(x.shape, 1700.0), x, z,
                    [(500.0, 10.0)], [(0.0, 0.0), (1000.0, 0.0)], 200.0)
    assert f.shape == (5,) + x.shape
    assert np.isclose(f[3].max(), 1.0) and np.isclose(f[4].max(), 1.0)
    assert np.allclose(f[0], 3000.0 / 4700.0)
