"""Pins of the oracle's learned-correction network: convolution against scipy, gradients by finite differences."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import unet
from paper_2009_02171_gb300.inputs import normals


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 4, 6, 8))
    w = rng.standard_normal((5, 3, 3, 3, 3))
    b = rng.standard_normal(5)
    out = unet.conv(x, w, b)
    for p in range(2):
        for co in range(5):
            ref = sum(ndimage.correlate(x[p, ci], w[co, ci], mode='constant', cval=0.0) for ci in range(3)) + b[co]
            assert np.allclose(out[p, co], ref, atol=1e-12)


def test_network_is_homogeneous_of_degree_one():
    C = 4
    params = unet.init(C, normals(7, 200000))
    r = np.random.default_rng(1).standard_normal((6, 2, 4, 4, 4))
    assert np.allclose(unet.forward(params, 3.5 * r), 3.5 * unet.forward(params, r), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize('layer', ['c1', 'c3', 'c5', 'c6'])
def test_gradients_match_finite_differences(layer):
    C = 3
    params = unet.init(C, normals(3, 200000))
    for k in params:  # nonzero biases so every ReLU branch is exercised
        params[k] = (params[k][0], 0.05 * np.arange(params[k][1].size))
    rng = np.random.default_rng(2)
    r = rng.standard_normal((2, 2, 4, 4, 4))
    e = rng.standard_normal((2, 2, 4, 4, 4))
    L, grads = unet.loss_and_grads(params, r, e)
    w, b = params[layer]
    h = 1e-6
    for idx in [(0, 0, 1, 1, 1), (w.shape[0] - 1, w.shape[1] - 1, 0, 2, 1)]:
        wp = w.copy(); wp[idx] += h
        wm = w.copy(); wm[idx] -= h
        Lp = unet.loss_and_grads(dict(params, **{layer: (wp, b)}), r, e)[0]
        Lm = unet.loss_and_grads(dict(params, **{layer: (wm, b)}), r, e)[0]
        assert abs((Lp - Lm) / (2 * h) - grads[layer][0][idx]) < 1e-6 * max(1.0, abs(grads[layer][0][idx]))
    bp = b.copy(); bp[0] += h
    bm = b.copy(); bm[0] -= h
    fd = (unet.loss_and_grads(dict(params, **{layer: (w, bp)}), r, e)[0] -
          unet.loss_and_grads(dict(params, **{layer: (w, bm)}), r, e)[0]) / (2 * h)
    assert abs(fd - grads[layer][1][0]) < 1e-6 * max(1.0, abs(fd))


def test_flatten_round_trip_and_count():
    params = unet.init(16, normals(5, 200000))
    flat = unet.flatten(params)
    C = 16
    expect = 27 * (2 * C + C * C + C * 2 * C + 4 * C * C + 3 * C * C + 2 * C) + (C + C + 2 * C + 2 * C + C + 2)
    assert flat.size == expect
    back = unet.unflatten(flat, C)
    for k in params:
        assert np.array_equal(back[k][0], params[k][0]) and np.array_equal(back[k][1], params[k][1])


def test_adam_constant_gradient_moves_lr_per_step():
    # with bias correction, a constant gradient g gives mhat = g and vhat = g^2 at every step
    rng = np.random.default_rng(4)
    g = rng.standard_normal(50)
    w0 = rng.standard_normal(50)
    w, m, v = w0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 6):
        w, m, v = unet.adam_step(w, g, m, v, t, 1e-2, 0.9, 0.999, 1e-8)
    assert np.allclose(w, w0 - 5 * 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)


def test_adam_two_steps_worked_example():
    # g1 = 1, g2 = -3 with beta1 = 0.5, beta2 = 0.75, lr = 0.1, eps = 0:
    # m2 = 0.5 * 0.5 + 0.5 * -3 = -1.25, mhat2 = -1.25 / 0.75; v2 = 0.75 * 0.25 + 0.25 * 9 = 2.4375, vhat2 = 2.4375 / 0.4375
    w = np.array([0.0])
    w, m, v = unet.adam_step(w, np.array([1.0]), np.zeros(1), np.zeros(1), 1, 0.1, 0.5, 0.75, 0.0)
    assert np.allclose(w, [-0.1])
    w, m, v = unet.adam_step(w, np.array([-3.0]), m, v, 2, 0.1, 0.5, 0.75, 0.0)
    assert np.allclose(w, [-0.1 - 0.1 * (-1.25 / 0.75) / np.sqrt(2.4375 / 0.4375)])


def test_pool_upsample_adjoint():
    # <pool(a), b> = <a, upsample(b)> / 8: the pooling's adjoint used by the backward pass
    rng = np.random.default_rng(6)
    a = rng.standard_normal((2, 3, 4, 6, 8))
    b = rng.standard_normal((2, 3, 2, 3, 4))
    assert np.isclose((unet.pool(a) * b).sum(), (a * unet.upsample(b)).sum() / 8)
