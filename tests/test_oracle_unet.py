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
