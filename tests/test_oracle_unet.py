"""Pins of the oracle's learned-correction network: convolution against scipy, the
cubed-sphere padding against the grid geometry and its adjoint, gradients by finite
differences, Adam against closed forms."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import unet
from oracle.grid import unit_vector
from paper_2009_02171_gb300.inputs import normals


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    xp = rng.standard_normal((2, 3, 4, 8, 10))   # padded (eta, xi) planes 6 x 8
    w = rng.standard_normal((5, 3, 3, 3, 3))
    b = rng.standard_normal(5)
    out = unet.conv(xp, w, b)
    for p in range(2):
        for co in range(5):
            ref = sum(ndimage.correlate(xp[p, ci], w[co, ci], mode='constant', cval=0.0) for ci in range(3)) + b[co]
            assert np.allclose(out[p, co], ref[:, 1:-1, 1:-1], atol=1e-12)


@pytest.mark.parametrize('n', [4, 8])
def test_halo_sources_are_the_adjacent_cells(n):
    """The ring cell beyond each edge takes the neighbour cell centred about one cell width away."""
    q, jq, iq = unet.halo_map(n)
    h = np.pi / 2 / n
    c = -np.pi / 4 + (np.arange(n) + 0.5) * h
    for p in range(6):
        for side in range(4):
            for t in range(n):
                # ring cell centre: half a cell beyond the edge
                xi, eta = {0: (-np.pi / 4 - h / 2, c[t]), 1: (np.pi / 4 + h / 2, c[t]),
                           2: (c[t], -np.pi / 4 - h / 2), 3: (c[t], np.pi / 4 + h / 2)}[side]
                v = unit_vector(p, np.array(xi), np.array(eta))
                src = unit_vector(q[p, side, t], np.array(c[iq[p, side, t]]), np.array(c[jq[p, side, t]]))
                assert q[p, side, t] != p
                assert np.arccos(np.clip(v @ src, -1, 1)) < 0.75 * h


@pytest.mark.parametrize('n', [2, 4, 6])
def test_halo_map_is_symmetric_and_covers_every_edge_cell_once(n):
    q, jq, iq = unet.halo_map(n)
    count = np.zeros((6, n, n), dtype=int)
    for p in range(6):
        for side in range(4):
            for t in range(n):
                count[q[p, side, t], jq[p, side, t], iq[p, side, t]] += 1
    edge = np.zeros((n, n), dtype=int)
    edge[0, :] += 1
    edge[-1, :] += 1
    edge[:, 0] += 1
    edge[:, -1] += 1
    assert np.array_equal(count, np.broadcast_to(edge, (6, n, n)))
    # the neighbour of the neighbour across the same face is the original edge cell
    cell_of = {0: lambda t: (t, 0), 1: lambda t: (t, n - 1), 2: lambda t: (0, t), 3: lambda t: (n - 1, t)}
    for p in range(6):
        for side in range(4):
            for t in range(n):
                qq, j, i = q[p, side, t], jq[p, side, t], iq[p, side, t]
                back = [(s2, t2) for s2 in range(4) for t2 in range(n)
                        if q[qq, s2, t2] == p and (jq[qq, s2, t2], iq[qq, s2, t2]) == cell_of[side](t)
                        and cell_of[s2](t2) == (j, i)]
                assert len(back) == 1


def test_pad_adjoint():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((12, 2, 3, 4, 4))
    g = rng.standard_normal((12, 2, 3, 6, 6))
    assert np.isclose((unet.pad(a) * g).sum(), (a * unet.pad_adjoint(g)).sum())
    assert np.all(unet.pad(a)[:, :, :, 0, 0] == 0)


def test_pool_upsample_adjoint():
    rng = np.random.default_rng(6)
    a = rng.standard_normal((2, 3, 4, 6, 8))
    b = rng.standard_normal((2, 3, 2, 3, 4))
    assert np.isclose((unet.pool(a) * b).sum(), (a * unet.upsample(b)).sum() / 8)


def _small(seed, C=3, levels=2):
    params = unet.init(C, levels, normals(seed, 27 * 8 * C * C * (levels + 2)))
    for i, k in enumerate(params):  # nonzero biases so every ReLU branch is exercised
        params[k] = (params[k][0], 0.05 * np.arange(params[k][1].size) - 0.02 * i)
    return params


def test_network_is_homogeneous_per_sample():
    params = _small(7)
    r = np.random.default_rng(1).standard_normal((12, 2, 4, 4, 4))
    r2 = r.copy()
    r2[:6] *= 3.5
    r2[6:] *= 0.25
    e, e2 = unet.forward(params, r, 2), unet.forward(params, r2, 2)
    assert np.allclose(e2[:6], 3.5 * e[:6], rtol=1e-12, atol=1e-14)
    assert np.allclose(e2[6:], 0.25 * e[6:], rtol=1e-12, atol=1e-14)
    assert np.all(unet.forward(params, np.zeros_like(r), 2) == 0)


@pytest.mark.parametrize('layer', ['e0a', 'e1b', 'e2a', 'd1', 'd0', 'out'])
def test_gradients_match_finite_differences(layer):
    params = _small(3)
    rng = np.random.default_rng(2)
    r = rng.standard_normal((12, 2, 4, 4, 4))
    e = rng.standard_normal((12, 2, 4, 4, 4))
    L, grads = unet.loss_and_grads(params, r, e, 2)
    w, b = params[layer]
    h = 1e-6
    for idx in [(0, 0, 1, 1, 1), (w.shape[0] - 1, w.shape[1] - 1, 0, 2, 1), (1, 0, 2, 0, 2)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        fd = (unet.loss_and_grads(dict(params, **{layer: (wp, b)}), r, e, 2)[0] -
              unet.loss_and_grads(dict(params, **{layer: (wm, b)}), r, e, 2)[0]) / (2 * h)
        assert abs(fd - grads[layer][0][idx]) < 1e-6 * max(1.0, abs(fd)), (layer, idx, fd, grads[layer][0][idx])
    bp, bm = b.copy(), b.copy()
    bp[-1] += h
    bm[-1] -= h
    fd = (unet.loss_and_grads(dict(params, **{layer: (w, bp)}), r, e, 2)[0] -
          unet.loss_and_grads(dict(params, **{layer: (w, bm)}), r, e, 2)[0]) / (2 * h)
    assert abs(fd - grads[layer][1][-1]) < 1e-6 * max(1.0, abs(fd))


def test_flatten_round_trip_and_count():
    C, levels = 16, 3
    params = unet.init(C, levels, normals(5, 27 * C * C * 20))
    flat = unet.flatten(params)
    expect = 27 * (2 * C + C * C * (2 * levels + 1) + 2 * C * C * levels + 2 * C) + C * (2 * levels + 2 + levels) + 2
    assert flat.size == expect
    back = unet.unflatten(flat, C, levels)
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
