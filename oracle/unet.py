"""FP64 reference of the learned coarse correction network (oracle; test infrastructure).

Not from the paper: the project's learned stand-in for the coarse-level solve of
the two-level preconditioner (eqn:coarsesolve).  A cubed-sphere U-Net maps the
coarse right-hand side r_c (2 channels: P, P_b; array [6 nb][2][Z][Y][X] with Z
radial, Y = eta, X = xi cells of each panel) to a coarse correction e_c.

Cubed-sphere padding: before every 3x3x3 convolution each panel is padded by one
cell in xi and eta with the values of the neighbouring panel's cells across the
edge (the cell sharing the edge face: `Grid.pair` of the oracle grid), zero at
the four ring corners; radially the padding is zero.  The convolution is then
a valid cross-correlation in (eta, xi) and a zero-padded one radially, plus a
bias.  Weights W[co][ci][dz][dy][dx], bias b[co].

Network with `levels` = L poolings and width C:
  s = RMS of r_c (per sample of 6 panels);  a = r_c / s
  level l = 0..L:  (l > 0: a = 2x2x2 mean pooling of E_{l-1})
                   A_l = relu(conv_{e l a}(pad a));  E_l = relu(conv_{e l b}(pad A_l))
  D_L = E_L;  level l = L-1..0:  D_l = relu(conv_{d l}(pad [E_l, up(D_{l+1})]))
  y = conv_out(pad D_0);  e_c = s y
(up = nearest upsampling by 2; channels: e0a 2 -> C, every other e C -> C,
d 2C -> C, out C -> 2.)  Loss: mean squared error of y against t = e_c / s.
The backward pass applies the chain rule, with the adjoint of the padding
(ring values scattered back to the neighbour cells they came from); it is pinned
by finite differences.
"""
from functools import lru_cache

import numpy as np

from oracle.grid import ETA_MAX, ETA_MIN, XI_MAX, XI_MIN, Grid


def layer_shapes(C, levels):
    """Ordered {name: (cin, cout)} of the convolutions (the flat parameter order)."""
    sh = {}
    for l in range(levels + 1):
        sh['e%da' % l] = (2 if l == 0 else C, C)
        sh['e%db' % l] = (C, C)
    for l in range(levels - 1, -1, -1):
        sh['d%d' % l] = (2 * C, C)
    sh['out'] = (C, 2)
    return sh


def init(C, levels, normals):
    """Weights from a stream of standard normals (He scaling), zero biases."""
    params, off = {}, 0
    for name, (ci, co) in layer_shapes(C, levels).items():
        n = co * ci * 27
        params[name] = (normals[off:off + n].reshape(co, ci, 3, 3, 3) * np.sqrt(2.0 / (ci * 27)), np.zeros(co))
        off += n
    return params


def flatten(params):
    """Flat parameter vector: layer by layer in layer_shapes order, W[co][ci][dz][dy][dx] then b[co]."""
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params.values()])


def unflatten(flat, C, levels):
    params, off = {}, 0
    for name, (ci, co) in layer_shapes(C, levels).items():
        n = co * ci * 27
        w = np.asarray(flat[off:off + n], dtype=np.float64).reshape(co, ci, 3, 3, 3)
        off += n
        params[name] = (w, np.asarray(flat[off:off + co], dtype=np.float64))
        off += co
    assert off == len(flat)
    return params


@lru_cache(maxsize=None)
def halo_map(n):
    """Neighbour cells across each panel edge of an n x n panel grid.

    Returns (q, jq, iq) arrays of shape [6][4][n]: the ring cell beyond `side` of
    panel p at tangential index t takes the value of cell (jq, iq) of panel q, the
    cell on the other side of the same edge face."""
    # face pairing of a 4n x 4n grid (the geometry needs >= 3 cells a side), coarsened:
    # face t of the n-grid is faces 4t .. 4t+3 of the fine one
    g = Grid(4 * n, 2)
    q = np.zeros((6, 4, n), dtype=np.int64)
    jq, iq = np.zeros_like(q), np.zeros_like(q)
    for p in range(6):
        for side in range(4):
            qq, sq, tmap, _ = g.pair[p][side]
            for t in range(n):
                tt = tmap[4 * t] // 4
                q[p, side, t] = qq
                if sq == XI_MIN:
                    jq[p, side, t], iq[p, side, t] = tt, 0
                elif sq == XI_MAX:
                    jq[p, side, t], iq[p, side, t] = tt, n - 1
                elif sq == ETA_MIN:
                    jq[p, side, t], iq[p, side, t] = 0, tt
                else:
                    jq[p, side, t], iq[p, side, t] = n - 1, tt
    return q, jq, iq


def _ring(side, n):
    """(y, x) index arrays of the ring cells beyond `side` in the padded (n+2) x (n+2) plane."""
    t = np.arange(n)
    if side == XI_MIN:
        return t + 1, np.zeros(n, dtype=np.int64)
    if side == XI_MAX:
        return t + 1, np.full(n, n + 1)
    if side == ETA_MIN:
        return np.zeros(n, dtype=np.int64), t + 1
    return np.full(n, n + 1), t + 1


def pad(a):
    """[6 nb][C][Z][n][n] -> [6 nb][C][Z][n+2][n+2] with the cubed-sphere ring (corners zero)."""
    P, C, Z, n, _ = a.shape
    q, jq, iq = halo_map(n)
    out = np.zeros((P, C, Z, n + 2, n + 2))
    out[:, :, :, 1:-1, 1:-1] = a
    for P0 in range(0, P, 6):
        for p in range(6):
            for side in range(4):
                y, x = _ring(side, n)
                out[P0 + p][:, :, y, x] = a[P0 + q[p, side], :, :, jq[p, side], iq[p, side]].transpose(1, 2, 0)
    return out


def pad_adjoint(g):
    """Adjoint of pad: interior plus the ring values added to the cells they were copied from."""
    P, C, Z, n2, _ = g.shape
    n = n2 - 2
    q, jq, iq = halo_map(n)
    out = g[:, :, :, 1:-1, 1:-1].copy()
    for P0 in range(0, P, 6):
        for p in range(6):
            for side in range(4):
                y, x = _ring(side, n)
                for t in range(n):
                    out[P0 + q[p, side, t], :, :, jq[p, side, t], iq[p, side, t]] += g[P0 + p, :, :, y[t], x[t]]
    return out


def conv(xp, w, b):
    """Padded input [P][ci][Z][n+2][n+2] -> [P][co][Z][n][n]: valid in (eta, xi), zero-padded radially."""
    P, ci, Z, Y2, X2 = xp.shape
    Y, X = Y2 - 2, X2 - 2
    xz = np.pad(xp, ((0, 0), (0, 0), (1, 1), (0, 0), (0, 0)))
    out = np.zeros((P, w.shape[0], Z, Y, X))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                out += np.einsum('oi,pizyx->pozyx', w[:, :, dz, dy, dx], xz[:, :, dz:dz + Z, dy:dy + Y, dx:dx + X])
    return out + b[None, :, None, None, None]


def conv_backward(xp, w, g):
    """Gradients of sum(g * conv(xp, w, b)) with respect to xp (padded, ring included), w and b."""
    P, ci, Z, Y2, X2 = xp.shape
    Y, X = Y2 - 2, X2 - 2
    xz = np.pad(xp, ((0, 0), (0, 0), (1, 1), (0, 0), (0, 0)))
    gx = np.zeros_like(xz)
    gw = np.zeros_like(w)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                sl = (slice(None), slice(None), slice(dz, dz + Z), slice(dy, dy + Y), slice(dx, dx + X))
                gw[:, :, dz, dy, dx] = np.einsum('pozyx,pizyx->oi', g, xz[sl])
                gx[sl] += np.einsum('oi,pozyx->pizyx', w[:, :, dz, dy, dx], g)
    return gx[:, :, 1:-1], gw, g.sum(axis=(0, 2, 3, 4))


def pool(a):
    P, C, Z, Y, X = a.shape
    return a.reshape(P, C, Z // 2, 2, Y // 2, 2, X // 2, 2).mean(axis=(3, 5, 7))


def upsample(a):
    return a.repeat(2, axis=2).repeat(2, axis=3).repeat(2, axis=4)


def _down_sum(g):
    P, C, Z, Y, X = g.shape
    return g.reshape(P, C, Z // 2, 2, Y // 2, 2, X // 2, 2).sum(axis=(3, 5, 7))


def forward(params, r, levels, keep=False):
    """e_c = N(r_c) per sample of 6 panels (r: [6 nb][2][Z][n][n]); keep=True also returns the cache."""
    P = r.shape[0]
    s = np.sqrt((r.reshape(P // 6, -1) ** 2).mean(axis=1))            # RMS per sample
    sp = np.repeat(s, 6)[:, None, None, None, None]
    x = np.where(sp > 0, r / np.where(sp > 0, sp, 1.0), 0.0)
    c = {'s': sp, 'in': [], 'A': [], 'E': [], 'cat': [], 'D': {}}
    a = x
    for l in range(levels + 1):
        if l > 0:
            a = pool(c['E'][l - 1])
        c['in'].append(a)
        A = np.maximum(conv(pad(a), *params['e%da' % l]), 0)
        E = np.maximum(conv(pad(A), *params['e%db' % l]), 0)
        c['A'].append(A)
        c['E'].append(E)
    d = c['E'][levels]
    for l in range(levels - 1, -1, -1):
        cat = np.concatenate([c['E'][l], upsample(d)], axis=1)
        c['cat'].append(cat)
        d = np.maximum(conv(pad(cat), *params['d%d' % l]), 0)
        c['D'][l] = d
    y = conv(pad(d), *params['out'])
    c['y'] = y
    e = sp * y
    return (e, c) if keep else e


def loss_and_grads(params, r, e, levels):
    """MSE of y against t = e / s (mean over all entries) and its parameter gradients."""
    _, c = forward(params, r, levels, keep=True)
    sp = c['s']
    t = np.where(sp > 0, e / np.where(sp > 0, sp, 1.0), 0.0)
    diff = c['y'] - t
    L = float((diff * diff).mean())
    gy = 2.0 * diff / diff.size
    grads = {}
    gxp, gw, gb = conv_backward(pad(c['D'][0]), params['out'][0], gy)
    grads['out'] = (gw, gb)
    gd = pad_adjoint(gxp) * (c['D'][0] > 0)
    gE = [np.zeros_like(E) for E in c['E']]
    C = c['E'][0].shape[1]
    # decoder in reverse order of the forward pass: l = 0 .. levels-1
    cats = {l: c['cat'][levels - 1 - l] for l in range(levels)}
    for l in range(levels):
        gxp, gw, gb = conv_backward(pad(cats[l]), params['d%d' % l][0], gd)
        grads['d%d' % l] = (gw, gb)
        gcat = pad_adjoint(gxp)
        gE[l] += gcat[:, :C]
        gnext = _down_sum(gcat[:, C:])
        if l + 1 < levels:
            gd = gnext * (c['D'][l + 1] > 0)
        else:
            gE[levels] += gnext
    for l in range(levels, -1, -1):
        g = gE[l] * (c['E'][l] > 0)
        gxp, gw, gb = conv_backward(pad(c['A'][l]), params['e%db' % l][0], g)
        grads['e%db' % l] = (gw, gb)
        g = pad_adjoint(gxp) * (c['A'][l] > 0)
        gxp, gw, gb = conv_backward(pad(c['in'][l]), params['e%da' % l][0], g)
        grads['e%da' % l] = (gw, gb)
        if l > 0:
            gE[l - 1] += upsample(pad_adjoint(gxp)) / 8.0
    return L, {k: grads[k] for k in params}


def adam_step(w, g, m, v, t, lr, beta1, beta2, eps):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) of flat arrays; t is the new step count (>= 1).
    Returns (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v
