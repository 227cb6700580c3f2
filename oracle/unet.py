"""FP64 reference of the learned coarse correction network (oracle; test infrastructure).

Not from the paper: the project's learned stand-in for the coarse-level solve of
the two-level preconditioner.  Per cubed-sphere panel, a small 3-D U-Net maps the
coarse right-hand side r_c (2 channels: P, P_b; shape [6][2][Z][Y][X]) to a
coarse correction e_c:
  s   = ||r_c||_2 (all panels and channels; homogeneity: N(a r) = a N(r))
  a1  = relu(conv(r_c / s; 2 -> C));     a2 = relu(conv(a1; C -> C))
  p   = mean over 2x2x2 blocks of a2
  a3  = relu(conv(p; C -> 2C));          a4 = relu(conv(a3; 2C -> 2C))
  u   = a4 repeated over 2x2x2 blocks (nearest upsampling)
  a5  = relu(conv([a2, u]; 3C -> C));    y  = conv(a5; C -> 2)
  e_c = s y
conv: 3x3x3 cross-correlation, stride 1, zero padding 1 inside each panel, plus bias.
Weights W[co][ci][dz][dy][dx], bias b[co].  Loss: mean squared error of y against
t = e_c / s.  Backward pass by the chain rule, pinned by finite differences.
"""
import numpy as np

LAYERS = (('c1', 2, 1), ('c2', 1, 1), ('c3', 1, 2), ('c4', 2, 2), ('c5', 3, 1), ('c6', 1, 0))


def shapes(C):
    """(cin, cout) of the six convolutions for base width C."""
    return {'c1': (2, C), 'c2': (C, C), 'c3': (C, 2 * C), 'c4': (2 * C, 2 * C), 'c5': (3 * C, C), 'c6': (C, 2)}


def init(C, normals):
    """Weights from a stream of standard normals (He scaling), zero biases."""
    params, off = {}, 0
    for name, (ci, co) in shapes(C).items():
        n = co * ci * 27
        w = normals[off:off + n].reshape(co, ci, 3, 3, 3) * np.sqrt(2.0 / (ci * 27))
        off += n
        params[name] = (w, np.zeros(co))
    return params


def conv(x, w, b):
    """x [P][ci][Z][Y][X] -> [P][co][Z][Y][X]; 3x3x3 cross-correlation, zero padding 1."""
    P, ci, Z, Y, X = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1), (1, 1)))
    out = np.zeros((P, w.shape[0], Z, Y, X))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                out += np.einsum('oi,pizyx->pozyx', w[:, :, dz, dy, dx], xp[:, :, dz:dz + Z, dy:dy + Y, dx:dx + X])
    return out + b[None, :, None, None, None]


def conv_backward(x, w, g):
    """Gradients of sum(g * conv(x, w, b)) with respect to x, w and b."""
    P, ci, Z, Y, X = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1), (1, 1)))
    gx = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                sl = (slice(None), slice(None), slice(dz, dz + Z), slice(dy, dy + Y), slice(dx, dx + X))
                gw[:, :, dz, dy, dx] = np.einsum('pozyx,pizyx->oi', g, xp[sl])
                gx[sl] += np.einsum('oi,pozyx->pizyx', w[:, :, dz, dy, dx], g)
    return gx[:, :, 1:-1, 1:-1, 1:-1], gw, g.sum(axis=(0, 2, 3, 4))


def pool(a):
    P, C, Z, Y, X = a.shape
    return a.reshape(P, C, Z // 2, 2, Y // 2, 2, X // 2, 2).mean(axis=(3, 5, 7))


def upsample(a):
    return a.repeat(2, axis=2).repeat(2, axis=3).repeat(2, axis=4)


def forward(params, r, keep=False):
    """e_c = N(r_c); with keep=True also the activations needed by backward()."""
    s = float(np.sqrt((r * r).sum()))
    if s == 0.0:
        return (np.zeros_like(r), None) if keep else np.zeros_like(r)
    x = r / s
    a1 = np.maximum(conv(x, *params['c1']), 0)
    a2 = np.maximum(conv(a1, *params['c2']), 0)
    p = pool(a2)
    a3 = np.maximum(conv(p, *params['c3']), 0)
    a4 = np.maximum(conv(a3, *params['c4']), 0)
    cat = np.concatenate([a2, upsample(a4)], axis=1)
    a5 = np.maximum(conv(cat, *params['c5']), 0)
    y = conv(a5, *params['c6'])
    if keep:
        return s * y, dict(s=s, x=x, a1=a1, a2=a2, p=p, a3=a3, a4=a4, cat=cat, a5=a5, y=y)
    return s * y


def loss_and_grads(params, r, e):
    """MSE of y against t = e / ||r|| (mean over all entries) and its parameter gradients."""
    _, st = forward(params, r, keep=True)
    t = e / st['s']
    diff = st['y'] - t
    L = float((diff * diff).mean())
    gy = 2.0 * diff / diff.size
    grads = {}
    g5, grads['c6'] = None, None
    gx, gw, gb = conv_backward(st['a5'], params['c6'][0], gy)
    grads['c6'] = (gw, gb)
    g = gx * (st['a5'] > 0)
    gx, gw, gb = conv_backward(st['cat'], params['c5'][0], g)
    grads['c5'] = (gw, gb)
    C = st['a2'].shape[1]
    g_a2 = gx[:, :C]
    g_u = gx[:, C:]
    P, C2, Z, Y, X = g_u.shape
    g_a4 = g_u.reshape(P, C2, Z // 2, 2, Y // 2, 2, X // 2, 2).sum(axis=(3, 5, 7))
    g = g_a4 * (st['a4'] > 0)
    gx, gw, gb = conv_backward(st['a3'], params['c4'][0], g)
    grads['c4'] = (gw, gb)
    g = gx * (st['a3'] > 0)
    gx, gw, gb = conv_backward(st['p'], params['c3'][0], g)
    grads['c3'] = (gw, gb)
    g_a2 = g_a2 + upsample(gx) / 8.0
    g = g_a2 * (st['a2'] > 0)
    gx, gw, gb = conv_backward(st['a1'], params['c2'][0], g)
    grads['c2'] = (gw, gb)
    g = gx * (st['a1'] > 0)
    _, gw, gb = conv_backward(st['x'], params['c1'][0], g)
    grads['c1'] = (gw, gb)
    return L, grads


def flatten(params):
    """Flat parameter vector: layer by layer, W[co][ci][dz][dy][dx] then b[co]."""
    return np.concatenate([np.concatenate([params[k][0].ravel(), params[k][1].ravel()]) for k, _, _ in LAYERS])


def unflatten(flat, C):
    params, off = {}, 0
    for name, (ci, co) in shapes(C).items():
        n = co * ci * 27
        w = np.asarray(flat[off:off + n], dtype=np.float64).reshape(co, ci, 3, 3, 3)
        off += n
        params[name] = (w, np.asarray(flat[off:off + co], dtype=np.float64))
        off += co
    assert off == len(flat)
    return params


def adam_step(w, g, m, v, t, lr, beta1, beta2, eps):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) of flat arrays; t is the new step count (>= 1).
    Returns (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v
