"""Seeded synthetic inputs for the shell dynamo solve (shared by tests and bench).

This module holds no arithmetic of the solver: it only samples fields at the
cell centres of a 6 x Ns x Ns x Nr equiangular cubed-sphere shell (panel p's
unit vector is M_p (1, tan xi, tan eta) / norm; panels 0..3 centred on
+x, +y, -x, -y, 4 on +z, 5 on -z) and draws random numbers.

* RNG: SplitMix64 (Steele, Lea, Flood 2014) -> uniforms in (0, 1) ->
  Box-Muller normals; `seed` selects the stream.
* Initial state (Theta = T - T0, Cartesian u and B, arrays [c][p][k][j][i]):
  Theta = 1e-2 b(r) q(x/r) / max|b q|, with b(r) = (r - r_i)(r_o - r) and q a
  random polynomial of total degree <= 3;
  u = 1e-2 curl(b(r)^2 a(x)) / max|.|, a a random degree-<=3 vector polynomial
  (divergence free, zero at both walls);
  B = B0 of the paper's benchmark initial condition (eqn:initial) plus
  1e-2 curl(b^2 a'(x)) / max|.| (pseudo-vacuum walls hold for both parts);
  P = P_b = 0.
"""
import numpy as np

_M = np.array([
    [[1, 0, 0], [0, 1, 0], [0, 0, 1]],
    [[0, -1, 0], [1, 0, 0], [0, 0, 1]],
    [[-1, 0, 0], [0, -1, 0], [0, 0, 1]],
    [[0, 1, 0], [-1, 0, 0], [0, 0, 1]],
    [[0, 0, -1], [0, 1, 0], [1, 0, 0]],
    [[0, 0, 1], [0, 1, 0], [-1, 0, 0]],
], dtype=np.float64)

RI, RO = 7.0 / 13.0, 20.0 / 13.0
_MASK64 = (1 << 64) - 1


def splitmix64(seed, n):
    """n successive SplitMix64 outputs (uint64) of the stream started at `seed`."""
    out = np.empty(n, dtype=np.uint64)
    s = seed & _MASK64
    for i in range(n):
        s = (s + 0x9E3779B97F4A7C15) & _MASK64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        out[i] = z ^ (z >> 31)
    return out


def normals(seed, n):
    """n standard normals by Box-Muller from SplitMix64 uniforms (53-bit, open interval)."""
    m = (n + 1) // 2
    u = (splitmix64(seed, 2 * m) >> np.uint64(11)).astype(np.float64)
    u = (u + 0.5) / float(1 << 53)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    z = np.concatenate([r * np.cos(2 * np.pi * u[1::2]), r * np.sin(2 * np.pi * u[1::2])])
    return z[:n]


def random_vector(n, seed):
    """Fast seeded standard-normal vector (numpy PCG64) for operator and solver inputs."""
    return np.random.default_rng(seed).standard_normal(n)


def cell_centres(Ns, Nr, ri=RI, ro=RO):
    """Cartesian cell centres, shape (3, 6, Nr, Ns, Ns)."""
    hs, hr = np.pi / (2 * Ns), (ro - ri) / Nr
    t = np.tan(-np.pi / 4 + (np.arange(Ns) + 0.5) * hs)
    r = ri + (np.arange(Nr) + 0.5) * hr
    Y, X = np.meshgrid(t, t, indexing='ij')          # [j][i]
    v = np.stack([np.ones_like(X), X, Y], -1) / np.sqrt(1 + X * X + Y * Y)[..., None]
    out = np.empty((3, 6, Nr, Ns, Ns))
    for p in range(6):
        w = v @ _M[p].T
        out[:, p] = r[None, :, None, None] * np.moveaxis(w, -1, 0)[:, None]
    return out


_MONO = [(a, b, c) for a in range(4) for b in range(4) for c in range(4) if a + b + c <= 3]


def _poly(coef, x, y, z, dx=(0, 0, 0)):
    """Polynomial sum_m coef[m] x^a y^b z^c (or one partial derivative of it)."""
    out = np.zeros_like(x)
    for cm, (a, b, c) in zip(coef, _MONO):
        e, f = [a, b, c], 1.0
        for ax in range(3):
            for _ in range(dx[ax]):
                f *= e[ax]
                e[ax] -= 1
        if f == 0.0 or min(e) < 0:
            continue
        out += cm * f * x ** e[0] * y ** e[1] * z ** e[2]
    return out


def _curl_b2a(coef3, x, y, z, ri, ro):
    """curl(b(r)^2 a(x)) = grad(b^2) x a + b^2 curl a, b = (r - ri)(ro - r)."""
    r = np.sqrt(x * x + y * y + z * z)
    b = (r - ri) * (ro - r)
    db = (ro + ri - 2 * r)
    gpsi = [2 * b * db * c / r for c in (x, y, z)]
    a = [_poly(coef3[i], x, y, z) for i in range(3)]
    d = lambda i, ax: _poly(coef3[i], x, y, z, tuple(1 if q == ax else 0 for q in range(3)))
    curl_a = [d(2, 1) - d(1, 2), d(0, 2) - d(2, 0), d(1, 0) - d(0, 1)]
    cross = [gpsi[1] * a[2] - gpsi[2] * a[1], gpsi[2] * a[0] - gpsi[0] * a[2], gpsi[0] * a[1] - gpsi[1] * a[0]]
    return np.stack([cross[c] + b * b * curl_a[c] for c in range(3)])


def benchmark_B0(x, y, z, ri=RI, ro=RO):
    """Cartesian B0 of the paper's benchmark initial condition (eqn:initial)."""
    r = np.sqrt(x * x + y * y + z * z)
    th = np.arccos(np.clip(z / r, -1, 1))
    ph = np.arctan2(y, x)
    Br = 5.0 / 8.0 * (9 * r ** 3 - 4 * (4 + 3 * (ri + ro)) * r ** 2 + (4 * ro + ri * (4 + 3 * ro)) * 6 * r
                      - 48 * ri * ro) / r * np.cos(th)
    Bt = -15.0 / 4.0 * (r - ri) * (r - ro) * (3 * r - 4) / r * np.sin(th)
    Bp = 15.0 / 8.0 * np.sin(np.pi * (r - ri)) * np.sin(2 * th)
    st, ct, sp_, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
    return np.stack([Br * st * cp + Bt * ct * cp - Bp * sp_,
                     Br * st * sp_ + Bt * ct * sp_ + Bp * cp,
                     Br * ct - Bt * st])


def initial_state(Ns, Nr, seed, amp=1e-2, ri=RI, ro=RO):
    """Seeded initial fields, flattened per component: u (3, N), T (N,), B (3, N), P, Pb."""
    X = cell_centres(Ns, Nr, ri, ro)
    x, y, z = X[0], X[1], X[2]
    r = np.sqrt(x * x + y * y + z * z)
    nm = len(_MONO)
    c = normals(seed, 7 * nm).reshape(7, nm)
    b = (r - ri) * (ro - r)
    th = b * _poly(c[0], x / r, y / r, z / r)
    th = amp * th / np.abs(th).max()
    u = _curl_b2a(c[1:4], x, y, z, ri, ro)
    u = amp * u / np.abs(u).max()
    dB = _curl_b2a(c[4:7], x, y, z, ri, ro)
    B = benchmark_B0(x, y, z, ri, ro) + amp * dB / np.abs(dB).max()
    N = x.size
    return dict(u=u.reshape(3, N), T=th.reshape(N), B=B.reshape(3, N), P=np.zeros(N), Pb=np.zeros(N))


def benchmark_Theta0(x, y, z, ri=RI, ro=RO):
    """Theta0 of the paper's benchmark initial condition (eqn:initial)."""
    r = np.sqrt(x * x + y * y + z * z)
    th = np.arccos(np.clip(z / r, -1, 1))
    ph = np.arctan2(y, x)
    s = 2 * r - ri - ro
    return 21.0 / np.sqrt(17920 * np.pi) * (1 - 3 * s ** 2 + 3 * s ** 4 - s ** 6) * np.sin(th) ** 4 * np.cos(4 * ph)


def benchmark_state(Ns, Nr, ri=RI, ro=RO):
    """The paper's benchmark initial condition (eqn:initial): u = 0, Theta0, B0; P = P_b = 0."""
    X = cell_centres(Ns, Nr, ri, ro)
    N = X[0].size
    return dict(u=np.zeros((3, N)), T=benchmark_Theta0(*X, ri, ro).reshape(N),
                B=benchmark_B0(*X, ri, ro).reshape(3, N), P=np.zeros(N), Pb=np.zeros(N))


def _edge_sequences(n, sizes):
    """All ordered sequences of edges from `sizes` summing to n, grouped by length."""
    out = {}

    def rec(rem, seq):
        if rem == 0:
            out.setdefault(len(seq), []).append(tuple(seq))
            return
        for s in sizes:
            if s <= rem:
                rec(rem - s, seq + [s])
    rec(n, [])
    return out


def uneven_boxes(Ns, Nr, sizes=(8, 12, 16, 24), target=None, seed=0):
    """An uneven decomposition of every panel into boxes with edges from `sizes`.

    Each panel's (i, j) square is cut along i and along j into seeded random edge
    sequences (Ns must be a sum of edges from `sizes`); every resulting rectangle's
    radial column is cut into its own random edge sequence.  With `target`, the
    number of radial pieces per rectangle is chosen so that the total box count is
    exactly `target`.  Returns owned boxes (panel, i0, i1, j0, j1, k0, k1) that
    tile the shell.  Input synthesis only."""
    rng = np.random.default_rng(seed)
    hseq = _edge_sequences(Ns, sizes)
    rseq = _edge_sequences(Nr, sizes)
    hlens = sorted(hseq)
    rects = []
    for p in range(6):
        li, lj = int(rng.choice(hlens)), int(rng.choice(hlens))
        ei = hseq[li][int(rng.integers(len(hseq[li])))]
        ej = hseq[lj][int(rng.integers(len(hseq[lj])))]
        ci, cj = np.concatenate([[0], np.cumsum(ei)]), np.concatenate([[0], np.cumsum(ej)])
        rects += [(p, int(ci[a]), int(ci[a + 1]), int(cj[b]), int(cj[b + 1]))
                  for a in range(len(ei)) for b in range(len(ej))]
    rlens = sorted(rseq)
    if target is None:
        counts = [int(rng.choice(rlens)) for _ in rects]
    else:
        lo, hi = rlens[0], rlens[-1]
        if not lo * len(rects) <= target <= hi * len(rects):
            raise ValueError('target %d not reachable with %d rectangles' % (target, len(rects)))
        counts = [lo] * len(rects)
        extra = target - lo * len(rects)
        order = rng.permutation(len(rects))
        while extra > 0:
            for r in order:
                if extra == 0:
                    break
                nxt = [c for c in rlens if c > counts[r]]
                if nxt and nxt[0] - counts[r] <= extra:
                    extra -= nxt[0] - counts[r]
                    counts[r] = nxt[0]
    boxes = []
    for (p, i0, i1, j0, j1), c in zip(rects, counts):
        seq = rseq[c][int(rng.integers(len(rseq[c])))]
        ck = np.concatenate([[0], np.cumsum(seq)])
        boxes += [(p, i0, i1, j0, j1, int(ck[q]), int(ck[q + 1])) for q in range(len(seq))]
    return boxes


def multiscale_fields(Ns, Nr, nsamples, seed, d=2, widths=(0.0, 0.5, 1.0, 2.0, 4.0, 8.0)):
    """nsamples random d-component fields on a 6 x Ns x Ns x Nr grid, each row of the
    result one sample laid out [c][p][k][j][i]: per sample, white noise on every
    (component, panel) block filtered by the Gaussian of a width (in cells) drawn from
    `widths` (periodic FFT filter over the block, 0 = white), scaled to unit RMS.
    Training and test inputs of the learned coarse correction."""
    rng = np.random.default_rng(seed)
    out = np.empty((nsamples, d * 6 * Nr * Ns * Ns))
    kz = np.fft.fftfreq(Nr)[:, None, None]
    ky = np.fft.fftfreq(Ns)[None, :, None]
    kx = np.fft.rfftfreq(Ns)[None, None, :]
    k2 = (2 * np.pi) ** 2 * (kz * kz + ky * ky + kx * kx)
    for s in range(nsamples):
        f = rng.standard_normal((d, 6, Nr, Ns, Ns))
        w = float(rng.choice(widths))
        if w > 0:
            f = np.fft.irfftn(np.fft.rfftn(f, axes=(2, 3, 4)) * np.exp(-0.5 * w * w * k2), s=(Nr, Ns, Ns),
                              axes=(2, 3, 4))
        out[s] = (f / np.sqrt((f * f).mean())).ravel()
    return out
