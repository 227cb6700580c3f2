"""Right-preconditioned restarted (flexible) GMRES (oracle; test infrastructure).

Paper Sec. 3.3, eqn:newlinear: A M^{-1} (M x) = b, restarted GMRES(m), stop
when ||A' x' - b|| <= max(eps_a, eps_r ||A' x'_0 - b||); with right
preconditioning A' x' - b = A x - b, the true residual.  Readings (design
notes): flexible GMRES (Z_j = M^{-1} v_j stored, x = x_0 + Z y) so that a
variable preconditioner (inner GMRES on the coarse level) is allowed;
classical Gram-Schmidt applied twice (CGS2); Givens rotations for the
least-squares problem; explicit residual recomputed at each restart.
"""
import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class GmresResult:
    x: np.ndarray
    iters: int
    converged: bool
    r0: float
    rfinal: float
    history: list = field(default_factory=list)


def fgmres(A, M, b, x0, restart=30, rtol=1e-8, atol=0.0, maxit=10000):
    """Solve A x = b; A and M are callables returning new arrays."""
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - A(x)
    beta = float(np.sqrt(r @ r))
    r0 = beta
    target = max(atol, rtol * r0)
    its = 0
    hist = [beta]
    while beta > target and its < maxit:
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        gvec = np.zeros(restart + 1)
        gvec[0] = beta
        breakdown = False
        for j in range(restart):
            z = M(V[j])
            Z.append(z)
            w = A(z)
            h = np.zeros(j + 2)
            for _ in range(2):                       # CGS2
                c = np.array([v @ w for v in V])
                for ci, v in zip(c, V):
                    w = w - ci * v
                h[:j + 1] += c
            hn = float(np.sqrt(w @ w))
            h[j + 1] = hn
            for i in range(j):                       # previous rotations
                t0 = cs[i] * h[i] + sn[i] * h[i + 1]
                h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1]
                h[i] = t0
            den = math.hypot(h[j], h[j + 1])
            cs[j], sn[j] = h[j] / den, h[j + 1] / den
            h[j], h[j + 1] = den, 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            H[:j + 2, j] = h
            its += 1
            hist.append(abs(gvec[j + 1]))
            if hn == 0.0:
                breakdown = True
            if abs(gvec[j + 1]) <= target or its >= maxit or breakdown:
                break
            V.append(w / hn)
        k = len(Z)
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):               # back substitution
            y[i] = (gvec[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        for yi, z in zip(y, Z):
            x = x + yi * z
        r = b - A(x)
        beta = float(np.sqrt(r @ r))
        hist[-1] = beta
        if breakdown:
            break
    return GmresResult(x, its, beta <= target, r0, beta, hist)
