"""Diagnostics of the paper's results section (oracle; test infrastructure).

* L2 error (Sec. 4.1): sqrt(sum_l sum_ijk sum_c (v - v_ref)^2 V_ijk).
* Alfven CFL number (Sec. 4.2): CFL_A = max(|v_A^1/h_s| + |v_A^2/h_s| +
  |v_A^3/h_r|) dt, v_A = B / sqrt(E Pm), contravariant components
  v^1 = v . grad(xi), v^2 = v . grad(eta), v^3 = v . rhat.
* Energies (Sec. 4.2): E_kin = Pm^2/2 int u^2 dV, E_mag = Pm/(2E) int B^2 dV.
"""
import numpy as np

from .grid import metric_angular, tangent_vectors


def l2_error(V, v, vref):
    d = (np.asarray(v) - np.asarray(vref)).reshape(-1, V.size)
    return float(np.sqrt(((d * d) * V[None]).sum()))


def contravariant_basis(grid, p):
    """grad(xi) * r and grad(eta) * r at the cell centres of panel p, each (Ns, Ns, 3) [j][i]."""
    XI, ETA = np.meshgrid(grid.xi, grid.xi, indexing='xy')
    sigma, a11, a22, a12 = metric_angular(XI, ETA)
    e1, e2 = tangent_vectors(p, XI, ETA)
    g1 = (a11[..., None] * e1 + a12[..., None] * e2) / sigma[..., None]
    g2 = (a12[..., None] * e1 + a22[..., None] * e2) / sigma[..., None]
    return g1, g2


def cfl_alfven(grid, B, E, Pm, dt):
    """Alfven CFL number of a Cartesian field B (3, N) on `grid` (Sec. 4.2, tab:gridlevels)."""
    Ns, Nr = grid.Ns, grid.Nr
    Bv = np.asarray(B).reshape(3, 6, Nr, Ns, Ns) / np.sqrt(E * Pm)
    rhat = grid.rhat()
    best = 0.0
    for p in range(6):
        g1, g2 = contravariant_basis(grid, p)
        v = Bv[:, p]                                            # (3, Nr, Ns, Ns)
        v1 = np.einsum('ckji,jic->kji', v, g1) / grid.r[:, None, None]
        v2 = np.einsum('ckji,jic->kji', v, g2) / grid.r[:, None, None]
        v3 = np.einsum('ckji,cji->kji', v, rhat[:, p])
        best = max(best, float((np.abs(v1) / grid.hs + np.abs(v2) / grid.hs + np.abs(v3) / grid.hr).max()))
    return best * dt


def energies(V, u, B, E, Pm):
    return 0.5 * Pm ** 2 * float((np.asarray(u).reshape(3, -1) ** 2 * V).sum()), \
        0.5 * Pm / E * float((np.asarray(B).reshape(3, -1) ** 2 * V).sum())
