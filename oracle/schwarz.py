"""Restricted additive Schwarz preconditioners (oracle; test infrastructure).

Paper Sec. 3.3:
* each panel is split into p = p1 p2 p3 non-overlapping boxes Omega_i
  (structured, 6p subdomains); Omega_i^delta extends Omega_i by delta cell
  layers, across panel edges into the neighbouring panel (fig:decomposition);
* one-level RAS (eqn:onelevel): M^{-1} = sum_i (R_i^0)^T (A_i^delta)^{-1} R_i^delta,
  A_i^delta = R_i^delta A (R_i^delta)^T, inverse approximated by ILU(0);
* hybrid two-level (eqn:twolevel, eqn:coarsesolve, eqn:finesolve):
  w = I_c^f A_c^{-1} I_f^c x, y = w + M_one^{-1} (x - A_f w); coarse mesh 1:2
  per direction, linear-average restriction, piecewise-constant prolongation,
  coarse system by inner GMRES to relative tolerance eta_c preconditioned by
  one-level RAS on the coarse mesh (eqn:coarsepreconditioner).

Readings (design notes):
* box sizes: N split into p parts as evenly as possible, remainders to the
  lowest-index boxes; radial overlap stops at the walls;
* R5: each subdomain is indexed as a box in its panel's extended index space
  (cells across an edge are the neighbour panel's cells, mapped through the
  edge correspondence; the box positions beyond a cube corner hold no cell).
  A_i^delta keeps, for each cell, the 11 structured stencil neighbours
  (i+-1, j+-1, (i+-1, j+-1), k+-1) with the diagonal d x d block dense and the
  off-diagonal blocks component-diagonal; other couplings of A are dropped.
  ILU(0) runs on this pattern in natural box order (k, j, i) with the
  components innermost.  Positions without a cell are identity rows.
* R7 restriction = arithmetic mean of the 8 children; R6 the coarse matrix is
  the same discretization on the coarse grid.
"""
import numpy as np
import scipy.sparse as sp

from .grid import Grid, XI_MIN, XI_MAX, ETA_MIN, ETA_MAX
from .ilu import ILU0
from .krylov import fgmres

# structured pattern offsets (di, dj, dk), in ascending natural order of the neighbour
OFFSETS = [(0, 0, -1), (-1, -1, 0), (0, -1, 0), (1, -1, 0), (-1, 0, 0), (0, 0, 0),
           (1, 0, 0), (-1, 1, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1)]


def split(n, parts):
    """Start offsets of `parts` boxes covering n cells as evenly as possible."""
    sizes = [n // parts + (1 if b < n % parts else 0) for b in range(parts)]
    return np.concatenate([[0], np.cumsum(sizes)])


def ext_cell(grid, p, k, j, i):
    """Global cell at (k, j, i) of panel p's extended index space, or -1 past a cube corner."""
    Ns = grid.Ns
    in_i, in_j = 0 <= i < Ns, 0 <= j < Ns
    if in_i and in_j:
        return grid.cell(p, k, j, i)
    if not in_i and not in_j:
        return -1
    if i < 0:
        side, m, t = XI_MIN, -1 - i, j
    elif i >= Ns:
        side, m, t = XI_MAX, i - Ns, j
    elif j < 0:
        side, m, t = ETA_MIN, -1 - j, i
    else:
        side, m, t = ETA_MAX, j - Ns, i
    assert m < Ns
    q, sq, tmap, _ = grid.pair[p][side]
    tq = int(tmap[t])
    if sq == XI_MIN:
        return grid.cell(q, k, tq, m)
    if sq == XI_MAX:
        return grid.cell(q, k, tq, Ns - 1 - m)
    if sq == ETA_MIN:
        return grid.cell(q, k, m, tq)
    return grid.cell(q, k, Ns - 1 - m, tq)


class Subdomain:
    def __init__(self, grid, p, own, delta):
        (i0, i1), (j0, j1), (k0, k1) = own
        self.panel, self.own = p, own
        self.lo = (i0 - delta, j0 - delta, max(0, k0 - delta))
        hi = (i1 + delta, j1 + delta, min(grid.Nr, k1 + delta))
        self.nx, self.ny, self.nz = hi[0] - self.lo[0], hi[1] - self.lo[1], hi[2] - self.lo[2]
        n = self.nx * self.ny * self.nz
        self.gmap = np.empty(n, dtype=np.int64)
        self.owned = np.zeros(n, dtype=bool)
        for lk in range(self.nz):
            for lj in range(self.ny):
                for li in range(self.nx):
                    i, j, k = self.lo[0] + li, self.lo[1] + lj, self.lo[2] + lk
                    loc = (lk * self.ny + lj) * self.nx + li
                    self.gmap[loc] = ext_cell(grid, p, k, j, i)
                    self.owned[loc] = i0 <= i < i1 and j0 <= j < j1 and k0 <= k < k1

    def local_matrix(self, A, d, N):
        """A_i^delta on the structured pattern (reading R5), CSR in natural order."""
        nx, ny, nz = self.nx, self.ny, self.nz
        LK, LJ, LI = [a.ravel() for a in np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing='ij')]
        loc = (LK * ny + LJ) * nx + LI
        rows, cols, gr, gc, real = [], [], [], [], []
        for (di, dj, dk) in OFFSETS:
            ok = (LI + di >= 0) & (LI + di < nx) & (LJ + dj >= 0) & (LJ + dj < ny) & (LK + dk >= 0) & (LK + dk < nz)
            p_ = loc[ok]
            q_ = ((LK[ok] + dk) * ny + LJ[ok] + dj) * nx + LI[ok] + di
            comps = [(a, b) for a in range(d) for b in range(d)] if (di, dj, dk) == (0, 0, 0) else [(a, a) for a in range(d)]
            for a, b in comps:
                rows.append(p_ * d + a)
                cols.append(q_ * d + b)
                g_p, g_q = self.gmap[p_], self.gmap[q_]
                gr.append(a * N + np.maximum(g_p, 0))
                gc.append(b * N + np.maximum(g_q, 0))
                real.append((g_p >= 0) & (g_q >= 0))
        rows, cols = np.concatenate(rows), np.concatenate(cols)
        gr, gc, real = np.concatenate(gr), np.concatenate(gc), np.concatenate(real)
        vals = np.zeros(rows.size)
        vals[real] = np.asarray(A[gr[real], gc[real]]).ravel()
        hole = self.gmap < 0                       # identity rows past a cube corner
        hole_diag = np.isin(rows // d, np.nonzero(hole)[0]) & (rows == cols)
        vals[hole_diag] = 1.0
        n = nx * ny * nz * d
        M = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
        assert M.nnz == rows.size
        return M


def decompose_boxes(grid, boxes, delta):
    """Subdomains from an explicit list of owned boxes (panel, i0, i1, j0, j1, k0, k1) that tile
    every panel (uneven decompositions); overlap delta as in decompose()."""
    return [Subdomain(grid, p, ((i0, i1), (j0, j1), (k0, k1)), delta) for (p, i0, i1, j0, j1, k0, k1) in boxes]


def decompose(grid, parts, delta):
    """6 p1 p2 p3 structured subdomains with overlap delta (paper Sec. 3.3)."""
    p1, p2, p3 = parts
    bi, bj, bk = split(grid.Ns, p1), split(grid.Ns, p2), split(grid.Nr, p3)
    subs = []
    for p in range(6):
        for c in range(p3):
            for b in range(p2):
                for a in range(p1):
                    own = ((bi[a], bi[a + 1]), (bj[b], bj[b + 1]), (bk[c], bk[c + 1]))
                    subs.append(Subdomain(grid, p, own, delta))
    return subs


class OneLevelRAS:
    """M_one^{-1} r = sum_i (R_i^0)^T (ILU(0) of A_i^delta)^{-1} R_i^delta r (eqn:onelevel)."""

    def __init__(self, grid, A, d, parts, delta, subs=None, boxes=None):
        self.N, self.d = grid.N, d
        if subs is None:
            subs = decompose_boxes(grid, boxes, delta) if boxes is not None else decompose(grid, parts, delta)
        self.subs = subs
        self.ilus = [ILU0(s.local_matrix(A, d, self.N)) for s in self.subs]

    def apply(self, r):
        N, d = self.N, self.d
        R = r.reshape(d, N)
        z = np.zeros((d, N))
        for s, ilu in zip(self.subs, self.ilus):
            real = s.gmap >= 0
            rl = np.zeros((s.gmap.size, d))
            rl[real] = R[:, s.gmap[real]].T
            xl = ilu.solve(rl.ravel()).reshape(-1, d)
            z[:, s.gmap[s.owned]] = xl[s.owned].T
        return z.ravel()


def restrict(grid, x, d):
    """Coarse value = arithmetic mean of its 8 children (reading R7 of 'linear average')."""
    Ns, Nr = grid.Ns, grid.Nr
    X = x.reshape(d, 6, Nr // 2, 2, Ns // 2, 2, Ns // 2, 2)
    return X.mean(axis=(3, 5, 7)).ravel()


def prolong(grid, xc, d):
    """Piecewise-constant interpolation: each fine cell takes its parent's value."""
    Ns, Nr = grid.Ns, grid.Nr
    X = xc.reshape(d, 6, Nr // 2, 1, Ns // 2, 1, Ns // 2, 1)
    return np.broadcast_to(X, (d, 6, Nr // 2, 2, Ns // 2, 2, Ns // 2, 2)).reshape(-1).copy()


class TwoLevelRAS:
    """Hybrid two-level RAS, y = w + M_one^{-1}(x - A_f w), w = I_c^f A_c^{-1} I_f^c x."""

    def __init__(self, grid, A, grid_c, A_c, d, parts, delta, delta_c, rtol_c=0.1, restart_c=30, maxit_c=30,
                 neumann_first=False, coarse_pc=None, parts_c=None):
        self.g, self.A, self.Ac, self.d = grid, A, A_c, d
        # the Neumann pressure (first PPBE component) has a singular coarse matrix whose left null
        # vector is the coarse cell volumes; its restricted right-hand side is projected onto the range
        self.Vc = grid_c.volumes().ravel() if neumann_first else None
        self.fine = OneLevelRAS(grid, A, d, parts, delta)
        # the coarse GMRES's preconditioner: one-level RAS (eqn:coarsepreconditioner), or for more levels the
        # hybrid construction again on the next coarser mesh (Sec. 3.3)
        # (parts_c: the coarse box split when it is chosen apart from the fine one)
        self.coarse = coarse_pc if coarse_pc is not None else OneLevelRAS(grid_c, A_c, d, parts_c or parts, delta_c)
        self.rtol_c, self.restart_c, self.maxit_c = rtol_c, restart_c, maxit_c
        self.inner_iters = 0

    def apply(self, x):
        xc = restrict(self.g, x, self.d)
        if self.Vc is not None:
            n = self.Vc.size
            xc[:n] -= (self.Vc @ xc[:n]) / self.Vc.sum()
        res = fgmres(lambda v: self.Ac @ v, self.coarse.apply, xc, np.zeros_like(xc),
                     restart=self.restart_c, rtol=self.rtol_c, atol=0.0, maxit=self.maxit_c)
        self.inner_iters += res.iters
        w = prolong(self.g, res.x, self.d)
        return w + self.fine.apply(x - self.A @ w)


def coarse_parts(parts, grid_c):
    """Boxes per panel on a coarse mesh: the fine split, capped by the coarse cell counts."""
    return (min(parts[0], grid_c.Ns), min(parts[1], grid_c.Ns), min(parts[2], grid_c.Nr))


def hybrid_ras(grid, A, matrix_of, d, parts, delta, delta_c, levels, rtol_c=0.1, restart_c=30, maxit_c=30,
               neumann_first=False, parts_c=None):
    """levels-level hybrid RAS (Sec. 3.3): levels = 1 is one-level RAS (eqn:onelevel); otherwise
    eqn:twolevel with the coarse system (the same discretization on the 1:2 mesh, matrix_of(coarse grid))
    solved by GMRES preconditioned by the (levels - 1)-level construction on that mesh.  Every coarse level
    uses overlap delta_c and the same inner tolerance, restart and iteration cap; parts_c (optional) is the box
    split of every coarse level, capped by each coarse mesh (default: the fine split)."""
    if levels <= 1:
        return OneLevelRAS(grid, A, d, parts, delta)
    gc = Grid(grid.Ns // 2, grid.Nr // 2, grid.ri, grid.ro)
    Ac = matrix_of(gc)
    pc = coarse_parts(parts_c or parts, gc)
    inner = hybrid_ras(gc, Ac, matrix_of, d, pc, delta_c, delta_c, levels - 1, rtol_c, restart_c, maxit_c,
                       neumann_first, parts_c) if levels > 2 else None
    return TwoLevelRAS(grid, A, gc, Ac, d, parts, delta, delta_c, rtol_c, restart_c, maxit_c, neumann_first,
                       coarse_pc=inner, parts_c=pc if parts_c else None)
