"""Semi-implicit predictor-corrector time step (oracle; test infrastructure).

Paper Sec. 3.1:
* Crank-Nicolson on the linear operators, second-order Adams-Bashforth
  f^{n+1/2} = 3/2 f^n - 1/2 f^{n-1} on the nonlinear terms (f^{1/2} = f^0);
* hat fields u^ = u - (dt/2) G P^n, B^ = B - (dt/2) G P_b^n (eqn:ubhat),
  u^0 = u^0, B^0 = B^0 on the first step;
* Step 1: VTBE (eqn:tsvelocity, eqn:tstemperature, eqn:tsmag) for
  (u~, Theta^{n+1}, B~); right-hand side x^ + (dt/2) M x^ + dt f^{n+1/2},
  which equals 2 x^ - A_V x^ + dt f^{n+1/2} since A_V = I - (dt/2) M;
* Step 2: PPBE (eqn:tsp, eqn:tspb): (dt/2) D G (P, P_b) = (D u~, D B~);
* Step 3: u = u~ - (dt/2) G P, B = B~ - (dt/2) G P_b (eqn:ubtilde).
Nonlinear terms (eqn:nonlinearoperator) in conservative form (Cartesian
components, reading R1): f1 = -div(u u_k) + div(B B_k)/(E Pm),
f2 = -div(u Theta), f3 = div(B u_k) - div(u B_k).
Reading: the Neumann pressure is fixed to zero volume-weighted mean (its
right-hand side is projected onto zero mean); initial guesses are the
previous step's solutions (Sec. 3.3), the current state on the first step.
"""
from dataclasses import dataclass

import numpy as np

from .discrete import Discretization, ppbe_matrix, vtbe_matrix
from .grid import Grid
from .krylov import fgmres
from .schwarz import OneLevelRAS, hybrid_ras


@dataclass
class Physics:
    E: float = 1e-3
    Ra: float = 100.0
    Pr: float = 1.0
    Pm: float = 5.0
    dt: float = 1e-4


@dataclass
class SolverOptions:
    parts: tuple = (1, 1, 1)
    parts_c: tuple = None   # coarse box split (None: the fine split)
    delta: int = 1
    ppbe_levels: int = 1
    delta_c: int = 1
    rtol_c: float = 0.1
    restart: int = 30
    rtol: float = 1e-8
    atol: float = 0.0
    maxit: int = 3000


def nonlinear_terms(d: Discretization, E, Pm, u, T, B, Eu=None, EB=None):
    """(f1, f2, f3) of eqn:nonlinearoperator stacked as 7 x N, in the conservative form of eqn:nonlinearint
    with Cartesian components: f1_k = -div(u u_k) + div(B B_k)/(E Pm), f2 = -div(u Theta),
    f3_k = div(B u_k) - div(u B_k).  u, B: (3, N); T: (N,).  Eu, EB: the wall extensions (built if None)."""
    npd = d.n_pad
    Eu = d.extension('odd') if Eu is None else Eu
    EB = d.extension_B() if EB is None else EB
    up = [Eu @ u[c] for c in range(3)]
    Tp = Eu @ T
    Bpa = EB @ np.concatenate(B)
    Bp = [Bpa[c * npd:(c + 1) * npd] for c in range(3)]
    c = 1.0 / (E * Pm)
    f1 = [-d.advective_div(up, up[k]) + c * d.advective_div(Bp, Bp[k]) for k in range(3)]
    f2 = [-d.advective_div(up, Tp)]
    f3 = [d.advective_div(Bp, up[k]) - d.advective_div(up, Bp[k]) for k in range(3)]
    return np.stack(f1 + f2 + f3)


class Stepper:
    def __init__(self, grid: Grid, phys: Physics, opt: SolverOptions):
        self.g, self.ph, self.opt = grid, phys, opt
        self.d = Discretization(grid)
        self.AV = vtbe_matrix(self.d, phys.E, phys.Ra, phys.Pr, phys.Pm, phys.dt)
        self.AP = ppbe_matrix(self.d, phys.E, phys.dt)
        self.MV = OneLevelRAS(grid, self.AV, 7, opt.parts, opt.delta)
        if opt.ppbe_levels >= 2:
            self.MP = hybrid_ras(grid, self.AP, lambda g: ppbe_matrix(Discretization(g), phys.E, phys.dt), 2,
                                 opt.parts, opt.delta, opt.delta_c, opt.ppbe_levels, opt.rtol_c, neumann_first=True,
                                 parts_c=opt.parts_c)
        else:
            self.MP = OneLevelRAS(grid, self.AP, 2, opt.parts, opt.delta)
        self.Eu = self.d.extension('odd')
        self.EB = self.d.extension_B()

    def nonlinear(self, u, T, B):
        """(f1, f2, f3) stacked as 7 x N (eqn:nonlinearoperator, eqn:nonlinearint)."""
        return nonlinear_terms(self.d, self.ph.E, self.ph.Pm, u, T, B, self.Eu, self.EB)

    def divergence_diagnostics(self, state):
        """Norms of the divergence of u^{n+1}, B^{n+1} after a step (eqn:divtime): 'face' from the projected
        face fluxes (equal to the PPBE residual blocks), 'cell' from the cell-centred fields (O(h^2));
        'rhs' = ||D(u~)||, ||D(B~)||."""
        N, ph = self.g.N, self.ph
        xt = state['xV']
        ut, Bt = xt[:3 * N].reshape(3, N), xt[4 * N:].reshape(3, N)
        c = 0.5 * ph.dt / ph.E
        bu = self.d.divergence(ut, 'u')
        bu = bu - (self.d.V @ bu) / self.d.V.sum()
        du_f = bu - c * (self.d.laplacian('even') @ state['P'])
        dB_f = self.d.projected_divergence(Bt, 'B', state['Pb'], 'odd', c)
        n2 = np.linalg.norm
        return dict(divU_face=n2(du_f), divB_face=n2(dB_f), divU_rhs=n2(bu),
                    divB_rhs=n2(self.d.divergence(Bt, 'B')),
                    divU_cell=n2(self.d.divergence(state['u'], 'u')), divB_cell=n2(self.d.divergence(state['B'], 'B')))

    def vtbe_rhs(self, state):
        """x^ and the VTBE right-hand side of Step 1."""
        ph, N = self.ph, self.g.N
        f = self.nonlinear(state['u'], state['T'], state['B'])
        fh = f if state.get('f_prev') is None else 1.5 * f - 0.5 * state['f_prev']
        if state.get('first', True):
            uh, Bh = state['u'], state['B']
        else:
            uh = state['u'] - 0.5 * ph.dt * self.d.gradient(state['P'], 'even', ph.E)
            Bh = state['B'] - 0.5 * ph.dt * self.d.gradient(state['Pb'], 'odd', ph.E)
        xh = np.concatenate([uh.ravel(), state['T'], Bh.ravel()])
        return f, xh, 2.0 * xh - self.AV @ xh + ph.dt * fh.ravel()

    def ppbe_rhs(self, xt):
        N = self.g.N
        ut, Bt = xt[:3 * N].reshape(3, N), xt[4 * N:].reshape(3, N)
        bp = self.d.divergence(ut, 'u')
        bp = bp - (self.d.V @ bp) / self.d.V.sum()
        return np.concatenate([bp, self.d.divergence(Bt, 'B')])

    def step(self, state):
        ph, opt, N = self.ph, self.opt, self.g.N
        f, xh, bV = self.vtbe_rhs(state)
        x0 = state['xV'] if state.get('xV') is not None else np.concatenate([state['u'].ravel(), state['T'], state['B'].ravel()])
        rv = fgmres(lambda v: self.AV @ v, self.MV.apply, bV, x0, opt.restart, opt.rtol, opt.atol, opt.maxit)
        xt = rv.x
        bP = self.ppbe_rhs(xt)
        rp = fgmres(lambda v: self.AP @ v, self.MP.apply, bP, np.concatenate([state['P'], state['Pb']]),
                    opt.restart, opt.rtol, opt.atol, opt.maxit)
        P, Pb = rp.x[:N].copy(), rp.x[N:].copy()
        P -= (self.d.V @ P) / self.d.V.sum()
        u = xt[:3 * N].reshape(3, N) - 0.5 * ph.dt * self.d.gradient(P, 'even', ph.E)
        B = xt[4 * N:].reshape(3, N) - 0.5 * ph.dt * self.d.gradient(Pb, 'odd', ph.E)
        new = dict(u=u, T=xt[3 * N:4 * N].copy(), B=B, P=P, Pb=Pb, f_prev=f, xV=xt, first=False)
        return new, dict(vtbe=rv, ppbe=rp)
