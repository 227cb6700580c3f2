"""Finite-volume operators on the cubed-sphere shell (oracle; test infrastructure).

All linear operators are assembled as scipy sparse matrices from plain index
arithmetic, so the same object serves the matrix-free apply (A @ x), the
subdomain matrices of the Schwarz preconditioner and the dense-LU pins.

Paper passages followed:
* eqn:divdiscretization -- divergence by the Gauss theorem over the six cell
  faces, contravariant face fluxes (v^i sqrt(g)) h h, V = sqrt(g) h_s^2 h_r.
* eqn:linearoperator -- L1 = lap - (2/E) z x, R1 = Ra/(E r_o) Theta r,
  L2 = lap/Pr, R2 = r_i r_o / r^3 u . r, L3 = lap/Pm, G = grad/E, D = div.
* eqn:tsvelocity, eqn:tstemperature, eqn:tsmag -- VTBE: x - (dt/2) M x.
* eqn:tsp, eqn:tspb -- PPBE: (dt/2) D G (P, P_b), P Neumann, P_b Dirichlet.
* eqn:nonlinearint -- conservative fluxes of a b.

Readings (listed in the design notes):
* R1 vectors are stored as Cartesian components, so the vector Laplacian is
  three scalar Laplacians and a.grad(b) = div(a b_k) per component (the
  Christoffel source of the paper's contravariant form is identically absent).
* R2 the PPBE operator is the compact face-gradient Laplacian D_f G_f.
* R3 panel-edge face fluxes are the mean of the two panels' one-sided fluxes.
* Scalar face gradient on a xi-face: normal two-point difference, tangential
  derivative = mean of the central differences of the two adjacent cells.
* Wall ghosts at the mirror radius r_g = 2 r_w - r_c: 'odd' ghost = -cell
  (u, Theta, P_b: zero at the wall), 'even' ghost = +cell (P: Neumann), and
  for B: ghost = -B + (1 + (r_c/r_g)^2)(B.rhat) rhat (tangential part zero,
  r^2 B_r flat: eqn:pvc and the condition d(r^2 B^3)/dr = 0).
"""
import numpy as np
import scipy.sparse as sp

from .grid import Grid, metric_angular, tangent_vectors, unit_vector, XI_MIN, XI_MAX, ETA_MIN, ETA_MAX


def _coo(rows, cols, vals, shape):
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=shape)


class Discretization:
    def __init__(self, grid: Grid):
        g = self.g = grid
        Ns, Nr = g.Ns, g.Nr
        self.n_pad = 6 * (Nr + 2) * (Ns + 2) ** 2
        self.n_fx = 6 * Nr * Ns * (Ns + 1)
        self.n_fr = 6 * (Nr + 1) * Ns * Ns
        self.V = g.volumes().ravel()
        P, K, J, I = np.meshgrid(np.arange(6), np.arange(Nr), np.arange(Ns), np.arange(Ns), indexing='ij')
        self._PKJI = [a.ravel() for a in (P, K, J, I)]
        self._build_faces()

    # ------------------------------------------------------------ indices
    def pad(self, p, kk, jj, ii):
        Ns, Nr = self.g.Ns, self.g.Nr
        return ((p * (Nr + 2) + kk) * (Ns + 2) + jj) * (Ns + 2) + ii

    def fx(self, p, k, j, i_f):
        Ns, Nr = self.g.Ns, self.g.Nr
        return ((p * Nr + k) * Ns + j) * (Ns + 1) + i_f

    def fy(self, p, k, j_f, i):  # offset by n_fx inside the horizontal face vector
        Ns, Nr = self.g.Ns, self.g.Nr
        return self.n_fx + ((p * Nr + k) * (Ns + 1) + j_f) * Ns + i

    def fr(self, p, k_f, j, i):
        Ns = self.g.Ns
        return ((p * (self.g.Nr + 1) + k_f) * Ns + j) * Ns + i

    def side_face(self, p, k, side, t):
        Ns = self.g.Ns
        if side == XI_MIN:
            return self.fx(p, k, t, 0)
        if side == XI_MAX:
            return self.fx(p, k, t, Ns)
        if side == ETA_MIN:
            return self.fy(p, k, 0, t)
        return self.fy(p, k, Ns, t)

    # ------------------------------------------------------------ extension (ghosts)
    def _panel_ghost_rows(self):
        """Rows of the padded array filled by panel-edge interpolation (reading R3)."""
        g, Ns, Nr = self.g, self.g.Ns, self.g.Nr
        rows, cols, vals = [], [], []
        k = np.arange(Nr)
        for p in range(6):
            for side in range(4):
                for t, (q, src, w) in enumerate(g.ghost[p][side]):
                    if side == XI_MIN:
                        jj, ii = t + 1, 0
                    elif side == XI_MAX:
                        jj, ii = t + 1, Ns + 1
                    elif side == ETA_MIN:
                        jj, ii = 0, t + 1
                    else:
                        jj, ii = Ns + 1, t + 1
                    for (js, is_), wm in zip(src, w):
                        rows.append(self.pad(p, k + 1, jj, ii))
                        cols.append(g.cell(q, k, js, is_))
                        vals.append(np.full(Nr, wm))
        return rows, cols, vals

    def _interior_rows(self):
        p, k, j, i = self._PKJI
        return [self.pad(p, k + 1, j + 1, i + 1)], [self.g.cell(p, k, j, i)], [np.ones(p.size)]

    def _corner_matrix(self, E0):
        """Cube-corner ghosts: phi(-1,-1) = phi(-1,0) + phi(0,-1) - phi(0,0) (reading R3)."""
        Ns, Nr = self.g.Ns, self.g.Nr
        rows, cols, vals = [], [], []
        k = np.arange(Nr)
        for p in range(6):
            for ic, iin in ((0, 1), (Ns + 1, Ns)):
                for jc, jin in ((0, 1), (Ns + 1, Ns)):
                    r = self.pad(p, k + 1, jc, ic)
                    for (jj, ii), s in (((jin, ic), 1.0), ((jc, iin), 1.0), ((jin, iin), -1.0)):
                        rows.append(r)
                        cols.append(self.pad(p, k + 1, jj, ii))
                        vals.append(np.full(Nr, s))
        S = _coo(rows, cols, vals, (self.n_pad, self.n_pad))
        return S @ E0

    def extension(self, bc):
        """Sparse (n_pad x N) map from cell values to the padded array (ghosts filled).

        bc = 'odd' (ghost = -cell at the walls) or 'even' (ghost = +cell)."""
        Ns, Nr, N = self.g.Ns, self.g.Nr, self.g.N
        r1, c1, v1 = self._interior_rows()
        r2, c2, v2 = self._panel_ghost_rows()
        E0 = _coo(r1 + r2, c1 + c2, v1 + v2, (self.n_pad, N))
        s = {'odd': -1.0, 'even': 1.0}[bc]
        P, J, I = [a.ravel() for a in np.meshgrid(np.arange(6), np.arange(Ns), np.arange(Ns), indexing='ij')]
        rw = [self.pad(P, 0, J + 1, I + 1), self.pad(P, Nr + 1, J + 1, I + 1)]
        cw = [self.g.cell(P, 0, J, I), self.g.cell(P, Nr - 1, J, I)]
        vw = [np.full(P.size, s), np.full(P.size, s)]
        Ew = _coo(rw, cw, vw, (self.n_pad, N))
        return E0 + self._corner_matrix(E0) + Ew

    def extension_B(self):
        """(3 n_pad x 3 N) extension of the Cartesian magnetic field (pseudo-vacuum walls)."""
        g, Ns, Nr, N, npd = self.g, self.g.Ns, self.g.Nr, self.g.N, self.n_pad
        r1, c1, v1 = self._interior_rows()
        r2, c2, v2 = self._panel_ghost_rows()
        E0 = _coo(r1 + r2, c1 + c2, v1 + v2, (npd, N))
        E0 = E0 + self._corner_matrix(E0)
        rhat = g.rhat()                                  # (3, 6, Ns, Ns)
        P, J, I = [a.ravel() for a in np.meshgrid(np.arange(6), np.arange(Ns), np.arange(Ns), indexing='ij')]
        rows, cols, vals = [], [], []
        for kk, kc, rc, rg in ((0, 0, g.r[0], 2 * g.ri - g.r[0]), (Nr + 1, Nr - 1, g.r[-1], 2 * g.ro - g.r[-1])):
            fac = 1.0 + (rc / rg) ** 2
            for a in range(3):
                for b in range(3):
                    m = fac * rhat[a, P, J, I] * rhat[b, P, J, I] - (1.0 if a == b else 0.0)
                    rows.append(a * npd + self.pad(P, kk, J + 1, I + 1))
                    cols.append(b * N + g.cell(P, kc, J, I))
                    vals.append(m)
        Ew = _coo(rows, cols, vals, (3 * npd, 3 * N))
        return sp.block_diag([E0, E0, E0], format='csr') + Ew

    # ------------------------------------------------------------ faces
    def _build_faces(self):
        g, Ns, Nr = self.g, self.g.Ns, self.g.Nr
        hs, hr = g.hs, g.hr
        # xi-faces (p, k, j, i_f): xi = xif[i_f], eta = xi[j]
        P, K, J, IF = [a.ravel() for a in np.meshgrid(np.arange(6), np.arange(Nr), np.arange(Ns), np.arange(Ns + 1), indexing='ij')]
        _, a11, _, a12 = metric_angular(g.xif[IF], g.xi[J])
        rows = [self.fx(P, K, J, IF)] * 6
        cols = [self.pad(P, K + 1, J + 1, IF + 1), self.pad(P, K + 1, J + 1, IF),
                self.pad(P, K + 1, J + 2, IF), self.pad(P, K + 1, J, IF),
                self.pad(P, K + 1, J + 2, IF + 1), self.pad(P, K + 1, J, IF + 1)]
        vals = [a11 * hr, -a11 * hr, a12 * hr / 4, -a12 * hr / 4, a12 * hr / 4, -a12 * hr / 4]
        Fx = _coo(rows, cols, vals, (self.n_fx, self.n_pad))
        Mx = _coo(rows[:2], cols[:2], [np.full(P.size, 0.5)] * 2, (self.n_fx, self.n_pad))
        Sx = np.empty((3, self.n_fx))
        for p in range(6):
            m = P == p
            e1, e2 = tangent_vectors(p, g.xif[IF[m]], g.xi[J[m]])
            Sx[:, m] = ((hs * hr * g.r[K[m]])[:, None] * (a11[m, None] * e1 + a12[m, None] * e2)).T
        # eta-faces (p, k, j_f, i): xi = xi[i], eta = xif[j_f]
        P, K, JF, I = [a.ravel() for a in np.meshgrid(np.arange(6), np.arange(Nr), np.arange(Ns + 1), np.arange(Ns), indexing='ij')]
        _, _, a22, a12 = metric_angular(g.xi[I], g.xif[JF])
        rows = [self.fy(P, K, JF, I) - self.n_fx] * 6
        cols = [self.pad(P, K + 1, JF + 1, I + 1), self.pad(P, K + 1, JF, I + 1),
                self.pad(P, K + 1, JF, I + 2), self.pad(P, K + 1, JF, I),
                self.pad(P, K + 1, JF + 1, I + 2), self.pad(P, K + 1, JF + 1, I)]
        vals = [a22 * hr, -a22 * hr, a12 * hr / 4, -a12 * hr / 4, a12 * hr / 4, -a12 * hr / 4]
        Fy = _coo(rows, cols, vals, (self.n_fx, self.n_pad))
        My = _coo(rows[:2], cols[:2], [np.full(P.size, 0.5)] * 2, (self.n_fx, self.n_pad))
        Sy = np.empty((3, self.n_fx))
        for p in range(6):
            m = P == p
            e1, e2 = tangent_vectors(p, g.xi[I[m]], g.xif[JF[m]])
            Sy[:, m] = ((hs * hr * g.r[K[m]])[:, None] * (a12[m, None] * e1 + a22[m, None] * e2)).T
        self.F_h = sp.vstack([Fx, Fy]).tocsr()
        self.M_h = sp.vstack([Mx, My]).tocsr()
        self.S_h = np.concatenate([Sx, Sy], axis=1)
        # r-faces (p, k_f, j, i)
        P, KF, J, I = [a.ravel() for a in np.meshgrid(np.arange(6), np.arange(Nr + 1), np.arange(Ns), np.arange(Ns), indexing='ij')]
        sigma = metric_angular(g.xi[I], g.xi[J])[0]
        c = hs * hs * g.rf[KF] ** 2 * sigma
        rows = [self.fr(P, KF, J, I)] * 2
        cols = [self.pad(P, KF + 1, J + 1, I + 1), self.pad(P, KF, J + 1, I + 1)]
        self.F_r = _coo(rows, cols, [c / hr, -c / hr], (self.n_fr, self.n_pad))
        self.M_r = _coo(rows, cols, [np.full(P.size, 0.5)] * 2, (self.n_fr, self.n_pad))
        self.S_r = np.empty((3, self.n_fr))
        for p in range(6):
            m = P == p
            self.S_r[:, m] = (c[m, None] * unit_vector(p, g.xi[I[m]], g.xi[J[m]])).T
        # panel-edge averaging of horizontal face fluxes (reading R3)
        nh = 2 * self.n_fx
        rows, cols, vals = [], [], []
        edge = np.zeros(nh, dtype=bool)
        k = np.arange(Nr)
        for p in range(6):
            for side in range(4):
                q, sq, tmap, sgn = g.pair[p][side]
                for t in range(Ns):
                    f = self.side_face(p, k, side, t)
                    fq = self.side_face(q, k, sq, tmap[t])
                    edge[f] = True
                    rows += [f, f]
                    cols += [f, fq]
                    vals += [np.full(Nr, 0.5), np.full(Nr, 0.5 * sgn)]
        inner = np.nonzero(~edge)[0]
        rows.append(inner)
        cols.append(inner)
        vals.append(np.ones(inner.size))
        self.Avg = _coo(rows, cols, vals, (nh, nh))
        # divergence: cells x faces, scaled by 1/V
        p, kk, j, i = self._PKJI
        cell = self.g.cell(p, kk, j, i)
        iv = 1.0 / self.V
        self.Div_h = _coo([cell] * 4, [self.fx(p, kk, j, i + 1), self.fx(p, kk, j, i),
                                       self.fy(p, kk, j + 1, i), self.fy(p, kk, j, i)],
                          [iv, -iv, iv, -iv], (self.g.N, nh))
        self.Div_r = _coo([cell] * 2, [self.fr(p, kk + 1, j, i), self.fr(p, kk, j, i)], [iv, -iv],
                          (self.g.N, self.n_fr))

    # ------------------------------------------------------------ operators
    def flux_laplacian(self):
        """(N x n_pad): scalar Laplacian of a padded array (divergence of the face gradient)."""
        return (self.Div_h @ self.Avg @ self.F_h + self.Div_r @ self.F_r).tocsr()

    def laplacian(self, bc):
        """Scalar Laplacian (N x N) with wall rule bc ('odd' Dirichlet-0, 'even' Neumann)."""
        return (self.flux_laplacian() @ self.extension(bc)).tocsr()

    def laplacian_B(self):
        """Laplacian of the Cartesian magnetic field (3N x 3N), pseudo-vacuum walls."""
        L = self.flux_laplacian()
        return (sp.block_diag([L, L, L]) @ self.extension_B()).tocsr()

    def face_div_matrix(self, comp):
        """(N x n_pad): divergence of a vector whose padded component `comp` is the input."""
        return (self.Div_h @ self.Avg @ sp.diags(self.S_h[comp]) @ self.M_h
                + self.Div_r @ sp.diags(self.S_r[comp]) @ self.M_r).tocsr()

    def divergence(self, v, kind):
        """Face-flux divergence D(v) of a Cartesian vector field v (3, N) (eqn:divdiscretization).

        kind = 'u' (no-slip walls) or 'B' (pseudo-vacuum walls)."""
        N = self.g.N
        if kind == 'u':
            Eu = self.extension('odd')
            pads = [Eu @ v[c] for c in range(3)]
        else:
            vp = self.extension_B() @ np.concatenate([v[0], v[1], v[2]])
            pads = [vp[c * self.n_pad:(c + 1) * self.n_pad] for c in range(3)]
        return sum(self.face_div_matrix(c) @ pads[c] for c in range(3))

    def projected_divergence(self, v, kind, phi, bc, coef):
        """D_f of the projected face fluxes F_f(v) - coef (grad phi)_f . S_f (reading R2, eqn:ubtilde on faces).

        The face normal flux of v is (v_f . S_f) with v_f the mean of the two adjacent values (as in
        `divergence`); the face gradient flux of phi is the one of the compact Laplacian (F_h, F_r).
        With v = B~, phi = P_b, bc = 'odd' and coef = dt/(2E) this is the discrete divergence of
        B^{n+1} taken on the faces (eqn:divtime)."""
        if kind == 'u':
            Eu = self.extension('odd')
            pads = [Eu @ v[c] for c in range(3)]
        else:
            vp = self.extension_B() @ np.concatenate([v[0], v[1], v[2]])
            pads = [vp[c * self.n_pad:(c + 1) * self.n_pad] for c in range(3)]
        php = self.extension(bc) @ phi
        fh = sum(self.S_h[c] * (self.M_h @ pads[c]) for c in range(3)) - coef * (self.F_h @ php)
        fr = sum(self.S_r[c] * (self.M_r @ pads[c]) for c in range(3)) - coef * (self.F_r @ php)
        return self.Div_h @ (self.Avg @ fh) + self.Div_r @ fr

    def gradient(self, phi, bc, E_ekman):
        """Cell gradient G(phi) = (1/E) grad phi by the Gauss theorem, (3, N)."""
        ph = self.extension(bc) @ phi
        fh, fr = self.M_h @ ph, self.M_r @ ph
        return np.stack([(self.Div_h @ (self.Avg @ (self.S_h[c] * fh)) + self.Div_r @ (self.S_r[c] * fr)) / E_ekman
                         for c in range(3)])

    def advective_div(self, a_pads, b_pad):
        """div(a b) with conservative face fluxes (a.S)_f b_f (eqn:nonlinearint, Cartesian)."""
        an_h = sum((self.M_h @ a_pads[c]) * self.S_h[c] for c in range(3))
        an_r = sum((self.M_r @ a_pads[c]) * self.S_r[c] for c in range(3))
        return self.Div_h @ (self.Avg @ (an_h * (self.M_h @ b_pad))) + self.Div_r @ (an_r * (self.M_r @ b_pad))


def vtbe_matrix(disc: Discretization, E, Ra, Pr, Pm, dt):
    """VTBE coefficient matrix A_V = I - (dt/2) M (eqn:tsvelocity, eqn:tstemperature, eqn:tsmag).

    Unknowns, component-major: (u_x, u_y, u_z, Theta, B_x, B_y, B_z), each N cells.
    M = [[lap - (2/E) z x , Ra/(E r_o) r ], [r_i r_o / r^3 r . , lap/Pr], [lap_B / Pm]].
    """
    g = disc.g
    N = g.N
    Lu = disc.laplacian('odd')
    LB = disc.laplacian_B()
    x = g.positions().reshape(3, N)
    rr = np.sqrt((x * x).sum(0))
    blocks = [[None] * 4 for _ in range(4)]
    I = sp.identity(N, format='csr')
    for c in range(3):
        blocks[c][c] = Lu
        blocks[c][3] = sp.diags(Ra / (E * g.ro) * x[c])
        blocks[3][c] = sp.diags(g.ri * g.ro / rr ** 3 * x[c])
    blocks[0][1] = (2.0 / E) * I
    blocks[1][0] = (-2.0 / E) * I
    blocks[3][3] = Lu / Pr
    M = sp.block_diag([sp.bmat(blocks, format='csr'), LB / Pm], format='csr')
    return (sp.identity(7 * N, format='csr') - 0.5 * dt * M).tocsr()


def ppbe_matrix(disc: Discretization, E, dt):
    """PPBE coefficient matrix (dt/2) D G on (P, P_b) = (dt/(2E)) lap (eqn:tsp, eqn:tspb).

    P takes the Neumann (even) wall rule, P_b the Dirichlet-0 (odd) rule."""
    c = 0.5 * dt / E
    return sp.block_diag([c * disc.laplacian('even'), c * disc.laplacian('odd')], format='csr')
