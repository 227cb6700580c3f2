"""Equiangular gnomonic cubed-sphere shell grid (oracle; test infrastructure).

Paper Sec. 3.2 ("Finite volume spatial discretization"): six panels with
local coordinates (xi, eta, r), xi, eta in [-pi/4, pi/4]; cell centres
xi_i = -pi/4 + (i+1/2) h_s, eta_j likewise, r_k = r_i + (k+1/2) h_r with
h_s = pi/(2 N_s), h_r = (r_o - r_i)/N_r; sqrt(g) = r^2 sec^2 xi sec^2 eta /
(1 + tan^2 xi + tan^2 eta)^{3/2}.

Readings where the paper is silent (see the readings list in the design notes):
* R0 panel orientation: panels 0..3 are equatorial, centred on +x, +y, -x, -y
  with eta pointing north; panel 4 is +z, panel 5 is -z.  The unit position
  vector of panel p is M_p (1, tan xi, tan eta) / sqrt(delta).
* R3 panel-edge ghosts: one ghost layer; a ghost value is the 3-point
  Lagrange interpolation along the neighbour panel's grid line parallel to
  the edge (the ghost centre lands exactly on the neighbour's first cell
  line), evaluated at the ghost's exact tangential position; cube-corner
  ghosts use phi(-1,-1) = phi(-1,0) + phi(0,-1) - phi(0,0).
"""
import numpy as np

# Cartesian unit vector of panel p:  M[p] @ (1, X, Y) / sqrt(1 + X^2 + Y^2)
PANEL_M = np.array([
    [[1, 0, 0], [0, 1, 0], [0, 0, 1]],     # 0: ( 1,  X,  Y)  centred on +x
    [[0, -1, 0], [1, 0, 0], [0, 0, 1]],    # 1: (-X,  1,  Y)  centred on +y
    [[-1, 0, 0], [0, -1, 0], [0, 0, 1]],   # 2: (-1, -X,  Y)  centred on -x
    [[0, 1, 0], [-1, 0, 0], [0, 0, 1]],    # 3: ( X, -1,  Y)  centred on -y
    [[0, 0, -1], [0, 1, 0], [1, 0, 0]],    # 4: (-Y,  X,  1)  centred on +z
    [[0, 0, 1], [0, 1, 0], [-1, 0, 0]],    # 5: ( Y,  X, -1)  centred on -z
], dtype=np.float64)

# panel sides: 0 = xi-min, 1 = xi-max, 2 = eta-min, 3 = eta-max
XI_MIN, XI_MAX, ETA_MIN, ETA_MAX = 0, 1, 2, 3


def unit_vector(p, xi, eta):
    """Cartesian unit position vector on panel p at angular coordinates (xi, eta)."""
    X, Y = np.tan(xi), np.tan(eta)
    v = np.stack([np.ones_like(X), X, Y], axis=-1)
    v = v / np.sqrt(1.0 + X * X + Y * Y)[..., None]
    return v @ PANEL_M[p].T


def locate(v):
    """Panel and (xi, eta) of a Cartesian direction v (inverse of unit_vector)."""
    w = np.einsum('pij,i->pj', PANEL_M, np.asarray(v, dtype=np.float64))  # M_p^T v
    p = int(np.argmax(w[:, 0]))
    return p, np.arctan(w[p, 1] / w[p, 0]), np.arctan(w[p, 2] / w[p, 0])


def metric_angular(xi, eta):
    """Angular factors of the metric (Sec. 3.2).

    With X = tan xi, Y = tan eta, delta = 1 + X^2 + Y^2:
      sigma = sqrt(g) / r^2 = (1+X^2)(1+Y^2) / delta^{3/2}      (paper's sqrt(g))
      a11 = sqrt(g) g^{11} = (1+Y^2) / sqrt(delta)
      a22 = sqrt(g) g^{22} = (1+X^2) / sqrt(delta)
      a12 = sqrt(g) g^{12} = X Y / sqrt(delta)
    (g^{ij} is the inverse of the covariant metric of the gnomonic map;
    g^{13} = g^{23} = 0, g^{33} = 1.)
    """
    X, Y = np.tan(xi), np.tan(eta)
    d = 1.0 + X * X + Y * Y
    sigma = (1 + X * X) * (1 + Y * Y) / d ** 1.5
    return sigma, (1 + Y * Y) / np.sqrt(d), (1 + X * X) / np.sqrt(d), X * Y / np.sqrt(d)


def tangent_vectors(p, xi, eta):
    """e1 = d(xhat)/d(xi), e2 = d(xhat)/d(eta) on panel p (Cartesian; g_1 = r e1, g_2 = r e2)."""
    X, Y = np.tan(xi), np.tan(eta)
    d = 1.0 + X * X + Y * Y
    one = np.ones_like(X)
    e1 = ((1 + X * X) / d ** 1.5)[..., None] * np.stack([-X, 1 + Y * Y, -X * Y], axis=-1)
    e2 = ((1 + Y * Y) / d ** 1.5)[..., None] * np.stack([-Y, -X * Y, 1 + X * X * one], axis=-1)
    return e1 @ PANEL_M[p].T, e2 @ PANEL_M[p].T


class Grid:
    """Cell-centred shell grid of 6 x N_s x N_s x N_r cells (paper Sec. 3.2)."""

    def __init__(self, Ns, Nr, ri=7.0 / 13.0, ro=20.0 / 13.0):
        assert Ns >= 3 and Nr >= 1
        self.Ns, self.Nr, self.ri, self.ro = Ns, Nr, float(ri), float(ro)
        self.hs = np.pi / (2 * Ns)
        self.hr = (self.ro - self.ri) / Nr
        self.N = 6 * Ns * Ns * Nr
        self.xi = -np.pi / 4 + (np.arange(Ns) + 0.5) * self.hs        # centres
        self.xif = -np.pi / 4 + np.arange(Ns + 1) * self.hs           # faces
        self.r = self.ri + (np.arange(Nr) + 0.5) * self.hr
        self.rf = self.ri + np.arange(Nr + 1) * self.hr
        self._build_edges()

    # ---- indexing: cell fields are arrays (6, Nr, Ns, Ns) = [p][k][j][i] ----
    def cell(self, p, k, j, i):
        return ((p * self.Nr + k) * self.Ns + j) * self.Ns + i

    def volumes(self):
        """V_{ijk} = sqrt(g)_{ijk} h_s^2 h_r (paper, after eqn:divdiscretization)."""
        XI, ETA = np.meshgrid(self.xi, self.xi, indexing='xy')   # [j][i]
        sigma = metric_angular(XI, ETA)[0]
        V = self.r[:, None, None] ** 2 * sigma[None] * self.hs ** 2 * self.hr
        return np.broadcast_to(V, (6,) + V.shape).copy()

    def positions(self):
        """Cartesian cell-centre positions, shape (3, 6, Nr, Ns, Ns)."""
        XI, ETA = np.meshgrid(self.xi, self.xi, indexing='xy')
        out = np.empty((3, 6, self.Nr, self.Ns, self.Ns))
        for p in range(6):
            u = unit_vector(p, XI, ETA)                          # [j][i][3]
            out[:, p] = self.r[None, :, None, None] * np.moveaxis(u, -1, 0)[:, None]
        return out

    def rhat(self):
        """Cartesian radial unit vector at cell centres, shape (3, 6, Ns, Ns)."""
        XI, ETA = np.meshgrid(self.xi, self.xi, indexing='xy')
        return np.stack([np.moveaxis(unit_vector(p, XI, ETA), -1, 0) for p in range(6)], axis=1)

    # ---- panel-edge connectivity and ghost interpolation (reading R3) ----
    def _side_point(self, side, t, depth):
        """(xi, eta) of a point outside/inside `side` at tangential cell index t.

        depth = +1/2 h beyond the edge is the ghost centre, 0 is the face centre.
        """
        tang = self.xi[t]
        edge = np.pi / 4 + depth
        if side == XI_MIN:
            return -edge, tang
        if side == XI_MAX:
            return edge, tang
        if side == ETA_MIN:
            return tang, -edge
        return tang, edge

    def _build_edges(self):
        """Edge pairing and ghost interpolation tables, derived from the geometry.

        ghost[p][side][t] = (q, [(j, i) x 3], [w x 3]) : the ghost centre beyond
        `side` of panel p at tangential index t lies on panel q's first cell
        line next to the shared edge; its value is the quadratic Lagrange
        interpolant along that line.
        pair[p][side] = (q, side_q, tmap, sign): faces (p, side, t) and
        (q, side_q, tmap[t]) are the same physical face; F_p = sign * F_q for
        fluxes measured along each panel's own increasing coordinate.
        """
        Ns, h = self.Ns, self.hs
        self.ghost = [[None] * 4 for _ in range(6)]
        self.pair = [[None] * 4 for _ in range(6)]
        for p in range(6):
            for side in range(4):
                rows, tmap, q_side = [], np.empty(Ns, dtype=np.int64), None
                for t in range(Ns):
                    xi, eta = self._side_point(side, t, h / 2)
                    q, xq, yq = locate(unit_vector(p, np.array(xi), np.array(eta)))
                    assert q != p
                    # which side of q is it next to, and the tangential coordinate
                    lim = np.pi / 4 - h / 2
                    if abs(xq + lim) < 1e-9:
                        s_q, tau = XI_MIN, yq
                    elif abs(xq - lim) < 1e-9:
                        s_q, tau = XI_MAX, yq
                    elif abs(yq + lim) < 1e-9:
                        s_q, tau = ETA_MIN, xq
                    elif abs(yq - lim) < 1e-9:
                        s_q, tau = ETA_MAX, xq
                    else:
                        raise AssertionError('ghost centre off the neighbour cell line')
                    assert q_side in (None, (q, s_q))
                    q_side = (q, s_q)
                    frac = (tau + np.pi / 4) / h - 0.5            # fractional cell index
                    c = int(min(max(round(frac), 1), Ns - 2))
                    s = frac - c
                    w = [0.5 * s * (s - 1.0), 1.0 - s * s, 0.5 * s * (s + 1.0)]
                    n0 = 0 if s_q in (XI_MIN, ETA_MIN) else Ns - 1
                    src = [((c + m, n0) if s_q in (XI_MIN, XI_MAX) else (n0, c + m)) for m in (-1, 0, 1)]
                    rows.append((q, src, w))
                    # face centre on the edge: its tangential index on q
                    fxi, feta = self._side_point(side, t, 0.0)
                    v = unit_vector(p, np.array(fxi), np.array(feta))
                    wq = PANEL_M[q].T @ v
                    txq, tyq = np.arctan(wq[1] / wq[0]), np.arctan(wq[2] / wq[0])
                    ftau = tyq if s_q in (XI_MIN, XI_MAX) else txq
                    tf = (ftau + np.pi / 4) / h - 0.5
                    assert abs(tf - round(tf)) < 1e-8
                    tmap[t] = int(round(tf))
                q, s_q = q_side
                sig_p = 1 if side in (XI_MAX, ETA_MAX) else -1
                sig_q = 1 if s_q in (XI_MAX, ETA_MAX) else -1
                self.ghost[p][side] = rows
                self.pair[p][side] = (q, s_q, tmap, -sig_p * sig_q)
