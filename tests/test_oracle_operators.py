"""Pins of the oracle's finite-volume operators: manufactured solutions, invariants, dense solves."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla
import sympy as s

from oracle.discrete import Discretization, ppbe_matrix, vtbe_matrix
from oracle.grid import Grid
from paper_2009_02171_gb300.inputs import cell_centres, random_vector

x, y, z = s.symbols('x y z')
r = s.sqrt(x * x + y * y + z * z)
RI, RO = 7 / 13., 20 / 13.
sv = (r - RI) / (RO - RI)
ANG = (x / r) ** 2 * (y / r) + 0.7 * (z / r) ** 3 - 0.3 * (x / r) * (z / r) + 0.2 * (y / r)


def _lam(e):
    return s.lambdify((x, y, z), e, 'numpy')


def _solve(A, b):
    Mi = sla.spilu(A.tocsc(), drop_tol=1e-6, fill_factor=30)
    xs, info = sla.gmres(A, b, M=sla.LinearOperator(A.shape, Mi.solve), rtol=1e-13, restart=200, maxiter=50)
    assert info == 0
    return xs


def _rates(errs):
    return [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def test_dirichlet_poisson_solution_second_order():
    """Solution of lap_h phi = lap phi (Theta / u wall rule) converges at O(h^2) in L2 and max norm."""
    phi = s.sin(s.pi * sv) * ANG
    f, fl = _lam(phi), _lam(sum(s.diff(phi, q, 2) for q in (x, y, z)))
    l2, mx = [], []
    for n in (6, 12):
        g = Grid(n, n)
        d = Discretization(g)
        X = cell_centres(n, n).reshape(3, -1)
        e = _solve(d.laplacian('odd'), fl(*X)) - f(*X)
        l2.append(np.sqrt((e * e * d.V).sum()))
        mx.append(abs(e).max())
    assert _rates(l2)[0] > 1.85 and _rates(mx)[0] > 1.85


def test_neumann_poisson_solution_second_order():
    """Pressure wall rule (Neumann): bordered solve; O(h^2) after removing the mean."""
    phi = s.cos(s.pi * sv) * ANG
    f, fl = _lam(phi), _lam(sum(s.diff(phi, q, 2) for q in (x, y, z)))
    l2 = []
    for n in (6, 12):
        g = Grid(n, n)
        d = Discretization(g)
        X = cell_centres(n, n).reshape(3, -1)
        L = d.laplacian('even')
        ex = f(*X)
        Ab = sp.bmat([[L, sp.csr_matrix(np.ones((g.N, 1)))], [sp.csr_matrix(d.V[None]), None]]).tocsc()
        sol = sla.spsolve(Ab, np.concatenate([fl(*X), [d.V @ ex]]))[:g.N]
        e = sol - ex
        l2.append(np.sqrt((e * e * d.V).sum()))
    assert _rates(l2)[0] > 1.85


def test_magnetic_laplacian_solution_second_order():
    """Pseudo-vacuum wall rule: the paper's B0 (eqn:initial) is BC-exact; solve lap_B B = lap B0."""
    Bt = -15 / 4 * (r - RI) * (r - RO) * (3 * r - 4) / r
    Br = 5 / 8 * (9 * r ** 3 - 4 * (4 + 3 * (RI + RO)) * r ** 2 + (4 * RO + RI * (4 + 3 * RO)) * 6 * r - 48 * RI * RO) / r
    Bp = 15 / 4 * s.sin(s.pi * (r - RI)) * z / r ** 2
    B = [Br * z / r * x / r + Bt / r ** 2 * z * x - Bp * y,
         Br * z / r * y / r + Bt / r ** 2 * z * y + Bp * x,
         Br * z / r * z / r - Bt / r ** 2 * (x * x + y * y)]
    fB = [_lam(c) for c in B]
    fL = [_lam(sum(s.diff(c, q, 2) for q in (x, y, z))) for c in B]
    l2 = []
    for n in (6, 12):
        g = Grid(n, n)
        d = Discretization(g)
        X = cell_centres(n, n).reshape(3, -1)
        sol = _solve(d.laplacian_B(), np.concatenate([fl(*X) for fl in fL]))
        e = sol - np.concatenate([fb(*X) for fb in fB])
        l2.append(np.sqrt((e.reshape(3, -1) ** 2 * d.V).sum()))
    assert _rates(l2)[0] > 1.8


@pytest.mark.parametrize('n', [6, 9])
def test_neumann_laplacian_kills_constants_and_is_conservative(n):
    g = Grid(n, n + 1)
    d = Discretization(g)
    L = d.laplacian('even')
    scale = abs(L).max()
    assert abs(L @ np.ones(g.N)).max() < 1e-12 * scale
    xr = random_vector(g.N, 5)
    assert abs(d.V @ (L @ xr)) < 1e-13 * scale * d.V.sum()


def test_face_divergence_is_conservative_and_consistent():
    """sum_c V_c D(v)_c = 0 for no-slip fields (fluxes telescope); D of a solenoidal field -> 0."""
    a = [x * y + z, y * z * z - x, x * x * z + y]
    psi = ((r - RI) * (RO - r)) ** 2
    v = [s.diff(psi * a[2], y) - s.diff(psi * a[1], z), s.diff(psi * a[0], z) - s.diff(psi * a[2], x),
         s.diff(psi * a[1], x) - s.diff(psi * a[0], y)]
    fv = _lam(v)
    errs = []
    for n in (8, 16):
        g = Grid(n, n)
        d = Discretization(g)
        X = cell_centres(n, n).reshape(3, -1)
        vr = random_vector(3 * g.N, 7).reshape(3, -1)
        dv = d.divergence(vr, 'u')
        assert abs(d.V @ dv) < 1e-12 * abs(dv).max() * d.V.sum()
        dv = d.divergence(np.array(fv(*X)), 'u')
        errs.append(np.sqrt((dv * dv * d.V).sum()))
    assert _rates(errs)[0] > 1.1  # |u| ~ b at the walls: O(h) wall layer (test_noslip_wall_layer_lowers_the_order_of_u_fluxes)


def test_gradient_and_nonlinear_flux_second_order():
    """Cell Gauss gradient (G = grad/E) and conservative div(a b) (eqn:nonlinearint) vs analytic."""
    a = [x * y + z, y * z * z - x, x * x * z + y]
    psi = ((r - RI) * (RO - r)) ** 2
    v = [s.diff(psi * a[2], y) - s.diff(psi * a[1], z), s.diff(psi * a[0], z) - s.diff(psi * a[2], x),
         s.diff(psi * a[1], x) - s.diff(psi * a[0], y)]
    phi = s.cos(s.pi * sv) * (x * y / r ** 2 + z / r)
    T = s.sin(s.pi * sv) * (x / r + y * z / r ** 2)
    fv, fphi, fT = _lam(v), _lam(phi), _lam(T)
    fg = _lam([s.diff(phi, q) for q in (x, y, z)])
    fadv = _lam(sum(v[i] * s.diff(T, q) for i, q in enumerate((x, y, z))))
    eg, ea = [], []
    for n in (8, 16):
        g = Grid(n, n)
        d = Discretization(g)
        X = cell_centres(n, n).reshape(3, -1)
        G = d.gradient(fphi(*X), 'even', 2.0)
        eg.append(np.sqrt(((2.0 * G - np.array(fg(*X))) ** 2 * d.V).sum()))
        Eu = d.extension('odd')
        V = np.array(fv(*X))
        ad = d.advective_div([Eu @ V[c] for c in range(3)], Eu @ fT(*X))
        ea.append(np.sqrt(((ad - fadv(*X)) ** 2 * d.V).sum()))
    assert _rates(eg)[0] > 1.85 and _rates(ea)[0] > 1.7


def test_vtbe_structure():
    """VTBE = I - dt/2 M: Coriolis antisymmetric coupling, R1/R2 pointwise couplings (eqn:linearoperator)."""
    g = Grid(4, 4)
    d = Discretization(g)
    E, Ra, Pr, Pm, dt = 1e-3, 100.0, 1.0, 5.0, 1e-4
    A = vtbe_matrix(d, E, Ra, Pr, Pm, dt).tocsr()
    N = g.N
    X = g.positions().reshape(3, N)
    c = 7
    assert abs(A[0 * N + c, 1 * N + c] - (-dt / 2 * 2 / E)) < 1e-14
    assert abs(A[1 * N + c, 0 * N + c] - (dt / 2 * 2 / E)) < 1e-14
    assert abs(A[2 * N + c, 3 * N + c] - (-dt / 2 * Ra / (E * g.ro) * X[2, c])) < 1e-12
    rr = np.linalg.norm(X[:, c])
    assert abs(A[3 * N + c, 0 * N + c] - (-dt / 2 * g.ri * g.ro / rr ** 3 * X[0, c])) < 1e-14
    # u rows never see B; B rows never see u or Theta
    assert abs(A[:3 * N, 4 * N:]).max() == 0 and abs(A[4 * N:, :4 * N]).max() == 0
    Lu = d.laplacian('odd')
    assert abs((A[3 * N:4 * N, 3 * N:4 * N] - (sp.identity(N) - dt / 2 / Pr * Lu))).max() < 1e-12


def test_ppbe_is_scaled_compact_laplacian():
    g = Grid(4, 4)
    d = Discretization(g)
    A = ppbe_matrix(d, 1e-3, 1e-4)
    c = 0.5e-4 / 1e-3
    assert abs(A[:g.N, :g.N] - c * d.laplacian('even')).max() == 0
    assert abs(A[g.N:, g.N:] - c * d.laplacian('odd')).max() == 0
