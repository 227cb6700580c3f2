"""Pins of the oracle's nonlinear terms, face divergence and the divergence constraint of the projection.

* eqn:nonlinearoperator / eqn:nonlinearint: Lorentz term (1/(E Pm)) B.grad B of f1, induction term
  B.grad u - u.grad B of f3 and advection -u.grad Theta of f2, against sympy on manufactured fields.
* eqn:divdiscretization: the face divergence with the pseudo-vacuum wall rule (B) and the no-slip rule (u).
* eqn:divtime with the projection of eqn:ubtilde taken on faces (reading R2): D_f B^{n+1} equals the P_b
  block of the PPBE residual, so it stays at the solver tolerance.
"""
import numpy as np
import pytest
import sympy as s

from oracle.discrete import Discretization, ppbe_matrix
from oracle.grid import Grid
from oracle.timestep import Physics, SolverOptions, Stepper, nonlinear_terms
from paper_2009_02171_gb300.inputs import cell_centres, initial_state, random_vector

x, y, z = s.symbols('x y z')
r = s.sqrt(x * x + y * y + z * z)
RI, RO = 7 / 13., 20 / 13.
# the paper's benchmark initial field B0 (eqn:initial): solenoidal and exact for the pseudo-vacuum walls
_Bt = -15 / 4 * (r - RI) * (r - RO) * (3 * r - 4) / r
_Br = 5 / 8 * (9 * r ** 3 - 4 * (4 + 3 * (RI + RO)) * r ** 2 + (4 * RO + RI * (4 + 3 * RO)) * 6 * r - 48 * RI * RO) / r
_Bp = 15 / 4 * s.sin(s.pi * (r - RI)) * z / r ** 2
B0 = [_Br * z / r * x / r + _Bt / r ** 2 * z * x - _Bp * y,
      _Br * z / r * y / r + _Bt / r ** 2 * z * y + _Bp * x,
      _Br * z / r * z / r - _Bt / r ** 2 * (x * x + y * y)]
T0 = s.sin(s.pi * (r - RI) / (RO - RI)) * (x / r + y * z / r ** 2)


def _lam(e):
    return s.lambdify((x, y, z), e, 'numpy')


def _velocity(power):
    """curl((r - r_i)^p (r_o - r)^p a): solenoidal, zero at both walls, |u| ~ b^(p-1) there."""
    a = [x * y + z, y * z * z - x, x * x * z + y]
    psi = ((r - RI) * (RO - r)) ** power
    return [s.diff(psi * a[2], y) - s.diff(psi * a[1], z), s.diff(psi * a[0], z) - s.diff(psi * a[2], x),
            s.diff(psi * a[1], x) - s.diff(psi * a[0], y)]


def _adv(a, b):
    return sum(a[i] * s.diff(b, q) for i, q in enumerate((x, y, z)))


def _l2(d, e):
    return float(np.sqrt((np.asarray(e) ** 2 * d.V).sum()))


def test_benchmark_field_is_solenoidal():
    """B0 of eqn:initial has zero divergence (the premise of the pseudo-vacuum pins below)."""
    div = sum(s.diff(B0[i], q) for i, q in enumerate((x, y, z)))
    f = _lam(div)
    X = cell_centres(6, 6).reshape(3, -1)
    assert abs(f(*X)).max() < 1e-10


def test_lorentz_induction_and_advection_terms_second_order():
    """f1 = -u.grad u + B.grad B/(E Pm), f2 = -u.grad Theta, f3 = B.grad u - u.grad B through the oracle's
    conservative fluxes, E = 0.5, Pm = 3 (a 1/Pm for 1/(E Pm), a swapped sign or a dropped term fails)."""
    E, Pm = 0.5, 3.0
    u = _velocity(4)
    want = _lam([-_adv(u, u[k]) + _adv(B0, B0[k]) / (E * Pm) for k in range(3)] + [-_adv(u, T0)] +
                [_adv(B0, u[k]) - _adv(u, B0[k]) for k in range(3)])
    fu, fB, fT = _lam(u), _lam(B0), _lam(T0)
    errs = []
    for n in (8, 16):
        d = Discretization(Grid(n, n))
        X = cell_centres(n, n).reshape(3, -1)
        F = nonlinear_terms(d, E, Pm, np.array(fu(*X)), fT(*X), np.array(fB(*X)))
        W = np.array(want(*X))
        errs.append([_l2(d, F[c] - W[c]) for c in range(7)])
    rates = [np.log2(a / b) for a, b in zip(*errs)]
    assert min(rates[:4]) > 1.85, rates     # f1 (Lorentz dominated), f2
    assert min(rates[4:]) > 1.65, rates     # f3 (induction)


def test_noslip_wall_layer_lowers_the_order_of_u_fluxes():
    """Why the no-slip fluxes converge below second order for |u| ~ b at the walls: the odd mirror ghost
    makes the wall flux exact while the first interior face keeps the O(h^2) error of the two-cell mean, so
    the wall-adjacent cells carry an O(h) divergence error (L2 rate -> 1.5); a field that vanishes faster
    at the walls restores second order.  The pseudo-vacuum field B0 is second order throughout."""
    rates = {}
    for p in (2, 4):
        fu = _lam(_velocity(p))
        e = []
        for n in (8, 16):
            d = Discretization(Grid(n, n))
            X = cell_centres(n, n).reshape(3, -1)
            e.append(_l2(d, d.divergence(np.array(fu(*X)), 'u')))
        rates[p] = np.log2(e[0] / e[1])
    fB = _lam(B0)
    eB = []
    for n in (8, 16):
        d = Discretization(Grid(n, n))
        X = cell_centres(n, n).reshape(3, -1)
        eB.append(_l2(d, d.divergence(np.array(fB(*X)), 'B')))
    assert 1.0 < rates[2] < 1.7 and rates[4] > 1.85, rates
    assert np.log2(eB[0] / eB[1]) > 1.9


@pytest.mark.parametrize('n', [4, 6])
def test_face_projection_divergence_equals_ppbe_residual(n):
    """D_f(F(B~) - dt/(2E) (grad P_b)_f . S_f) = D(B~) - (dt/2) D_f G_f P_b = P_b block of b - A x for any
    B~, P_b (the invariant behind 'div B at solver tolerance'); the same for u~ and P."""
    g = Grid(n, n + 1)
    d = Discretization(g)
    N, E, dt = g.N, 1e-3, 1e-4
    A = ppbe_matrix(d, E, dt)
    Bt = random_vector(3 * N, 1).reshape(3, N)
    ut = random_vector(3 * N, 2).reshape(3, N)
    P, Pb = random_vector(N, 3), random_vector(N, 4)
    b = np.concatenate([d.divergence(ut, 'u'), d.divergence(Bt, 'B')])
    res = b - A @ np.concatenate([P, Pb])
    c = 0.5 * dt / E
    fB = d.projected_divergence(Bt, 'B', Pb, 'odd', c)
    fu = d.projected_divergence(ut, 'u', P, 'even', c)
    scale = np.linalg.norm(b) + np.linalg.norm(A @ np.concatenate([P, Pb]))
    assert np.linalg.norm(fB - res[N:]) < 1e-14 * scale
    assert np.linalg.norm(fu - res[:N]) < 1e-14 * scale


def test_oracle_step_keeps_face_divergence_at_solver_tolerance():
    """After a step, ||D_f B^{n+1}|| <= the PPBE solve's final residual (eqn:divtime on faces), while the
    cell-centred D B^{n+1} of eqn:ubtilde stays at the discretization error."""
    g = Grid(8, 8)
    st = Stepper(g, Physics(E=1e-3, Ra=100.0, Pr=1.0, Pm=5.0, dt=1e-4), SolverOptions(rtol=1e-8))
    s1, info = st.step(dict(initial_state(8, 8, 0), first=True))
    s2, info2 = st.step(s1)
    for state, inf in ((s1, info), (s2, info2)):
        dg = st.divergence_diagnostics(state)
        rf = inf['ppbe'].rfinal
        assert dg['divB_face'] <= rf * (1 + 1e-6) and dg['divU_face'] <= rf * (1 + 1e-6)
        assert dg['divB_face'] < 1e-6 * dg['divB_rhs']
        assert dg['divB_cell'] > 1e3 * dg['divB_face']
