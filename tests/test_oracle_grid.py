"""Pins of the oracle's grid and metric against the paper and against finite differences."""
import os

import numpy as np
import pytest

from oracle.grid import Grid, PANEL_M, locate, metric_angular, tangent_vectors, unit_vector
from oracle.diagnostics import cfl_alfven
from paper_2009_02171_gb300.inputs import benchmark_B0, cell_centres

GOLD = os.path.join(os.path.dirname(__file__), 'golden')


def _fd_basis(p, xi, eta, r, h=1e-6):
    x = lambda a, b, c: c * unit_vector(p, np.array(a), np.array(b))
    g1 = (x(xi + h, eta, r) - x(xi - h, eta, r)) / (2 * h)
    g2 = (x(xi, eta + h, r) - x(xi, eta - h, r)) / (2 * h)
    g3 = (x(xi, eta, r + h) - x(xi, eta, r - h)) / (2 * h)
    return g1, g2, g3


def test_sqrt_g_and_inverse_metric_match_finite_differences():
    """Paper Sec. 3.2, sqrt(g) formula; g^{ij} from inverting the FD metric."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        p = int(rng.integers(6))
        xi, eta = rng.uniform(-np.pi / 4, np.pi / 4, 2)
        r = rng.uniform(0.6, 1.5)
        g1, g2, g3 = _fd_basis(p, xi, eta, r)
        G = np.array([[a @ b for b in (g1, g2, g3)] for a in (g1, g2, g3)])
        sigma, a11, a22, a12 = metric_angular(np.array(xi), np.array(eta))
        sqrtg = r * r * sigma
        assert abs(np.sqrt(np.linalg.det(G)) / sqrtg - 1) < 1e-8
        assert np.linalg.det(np.array([g1, g2, g3])) > 0          # right-handed (xi, eta, r)
        Gi = np.linalg.inv(G)
        assert np.allclose([Gi[0, 0] * sqrtg, Gi[1, 1] * sqrtg, Gi[0, 1] * sqrtg], [a11, a22, a12], rtol=1e-7)
        assert np.allclose(Gi[:2, 2], 0, atol=1e-8) and abs(Gi[2, 2] - 1) < 1e-8
        e1, e2 = tangent_vectors(p, np.array(xi), np.array(eta))
        assert np.allclose(r * e1, g1, atol=1e-8) and np.allclose(r * e2, g2, atol=1e-8)


def test_christoffel_symbols_printed_in_paper():
    """Gamma^k_ij = g^k . d_j g_i (FD) equals the three matrices printed in Sec. 3.2."""
    rng = np.random.default_rng(2)
    h = 1e-5
    for _ in range(10):
        xi, eta = rng.uniform(-0.7, 0.7, 2)
        r = rng.uniform(0.6, 1.5)
        X, Y = np.tan(xi), np.tan(eta)
        d = 1 + X * X + Y * Y
        q = (xi, eta, r)
        def basis(a, b, c):
            e1, e2 = tangent_vectors(0, np.array(a), np.array(b))
            return np.array([c * e1, c * e2, unit_vector(0, np.array(a), np.array(b))])
        dG = []
        for j in range(3):
            qp, qm = list(q), list(q)
            qp[j] += h
            qm[j] -= h
            dG.append((basis(*qp) - basis(*qm)) / (2 * h))        # dG[j][i] = d_j g_i
        Gi = np.linalg.inv(basis(*q) @ basis(*q).T)
        gup = Gi @ basis(*q)                                       # contravariant basis
        Gam = np.array([[[gup[k] @ dG[j][i] for j in range(3)] for i in range(3)] for k in range(3)])
        s2x, s2y = 1 + X * X, 1 + Y * Y
        G1 = np.array([[2 * X * Y * Y / d, -Y * s2y / d, 1 / r], [-Y * s2y / d, 0, 0], [1 / r, 0, 0]])
        G2 = np.array([[0, -X * s2x / d, 0], [-X * s2x / d, 2 * Y * X * X / d, 1 / r], [0, 1 / r, 0]])
        G3 = r * s2x * s2y / d ** 2 * np.array([[-s2x, X * Y, 0], [X * Y, -s2y, 0], [0, 0, 0]])
        for k, ref in enumerate((G1, G2, G3)):
            assert np.allclose(Gam[k], ref, atol=1e-8), (k, Gam[k], ref)


def test_panels_tile_the_sphere_and_round_trip():
    rng = np.random.default_rng(3)
    v = rng.standard_normal((500, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    for w in v:
        p, xi, eta = locate(w)
        assert -np.pi / 4 - 1e-12 <= xi <= np.pi / 4 + 1e-12 and -np.pi / 4 - 1e-12 <= eta <= np.pi / 4 + 1e-12
        assert np.allclose(unit_vector(p, np.array(xi), np.array(eta)), w, atol=1e-12)
    for p in range(6):
        assert np.allclose(PANEL_M[p] @ PANEL_M[p].T, np.eye(3))


def test_cell_volumes_converge_to_shell_volume():
    """V = sqrt(g) h_s^2 h_r (Sec. 3.2) sums to 4 pi (r_o^3 - r_i^3)/3 at second order."""
    errs = []
    for n in (8, 16, 32):
        g = Grid(n, n)
        exact = 4 * np.pi * (g.ro ** 3 - g.ri ** 3) / 3
        errs.append(abs(g.volumes().sum() / exact - 1))
    assert errs[-1] < 1e-3
    assert np.log2(errs[0] / errs[1]) > 1.9 and np.log2(errs[1] / errs[2]) > 1.9


def test_cell_counts_table():
    for line in open(os.path.join(GOLD, 'cell_counts.txt')):
        if line.startswith('#'):
            continue
        _, ns, nr, tot, R = line.split()
        g = Grid(int(ns), int(nr))
        assert g.N == int(tot)
        assert round(g.N ** (1 / 3)) == int(R)


def test_ghost_tables_use_first_neighbour_line_and_partition_of_unity():
    g = Grid(10, 2)
    for p in range(6):
        for side in range(4):
            q, sq, tmap, sgn = g.pair[p][side]
            assert g.pair[q][sq][0] == p and g.pair[q][sq][1] == side
            assert np.array_equal(g.pair[q][sq][2][tmap], np.arange(10))
            for (qq, src, w) in g.ghost[p][side]:
                assert qq == q and abs(sum(w) - 1) < 1e-14


@pytest.mark.parametrize('row', [l.split() for l in open(os.path.join(GOLD, 'cfl_gridlevels.txt')) if not l.startswith('#')])
def test_cfl_alfven_table(row):
    """tab:gridlevels CFL_A column (and the 0.33 of Sec. 4.3) from eqn:initial."""
    name, ns, nr, dt5, c5, dt8, c8 = row
    g = Grid(int(ns), int(nr))
    B = benchmark_B0(*cell_centres(int(ns), int(nr))).reshape(3, -1)
    if float(dt5) > 0:
        assert round(cfl_alfven(g, B, 1e-3, 5.0, float(dt5)), 2) == float(c5)
    assert round(cfl_alfven(g, B, 1e-3, 8.0, float(dt8)), 2) == float(c8)
