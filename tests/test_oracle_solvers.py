"""Pins of the oracle's ILU(0), Schwarz preconditioners and FGMRES."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.discrete import Discretization, ppbe_matrix, vtbe_matrix
from oracle.grid import Grid
from oracle.ilu import ILU0
from oracle.krylov import fgmres
from oracle.schwarz import OFFSETS, OneLevelRAS, TwoLevelRAS, decompose, ext_cell, prolong, restrict
from paper_2009_02171_gb300.inputs import random_vector


def _lu_from_factors(f):
    n = f.n
    A = sp.csr_matrix((f.a, f.indices, f.indptr), shape=(n, n)).toarray()
    L = np.tril(A, -1) + np.eye(n)
    U = np.triu(A)
    return L, U


def test_ilu0_defining_property_on_subdomain_matrix():
    """ILU(0): (L U)_ij = A_ij on the pattern of A (Saad, Sec. 10.3), on a real VTBE subdomain."""
    g = Grid(6, 4)
    A = vtbe_matrix(Discretization(g), 1e-3, 100, 1, 5, 1e-4)
    sub = decompose(g, (2, 2, 1), 1)[3]
    Al = sub.local_matrix(A, 7, g.N)
    f = ILU0(Al)
    L, U = _lu_from_factors(f)
    LU = L @ U
    Ad = Al.toarray()
    mask = Al.copy()
    mask.data[:] = 1
    mask = mask.toarray() > 0
    assert abs(LU[mask] - Ad[mask]).max() < 1e-12 * abs(Ad).max()


def test_ilu0_exact_when_pattern_has_no_fill():
    rng = np.random.default_rng(0)
    n = 40
    A = sp.diags([rng.random(n - 1), 4 + rng.random(n), rng.random(n - 1)], [-1, 0, 1]).tocsr()
    b = rng.random(n)
    assert abs(ILU0(A).solve(b) - np.linalg.solve(A.toarray(), b)).max() < 1e-14
    blocks = [sp.csr_matrix(rng.random((5, 5)) + 5 * np.eye(5)) for _ in range(4)]
    A = sp.block_diag(blocks, format='csr')
    b = rng.random(20)
    assert abs(ILU0(A).solve(b) - np.linalg.solve(A.toarray(), b)).max() < 1e-13


def test_subdomain_matrix_is_restriction_of_A_on_structured_pattern():
    """A_i^delta = R_i^delta A (R_i^delta)^T (eqn:onelevel), brute force, kept on the pattern."""
    g = Grid(4, 3)
    A = ppbe_matrix(Discretization(g), 1e-3, 1e-4).toarray()
    for sub in decompose(g, (2, 1, 1), 1)[:4]:
        Al = sub.local_matrix(sp.csr_matrix(A), 2, g.N).toarray()
        n = sub.gmap.size
        for p in range(n):
            pk, rem = divmod(p, sub.nx * sub.ny)
            pj, pi = divmod(rem, sub.nx)
            for q in range(n):
                qk, rem = divmod(q, sub.nx * sub.ny)
                qj, qi = divmod(rem, sub.nx)
                inpat = (qi - pi, qj - pj, qk - pk) in OFFSETS
                for a in range(2):
                    for b in range(2):
                        val = Al[p * 2 + a, q * 2 + b]
                        if not inpat or (p != q and a != b):
                            assert val == 0
                        elif sub.gmap[p] < 0 or sub.gmap[q] < 0:
                            assert val == (1.0 if (p == q and a == b and sub.gmap[p] < 0) else 0.0)
                        else:
                            assert val == A[a * g.N + sub.gmap[p], b * g.N + sub.gmap[q]]


def test_decomposition_owned_cells_partition_and_overlap_is_adjacent():
    g = Grid(8, 4)
    subs = decompose(g, (2, 2, 2), 2)
    owned = np.concatenate([s.gmap[s.owned] for s in subs])
    assert np.array_equal(np.sort(owned), np.arange(g.N))
    X = g.positions().reshape(3, -1)
    for s in subs:
        real = s.gmap[s.gmap >= 0]
        assert len(np.unique(real)) == real.size
        # box neighbours along i are geometrically adjacent cells (distance ~ r h_s)
        G = s.gmap.reshape(s.nz, s.ny, s.nx)
        a, b = G[:, :, :-1], G[:, :, 1:]
        ok = (a >= 0) & (b >= 0)
        dist = np.linalg.norm(X[:, a[ok]] - X[:, b[ok]], axis=0)
        assert dist.max() < 2.0 * g.ro * g.hs


def test_ext_cell_across_edges_matches_geometry():
    """A cell one layer beyond a panel edge is the neighbour cell nearest to the ghost centre."""
    g = Grid(8, 1)
    X = g.positions().reshape(3, -1)
    from oracle.grid import unit_vector
    for p in range(6):
        for (i, j) in [(-1, 3), (8, 5), (2, -1), (6, 8)]:
            c = ext_cell(g, p, 0, j, i)
            xi, eta = -np.pi / 4 + (i + 0.5) * g.hs, -np.pi / 4 + (j + 0.5) * g.hs
            gh = g.r[0] * unit_vector(p, np.array(xi), np.array(eta))
            assert np.argmin(np.linalg.norm(X - gh[:, None], axis=0)) == c


def test_fgmres_diagonal_converges_in_k_iterations():
    k = 20
    D = np.arange(1, k + 1, dtype=float)
    b = np.ones(k)
    res = fgmres(lambda v: D * v, lambda v: v.copy(), b, np.zeros(k), restart=30, rtol=1e-12)
    assert res.converged and res.iters <= k
    assert abs(res.x - 1 / D).max() < 1e-10


def test_fgmres_restarted_matches_dense_solve():
    rng = np.random.default_rng(4)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    res = fgmres(lambda v: A @ v, lambda v: v.copy(), b, np.zeros(n), restart=7, rtol=1e-12)
    assert res.converged and res.rfinal <= 1e-12 * res.r0
    assert abs(res.x - np.linalg.solve(A, b)).max() < 1e-10


@pytest.mark.parametrize('kind,n', [('vtbe', 4), ('ppbe', 4), ('ppbe', 6)])
def test_preconditioned_fgmres_matches_dense_lu(kind, n):
    """x = A^{-1} b by brute-force dense LU on the tiniest grids (P part bordered for Neumann)."""
    g = Grid(n, n)
    d = Discretization(g)
    if kind == 'vtbe':
        A, dof = vtbe_matrix(d, 1e-3, 100, 1, 5, 1e-4), 7
    else:
        A, dof = ppbe_matrix(d, 1e-3, 1e-4), 2
    b = random_vector(dof * g.N, 11)
    if kind == 'ppbe':
        b[:g.N] -= (d.V @ b[:g.N]) / d.V.sum()
    M = OneLevelRAS(g, A, dof, (2, 1, 1), 1)
    res = fgmres(lambda v: A @ v, M.apply, b, np.zeros_like(b), restart=30, rtol=1e-13, maxit=2000)
    assert res.converged
    Ad = A.toarray()
    if kind == 'vtbe':
        ref = np.linalg.solve(Ad, b)
        x = res.x
    else:
        N = g.N
        Ab = np.zeros((N + 1, N + 1))
        Ab[:N, :N] = Ad[:N, :N]
        Ab[:N, N] = 1
        Ab[N, :N] = d.V
        refP = np.linalg.solve(Ab, np.concatenate([b[:N], [0]]))[:N]
        ref = np.concatenate([refP, np.linalg.solve(Ad[N:, N:], b[N:])])
        x = res.x.copy()
        x[:N] -= (d.V @ x[:N]) / d.V.sum()
    assert abs(x - ref).max() < 1e-9 * abs(ref).max()


def test_restriction_and_prolongation():
    g = Grid(8, 6)
    xc = random_vector(2 * 6 * 3 * 4 * 4, 3)
    assert np.array_equal(restrict(g, prolong(g, xc, 2), 2), xc)
    assert np.allclose(restrict(g, np.ones(2 * g.N), 2), 1.0)


def test_two_level_beats_one_level_on_ppbe():
    """Hybrid two-level RAS (eqn:twolevel) needs far fewer outer iterations than one-level."""
    g, gc = Grid(16, 16), Grid(8, 8)
    A = ppbe_matrix(Discretization(g), 1e-3, 1e-4)
    Ac = ppbe_matrix(Discretization(gc), 1e-3, 1e-4)
    b = random_vector(2 * g.N, 21)
    V = Discretization(g).V
    b[:g.N] -= (V @ b[:g.N]) / V.sum()
    r1 = fgmres(lambda v: A @ v, OneLevelRAS(g, A, 2, (1, 1, 1), 1).apply, b, np.zeros_like(b), rtol=1e-8)
    M2 = TwoLevelRAS(g, A, gc, Ac, 2, (1, 1, 1), 1, 1, neumann_first=True)
    r2 = fgmres(lambda v: A @ v, M2.apply, b, np.zeros_like(b), rtol=1e-8)
    assert r1.converged and r2.converged
    assert r2.iters * 2 < r1.iters
    assert np.linalg.norm(b - A @ r2.x) <= 1e-8 * np.linalg.norm(b) * 1.0001


def test_two_level_neumann_coarse_projection_prevents_stagnation():
    """Consecutive time steps with the two-level PPBE keep a steady iteration count (the coarse
    Neumann-pressure right-hand side is projected onto the range of the singular coarse matrix)."""
    from oracle.timestep import Physics, SolverOptions, Stepper
    from paper_2009_02171_gb300.inputs import initial_state
    st = Stepper(Grid(8, 8), Physics(), SolverOptions(parts=(2, 2, 1), delta=1, ppbe_levels=2, rtol=1e-10))
    s = dict(initial_state(8, 8, 0), first=True)
    its = []
    for _ in range(3):
        s, info = st.step(s)
        assert info['ppbe'].converged
        its.append(info['ppbe'].iters)
    assert max(its) <= 2 * min(its) + 2


def test_multilevel_with_exact_coarse_solves_equals_two_level():
    """Sec. 3.3 multilevel hybrid RAS: when each coarse GMRES is solved exactly (tiny coarse tolerance), the
    coarse preconditioner (one-level, or two-level on the next mesh) no longer matters, so the 3-level
    operator equals the 2-level one; with the default 0.1 coarse tolerance both stay valid preconditioners."""
    from oracle.schwarz import hybrid_ras
    E, dt = 1e-3, 1e-4
    g = Grid(16, 8)
    A = ppbe_matrix(Discretization(g), E, dt)
    mat = lambda gg: ppbe_matrix(Discretization(gg), E, dt)
    r = random_vector(A.shape[0], 11)
    r[:g.N] -= (g.volumes().ravel() @ r[:g.N]) / g.volumes().sum()
    z2 = hybrid_ras(g, A, mat, 2, (2, 2, 1), 1, 1, 2, rtol_c=1e-13, maxit_c=400, neumann_first=True).apply(r)
    z3 = hybrid_ras(g, A, mat, 2, (2, 2, 1), 1, 1, 3, rtol_c=1e-13, maxit_c=400, neumann_first=True).apply(r)
    # the coarse Neumann pressure matrix is singular: exact coarse solves agree up to a constant in P
    V = g.volumes().ravel()
    for z in (z2, z3):
        z[:g.N] -= (V @ z[:g.N]) / V.sum()
    assert np.abs(z3 - z2).max() < 1e-8 * np.abs(z2).max()
    its = {}
    for lv in (1, 2, 3):
        M = hybrid_ras(g, A, mat, 2, (2, 2, 1), 1, 1, lv, neumann_first=True)
        res = fgmres(lambda v: A @ v, M.apply, r, np.zeros_like(r), restart=30, rtol=1e-8, maxit=400)
        assert res.converged and np.linalg.norm(r - A @ res.x) <= 1.0001e-8 * np.linalg.norm(r)
        its[lv] = res.iters
    assert its[2] < its[1] and its[3] <= its[2] + 2


def test_coarse_box_split_changes_only_the_coarse_preconditioner():
    """Sec. 3.3: the coarse GMRES of eqn:coarsesolve is preconditioned by one-level RAS on the coarse mesh; its
    box split (parts_c) is a free parameter.  With exact coarse solves the two-level operator does not depend on
    it (up to the Neumann constant); parts_c equal to the fine split is the default operator bit for bit; at the
    default coarse tolerance both splits give valid preconditioners."""
    from oracle.schwarz import hybrid_ras
    E, dt = 1e-3, 1e-4
    g = Grid(16, 8)
    A = ppbe_matrix(Discretization(g), E, dt)
    mat = lambda gg: ppbe_matrix(Discretization(gg), E, dt)
    r = random_vector(A.shape[0], 13)
    V = g.volumes().ravel()
    r[:g.N] -= (V @ r[:g.N]) / V.sum()
    base = hybrid_ras(g, A, mat, 2, (2, 2, 1), 1, 1, 2, neumann_first=True).apply(r)
    same = hybrid_ras(g, A, mat, 2, (2, 2, 1), 1, 1, 2, neumann_first=True, parts_c=(2, 2, 1)).apply(r)
    assert np.array_equal(base, same)
    ze = [hybrid_ras(g, A, mat, 2, (2, 2, 1), 1, 1, 2, rtol_c=1e-13, maxit_c=400, neumann_first=True,
                     parts_c=pc).apply(r) for pc in (None, (4, 4, 2))]
    for z in ze:
        z[:g.N] -= (V @ z[:g.N]) / V.sum()
    assert np.abs(ze[1] - ze[0]).max() < 1e-8 * np.abs(ze[0]).max()
    M = hybrid_ras(g, A, mat, 2, (2, 2, 1), 1, 1, 2, neumann_first=True, parts_c=(4, 4, 2))
    assert len(M.coarse.subs) == 6 * 4 * 4 * 2
    res = fgmres(lambda v: A @ v, M.apply, r, np.zeros_like(r), restart=30, rtol=1e-8, maxit=400)
    assert res.converged and np.linalg.norm(r - A @ res.x) <= 1.0001e-8 * np.linalg.norm(r)
