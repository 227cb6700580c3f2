"""GPU path (through the C ABI) against the CPU oracle, element by element."""
import numpy as np
import pytest

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

from oracle.discrete import Discretization, ppbe_matrix, vtbe_matrix  # noqa: E402
from oracle.grid import Grid  # noqa: E402
from oracle.krylov import fgmres  # noqa: E402
from oracle.schwarz import OneLevelRAS, TwoLevelRAS  # noqa: E402
from oracle.timestep import Physics, SolverOptions, Stepper  # noqa: E402
from paper_2009_02171_gb300.inputs import initial_state, random_vector  # noqa: E402

PH = dict(E=1e-3, Ra=100.0, Pr=1.0, Pm=5.0, dt=1e-4)


@pytest.fixture(scope='module')
def fv():
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    from paper_2009_02171_gb300 import fv as f
    return f


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device='cuda')


def _oracle_matrix(kind, Ns, Nr):
    d = Discretization(Grid(Ns, Nr))
    if kind == 0:
        return vtbe_matrix(d, PH['E'], PH['Ra'], PH['Pr'], PH['Pm'], PH['dt']), 7, d
    return ppbe_matrix(d, PH['E'], PH['dt']), 2, d


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize('kind', [0, 1])
@pytest.mark.parametrize('Ns,Nr', [(8, 6), (13, 5), (40, 9), (33, 17)])
def test_apply_matches_oracle(fv, kind, Ns, Nr):
    """y = A x (matrix-free CUDA) vs the oracle's assembled A @ x: 1e-12 relative."""
    A, d, _ = _oracle_matrix(kind, Ns, Nr)
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, kind, **PH)
    x = random_vector(A.shape[0], 1 + kind)
    y = fv.fv_apply_op(s, _dev(x), torch.empty(A.shape[0], dtype=torch.float64, device='cuda')).cpu().numpy()
    assert _rel(y, A @ x) < 1e-12
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


@pytest.mark.parametrize('kind', [0, 1])
@pytest.mark.parametrize('Ns,Nr', [(8, 6), (40, 9), (33, 17)])
def test_fp32_apply_matches_oracle(fv, kind, Ns, Nr):
    """FP32 operator of the mixed-precision inner solves (FP32 tables and arithmetic) vs the oracle's FP64
    A @ x: 2e-5 of max |A x| (FP32 rounding of an 11-point stencil; an index error is O(1)).  The sizes
    span several 32-wide tiles, ragged tiles (33, 40) and several level chunks."""
    A, d, _ = _oracle_matrix(kind, Ns, Nr)
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, kind, **PH, precision=fv.FV_PREC_FP32, inner_maxit=2, coarse_maxit=2)
    x = random_vector(A.shape[0], 3 + kind)
    xt = torch.tensor(x, dtype=torch.float32, device='cuda')
    y = fv.fv_apply_op_fp32(s, xt, torch.empty_like(xt)).double().cpu().numpy()
    want = A @ xt.double().cpu().numpy()
    assert _rel(y, want) < 2e-5
    with pytest.raises(fv.FvError):
        s64 = fv.fv_assemble_system(g, kind, **PH)
        try:
            fv.fv_apply_op_fp32(s64, xt, torch.empty_like(xt))
        finally:
            fv.fv_free_system(s64)
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


# Sweep variants: VTBE (kind 0) boxes whose widest wavefront step fits the CTA (<= 384 cells) take the
# register-pipelined level-mapped sweeps.  PPBE boxes of that kind take the shared-memory staged sweeps,
# 8 steps deep (the small cases) or 4 (40 x 4: 42 x 42 x 4 boxes, 96 threads), or the register-pipelined
# ones when no 4-deep stage ring fits (32 x 12 with overlap 2: 36 x 36 x 12 boxes, 224 threads, 218 KB).
# 42 x 42 x 24 (504 cells in a step) takes the level-mapped sweeps with several cells a thread.
@pytest.mark.parametrize('kind,Ns,Nr,parts,delta', [(0, 8, 6, (2, 2, 2), 1), (1, 10, 8, (3, 2, 2), 2),
                                                     (1, 8, 8, (1, 1, 1), 1), (0, 9, 5, (2, 3, 1), 2),
                                                     (1, 16, 12, (1, 1, 1), 1), (1, 40, 4, (1, 1, 1), 1),
                                                     (1, 32, 12, (1, 1, 1), 2), (1, 40, 24, (1, 1, 1), 1)])
def test_one_level_ras_matches_oracle(fv, kind, Ns, Nr, parts, delta):
    """z = M_one^{-1} r (level-scheduled ILU(0) sweeps) vs the oracle's sequential ILU(0)."""
    A, d, _ = _oracle_matrix(kind, Ns, Nr)
    M = OneLevelRAS(Grid(Ns, Nr), A, d, parts, delta)
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, kind, **PH, p=parts, overlap=delta)
    r = random_vector(A.shape[0], 7)
    z = fv.fv_precond_apply(s, _dev(r), torch.empty(A.shape[0], dtype=torch.float64, device='cuda')).cpu().numpy()
    assert _rel(z, M.apply(r)) < 1e-11
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


def test_two_level_ras_matches_oracle(fv):
    """Hybrid two-level preconditioner (eqn:twolevel) with inner coarse FGMRES to 0.1."""
    Ns, Nr, parts = 12, 8, (2, 2, 1)
    A, d, _ = _oracle_matrix(1, Ns, Nr)
    Ac, _, _ = _oracle_matrix(1, Ns // 2, Nr // 2)
    M = TwoLevelRAS(Grid(Ns, Nr), A, Grid(Ns // 2, Nr // 2), Ac, 2, parts, 1, 1, 0.1, 30, 30, neumann_first=True)
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, 1, **PH, p=parts, overlap=1, levels=2, overlap_coarse=1)
    r = random_vector(A.shape[0], 9)
    z = fv.fv_precond_apply(s, _dev(r), torch.empty(A.shape[0], dtype=torch.float64, device='cuda')).cpu().numpy()
    assert _rel(z, M.apply(r)) < 1e-9
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


def test_two_level_ras_with_its_own_coarse_box_split_matches_oracle(fv):
    """The coarse one-level RAS (eqn:coarsepreconditioner) over boxes split apart from the fine ones
    (fv_pc_desc cp1..cp3 against the oracle's parts_c): 12 x 8 fine boxes (2, 2, 1), coarse (3, 3, 2)."""
    Ns, Nr, parts, cparts = 12, 8, (2, 2, 1), (3, 3, 2)
    A, d, _ = _oracle_matrix(1, Ns, Nr)
    Ac, _, _ = _oracle_matrix(1, Ns // 2, Nr // 2)
    M = TwoLevelRAS(Grid(Ns, Nr), A, Grid(Ns // 2, Nr // 2), Ac, 2, parts, 1, 1, 0.1, 30, 30, neumann_first=True,
                    parts_c=cparts)
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, 1, **PH, p=parts, overlap=1, levels=2, overlap_coarse=1, coarse_p=cparts)
    r = random_vector(A.shape[0], 9)
    z = fv.fv_precond_apply(s, _dev(r), torch.empty(A.shape[0], dtype=torch.float64, device='cuda')).cpu().numpy()
    assert _rel(z, M.apply(r)) < 1e-9
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


def test_three_level_ras_matches_oracle(fv):
    """Multilevel hybrid RAS (Sec. 3.3): the coarse GMRES of the two-level preconditioner is itself
    preconditioned by the two-level construction on the next 1:2 mesh (16 x 8 -> 8 x 4 -> 4 x 2)."""
    from oracle.schwarz import hybrid_ras
    Ns, Nr, parts = 16, 8, (2, 2, 1)
    A, d, _ = _oracle_matrix(1, Ns, Nr)
    mat = lambda gg: ppbe_matrix(Discretization(gg), PH['E'], PH['dt'])
    M = hybrid_ras(Grid(Ns, Nr), A, mat, 2, parts, 1, 1, 3, neumann_first=True)
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, 1, **PH, p=parts, overlap=1, levels=3, overlap_coarse=1)
    r = random_vector(A.shape[0], 9)
    z = fv.fv_precond_apply(s, _dev(r), torch.empty(A.shape[0], dtype=torch.float64, device='cuda')).cpu().numpy()
    assert _rel(z, M.apply(r)) < 1e-9
    # a 3-level FGMRES solve (Neumann P block of the right-hand side made consistent): solution to 1e-7 at a
    # 1e-8 residual after removing P's mean, iterations within one
    N, V = 6 * Ns * Ns * Nr, Grid(Ns, Nr).volumes().ravel()
    b = random_vector(A.shape[0], 12)
    b[:N] -= (V @ b[:N]) / V.sum()
    ref = fgmres(lambda v: A @ v, M.apply, b, np.zeros_like(b), restart=30, rtol=1e-8, maxit=500)
    x = torch.zeros(A.shape[0], dtype=torch.float64, device='cuda')
    st = fv.fv_gmres_solve(s, _dev(b), x, rtol=1e-8, max_it=500)
    assert st.converged and abs(st.iters - ref.iters) <= 1
    xs, rx = x.cpu().numpy(), ref.x.copy()
    for v in (xs, rx):
        v[:N] -= (V @ v[:N]) / V.sum()
    assert _rel(xs, rx) < 1e-7
    with pytest.raises(fv.FvError):   # 16 x 8 has no fourth 1:2 mesh with Nr >= 4 to coarsen
        fv.fv_assemble_system(g, 1, **PH, p=parts, overlap=1, levels=4, overlap_coarse=1)
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


@pytest.mark.parametrize('kind,levels', [(0, 1), (1, 1), (1, 2)])
def test_gmres_solution_matches_oracle(fv, kind, levels):
    """Solutions at a 1e-8 relative residual agree to 1e-7 (same algorithm, same ordering)."""
    Ns = Nr = 12
    parts = (2, 2, 2)
    A, d, disc = _oracle_matrix(kind, Ns, Nr)
    G = Grid(Ns, Nr)
    if levels == 2:
        Ac, _, _ = _oracle_matrix(1, Ns // 2, Nr // 2)
        M = TwoLevelRAS(G, A, Grid(Ns // 2, Nr // 2), Ac, d, parts, 1, 1, neumann_first=True)
    else:
        M = OneLevelRAS(G, A, d, parts, 1)
    b = random_vector(A.shape[0], 13)
    if kind == 1:
        b[:G.N] -= (disc.V @ b[:G.N]) / disc.V.sum()
    ref = fgmres(lambda v: A @ v, M.apply, b, np.zeros_like(b), restart=30, rtol=1e-8)
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, kind, **PH, p=parts, overlap=1, levels=levels)
    x = torch.zeros(A.shape[0], dtype=torch.float64, device='cuda')
    st = fv.fv_gmres_solve(s, _dev(b), x, rtol=1e-8)
    xs = x.cpu().numpy()
    assert st.converged and abs(st.iters - ref.iters) <= 1
    assert np.linalg.norm(b - A @ xs) <= 1.0001e-8 * np.linalg.norm(b)
    if kind == 1:
        xs[:G.N] -= (disc.V @ xs[:G.N]) / disc.V.sum()
        rx = ref.x.copy()
        rx[:G.N] -= (disc.V @ rx[:G.N]) / disc.V.sum()
    else:
        rx = ref.x
    assert _rel(xs, rx) < 1e-7
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


@pytest.mark.parametrize('levels', [1, 2])
def test_time_step_matches_oracle(fv, levels):
    """Two predictor-corrector steps (Sec. 3.1) from seeded synthetic fields."""
    Ns, Nr, parts = 8, 8, (2, 2, 1)
    s0 = initial_state(Ns, Nr, 0)
    N = 6 * Ns * Ns * Nr
    init = np.concatenate([s0['u'].ravel(), s0['T'], s0['B'].ravel(), s0['P'], s0['Pb']])
    st_o = Stepper(Grid(Ns, Nr), Physics(**PH), SolverOptions(parts=parts, delta=1, ppbe_levels=levels, rtol=1e-10))
    ref = dict(s0, first=True)
    for _ in range(2):
        ref, info = st_o.step(ref)
        assert info['vtbe'].converged and info['ppbe'].converged
    g = fv.fv_build_grid(Ns, Nr)
    V = fv.fv_assemble_system(g, 0, **PH, p=parts, overlap=1)
    P = fv.fv_assemble_system(g, 1, **PH, p=parts, overlap=1, levels=levels)
    st = fv.fv_state_create(g, _dev(init), **PH)
    stats = fv.fv_time_step(st, V, P, nsteps=2, rtol=1e-10)
    assert all(s.converged for s in stats)
    out = fv.fv_state_get(st, torch.empty(9 * N, dtype=torch.float64, device='cuda')).cpu().numpy()
    assert _rel(out[:3 * N], ref['u'].ravel()) < 1e-7
    assert _rel(out[3 * N:4 * N], ref['T']) < 1e-7
    assert _rel(out[4 * N:7 * N], ref['B'].ravel()) < 1e-7
    assert _rel(out[7 * N:8 * N], ref['P']) < 1e-6
    fv.fv_free_state(st)
    fv.fv_free_system(V)
    fv.fv_free_system(P)
    fv.fv_free_grid(g)


def test_bad_arguments_raise(fv):
    with pytest.raises(fv.FvError):
        fv.fv_build_grid(2, 1)
    g = fv.fv_build_grid(9, 6)
    with pytest.raises(fv.FvError):
        fv.fv_assemble_system(g, 1, **PH, p=(1, 1, 1), levels=2, overlap=1)  # odd Ns has no 1:2 coarse mesh
    with pytest.raises(fv.FvError):
        fv.fv_assemble_system(g, 1, **PH, p=(10, 1, 1), overlap=1)           # more boxes than cells
    fv.fv_free_grid(g)


@pytest.mark.parametrize('kind,levels,gs', [(0, 1, 2), (1, 2, 2), (0, 1, 1), (1, 2, 1)])
def test_mixed_precision_solve_reaches_fp64_residual(fv, kind, levels, gs):
    """FP32 inner FGMRES (FP32 operator, FP32 ILU(0) sweeps, FP32 coarse level) as the
    preconditioner of the FP64 outer FGMRES: the true FP64 residual (oracle matrix) reaches
    1e-8 and the solution matches the FP64 solution to the conditioning-limited accuracy."""
    Ns = Nr = 12
    parts = (2, 2, 2)
    A, d, disc = _oracle_matrix(kind, Ns, Nr)
    b = random_vector(A.shape[0], 17)
    if kind == 1:
        b[:disc.g.N] -= (disc.V @ b[:disc.g.N]) / disc.V.sum()
    g = fv.fv_build_grid(Ns, Nr)
    s64 = fv.fv_assemble_system(g, kind, **PH, p=parts, overlap=1, levels=levels)
    s32 = fv.fv_assemble_system(g, kind, **PH, p=parts, overlap=1, levels=levels, precision=fv.FV_PREC_FP32,
                                inner_maxit=6, coarse_maxit=8, inner_gs_passes=gs)
    x64 = torch.zeros(A.shape[0], dtype=torch.float64, device='cuda')
    x32 = torch.zeros_like(x64)
    st64 = fv.fv_gmres_solve(s64, _dev(b), x64, rtol=1e-8)
    st32 = fv.fv_gmres_solve(s32, _dev(b), x32, rtol=1e-8)
    assert st64.converged and st32.converged
    xs = x32.cpu().numpy()
    assert np.linalg.norm(b - A @ xs) <= 1.0001e-8 * np.linalg.norm(b)
    ref = x64.cpu().numpy()
    if kind == 1:
        for v in (xs, ref):
            v[:disc.g.N] -= (disc.V @ v[:disc.g.N]) / disc.V.sum()
    assert _rel(xs, ref) < 1e-6
    assert st32.iters <= st64.iters            # each outer step carries an FP32 inner solve
    for h in (s64, s32):
        fv.fv_free_system(h)
    fv.fv_free_grid(g)


def test_mixed_precision_time_step_matches_oracle(fv):
    Ns, Nr, parts = 8, 8, (2, 2, 1)
    s0 = initial_state(Ns, Nr, 0)
    N = 6 * Ns * Ns * Nr
    init = np.concatenate([s0['u'].ravel(), s0['T'], s0['B'].ravel(), s0['P'], s0['Pb']])
    st_o = Stepper(Grid(Ns, Nr), Physics(**PH), SolverOptions(parts=parts, delta=1, ppbe_levels=2, rtol=1e-10))
    ref, _ = st_o.step(dict(s0, first=True))
    g = fv.fv_build_grid(Ns, Nr)
    mp = dict(precision=fv.FV_PREC_FP32, inner_maxit=6, coarse_maxit=8)
    V = fv.fv_assemble_system(g, 0, **PH, p=parts, overlap=1, **mp)
    P = fv.fv_assemble_system(g, 1, **PH, p=parts, overlap=1, levels=2, **mp)
    st = fv.fv_state_create(g, _dev(init), **PH)
    stats = fv.fv_time_step(st, V, P, nsteps=1, rtol=1e-10)
    assert all(s.converged for s in stats)
    out = fv.fv_state_get(st, torch.empty(9 * N, dtype=torch.float64, device='cuda')).cpu().numpy()
    assert _rel(out[:3 * N], ref['u'].ravel()) < 1e-7
    assert _rel(out[3 * N:4 * N], ref['T']) < 1e-7
    assert _rel(out[4 * N:7 * N], ref['B'].ravel()) < 1e-7
    # second and third steps replay the captured inner-solve graphs
    ref2 = ref
    for _ in range(2):
        ref2, _ = st_o.step(ref2)
    stats = fv.fv_time_step(st, V, P, nsteps=2, rtol=1e-10)
    assert all(s.converged for s in stats)
    out = fv.fv_state_get(st, torch.empty(9 * N, dtype=torch.float64, device='cuda')).cpu().numpy()
    assert _rel(out[:3 * N], ref2['u'].ravel()) < 1e-7
    assert _rel(out[4 * N:7 * N], ref2['B'].ravel()) < 1e-7
    for h, f in ((st, fv.fv_free_state), (V, fv.fv_free_system), (P, fv.fv_free_system), (g, fv.fv_free_grid)):
        f(h)


def test_mixed_precision_three_level_solve_reaches_fp64_residual(fv):
    """FP32 inner FGMRES whose two-level preconditioner's coarse solve is itself two-level (three meshes,
    16 -> 8 -> 4): the true FP64 residual against the oracle matrix reaches 1e-8."""
    Ns = Nr = 16
    A, d, disc = _oracle_matrix(1, Ns, Nr)
    b = random_vector(A.shape[0], 21)
    b[:disc.g.N] -= (disc.V @ b[:disc.g.N]) / disc.V.sum()
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, 1, **PH, p=(2, 2, 2), overlap=1, levels=3, precision=fv.FV_PREC_FP32,
                              inner_maxit=6, coarse_maxit=6)
    x = torch.zeros(A.shape[0], dtype=torch.float64, device='cuda')
    st = fv.fv_gmres_solve(s, _dev(b), x, rtol=1e-8)
    assert st.converged
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1.0001e-8 * np.linalg.norm(b)
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


@pytest.mark.parametrize('kind,levels', [(0, 1), (1, 2)])
def test_bf16_factor_solve_reaches_fp64_residual(fv, kind, levels):
    """FV_PREC_BF16: the FP32 inner solves read their ILU(0) factors stored in BF16 (every level, staged and
    register-pipelined sweeps).  The outer FP64 FGMRES still reaches a true FP64 residual of 1e-8 against the
    oracle's matrix, in at most two more outer iterations than with FP32 factors."""
    Ns = Nr = 12
    A, d, disc = _oracle_matrix(kind, Ns, Nr)
    b = random_vector(A.shape[0], 23)
    if kind == 1:
        b[:disc.g.N] -= (disc.V @ b[:disc.g.N]) / disc.V.sum()
    g = fv.fv_build_grid(Ns, Nr)
    its = {}
    for prec in (fv.FV_PREC_FP32, fv.FV_PREC_BF16):
        s = fv.fv_assemble_system(g, kind, **PH, p=(2, 2, 2), overlap=1, levels=levels, precision=prec,
                                  inner_maxit=6, coarse_maxit=6)
        x = torch.zeros(A.shape[0], dtype=torch.float64, device='cuda')
        st = fv.fv_gmres_solve(s, _dev(b), x, rtol=1e-8)
        assert st.converged
        assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1.0001e-8 * np.linalg.norm(b)
        its[prec] = st.iters
        if prec == fv.FV_PREC_BF16 and kind == 1:
            with pytest.raises(fv.FvError):
                fv.fv_gmres_solve_batch(s, _dev(b[None]), torch.zeros(1, A.shape[0], dtype=torch.float64,
                                                                       device='cuda'))
        fv.fv_free_system(s)
    assert its[fv.FV_PREC_BF16] <= its[fv.FV_PREC_FP32] + 2
    fv.fv_free_grid(g)


def test_coarse_transfers_match_oracle(fv):
    """I_f^c (mean of the 8 children, P's volume-weighted mean removed for PPBE) and I_c^f (piecewise
    constant) of the two-level preconditioner (eqn:coarsesolve), through fv_restrict_coarse and
    fv_prolong_coarse, against the oracle's restrict and prolong: exact up to rounding of the mean."""
    from oracle.schwarz import prolong, restrict
    Ns, Nr = 12, 8
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, 1, **PH, p=(2, 2, 1), overlap=1, levels=2, overlap_coarse=1)
    n = fv.fv_system_size(s)
    x = random_vector(n, 21)
    xc = random_vector(n // 8, 22)
    gc = Grid(Ns // 2, Nr // 2)
    rc = fv.fv_restrict_coarse(s, _dev(x), torch.empty(n // 8, dtype=torch.float64, device='cuda')).cpu().numpy()
    ref = restrict(Grid(Ns, Nr), x, 2)
    Vc, Nc = gc.volumes().ravel(), gc.N
    ref[:Nc] -= (Vc @ ref[:Nc]) / Vc.sum()
    assert np.abs(rc - ref).max() < 1e-13 * np.abs(ref).max()
    xf = fv.fv_prolong_coarse(s, _dev(xc), torch.empty(n, dtype=torch.float64, device='cuda')).cpu().numpy()
    assert np.array_equal(xf, prolong(Grid(Ns, Nr), xc, 2))
    fv.fv_free_system(s)
    fv.fv_free_grid(g)
