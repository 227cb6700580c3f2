"""Batched solves (many right-hand sides, uneven subdomains) against the oracle and single solves."""
import numpy as np
import pytest

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

from oracle.discrete import Discretization, ppbe_matrix, vtbe_matrix  # noqa: E402
from oracle.grid import Grid  # noqa: E402
from oracle.krylov import fgmres  # noqa: E402
from oracle.schwarz import OneLevelRAS  # noqa: E402
from paper_2009_02171_gb300.inputs import random_vector, uneven_boxes  # noqa: E402

PH = dict(E=1e-3, Ra=100.0, Pr=1.0, Pm=5.0, dt=1e-4)


@pytest.fixture(scope='module')
def fv():
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    from paper_2009_02171_gb300 import fv as f
    return f


def test_uneven_boxes_tile_the_shell():
    for (Ns, Nr) in ((16, 16), (48, 48)):
        boxes = uneven_boxes(Ns, Nr, sizes=(4, 8, 12) if Ns == 16 else (8, 12, 16, 24), seed=3)
        cover = np.zeros((6, Nr, Ns, Ns), dtype=int)
        for (p, i0, i1, j0, j1, k0, k1) in boxes:
            cover[p, k0:k1, j0:j1, i0:i1] += 1
        assert (cover == 1).all()


@pytest.mark.parametrize('kind,prec', [(1, 0), (1, 1), (0, 1)])
def test_batch_matches_oracle_on_uneven_subdomains(fv, kind, prec):
    Ns = Nr = 16
    boxes = uneven_boxes(Ns, Nr, sizes=(4, 8, 12), seed=1)
    g_o = Grid(Ns, Nr)
    disc = Discretization(g_o)
    A = vtbe_matrix(disc, **{k: PH[k] for k in ('E', 'Ra', 'Pr', 'Pm', 'dt')}) if kind == 0 else ppbe_matrix(disc, PH['E'], PH['dt'])
    d = 7 if kind == 0 else 2
    M = OneLevelRAS(g_o, A, d, None, 1, boxes=boxes)
    nrhs = 5
    Bn = np.stack([random_vector(A.shape[0], 40 + r) for r in range(nrhs)])
    if kind == 1:
        Bn[:, :g_o.N] -= (Bn[:, :g_o.N] @ disc.V)[:, None] / disc.V.sum()
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, kind, **PH, overlap=1, boxes=boxes, precision=prec)
    B = torch.tensor(Bn, device='cuda')
    X = torch.zeros_like(B)
    stats = fv.fv_gmres_solve_batch(s, B, X, rtol=1e-8)
    Xn = X.cpu().numpy()
    for r in range(nrhs):
        assert stats[r].converged
        assert np.linalg.norm(Bn[r] - A @ Xn[r]) <= 1.0001e-8 * np.linalg.norm(Bn[r])
        ref = fgmres(lambda v: A @ v, M.apply, Bn[r], np.zeros(A.shape[0]), restart=30, rtol=1e-8)
        x, y = Xn[r].copy(), ref.x.copy()
        if kind == 1:
            x[:g_o.N] -= (disc.V @ x[:g_o.N]) / disc.V.sum()
            y[:g_o.N] -= (disc.V @ y[:g_o.N]) / disc.V.sum()
        assert np.abs(x - y).max() / np.abs(y).max() < (1e-7 if prec == 0 else 1e-6)
        if prec == 0:
            assert abs(stats[r].iters - ref.iters) <= 1
    # the batch gives the single-RHS answers
    x1 = torch.zeros(A.shape[0], dtype=torch.float64, device='cuda')
    fv.fv_gmres_solve(s, B[2].contiguous(), x1, rtol=1e-8)
    assert (x1 - X[2]).abs().max().item() / X[2].abs().max().item() < 1e-6
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


def test_batched_cycles_replay_as_one_graph(fv):
    """The batched FGMRES is driven on the device (Givens rotations and least squares per right-hand side):
    the first restart cycle runs eagerly, later cycles replay one captured CUDA graph.  FGMRES(5) needs
    several cycles; three calls on the same buffers give bitwise the same iterates and iteration counts, the
    true residuals reach 1e-8, and a call with other buffers recaptures."""
    Ns = Nr = 12
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, 1, **PH, p=(2, 2, 2), overlap=1, precision=1)
    n = fv.fv_system_size(s)
    A, _, disc = None, None, Discretization(Grid(Ns, Nr))
    A = ppbe_matrix(disc, PH['E'], PH['dt'])
    nrhs = 4
    Bn = np.stack([random_vector(n, 60 + r) for r in range(nrhs)])
    Bn[:, :disc.g.N] -= (Bn[:, :disc.g.N] @ disc.V)[:, None] / disc.V.sum()
    B = torch.tensor(Bn, device='cuda')
    X = torch.zeros_like(B)
    runs = []
    for _ in range(3):
        X.zero_()
        st = fv.fv_gmres_solve_batch(s, B, X, restart=5, rtol=1e-8, max_it=2000)
        runs.append((X.clone(), [t.iters for t in st]))
        assert all(t.converged for t in st) and max(t.iters for t in st) > 10
    for xr, its in runs[1:]:
        assert torch.equal(xr, runs[0][0]) and its == runs[0][1]
    Xn = runs[0][0].cpu().numpy()
    for r in range(nrhs):
        assert np.linalg.norm(Bn[r] - A @ Xn[r]) <= 1.0001e-8 * np.linalg.norm(Bn[r])
    B2, X2 = B.clone(), torch.zeros_like(B)
    st = fv.fv_gmres_solve_batch(s, B2, X2, restart=5, rtol=1e-8, max_it=2000)
    assert torch.equal(X2, runs[0][0]) and [t.iters for t in st] == runs[0][1]
    fv.fv_free_system(s)
    fv.fv_free_grid(g)
