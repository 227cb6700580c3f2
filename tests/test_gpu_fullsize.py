"""GPU path at the bench's full sizes and launch configurations, against the oracle.

Where the oracle can compute the whole result at that size (operator applies,
one-level RAS) the comparison is element by element with the small-size bars;
for the solves it checks what holds at any size: the true FP64 residual, from the
oracle's matrix, is at most the requested 1e-8."""
import numpy as np
import pytest

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

from oracle.discrete import Discretization, ppbe_matrix, vtbe_matrix  # noqa: E402
from oracle.grid import Grid  # noqa: E402
from oracle.schwarz import OneLevelRAS  # noqa: E402
from paper_2009_02171_gb300.inputs import random_vector, uneven_boxes  # noqa: E402

PH = dict(E=1e-3, Ra=100.0, Pr=1.0, Pm=5.0, dt=1e-4)
NS = NR = 64            # the bench's shell, 6 x 64^2 x 64
PARTS, DELTA = (2, 2, 4), 2


@pytest.fixture(scope='module')
def fv():
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    from paper_2009_02171_gb300 import fv as f
    return f


@pytest.fixture(scope='module')
def disc():
    return Discretization(Grid(NS, NR))


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device='cuda')


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize('kind', [0, 1])
def test_apply_at_bench_size(fv, disc, kind):
    A = vtbe_matrix(disc, PH['E'], PH['Ra'], PH['Pr'], PH['Pm'], PH['dt']) if kind == 0 else \
        ppbe_matrix(disc, PH['E'], PH['dt'])
    g = fv.fv_build_grid(NS, NR)
    s = fv.fv_assemble_system(g, kind, **PH, p=PARTS, overlap=DELTA)
    x = random_vector(A.shape[0], 3 + kind)
    y = fv.fv_apply_op(s, _dev(x), torch.empty(A.shape[0], dtype=torch.float64, device='cuda')).cpu().numpy()
    assert _rel(y, A @ x) < 1e-12
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


def test_one_level_ras_at_bench_size(fv, disc):
    A = ppbe_matrix(disc, PH['E'], PH['dt'])
    M = OneLevelRAS(Grid(NS, NR), A, 2, PARTS, DELTA)
    g = fv.fv_build_grid(NS, NR)
    s = fv.fv_assemble_system(g, 1, **PH, p=PARTS, overlap=DELTA)
    r = random_vector(A.shape[0], 5)
    z = fv.fv_precond_apply(s, _dev(r), torch.empty(A.shape[0], dtype=torch.float64, device='cuda')).cpu().numpy()
    assert _rel(z, M.apply(r)) < 1e-11
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


def test_mixed_learned_solve_at_bench_size(fv, disc):
    """The bench's headline PPBE configuration (FP32 inner solves with one Gram-Schmidt pass, learned
    coarse correction + 6 coarse iterations) reaches a true FP64 1e-8 residual without the fallback."""
    from paper_2009_02171_gb300.learned import train_learned_correction
    A = ppbe_matrix(disc, PH['E'], PH['dt'])
    g = fv.fv_build_grid(NS, NR)
    s = fv.fv_assemble_system(g, 1, **PH, p=PARTS, overlap=DELTA, levels=2, overlap_coarse=1,
                              precision=fv.FV_PREC_FP32, inner_maxit=8, coarse_maxit=10, inner_gs_passes=1)
    net, info = train_learned_correction(s, NS, NR, npairs=64, epochs=10)
    xt = random_vector(A.shape[0], 11)
    b = A @ xt                     # consistent with the singular Neumann pressure block
    x = torch.zeros(A.shape[0], dtype=torch.float64, device='cuda')
    st = fv.fv_gmres_solve(s, _dev(b), x, rtol=1e-8)
    xs = x.cpu().numpy()
    assert st.converged and st.fallback == 0
    assert np.linalg.norm(b - A @ xs) <= 1.0001e-8 * np.linalg.norm(b)
    fv.fv_pc_set_learned(s, None)
    fv.fv_net_free(net)
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


def test_batch_at_bench_size(fv):
    """32 right-hand sides on the PPBE 6 x 48^2 x 48 shell with 512 uneven boxes (the batch bench)."""
    Ns = Nr = 48
    A = ppbe_matrix(Discretization(Grid(Ns, Nr)), PH['E'], PH['dt'])
    boxes = uneven_boxes(Ns, Nr, target=512, seed=0)
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, 1, **PH, overlap=2, boxes=boxes, precision=fv.FV_PREC_FP32)
    n = A.shape[0]
    Xt = np.stack([random_vector(n, 100 + r) for r in range(32)])
    B = np.ascontiguousarray((A @ Xt.T).T)
    X = torch.zeros(32, n, dtype=torch.float64, device='cuda')
    st = fv.fv_gmres_solve_batch(s, _dev(B), X, rtol=1e-8)
    Xs = X.cpu().numpy()
    for r in range(32):
        assert st[r].converged
        assert np.linalg.norm(B[r] - A @ Xs[r]) <= 1.0001e-8 * np.linalg.norm(B[r])
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


def test_learned_solve_at_9m_cells(fv):
    """The learned-correction case at 6 x 128^2 x 96 (9.4M cells, coarse 6 x 64^2 x 48): plain two-level RAS
    and the learned coarse correction (4 levels, a short training, + 8 coarse iterations), both to a true
    1e-8 residual; prints the iterations and times of both."""
    from paper_2009_02171_gb300.learned import train_learned_correction
    Ns, Nr, parts = 128, 96, (4, 4, 6)
    A = ppbe_matrix(Discretization(Grid(Ns, Nr)), PH['E'], PH['dt'])
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, 1, **PH, p=parts, overlap=DELTA, levels=2, overlap_coarse=1,
                              precision=fv.FV_PREC_FP32, inner_maxit=8, coarse_maxit=10, inner_gs_passes=1)
    xt = random_vector(A.shape[0], 13)
    b = A @ xt
    bd = _dev(b)
    out = {}
    for mode in ('plain', 'learned'):
        net = None
        if mode == 'learned':
            net, info = train_learned_correction(s, Ns, Nr, levels=4, npairs=64, epochs=10, coarse_its=8)
        x = torch.zeros(A.shape[0], dtype=torch.float64, device='cuda')
        fv.fv_gmres_solve(s, bd, x, rtol=1e-8)  # warm-up (captures the inner solve)
        x.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = fv.fv_gmres_solve(s, bd, x, rtol=1e-8)
        e1.record()
        torch.cuda.synchronize()
        xs = x.cpu().numpy()
        assert st.converged and st.fallback == 0
        assert np.linalg.norm(b - A @ xs) <= 1.0001e-8 * np.linalg.norm(b)
        out[mode] = (st.iters, st.inner_iters, e0.elapsed_time(e1))
        if net is not None:
            fv.fv_pc_set_learned(s, None)
            fv.fv_net_free(net)
    print('\nPPBE 6x128^2x96 to 1e-8: plain %d outer / %d inner iterations, %.1f ms; learned %d / %d, %.1f ms' %
          (*out['plain'], *out['learned']))
    fv.fv_free_system(s)
    fv.fv_free_grid(g)
