"""Learned coarse correction on the GPU (through the C ABI) against the FP64 oracle network.

The CUDA network stores weights, activations and gradients in BF16 (unit
roundoff 2^-9) and accumulates in FP32; the oracle runs in FP64 on the same
BF16-rounded weights.  Along the convolutions each value is rounded about a
dozen times and every rounding can flip a ReLU decision near zero.  Measured
sensitivity: rounding only the input to BF16 moves the oracle's own layer
gradients by up to 3.5 %.  Bars: relative L2 error 2e-2 for the output; for
the gradient, 5e-2 on the whole parameter vector and, per layer, 0.2 with a
cosine similarity of at least 0.98 (the deepest levels have few cells, so their
sums average few roundings).  An indexing mistake gives O(1) errors."""
import numpy as np
import pytest

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

from oracle import unet  # noqa: E402
from paper_2009_02171_gb300.inputs import multiscale_fields, normals, random_vector  # noqa: E402

PH = dict(E=1e-3, Ra=100.0, Pr=1.0, Pm=5.0, dt=1e-4)


@pytest.fixture(scope='module')
def fv():
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    from paper_2009_02171_gb300 import fv as f
    return f


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device='cuda')


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _params(C, levels, seed):
    p = unet.init(C, levels, normals(seed, 27 * C * C * (3 * levels + 3) * 2))
    for i, k in enumerate(p):
        p[k] = (p[k][0], 0.05 * normals(seed + 100 + i, p[k][1].size))
    flat = unet.flatten(p).astype(np.float32)
    ref = unet.unflatten(flat.astype(np.float64), C, levels)
    ref = {k: (bf16(w), b) for k, (w, b) in ref.items()}  # the GPU multiplies BF16 weights
    return flat, ref


def _to_oracle(v, Ns, Nr):
    """Rows of samples laid out [c][p][k][j][i] -> oracle panels [6 nb][c][k][j][i]."""
    v = np.asarray(v).reshape(-1, 2, 6, Nr, Ns, Ns)
    return v.transpose(0, 2, 1, 3, 4, 5).reshape(-1, 2, Nr, Ns, Ns)


def _from_oracle(a, nb):
    return a.reshape(nb, 6, 2, *a.shape[2:]).transpose(0, 2, 1, 3, 4, 5).reshape(nb, -1)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# (C, Ns, Nr, levels): ragged bricks in every pass (padded planes 10 = 8 + 2 and 6 = 4 + 2,
# radial 2 and 1 below a 4-deep brick) and a one-cell panel at the bottom level
CASES = [(16, 8, 8, 3), (32, 8, 4, 2)]


@pytest.mark.parametrize('C,Ns,Nr,levels', CASES)
def test_forward_matches_oracle(fv, C, Ns, Nr, levels):
    flat, ref = _params(C, levels, 11)
    net = fv.fv_net_create(C, Ns, Nr, levels=levels, max_batch=3)
    fv.fv_net_set_params(net, flat)
    n1 = 2 * 6 * Ns * Ns * Nr
    r = multiscale_fields(Ns, Nr, 3, seed=3)
    r[1] *= 1e3       # each sample is normalised by its own norm
    r[2] = 0.0        # zero input -> zero output
    e = fv.fv_net_forward(net, 3, _dev(r.ravel()), torch.empty(3 * n1, dtype=torch.float64, device='cuda'))
    e = e.cpu().numpy().reshape(3, n1)
    want = _from_oracle(unet.forward(ref, _to_oracle(r[:2], Ns, Nr), levels), 2)
    for s in range(2):
        assert _rel(e[s], want[s]) < 2e-2, (s, _rel(e[s], want[s]))
    assert np.all(e[2] == 0.0)
    fv.fv_net_free(net)


@pytest.mark.parametrize('C,Ns,Nr,levels', CASES)
def test_gradients_match_oracle(fv, C, Ns, Nr, levels):
    flat, ref = _params(C, levels, 12)
    net = fv.fv_net_create(C, Ns, Nr, levels=levels, max_batch=2)
    fv.fv_net_set_params(net, flat)
    r = multiscale_fields(Ns, Nr, 2, seed=5)
    e = multiscale_fields(Ns, Nr, 2, seed=6) * np.array([[0.3], [2.0]])
    loss, g = fv.fv_net_loss_grad(net, 2, _dev(r.ravel()), _dev(e.ravel()))
    L, gr = unet.loss_and_grads(ref, _to_oracle(r, Ns, Nr), _to_oracle(e, Ns, Nr), levels)
    assert abs(loss - L) < 1e-2 * L
    assert _rel(g.astype(np.float64), unet.flatten(gr)) < 5e-2
    got = unet.unflatten(g.astype(np.float64), C, levels)
    for k in gr:
        for a, b in ((got[k][0], gr[k][0]), (got[k][1], gr[k][1])):
            cos = (a * b).sum() / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-300)
            assert _rel(a, b) < 0.2 and cos > 0.98, (k, _rel(a, b), cos)
    fv.fv_net_free(net)


def test_he_initialisation(fv):
    net = fv.fv_net_create(32, 8, 8, levels=3)
    fv.fv_net_init(net, 7)
    w = fv.fv_net_get_params(net).astype(np.float64)
    fv.fv_net_init(net, 7)
    assert np.array_equal(fv.fv_net_get_params(net), w.astype(np.float32))
    for k, (W, b) in unet.unflatten(w, 32, 3).items():
        ci = W.shape[1]
        assert np.all(b == 0)
        assert abs(W.std() / np.sqrt(2.0 / (27 * ci)) - 1) < 0.1 and abs(W.mean()) < 0.1 * W.std(), k
    fv.fv_net_free(net)


def test_adam_matches_oracle(fv):
    flat, _ = _params(16, 2, 13)
    net = fv.fv_net_create(16, 8, 8, levels=2)
    fv.fv_net_set_params(net, flat)
    w, m, v = flat.astype(np.float64), np.zeros(flat.size), np.zeros(flat.size)
    for t in range(1, 4):
        g = normals(200 + t, flat.size).astype(np.float32)
        fv.fv_net_adam_step(net, g, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8)
        w, m, v = unet.adam_step(w, g.astype(np.float64), m, v, t, 1e-3, 0.9, 0.999, 1e-8)
    got = fv.fv_net_get_params(net).astype(np.float64)
    assert np.abs(got - w).max() < 1e-6 * (1 + np.abs(w).max())
    fv.fv_net_free(net)


def test_training_is_bitwise_reproducible(fv):
    """Gradients are summed in a fixed order (no floating-point atomics): the same data, seed and
    initialisation give the same weights bit for bit."""
    R = _dev(multiscale_fields(8, 8, 8, seed=9))
    E = _dev(multiscale_fields(8, 8, 8, seed=10))
    out = []
    for _ in range(2):
        net = fv.fv_net_create(16, 8, 8, levels=3, max_batch=4)
        fv.fv_net_init(net, 3)
        fv.fv_net_train(net, R, E, epochs=3, batch=4, seed=1, lr=1e-3)
        out.append(fv.fv_net_get_params(net))
        fv.fv_net_free(net)
    assert np.array_equal(out[0], out[1])


def test_training_reduces_the_loss(fv):
    flat, _ = _params(16, 2, 14)
    net = fv.fv_net_create(16, 8, 8, levels=2, max_batch=4)
    fv.fv_net_set_params(net, flat)
    R = _dev(multiscale_fields(8, 8, 16, seed=7))
    losses = fv.fv_net_train(net, R, R.clone(), epochs=25, batch=4, seed=1, lr=3e-3)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.5 * losses[0], losses
    fv.fv_net_free(net)


@pytest.fixture(scope='module')
def ppbe(fv):
    """Two-level PPBE system on 6 x 16^2 x 16 and a network trained on its coarse solves."""
    Ns = Nr = 16
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, 1, **PH, p=(2, 2, 2), overlap=1, levels=2, overlap_coarse=1)
    c = fv.fv_coarse_system(s)
    n, nc = fv.fv_system_size(s), fv.fv_system_size(c)
    X = _dev(multiscale_fields(Ns, Nr, 48, seed=21))
    Rc = torch.empty(48, nc, dtype=torch.float64, device='cuda')
    for i in range(48):
        fv.fv_restrict_coarse(s, X[i].contiguous(), Rc[i])
    Ec = torch.zeros_like(Rc)
    for i in range(0, 48, 16):
        st = fv.fv_gmres_solve_batch(c, Rc[i:i + 16].contiguous(), Ec[i:i + 16], rtol=1e-6)
        assert all(t.converged for t in st)
    net = fv.fv_net_create(16, Ns // 2, Nr // 2, levels=3, max_batch=8)
    fv.fv_net_set_params(net, _params(16, 3, 15)[0])
    losses = fv.fv_net_train(net, Rc, Ec, epochs=40, batch=8, seed=2, lr=2e-3)
    yield fv, s, net, n, losses
    fv.fv_pc_set_learned(s, None)
    fv.fv_net_free(net)
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


def _solve(fv, s, n, seed, **kw):
    xt = random_vector(n, seed)
    b = torch.empty(n, dtype=torch.float64, device='cuda')
    fv.fv_apply_op(s, _dev(xt), b)
    x = torch.zeros(n, dtype=torch.float64, device='cuda')
    st = fv.fv_gmres_solve(s, b, x, rtol=1e-8, **kw)
    r = torch.empty_like(b)
    fv.fv_apply_op(s, x, r)
    return st, (torch.linalg.norm(b - r) / torch.linalg.norm(b)).item()


def test_learned_preconditioner_converges_and_reports_gain(fv, ppbe):
    fv, s, net, n, losses = ppbe
    assert losses[-1] < losses[0]
    plain, res_p = _solve(fv, s, n, 31)
    fv.fv_pc_set_learned(s, net, coarse_its=0)
    learned, res_l = _solve(fv, s, n, 31, max_it=200)
    fv.fv_pc_set_learned(s, net, coarse_its=2, flags=fv.FV_LEARN_GUESS)
    hybrid, res_h = _solve(fv, s, n, 31)
    fv.fv_pc_set_learned(s, None)
    print('\nlearned coarse correction, PPBE 6x16^2x16: loss %.3g -> %.3g; outer iterations plain %d '
          '(coarse its %d), learned %d (coarse its 0, fallback %d), learned+2 its+guess %d (coarse its %d)' %
          (losses[0], losses[-1], plain.iters, plain.inner_iters, learned.iters, learned.fallback, hybrid.iters,
           hybrid.inner_iters))
    # the learned correction alone may stall FGMRES: the plain fallback then finishes the solve
    for st, res in ((plain, res_p), (learned, res_l), (hybrid, res_h)):
        assert st.converged and res < 1.0001e-8
    assert hybrid.fallback == 0


def test_learned_correction_gains_over_the_same_coarse_budget(fv, ppbe):
    """What the trained network gains over the method without it, at the same coarse work per application:
    the plain two-level preconditioner with exactly 2 coarse FGMRES iterations against the network's
    correction followed by the same 2 iterations (seeded right-hand sides, FGMRES(30) to 1e-8)."""
    fv, s, net, n, _ = ppbe
    g = fv.fv_build_grid(16, 16)
    s2 = fv.fv_assemble_system(g, 1, **PH, p=(2, 2, 2), overlap=1, levels=2, overlap_coarse=1, coarse_maxit=2,
                               coarse_rtol=1e-30)
    plain, learned = [], []
    for seed in (31, 33, 35):
        st, res = _solve(fv, s2, n, seed)
        assert st.converged and res < 1.0001e-8
        plain.append(st.iters)
        fv.fv_pc_set_learned(s2, net, coarse_its=2)
        st, res = _solve(fv, s2, n, seed)
        fv.fv_pc_set_learned(s2, None)
        assert st.converged and res < 1.0001e-8 and st.fallback == 0
        learned.append(st.iters)
    print('\nsame coarse budget (2 coarse iterations per application): outer iterations plain %s, learned %s'
          % (plain, learned))
    assert sum(learned) < sum(plain) and all(a <= b for a, b in zip(learned, plain))
    fv.fv_free_system(s2)
    fv.fv_free_grid(g)


@pytest.mark.parametrize('bad', ['zero', 'nan'])
def test_plain_fallback_finishes_a_failed_learned_solve(fv, ppbe, bad):
    fv, s, _, n, _ = ppbe
    plain, _ = _solve(fv, s, n, 32)
    net = fv.fv_net_create(16, 8, 8, levels=3)
    k = fv.fv_net_param_count(net)
    fv.fv_net_set_params(net, np.zeros(k, np.float32) if bad == 'zero' else np.full(k, np.nan, np.float32))
    fv.fv_pc_set_learned(s, net, coarse_its=0)
    st, res = _solve(fv, s, n, 32, restart=plain.iters + 1, max_it=100, raise_on_noconv=False)
    fv.fv_pc_set_learned(s, None)
    fv.fv_net_free(net)
    assert st.fallback == 1 and st.converged and res < 1.0001e-8


def test_learned_mixed_precision_inner_solve(fv):
    """The FP32 inner path (graph-captured) with the learned coarse solve reaches the FP64 residual."""
    Ns = Nr = 16
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, 1, **PH, p=(2, 2, 2), overlap=1, levels=2, overlap_coarse=1,
                              precision=fv.FV_PREC_FP32, inner_maxit=8, coarse_maxit=8)
    net = fv.fv_net_create(16, 8, 8, levels=3)
    fv.fv_net_set_params(net, _params(16, 3, 16)[0])
    n = fv.fv_system_size(s)
    for its in (0, 3):
        fv.fv_pc_set_learned(s, net, coarse_its=its)
        for seed in (41, 42):  # second solve replays the captured inner graph
            st, res = _solve(fv, s, n, seed)
            assert st.converged and res < 1.0001e-8
    fv.fv_pc_set_learned(s, None)
    fv.fv_net_free(net)
    fv.fv_free_system(s)
    fv.fv_free_grid(g)
