"""Time-stepping state through the C ABI: reset, diagnostics against the oracle, and long runs of the bench
workload (stability at the CFL-limited time step)."""
import numpy as np
import pytest

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

from oracle.diagnostics import cfl_alfven, energies  # noqa: E402
from oracle.grid import Grid  # noqa: E402
from oracle.timestep import Physics, SolverOptions, Stepper  # noqa: E402
from paper_2009_02171_gb300.inputs import initial_state  # noqa: E402

PH = dict(E=1e-3, Ra=100.0, Pr=1.0, Pm=5.0, dt=1e-4)


@pytest.fixture(scope='module')
def fv():
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    from paper_2009_02171_gb300 import fv as f
    return f


def _init(Ns, Nr, seed=0):
    s0 = initial_state(Ns, Nr, seed)
    return s0, np.concatenate([s0['u'].ravel(), s0['T'], s0['B'].ravel(), s0['P'], s0['Pb']])


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device='cuda')


def test_reset_then_step_reproduces_a_fresh_first_step(fv):
    """fv_state_reset drops the Adams-Bashforth history and the previous guesses: reset + step is bitwise
    the first step of a newly created state; fv_state_set keeps the history (it continues a trajectory)."""
    Ns = Nr = 8
    _, init = _init(Ns, Nr)
    N = init.size // 9
    g = fv.fv_build_grid(Ns, Nr)
    V = fv.fv_assemble_system(g, 0, **PH, p=(2, 2, 1), overlap=1)
    P = fv.fv_assemble_system(g, 1, **PH, p=(2, 2, 1), overlap=1, levels=2)
    a = fv.fv_state_create(g, _dev(init), **PH)
    fv.fv_time_step(a, V, P, nsteps=1)
    first = fv.fv_state_get(a, torch.empty(9 * N, dtype=torch.float64, device='cuda')).clone()
    fv.fv_time_step(a, V, P, nsteps=2)
    fv.fv_state_reset(a, _dev(init))
    assert fv.fv_state_diagnostics(a)['steps'] == 0
    fv.fv_time_step(a, V, P, nsteps=1)
    again = fv.fv_state_get(a, torch.empty(9 * N, dtype=torch.float64, device='cuda'))
    assert torch.equal(first, again)
    # set (history kept) from the step-1 fields continues like the trajectory's second step
    b = fv.fv_state_create(g, _dev(init), **PH)
    fv.fv_time_step(b, V, P, nsteps=2)
    two = fv.fv_state_get(b, torch.empty(9 * N, dtype=torch.float64, device='cuda')).clone()
    fv.fv_state_set(a, first)
    fv.fv_time_step(a, V, P, nsteps=1)
    assert torch.equal(two, fv.fv_state_get(a, torch.empty(9 * N, dtype=torch.float64, device='cuda')))
    for h, f in ((a, fv.fv_free_state), (b, fv.fv_free_state), (V, fv.fv_free_system), (P, fv.fv_free_system),
                 (g, fv.fv_free_grid)):
        f(h)


@pytest.mark.parametrize('levels', [1, 2])
def test_time_step_diagnostics_and_pb_match_oracle(fv, levels):
    """Two steps against the oracle: P_b, energies, CFL_A and the cell divergences elementwise; the face
    divergence of B^{n+1} (eqn:divtime on faces) bounded by the PPBE final residual on both sides."""
    Ns, Nr, parts = 8, 8, (2, 2, 1)
    s0, init = _init(Ns, Nr)
    N = init.size // 9
    grid = Grid(Ns, Nr)
    st_o = Stepper(grid, Physics(**PH), SolverOptions(parts=parts, delta=1, ppbe_levels=levels, rtol=1e-10))
    ref = dict(s0, first=True)
    for _ in range(2):
        ref, info = st_o.step(ref)
    g = fv.fv_build_grid(Ns, Nr)
    V = fv.fv_assemble_system(g, 0, **PH, p=parts, overlap=1)
    P = fv.fv_assemble_system(g, 1, **PH, p=parts, overlap=1, levels=levels)
    st = fv.fv_state_create(g, _dev(init), **PH)
    d0 = fv.fv_state_diagnostics(st, P)
    assert d0['divB_face'] == -1 and d0['steps'] == 0
    ek0, em0 = energies(st_o.d.V, s0['u'], s0['B'], PH['E'], PH['Pm'])
    assert abs(d0['E_kin'] - ek0) < 1e-12 * ek0 and abs(d0['E_mag'] - em0) < 1e-12 * em0
    c0 = cfl_alfven(grid, s0['B'], PH['E'], PH['Pm'], PH['dt'])
    assert abs(d0['cfl_alfven'] - c0) < 1e-12 * c0
    stats = fv.fv_time_step(st, V, P, nsteps=2, rtol=1e-10)
    out = fv.fv_state_get(st, torch.empty(9 * N, dtype=torch.float64, device='cuda')).cpu().numpy()
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(out[8 * N:], ref['Pb']) < 1e-6
    d = fv.fv_state_diagnostics(st, P)
    do = st_o.divergence_diagnostics(ref)
    ek, em = energies(st_o.d.V, ref['u'], ref['B'], PH['E'], PH['Pm'])
    assert abs(d['E_kin'] - ek) < 1e-7 * ek and abs(d['E_mag'] - em) < 1e-9 * em
    for k in ('divU_cell', 'divB_cell', 'divB_rhs', 'divU_rhs'):
        assert abs(d[k] - do[k]) < 1e-6 * do[k], (k, d[k], do[k])
    assert d['divB_face'] <= stats[3].rfinal * (1 + 1e-6)
    assert do['divB_face'] <= info['ppbe'].rfinal * (1 + 1e-6)
    assert d['divB_face'] < 1e-8 * d['divB_rhs'] and d['divB_cell'] > 1e3 * d['divB_face']
    assert d['steps'] == 2
    for h, f in ((st, fv.fv_free_state), (V, fv.fv_free_system), (P, fv.fv_free_system), (g, fv.fv_free_grid)):
        f(h)


@pytest.mark.parametrize('mode', ['fp64', 'mixed', 'learned'])
def test_bench_workload_stays_stable_for_60_steps(fv, mode):
    """The bench's 6 x 64^2 x 64 step at its CFL-limited dt (Alfven CFL <= 0.9, Sec. 4.2) for 60 steps, more
    than one pass of the driver's run (warm-up + steps): every solve converges and D_f B stays at the PPBE
    residual.  In the paper's units E_kin + E_mag = Pm^2 (1/2 int u^2 + 1/(E Pm) 1/2 int B^2), which the
    Lorentz and induction terms only exchange; viscous and ohmic dissipation lower it and the buoyancy work
    at Ra = 100 is small over 60 steps, while an Alfven-unstable step makes it grow exponentially."""
    import bench
    c = dict(bench.CFG)
    s0, host = _init(c['Ns'], c['Nr'], c['seed'])
    cfl_unit = cfl_alfven(Grid(c['Ns'], c['Nr']), s0['B'], c['E'], c['Pm'], 1.0)
    dt = bench.stable_dt(cfl_unit)
    assert 0.8 < cfl_unit * dt <= bench.CFL_TARGET
    h, _, _ = bench.build_arm(fv, torch, c, dt, mode, host)
    d = fv.fv_state_diagnostics(h['st'], h['P'])
    assert abs(d['cfl_alfven'] - cfl_unit * dt) < 1e-9
    ek, em = [d['E_kin']], [d['E_mag']]
    for _ in range(60):
        s = fv.fv_time_step(h['st'], h['V'], h['P'], 1, restart=c['restart'], rtol=c['rtol'])
        assert s[0].converged and s[1].converged
        d = fv.fv_state_diagnostics(h['st'], h['P'])
        assert np.isfinite(d['E_kin']) and np.isfinite(d['E_mag'])
        assert d['divB_face'] <= s[1].rfinal * (1 + 1e-6)
        ek.append(d['E_kin'])
        em.append(d['E_mag'])
    tot = np.array(ek) + np.array(em)
    assert tot.max() < 1.01 * tot[0], (tot[0], tot.max())
    bench.free_arm(fv, h)
