#!/usr/bin/env python
"""Time per time step of the shell dynamo solve path on GB300 (prints one JSON line).

Workload (the mid-size mixed-vs-plain shell of the project's configuration
list): 6 x 64^2 x 64 cells (1,572,864), E = 1e-3, Pm = 5, Ra = 100, Pr = 1,
seeded synthetic fields (seed 1 + rank).  The time step dt is chosen from the
seeded field so that the Alfven CFL number is at most 0.9 (dt = 0.9 / CFL_A
per unit dt, rounded down to two significant digits; 5.7e-5 on this shell),
the stability margin the paper keeps on every grid of its Table of grid
levels (Sec. 4.2).  One step = the paper's predictor-corrector time step
(Sec. 3.1): nonlinear terms, VTBE solve (FGMRES(30), one-level RAS,
96 subdomains = 6 x (2 x 2 x 4), overlap 2), PPBE solve (FGMRES(30), hybrid
two-level RAS, coarse 32^3 x 6 with overlap 1), projection; both systems to a
1e-8 relative FP64 residual.  Three arms, each timed on the same steps of the
same trajectory (every pass restarts from the seeded fields with a fresh
history): fp64 (FP64 throughout, coarse inner GMRES to 0.1), mixed (FP32
inner FGMRES in FP64 outer FGMRES, 10 coarse iterations) and the headline
learned (mixed, with the coarse solve replaced by a BF16 cubed-sphere U-Net
followed by 6 coarse iterations; its training on seeded pairs from the plain
coarse solver is setup, reported in `learned`).

value       -- ms per time step (max over ranks; one independent shell per GPU)
e2e         -- the same through the C ABI with the state copied host->device
               before and device->host after every step (pinned host buffers)
roofline    -- live CUDA-event duration of the dominant kernel category over
               the timed region against its algorithmic bytes
stencil     -- the same for the FP32 operator applies (VTBE, PPBE)
cpu_baseline-- the CPU oracle (rank 0, N = 1): real time steps of the same
               workload (fewer than --steps; the count is stated)
--impl reference runs only the oracle arm, on the same workload.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# the shells of the project's configuration list (seeded synthetic fields, E = 1e-3, Pm = 5, Ra = 100, Pr = 1):
# boxes of 32 x 32 x 16 cells + overlap 2 in every case but the tiny one
COMMON = dict(overlap_coarse=1, E=1e-3, Ra=100.0, Pr=1.0, Pm=5.0, rtol=1e-8, vtbe_inner=4, ppbe_inner=8,
              coarse_its=10, inner_gs=1)
CONFIGS = {
    'shell16': dict(COMMON, Ns=16, Nr=16, p=(1, 1, 1), overlap=1, levels=1, restart=30, seed=0),
    # coarse boxes 8 x 8 x 16 (4 x 4 x 2 a panel, 384 in all): 45 wavefront steps a sweep instead of 61
    'shell64': dict(COMMON, Ns=64, Nr=64, p=(2, 2, 4), overlap=2, levels=2, restart=30, seed=1, coarse_p=(4, 4, 2)),
    'shell128': dict(COMMON, Ns=128, Nr=96, p=(4, 4, 6), overlap=2, levels=2, restart=30, seed=3),
    # three PPBE meshes (192 -> 96 -> 48): the learned correction's training generates its targets with the
    # batched one-level coarse solver, so this shell's arms are FP64 and mixed precision
    'shell192': dict(COMMON, Ns=192, Nr=128, p=(6, 6, 8), overlap=2, levels=3, restart=20, seed=4, coarse_its=4,
                     arms=('fp64', 'mixed')),
}
CFG = CONFIGS['shell64']
# largest Alfven CFL number of the seeded field the time step may give (paper Sec. 4.2 keeps <= 1.19 and
# notes instability about 10 % above its choices)
CFL_TARGET = 0.9
# learned coarse correction of the headline arm: network and training (seeded synthetic pairs from the plain
# coarse solver; data generation and training are counted in setup_s); deeper networks on larger coarse grids
LEARN = dict(C=16, levels=3, pairs=256, epochs=40, batch=8, lr=3e-4, coarse_its=6)
LEARN_BY_CONFIG = {'shell128': dict(LEARN, levels=4, coarse_its=8), 'shell192': dict(LEARN, levels=4, coarse_its=8)}
METRIC = 'wall time per time step at 1e-8 residual'
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a kernel category at the default
# workload, from the ncu capture in the file named beside it; a category leaves this table when its kernels
# change, until they are captured again
TRAFFIC = {'net_fwd': (49537707, 'profiles/launches_net_forward_c16_coarse32.md'),
           'apply_vtbe_fp32': (57991936, 'profiles/ncu_apply_vtbe_fp32_shell64.md')}
# CPU oracle: wall-clock budget for its real time steps (after its setup); at least one step always runs
ORACLE_BUDGET_S = float(os.environ.get('FV_ORACLE_BUDGET_S', '100'))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=5)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--precision', default=None, choices=['learned', 'mixed', 'bf16', 'fp64'],
                    help='headline arm (learned = mixed precision with the learned coarse correction; default: the '
                         'last arm of the shell, learned where it has one); the other arms are timed beside it')
    ap.add_argument('--single', action='store_true', help='time the headline arm only (profiling runs)')
    ap.add_argument('--ns', type=int, default=0, help='override Ns = Nr (small profiling cases)')
    ap.add_argument('--config', default='shell64', choices=sorted(CONFIGS),
                    help='shell of the time-step workload (shell64: the mid-size mixed-vs-plain shell; shell128, '
                         'shell192: the learned-correction and full-scale shells)')
    ap.add_argument('--levels', type=int, default=0, help='override the PPBE preconditioner levels')
    ap.add_argument('--coarse-its', type=int, default=0, help='override the fixed coarse iterations (mixed precision)')
    ap.add_argument('--ppbe-inner', type=int, default=0, help='override the PPBE inner iterations (mixed precision)')
    ap.add_argument('--coarse-p', default='', help='coarse-level box split a,b,c per panel (default: the fine split)')
    ap.add_argument('--learned-its', type=int, default=0, help='override the coarse iterations after the network (learned arm)')
    ap.add_argument('--learn-guess', action='store_true', help='learned arm: also correct each initial guess with the network')
    ap.add_argument('--vtbe-inner', type=int, default=0, help='override the VTBE inner iterations (mixed precision)')
    ap.add_argument('--workload', default='step', choices=['step', 'batch', 'net', 'trajectory', 'apply', 'strong',
                                                           'p8', 'convergence'],
                    help='step: the time step (headline); batch: 32 right-hand sides on uneven subdomains; '
                         'trajectory: one arm (--precision) for --steps steps from the seeded fields, one JSON '
                         'line of diagnostics per step; apply: the operator applies alone (FP64 and FP32); strong: '
                         'the strong-scaling workload of the paper replayed on one GPU; p8: benchmark P8 on grid '
                         'G48 (--steps steps, energies every --every steps); convergence: the spatial and temporal '
                         'convergence study of Sec. 4.1')
    ap.add_argument('--every', type=int, default=1000, help='p8: steps between diagnostics lines')
    ap.add_argument('--budget-min', type=float, default=0.0, help='p8: stop after this many minutes (0: none)')
    ap.add_argument('--dt', type=float, default=0.0, help='trajectory: time step (default: the CFL-limited dt)')
    return ap.parse_args()


def floor2(x):
    """x > 0 rounded down to two significant digits (exact decimal, e.g. 5.7e-05)."""
    e = math.floor(math.log10(x)) - 1
    m = math.floor(x / 10.0 ** e + 1e-9)
    return float('%de%d' % (m, e))


def stable_dt(cfl_per_unit_dt):
    """The step whose Alfven CFL number is at most CFL_TARGET, rounded down to two significant digits."""
    return floor2(CFL_TARGET / cfl_per_unit_dt)


def max_over_ranks(value, device):
    """The largest of the ranks' values (the job's time is its slowest rank's); every rank gets it."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup(backend):
    import torch.distributed as dist
    ws = int(os.environ.get('WORLD_SIZE', '1'))
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault('MASTER_ADDR', '127.0.0.1')
        dist.init_process_group(backend)
    return int(os.environ.get('RANK', '0')), ws, int(os.environ.get('LOCAL_RANK', '0'))


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""
    FIELDS = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
              'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
              'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, gpu):
        self.gpu, self.proc, self.path = gpu, None, '/tmp/fv_clocks_%d_%d.csv' % (os.getpid(), gpu)

    def __enter__(self):
        try:
            self.f = open(self.path, 'w')
            self.proc = subprocess.Popen(['nvidia-smi', '-i', str(self.gpu), '--query-gpu=' + self.FIELDS,
                                          '--format=csv,noheader,nounits', '-lms', '200'], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        # let nvidia-smi finish initialising (its driver calls can stall CUDA calls) before timing starts
        deadline = time.time() + 5.0
        while self.proc and time.time() < deadline and os.path.getsize(self.path) == 0:
            time.sleep(0.05)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['nvidia-smi unavailable']}
        rows = [l.split(',') for l in open(self.path).read().strip().splitlines() if l.count(',') >= 8]
        if not rows:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['no samples']}
        sm = sorted(float(r[1]) for r in rows)
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.strip() == 'Active'})
        return {'sm_mhz': sm[len(sm) // 2], 'sm_max_mhz': float(rows[0][2]), 'samples': len(rows),
                'power_w_max': max(float(r[3]) for r in rows if r[3].strip() not in ('', '[N/A]')),
                'reasons': reasons}


def oracle_cfl_per_unit_dt(c):
    """Alfven CFL number of the seeded field per unit dt, from the oracle's diagnostic (CPU)."""
    from oracle.diagnostics import cfl_alfven
    from oracle.grid import Grid
    from paper_2009_02171_gb300.inputs import initial_state
    s = initial_state(c['Ns'], c['Nr'], c['seed'])
    return cfl_alfven(Grid(c['Ns'], c['Nr']), s['B'], c['E'], c['Pm'], 1.0)


def oracle_step_time(c, max_steps, budget_s=ORACLE_BUDGET_S):
    """Real time steps of the CPU oracle (FP64, numpy/scipy + plain-C ILU(0), one thread) on workload c:
    its setup (matrices, subdomain ILU(0) factors) untimed, then steps 1, 2, ... of the trajectory until
    max_steps or budget_s seconds (at least one).  Returns (ms per step, description)."""
    os.environ.setdefault('OMP_NUM_THREADS', '1')
    os.environ.setdefault('OPENBLAS_NUM_THREADS', '1')
    from oracle.grid import Grid
    from oracle.timestep import Physics, SolverOptions, Stepper
    from paper_2009_02171_gb300.inputs import initial_state
    t0 = time.perf_counter()
    dt = stable_dt(oracle_cfl_per_unit_dt(c))
    st = Stepper(Grid(c['Ns'], c['Nr']), Physics(c['E'], c['Ra'], c['Pr'], c['Pm'], dt),
                 SolverOptions(parts=c['p'], delta=c['overlap'], ppbe_levels=c['levels'],
                               delta_c=c['overlap_coarse'], rtol=c['rtol'], restart=c['restart'],
                               parts_c=c.get('coarse_p')))
    setup = time.perf_counter() - t0
    s = dict(initial_state(c['Ns'], c['Nr'], c['seed']), first=True)
    times, its = [], []
    t_all = time.perf_counter()
    while len(times) < max(1, max_steps) and (not times or time.perf_counter() - t_all < budget_s):
        t = time.perf_counter()
        s, info = st.step(s)
        times.append(time.perf_counter() - t)
        its.append((info['vtbe'].iters, info['ppbe'].iters))
    ms = sum(times) / len(times) * 1e3
    cells = 6 * c['Ns'] ** 2 * c['Nr']
    return ms, dict(kind='oracle', cores=1, unit='ms/step', timed_steps=len(times), setup_s=round(setup, 1),
                    dt=dt, iterations_vtbe_ppbe=its, nproc=os.cpu_count(),
                    sample='oracle time steps 1..%d of the same workload (6x%d^2x%d, %d cells, dt %.2g, same solver '
                           'options), no warm-up, one thread; setup (matrices, ILU(0) factors) %.0f s untimed'
                           % (len(times), c['Ns'], c['Nr'], cells, dt, setup))


def reference_arm(args, rank, ws):
    if rank != 0:
        return
    c = config_of(args)
    ms, cb = oracle_step_time(c, args.steps)
    cb['value'] = ms
    print(json.dumps({'impl': 'reference', 'metric': METRIC, 'value': ms, 'unit': 'ms/step', 'n_gpus': args.gpus,
                      'steps': cb['timed_steps'], 'requested_steps': args.steps, 'warmup': 0,
                      'requested_warmup': args.warmup, 'ms_per_step': ms, 'higher_is_better': False,
                      'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
                      'config': {'workload': workload_name(c), 'dt': cb['dt']}, 'cpu_baseline': cb,
                      'e2e': {'value': ms, 'unit': 'ms/step', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}}))


BATCH = dict(Ns=48, Nr=48, nrhs=32, nboxes=512, overlap=2, rtol=1e-8, restart=30, dt=1e-4)


def batch_workload(args, fv, torch, rank, ws):
    """32 PPBE right-hand sides (seeds 100..131) on 6 x 48^2 x 48 with 512 uneven subdomains
    (edges 8..24 cells, overlap 2), FP32 subdomain solves in the FP64 outer FGMRES."""
    import numpy as np
    from paper_2009_02171_gb300.inputs import random_vector, uneven_boxes
    c = BATCH
    boxes = uneven_boxes(c['Ns'], c['Nr'], target=c['nboxes'], seed=0)
    g = fv.fv_build_grid(c['Ns'], c['Nr'])
    s = fv.fv_assemble_system(g, fv.FV_PPBE, E=CFG['E'], Ra=CFG['Ra'], Pr=CFG['Pr'], Pm=CFG['Pm'], dt=c['dt'],
                              overlap=c['overlap'], boxes=boxes, precision=fv.FV_PREC_FP32)
    n = fv.fv_system_size(s)
    # right-hand sides b = A x for seeded random x: in the range of A, so consistent for the
    # singular Neumann pressure block
    Xt = torch.tensor(np.stack([random_vector(n, 100 + r) for r in range(c['nrhs'])]), device='cuda')
    Bd = torch.empty_like(Xt)
    for r in range(c['nrhs']):
        fv.fv_apply_op(s, Xt[r], Bd[r])
    X = torch.zeros_like(Bd)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        X.zero_()
        fv.fv_gmres_solve_batch(s, Bd, X, restart=c['restart'], rtol=c['rtol'])
    with ClockSampler(int(os.environ.get('LOCAL_RANK', '0'))) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            X.zero_()
            st = fv.fv_gmres_solve_batch(s, Bd, X, restart=c['restart'], rtol=c['rtol'])
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # the same 32 right-hand sides one at a time (batches of one: same preconditioner, no sharing)
    x1 = torch.zeros(1, n, dtype=torch.float64, device='cuda')
    fv.fv_gmres_solve_batch(s, Bd[:1].contiguous(), x1, restart=c['restart'], rtol=c['rtol'])  # tune G for nrhs = 1
    e0.record(stream)
    its1 = []
    for r in range(c['nrhs']):
        x1.zero_()
        its1.append(fv.fv_gmres_solve_batch(s, Bd[r:r + 1].contiguous(), x1, restart=c['restart'],
                                            rtol=c['rtol'])[0].iters)
    e1.record(stream)
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1)
    if rank == 0:
        print(json.dumps({'metric': 'wall time per batched solve of 32 right-hand sides at 1e-8 residual',
                          'value': round(ms, 3), 'unit': 'ms/solve', 'n_gpus': ws, 'steps': args.steps,
                          'warmup': args.warmup, 'higher_is_better': False, 'scaling': 'weak',
                          'dtype': 'f32 subdomain solves / f64 outer', 'data': 'synthetic',
                          'config': {'workload': 'PPBE 6x48^2x48, 32 RHS b = A x (x seeded 100..131), 512 uneven '
                                                 'subdomains (edges 8..24) + overlap 2, one-level RAS, FGMRES(30) '
                                                 'to 1e-8'},
                          'iterations': [x.iters for x in st], 'converged': all(x.converged for x in st),
                          'unbatched_ms': round(ms1, 3), 'unbatched_iterations': its1,
                          'clocks': clk.summary()}))
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


def net_workload(args, fv, torch, rank, ws):
    """The learned correction's network alone on the bench's coarse grid (6 x 32^3, C = 16, 3 levels):
    forward of one sample (as inside the preconditioner) and one training step of a batch of 8."""
    from paper_2009_02171_gb300.inputs import multiscale_fields
    c = config_of(args)
    ns, nr, L = c['Ns'] // 2, c['Nr'] // 2, c['learn']
    net = fv.fv_net_create(L['C'], ns, nr, levels=L['levels'], max_batch=L['batch'])
    fv.fv_net_init(net, 1)
    R = torch.tensor(multiscale_fields(ns, nr, L['batch'], seed=1), device='cuda')
    E = torch.empty_like(R)
    r0, e_0 = R[0].contiguous(), E[0].contiguous()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        fv.fv_net_forward(net, 1, r0, e_0)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push('net_forward')  # ncu --nvtx --nvtx-include net_forward/: the timed forwards
    e0.record(stream)
    for _ in range(args.steps):
        fv.fv_net_forward(net, 1, r0, e_0)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms_f = e0.elapsed_time(e1) / args.steps
    fv.fv_net_train(net, R, R.clone(), epochs=max(1, args.warmup), batch=L['batch'], seed=1, lr=L['lr'])
    torch.cuda.synchronize()
    e0.record(stream)
    fv.fv_net_train(net, R, R.clone(), epochs=args.steps, batch=L['batch'], seed=2, lr=L['lr'])
    e1.record(stream)
    torch.cuda.synchronize()
    ms_t = e0.elapsed_time(e1) / args.steps
    flops = network_flops(c)
    peaks = json.load(open(os.path.join(ROOT, 'MEASURED_PEAKS.json'))) if os.path.exists(
        os.path.join(ROOT, 'MEASURED_PEAKS.json')) else {}
    pk = peaks.get('bf16_tflops', 1869.0)
    ach = flops / (ms_f * 1e-3) / 1e12
    if rank == 0:
        print(json.dumps({'metric': 'learned-correction network forward time (one sample)', 'value': round(ms_f, 4),
                          'unit': 'ms/forward', 'n_gpus': ws, 'steps': args.steps, 'warmup': args.warmup,
                          'higher_is_better': False, 'scaling': 'weak', 'dtype': 'bf16 x bf16 -> f32',
                          'data': 'synthetic', 'config': {'workload': 'cubed-sphere U-Net C=%d, %d levels, grid 6x%d^2x%d'
                                                          % (L['C'], L['levels'], ns, nr)},
                          'train_step_ms_batch8': round(ms_t, 3),
                          # per forward: sumsq + ordered sum, pack, ring; per level 2 convolutions (+ pool and its
                          # ring below level 0); per decoder level 1 convolution; output conv; unpack
                          'gpu_launches': args.steps * (8 + 5 * L['levels']),
                          'roofline': {'kernel': 'net_fwd', 'bound': 'tensor', 'achieved': round(ach, 2), 'peak': pk,
                                       'unit': 'TFLOP/s', 'frac': round(ach / pk, 4),
                                       'traffic': TRAFFIC['net_fwd'][0] if not args.ns else None,
                                       'traffic_source': TRAFFIC['net_fwd'][1] if not args.ns else None,
                                       'flops_per_launch': flops,
                                       'peak_source': 'MEASURED_PEAKS.json bf16_tflops (of measured; timed alone)'}}))
    fv.fv_net_free(net)


def trajectory_workload(args, fv, torch, rank, ws, c, host, dt):
    """Per-step metrics of one arm (JSON lines): iterations, final residuals, E_kin, E_mag, Alfven CFL number,
    face and cell divergence of B (fv_state_diagnostics); stops at the first failed step and reports it."""
    h, t_setup, _ = build_arm(fv, torch, c, dt, args.precision or 'fp64', host)
    d = fv.fv_state_diagnostics(h['st'], h['P'])
    if rank == 0:
        print(json.dumps({'step': 0, 'dt': dt, 'precision': args.precision or 'fp64', 'workload': workload_name(c),
                          'setup_s': round(t_setup, 2), 'E_kin': d['E_kin'], 'E_mag': d['E_mag'],
                          'cfl_alfven': d['cfl_alfven']}), flush=True)
    for n in range(1, args.steps + 1):
        try:
            s = fv.fv_time_step(h['st'], h['V'], h['P'], 1, restart=c['restart'], rtol=c['rtol'])
        except fv.FvError as e:
            if rank == 0:
                print(json.dumps({'step': n, 'error': str(e)}), flush=True)
            break
        d = fv.fv_state_diagnostics(h['st'], h['P'])
        if rank == 0:
            print(json.dumps({'step': n, 'iters_vtbe': s[0].iters, 'iters_ppbe': s[1].iters,
                              'rfinal_vtbe': s[0].rfinal, 'rfinal_ppbe': s[1].rfinal, 'E_kin': d['E_kin'],
                              'E_mag': d['E_mag'], 'cfl_alfven': d['cfl_alfven'], 'divB_face': d['divB_face'],
                              'divB_rhs': d['divB_rhs'], 'divB_cell': d['divB_cell']}), flush=True)
    free_arm(fv, h)


def apply_workload(args, fv, torch, rank, ws, c, dt):
    """y = A x alone, VTBE and PPBE, FP64 (fv_apply_op) and FP32 (fv_apply_op_fp32), on workload c: CUDA-event
    time per apply over --steps applies (after --warmup) on inputs larger than L2 (a ring of vectors whose
    total exceeds 129 MB, so every apply reads x from HBM), kernel split from the library's timers."""
    from paper_2009_02171_gb300.inputs import random_vector
    g = fv.fv_build_grid(c['Ns'], c['Nr'])
    peaks = json.load(open(os.path.join(ROOT, 'MEASURED_PEAKS.json'))) if os.path.exists(
        os.path.join(ROOT, 'MEASURED_PEAKS.json')) else {}
    hbm = peaks.get('hbm_gbs', 6800.0)
    out = {}
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    N = 6 * c['Ns'] ** 2 * c['Nr']
    for kind, name in ((fv.FV_VTBE, 'vtbe'), (fv.FV_PPBE, 'ppbe')):
        s = fv.fv_assemble_system(g, kind, E=c['E'], Ra=c['Ra'], Pr=c['Pr'], Pm=c['Pm'], dt=dt,
                                  precision=fv.FV_PREC_FP32, inner_maxit=1, coarse_maxit=1)
        n = fv.fv_system_size(s)
        for dtype, es, call in ((torch.float64, 8, fv.fv_apply_op), (torch.float32, 4, fv.fv_apply_op_fp32)):
            ring = max(2, int(3 * 129e6 / (2 * n * es)) + 1)
            X = [torch.tensor(random_vector(n, 7 + q), dtype=dtype, device='cuda') for q in range(ring)]
            Y = [torch.empty_like(X[0]) for _ in range(ring)]
            for q in range(args.warmup):
                call(s, X[q % ring], Y[q % ring])
            torch.cuda.synchronize()
            e0.record(stream)
            for q in range(args.steps):
                call(s, X[q % ring], Y[q % ring])
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            fv.fv_profile_enable(True)
            for q in range(args.steps):
                call(s, X[q % ring], Y[q % ring])
            kern = {}
            for cat in (fv.K_NAMES_INV['ghost'], fv.K_NAMES_INV['apply_' + name]):
                cat += fv.K_FP32 if es == 4 else 0
                nl, t = fv.fv_profile_read(cat)
                kern[fv.category_name(cat)] = round(t / max(nl, 1) * 1e3, 2)
            fv.fv_profile_enable(False)
            d = 7 if kind == fv.FV_VTBE else 2
            nbytes = 2 * d * N * es
            out['%s_%s' % (name, 'fp64' if es == 8 else 'fp32')] = {
                'us_per_apply': round(ms * 1e3, 2), 'bytes': nbytes, 'GBps': round(nbytes / (ms * 1e-3) / 1e9, 1),
                'frac_of_hbm': round(nbytes / (ms * 1e-3) / 1e9 / hbm, 4), 'kernel_us_edge_tile': kern}
            del X, Y
        fv.fv_free_system(s)
    fv.fv_free_grid(g)
    if rank == 0:
        print(json.dumps({'metric': 'operator apply time and algorithmic HBM bandwidth', 'workload':
                          'y = A x on 6x%d^2x%d (%d cells), dt %.2g' % (c['Ns'], c['Nr'], N, dt),
                          'steps': args.steps, 'warmup': args.warmup, 'hbm_peak_gbs': hbm,
                          'peak_source': 'MEASURED_PEAKS.json hbm_gbs (of measured)',
                          'l2': 'ring of input vectors > 3 x L2', 'applies': out}))


# the paper's strong-scaling workload (Sec. 4.3, tab:strong): benchmark P8 (E = 1e-3, Pr = 1, Ra = 100,
# Pm = 8) from its initial condition (eqn:initial) on 6 x 144^2 x 168 at dt = 1e-5, overlap 1, ILU(0),
# GMRES(30), VTBE one-level RAS, PPBE one- and two-level (coarse inner GMRES to 0.1); tolerances
# eps_a / eps_r 1e-10 / 1e-8 (VTBE) and 1e-8 / 1e-6 (PPBE); one subdomain per processor core of the
# paper's runs: np = 6 p1 p2 p3.  Printed averages over the first ten steps (tab:strong) for context:
# np -> (VTBE its, VTBE s, PPBE one-level its, s, two-level its, inner its, s).
STRONG = dict(Ns=144, Nr=168, E=1e-3, Ra=100.0, Pr=1.0, Pm=8.0, dt=1e-5, overlap=1, restart=30,
              vtbe=dict(atol=1e-10, rtol=1e-8), ppbe=dict(atol=1e-8, rtol=1e-6),
              decomps={1296: (6, 6, 6), 2592: (6, 6, 12), 5184: (12, 6, 12), 10368: (12, 12, 12)})
STRONG_PAPER = {1296: (3.0, 6.65, 144.9, 29.69, 22.0, 13.4, 15.80), 2592: (3.0, 3.41, 154.0, 16.90, 22.2, 16.0, 10.18),
                5184: (3.0, 1.77, 158.0, 9.60, 22.1, 14.0, 5.72), 10368: (3.0, 0.92, 151.1, 5.24, 22.4, 16.1, 4.20)}


def strong_workload(args, fv, torch, rank, ws):
    """tab:strong replayed on one GB300, FP64 throughout: for each of the paper's subdomain counts, --steps time
    steps (first steps of the trajectory) with one-level and with two-level PPBE; averages of the outer
    iterations, coarse inner iterations and GPU solve times per step of each system."""
    import numpy as np
    from paper_2009_02171_gb300.inputs import benchmark_state
    c = STRONG
    ph = dict(E=c['E'], Ra=c['Ra'], Pr=c['Pr'], Pm=c['Pm'], dt=c['dt'])
    s0 = benchmark_state(c['Ns'], c['Nr'])
    host = np.concatenate([s0['u'].ravel(), s0['T'], s0['B'].ravel(), s0['P'], s0['Pb']])
    g = fv.fv_build_grid(c['Ns'], c['Nr'])
    init = torch.tensor(host, device='cuda')
    st = fv.fv_state_create(g, init, **ph)
    cfl = fv.fv_state_diagnostics(st)['cfl_alfven']
    rows = {}
    for npc, parts in c['decomps'].items():
        t0 = time.perf_counter()
        V = fv.fv_assemble_system(g, fv.FV_VTBE, **ph, p=parts, overlap=c['overlap'], levels=1)
        row = {'subdomains': 6 * parts[0] * parts[1] * parts[2], 'boxes': [c['Ns'] // parts[0], c['Ns'] // parts[1],
                                                                           c['Nr'] // parts[2]]}
        for lv in (1, 2):
            P = fv.fv_assemble_system(g, fv.FV_PPBE, **ph, p=parts, overlap=c['overlap'], levels=lv, overlap_coarse=1,
                                      coarse_rtol=0.1)
            fv.fv_state_reset(st, init)
            vi, vt, pi, pin, pt = [], [], [], [], []
            for _ in range(args.steps):
                sv, sp = fv.fv_time_step_opts(st, V, P, 1, vtbe_opts=dict(c['vtbe'], restart=c['restart']),
                                              ppbe_opts=dict(c['ppbe'], restart=c['restart']))
                vi.append(sv.iters), vt.append(sv.time_ms), pi.append(sp.iters), pin.append(sp.inner_iters)
                pt.append(sp.time_ms)
            mean = lambda a: round(sum(a) / len(a), 2)
            if lv == 1:
                row.update(vtbe_its=mean(vi), vtbe_ms=mean(vt), ppbe1_its=mean(pi), ppbe1_ms=mean(pt))
            else:
                row.update(ppbe2_its=mean(pi), ppbe2_inner_per_outer=round(sum(pin) / max(sum(pi), 1), 1),
                           ppbe2_ms=mean(pt))
            fv.fv_free_system(P)
        fv.fv_free_system(V)
        row['setup_s'] = round(time.perf_counter() - t0, 1)
        pp = STRONG_PAPER[npc]
        row['paper_taihulight'] = dict(vtbe_its=pp[0], vtbe_s=pp[1], ppbe1_its=pp[2], ppbe1_s=pp[3], ppbe2_its=pp[4],
                                       ppbe2_inner=pp[5], ppbe2_s=pp[6])
        rows[npc] = row
        if rank == 0:
            print(json.dumps({'np': npc, **row}), flush=True)
    fv.fv_free_state(st)
    fv.fv_free_grid(g)
    if rank == 0:
        print(json.dumps({'metric': 'strong-scaling workload replayed on one GPU (tab:strong)', 'workload':
                          'P8 on 6x144^2x168 (20.9M cells), dt 1e-5, FP64, GMRES(30), overlap 1, ILU(0)',
                          'cfl_alfven': round(cfl, 3), 'steps': args.steps, 'rows': rows}))


# benchmark P8 (Sec. 4.2, tab:gridlevels, tab:comparison): E = 1e-3, Pr = 1, Ra = 100, Pm = 8 from the
# initial condition eqn:initial on grid G48 (6 x 48^2 x 72), dt = 8e-5 (CFL_A 1.12), run to t = 8 (one magnetic
# diffusion time, 100,000 steps); the paper's G48 energies at the quasi-steady state and the pseudospectral
# reference (tab:comparison)
P8 = dict(Ns=48, Nr=72, E=1e-3, Ra=100.0, Pr=1.0, Pm=8.0, dt=8e-5, p=(3, 3, 3), overlap=2, overlap_coarse=1,
          levels=2, vtbe_inner=4, ppbe_inner=8, coarse_its=10, inner_gs=1,
          vtbe=dict(atol=1e-10, rtol=1e-8), ppbe=dict(atol=1e-8, rtol=1e-6))
P8_PAPER = dict(G48=dict(E_mag=313663.1, E_kin=21928.4), PS=dict(E_mag=312754.7, E_kin=21634.9))


def p8_workload(args, fv, torch, rank, ws):
    """Benchmark P8 on G48 with the mixed-precision solver (both systems to the paper's stopping rules):
    E_kin and E_mag (Sec. 4.2 definitions) every --every steps, to compare with tab:comparison."""
    import numpy as np
    from paper_2009_02171_gb300.inputs import benchmark_state
    c = dict(P8)
    for k, a in (('coarse_its', args.coarse_its), ('ppbe_inner', args.ppbe_inner), ('vtbe_inner', args.vtbe_inner)):
        if a:
            c[k] = a
    ph = dict(E=c['E'], Ra=c['Ra'], Pr=c['Pr'], Pm=c['Pm'], dt=c['dt'])
    s0 = benchmark_state(c['Ns'], c['Nr'])
    host = np.concatenate([s0['u'].ravel(), s0['T'], s0['B'].ravel(), s0['P'], s0['Pb']])
    t0 = time.perf_counter()
    g = fv.fv_build_grid(c['Ns'], c['Nr'])
    mv = dict(precision=fv.FV_PREC_FP32, inner_maxit=c['vtbe_inner'], inner_gs_passes=c['inner_gs'])
    mp = dict(precision=fv.FV_PREC_FP32, inner_maxit=c['ppbe_inner'], coarse_maxit=c['coarse_its'],
              inner_gs_passes=c['inner_gs'])
    V = fv.fv_assemble_system(g, fv.FV_VTBE, **ph, p=c['p'], overlap=c['overlap'], levels=1, **mv)
    P = fv.fv_assemble_system(g, fv.FV_PPBE, **ph, p=c['p'], overlap=c['overlap'], levels=c['levels'],
                              overlap_coarse=c['overlap_coarse'], **mp)
    st = fv.fv_state_create(g, torch.tensor(host, device='cuda'), **ph)
    d = fv.fv_state_diagnostics(st, P)
    if rank == 0:
        print(json.dumps({'step': 0, 't': 0.0, 'E_kin': d['E_kin'], 'E_mag': d['E_mag'], 'cfl_alfven': d['cfl_alfven'],
                          'setup_s': round(time.perf_counter() - t0, 1)}), flush=True)
    vo, po = dict(c['vtbe'], restart=30), dict(c['ppbe'], restart=30)
    t_run, n, its, hist = time.perf_counter(), 0, [0, 0], []
    while n < args.steps:
        k = min(args.every, args.steps - n)
        ss = fv.fv_time_step_opts(st, V, P, k, vtbe_opts=vo, ppbe_opts=po)
        n += k
        its[0] += sum(x.iters for x in ss[0::2])
        its[1] += sum(x.iters for x in ss[1::2])
        d = fv.fv_state_diagnostics(st, P)
        el = time.perf_counter() - t_run
        hist.append((n * c['dt'], d['E_kin'], d['E_mag']))
        if rank == 0:
            print(json.dumps({'step': n, 't': round(n * c['dt'], 5), 'E_kin': d['E_kin'], 'E_mag': d['E_mag'],
                              'cfl_alfven': d['cfl_alfven'], 'divB_face_over_rhs': d['divB_face'] / d['divB_rhs'],
                              'its_vtbe_ppbe_mean': [round(its[0] / n, 2), round(its[1] / n, 2)],
                              'ms_per_step': round(el / n * 1e3, 2)}), flush=True)
        if not (np.isfinite(d['E_kin']) and np.isfinite(d['E_mag'])):
            break
        if args.budget_min and el > args.budget_min * 60:
            break
    # time averages over the last quarter of the run (t_m = t / Pm in [0.75, 1] for the full run to t = 8:
    # the quasi-steady part of the P8 solution), the form the table's global quantities take
    t_end = n * c['dt']
    tail = [h for h in hist if h[0] >= 0.75 * t_end] or hist[-1:]
    avg = {'E_kin': float(np.mean([h[1] for h in tail])), 'E_mag': float(np.mean([h[2] for h in tail])),
           'samples': len(tail), 't_from': tail[0][0] if tail else None}
    if rank == 0:
        print(json.dumps({'metric': 'benchmark P8 on G48 (tab:comparison)', 'steps': n, 't': n * c['dt'],
                          'mean_last_quarter': avg,
                          'rel_mean_vs_paper_G48': {k: avg[k] / P8_PAPER['G48'][k] - 1 for k in ('E_mag', 'E_kin')},
                          'rel_mean_vs_PS': {k: avg[k] / P8_PAPER['PS'][k] - 1 for k in ('E_mag', 'E_kin')},
                          'inner_iterations_vtbe_ppbe_coarse': [c['vtbe_inner'], c['ppbe_inner'], c['coarse_its']],
                          't_magnetic': n * c['dt'] / c['Pm'], 'E_kin': d['E_kin'], 'E_mag': d['E_mag'],
                          'paper': P8_PAPER, 'rel_vs_paper_G48': {k: d[k] / P8_PAPER['G48'][k] - 1 for k in
                                                                  ('E_mag', 'E_kin')},
                          'ms_per_step': round((time.perf_counter() - t_run) / max(n, 1) * 1e3, 2)}), flush=True)
    for h, f in ((st, fv.fv_free_state), (V, fv.fv_free_system), (P, fv.fv_free_system), (g, fv.fv_free_grid)):
        f(h)


# convergence study (Sec. 4.1): Pr = 1, Ra = 100, E = 0.1, Pm = 1000, initial condition eqn:initial.  Space:
# dt = 1e-5 to t = 1e-3 on 6 x N^3 against N = 128 (reference restricted by 2 x 2 x 2 means).  Time: 6 x 32^3 to
# t = 1 against the smallest step (the paper's printed reference step is read as garbled).  FP64 solves to a
# 1e-10 relative residual; boxes of 16^3 cells, two-level PPBE.
CONV = dict(E=0.1, Ra=100.0, Pr=1.0, Pm=1000.0, rtol=1e-10, space_grids=(16, 32, 64), space_ref=128,
            space_dt=1e-5, space_t=1e-3, time_grid=32, time_dts=(8e-3, 4e-3, 2e-3, 1e-3), time_ref_dt=2.5e-4,
            time_t=1.0)


def convergence_workload(args, fv, torch, rank, ws):
    """L2 errors (Sec. 4.1 definition, sqrt(sum_c sum_cells (v - v_ref)^2 V)) of u, Theta and B against a
    finer reference, in space and in time, and the observed orders."""
    import numpy as np
    from paper_2009_02171_gb300.inputs import benchmark_state
    c = CONV
    ph0 = dict(E=c['E'], Ra=c['Ra'], Pr=c['Pr'], Pm=c['Pm'])

    def run(n, dt, t_end):
        g = fv.fv_build_grid(n, n)
        ph = dict(ph0, dt=dt)
        parts = (max(1, n // 16),) * 3
        V = fv.fv_assemble_system(g, fv.FV_VTBE, **ph, p=parts, overlap=1, levels=1)
        P = fv.fv_assemble_system(g, fv.FV_PPBE, **ph, p=parts, overlap=1, levels=2 if n >= 16 else 1,
                                  overlap_coarse=1)
        s0 = benchmark_state(n, n)
        host = np.concatenate([s0['u'].ravel(), s0['T'], s0['B'].ravel(), s0['P'], s0['Pb']])
        st = fv.fv_state_create(g, torch.tensor(host, device='cuda'), **ph)
        steps = int(round(t_end / dt))
        t0 = time.perf_counter()
        left = steps
        while left:
            k = min(left, 100)
            fv.fv_time_step(st, V, P, k, rtol=c['rtol'])
            left -= k
        out = torch.empty(host.size, dtype=torch.float64, device='cuda')
        x = fv.fv_state_get(st, out).cpu().numpy()
        el = time.perf_counter() - t0
        for h, f in ((st, fv.fv_free_state), (V, fv.fv_free_system), (P, fv.fv_free_system), (g, fv.fv_free_grid)):
            f(h)
        return x, steps, el

    def volumes(n, ri=7.0 / 13.0, ro=20.0 / 13.0):
        """Cell volumes sqrt(g)(centre) h_s^2 h_r (Sec. 3.2), [panel][k][j][i]."""
        hs, hr = np.pi / (2 * n), (ro - ri) / n
        xi = -np.pi / 4 + (np.arange(n) + 0.5) * hs
        X, Y = np.tan(xi)[None, :], np.tan(xi)[:, None]
        d = 1 + X * X + Y * Y
        sig = (1 + X * X) * (1 + Y * Y) / d ** 1.5
        r = ri + (np.arange(n) + 0.5) * hr
        v = (r ** 2)[:, None, None] * sig[None] * hs * hs * hr
        return np.broadcast_to(v, (6, n, n, n)).ravel()

    def restrict(x, n, levels):
        """Mean of the 2 x 2 x 2 children, `levels` times, per field ([comp][panel][k][j][i])."""
        a = x.reshape(-1, 6, n, n, n)
        for _ in range(levels):
            m = a.shape[2] // 2
            a = a.reshape(a.shape[0], 6, m, 2, m, 2, m, 2).mean(axis=(3, 5, 7))
        return a.reshape(a.shape[0], -1)

    def l2(x, ref, n):
        v = volumes(n)
        xa, ra = x.reshape(9, -1), ref.reshape(9, -1)
        out = {}
        for name, sl in (('u', slice(0, 3)), ('T', slice(3, 4)), ('B', slice(4, 7))):
            out[name] = float(np.sqrt((((xa[sl] - ra[sl]) ** 2) * v).sum()))
        return out

    res = {'space': {}, 'time': {}}
    ref, _, el = run(c['space_ref'], c['space_dt'], c['space_t'])
    res['space']['reference'] = dict(n=c['space_ref'], seconds=round(el, 1))
    lev = {n: int(round(np.log2(c['space_ref'] / n))) for n in c['space_grids']}
    errs = {}
    for n in c['space_grids']:
        x, steps, el = run(n, c['space_dt'], c['space_t'])
        errs[n] = l2(x, restrict(ref, c['space_ref'], lev[n]).ravel(), n)
        res['space'][n] = dict(errs[n], steps=steps, seconds=round(el, 1))
    ns = list(c['space_grids'])
    res['space']['orders'] = {f: [round(np.log2(errs[a][f] / errs[b][f]), 2) for a, b in zip(ns, ns[1:])]
                              for f in ('u', 'T', 'B')}
    n = c['time_grid']
    ref, steps, el = run(n, c['time_ref_dt'], c['time_t'])
    res['time']['reference'] = dict(dt=c['time_ref_dt'], steps=steps, seconds=round(el, 1))
    errs = {}
    for dt in c['time_dts']:
        x, steps, el = run(n, dt, c['time_t'])
        errs[dt] = l2(x, ref, n)
        res['time'][dt] = dict(errs[dt], steps=steps, seconds=round(el, 1))
    ds = list(c['time_dts'])
    res['time']['orders'] = {f: [round(np.log2(errs[a][f] / errs[b][f]), 2) for a, b in zip(ds, ds[1:])]
                             for f in ('u', 'T', 'B')}
    if rank == 0:
        print(json.dumps({'metric': 'convergence study (Sec. 4.1): L2 errors and orders', 'physics': ph0,
                          'results': {k: {str(kk): vv for kk, vv in v.items()} for k, v in res.items()}}))


def build_arm(fv, torch, c, dt, mode, host):
    """(handles, setup seconds, learned-correction info) of arm mode in {fp64, mixed, bf16, learned} on workload c
    (bf16: mixed precision with the ILU(0) factors stored in BF16)."""
    ph = dict(E=c['E'], Ra=c['Ra'], Pr=c['Pr'], Pm=c['Pm'], dt=dt)
    t = time.perf_counter()
    mixed = mode != 'fp64'
    prec = fv.FV_PREC_BF16 if mode == 'bf16' else fv.FV_PREC_FP32
    g = fv.fv_build_grid(c['Ns'], c['Nr'])
    mv = dict(precision=prec, inner_maxit=c['vtbe_inner'], inner_gs_passes=c['inner_gs']) if mixed else {}
    mpp = dict(precision=prec, inner_maxit=c['ppbe_inner'], coarse_maxit=c['coarse_its'],
               inner_gs_passes=c['inner_gs']) if mixed else {}
    V = fv.fv_assemble_system(g, fv.FV_VTBE, **ph, p=c['p'], overlap=c['overlap'], levels=1, **mv)
    P = fv.fv_assemble_system(g, fv.FV_PPBE, **ph, p=c['p'], overlap=c['overlap'], levels=c['levels'],
                              overlap_coarse=c['overlap_coarse'], coarse_p=c.get('coarse_p', (0, 0, 0)), **mpp)
    net, info = None, None
    if mode == 'learned':
        from paper_2009_02171_gb300.learned import train_learned_correction
        L = c.get('learn', LEARN)
        net, info = train_learned_correction(P, c['Ns'], c['Nr'], C=L['C'], levels=L['levels'], npairs=L['pairs'],
                                             epochs=L['epochs'], batch=L['batch'], lr=L['lr'],
                                             coarse_its=L['coarse_its'],
                                             flags=fv.FV_LEARN_GUESS if L.get('guess') else 0)
    init = torch.tensor(host, device='cuda')
    st = fv.fv_state_create(g, init, **ph)
    torch.cuda.synchronize()
    return dict(g=g, V=V, P=P, st=st, net=net, init=init), time.perf_counter() - t, info


def free_arm(fv, h):
    if h['net'] is not None:
        fv.fv_pc_set_learned(h['P'], None)
        fv.fv_net_free(h['net'])
    fv.fv_free_state(h['st'])
    fv.fv_free_system(h['V'])
    fv.fv_free_system(h['P'])
    fv.fv_free_grid(h['g'])


def main():
    args = parse()
    if args.impl == 'reference':
        import torch.distributed as dist
        rank, ws, _ = dist_setup('gloo')
        reference_arm(args, rank, ws)
        if ws > 1:
            dist.destroy_process_group()
        return
    import numpy as np
    import torch
    import torch.distributed as dist
    rank, ws, local = dist_setup('nccl')
    torch.cuda.set_device(local)
    from paper_2009_02171_gb300 import fv
    from paper_2009_02171_gb300.inputs import initial_state
    if args.workload in ('batch', 'net', 'strong', 'p8', 'convergence'):
        {'batch': batch_workload, 'net': net_workload, 'strong': strong_workload, 'p8': p8_workload,
         'convergence': convergence_workload}[args.workload](args, fv, torch, rank, ws)
        if ws > 1:
            dist.destroy_process_group()
        return

    c = config_of(args)
    s0 = initial_state(c['Ns'], c['Nr'], c['seed'] + rank)
    host = np.concatenate([s0['u'].ravel(), s0['T'], s0['B'].ravel(), s0['P'], s0['Pb']])
    N = host.size // 9
    # time step from the live Alfven CFL number of the seeded field (computed by the library on the GPU)
    g0 = fv.fv_build_grid(c['Ns'], c['Nr'])
    st0 = fv.fv_state_create(g0, torch.tensor(host, device='cuda'), E=c['E'], Ra=c['Ra'], Pr=c['Pr'], Pm=c['Pm'],
                             dt=1.0)
    cfl_unit = fv.fv_state_diagnostics(st0)['cfl_alfven']
    fv.fv_free_state(st0)
    fv.fv_free_grid(g0)
    dt = stable_dt(cfl_unit)
    if args.workload in ('trajectory', 'apply'):
        if args.workload == 'trajectory':
            trajectory_workload(args, fv, torch, rank, ws, c, host, args.dt or dt)
        else:
            apply_workload(args, fv, torch, rank, ws, c, args.dt or dt)
        if ws > 1:
            dist.destroy_process_group()
        return
    opts = dict(restart=c['restart'], rtol=c['rtol'])
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(h, steps, warmup, profile=False, label=None):
        """Restart from the seeded fields (fresh history), `warmup` untimed steps, `steps` timed steps."""
        V, P, st = h['V'], h['P'], h['st']
        fv.fv_state_reset(st, h['init'])
        for _ in range(warmup):
            fv.fv_time_step(st, V, P, 1, **opts)
        iters = []
        with ClockSampler(local) as clk:
            if ws > 1:
                dist.barrier()
            torch.cuda.synchronize()
            if profile:
                fv.fv_profile_enable(True)
            if label:  # NVTX range: ncu --nvtx --nvtx-include <label>/ captures exactly these launches
                torch.cuda.nvtx.range_push(label)
            e0.record(stream)
            for _ in range(steps):
                s = fv.fv_time_step(st, V, P, 1, **opts)
                iters.append((s[0].iters, s[1].iters, s[0].inner_iters, s[1].inner_iters, s[1].rfinal))
            e1.record(stream)
            if label:
                torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            if ws > 1:
                dist.barrier()
        ms = e0.elapsed_time(e1) / steps
        if ws > 1:
            ms = max_over_ranks(ms, 'cuda')
        return ms, iters, clk.summary()

    def final_fields(h):
        out = torch.empty(9 * N, dtype=torch.float64, device='cuda')
        fv.fv_state_get(h['st'], out)
        return out.cpu().numpy()

    def errors(x, ref):
        """max |x - ref| / max |ref| per field against the FP64 arm after the same steps."""
        sl = {'u': slice(0, 3 * N), 'T': slice(3 * N, 4 * N), 'B': slice(4 * N, 7 * N), 'P': slice(7 * N, 8 * N),
              'Pb': slice(8 * N, 9 * N)}
        return {k: float(np.abs(x[v] - ref[v]).max() / max(np.abs(ref[v]).max(), 1e-300)) for k, v in sl.items()}

    def diag_summary(h, iters):
        d = fv.fv_state_diagnostics(h['st'], h['P'])
        return {'E_kin': d['E_kin'], 'E_mag': d['E_mag'], 'cfl_alfven': d['cfl_alfven'],
                'divB_face': d['divB_face'], 'divB_face_over_rhs': d['divB_face'] / d['divB_rhs'],
                'divB_face_le_ppbe_rfinal': bool(d['divB_face'] <= iters[-1][4] * (1 + 1e-6)),
                'divB_cell_over_rhs': d['divB_cell'] / d['divB_rhs'], 'steps': d['steps']}

    arms = c.get('arms', ('fp64', 'mixed', 'learned'))
    head = args.precision or arms[-1]
    others, ref_fields = {}, None
    # the other arms first (same steps), fp64 first so its final fields are the reference of the others
    if not args.single:
        for mode in [m for m in arms if m != head]:
            other, t_other, info_o = build_arm(fv, torch, c, dt, mode, host)
            ms_o, it_o, _ = timed(other, args.steps, args.warmup)
            x = final_fields(other)
            others[mode] = {'ms_per_step': round(ms_o, 3), 'iterations_vtbe_ppbe': [(i[0], i[1]) for i in it_o],
                            'setup_s': round(t_other, 2), 'diag': diag_summary(other, it_o)}
            if mode == 'fp64':
                ref_fields = x
            elif ref_fields is not None:
                others[mode]['error_vs_fp64'] = errors(x, ref_fields)
            if info_o:
                others[mode]['learned'] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in info_o.items()}
            free_arm(fv, other)
    h, t_setup, info = build_arm(fv, torch, c, dt, head, host)
    ms, iters, clocks = timed(h, args.steps, args.warmup, label='timed_steps')
    x_head = final_fields(h)
    diag = diag_summary(h, iters)
    err = errors(x_head, ref_fields) if ref_fields is not None and head != 'fp64' else None
    ms_prof, _, _ = timed(h, args.steps, args.warmup, profile=True)
    kern = {}
    for cat in range(fv.K_COUNT):
        if cat % 16 not in fv.K_NAMES:
            continue
        n, t = fv.fv_profile_read(cat)
        if n:
            kern[fv.category_name(cat)] = {'launches': n, 'ms_total': round(t, 3),
                                           'ms_per_step': round(t / args.steps, 3)}
    fv.fv_profile_enable(False)

    # end to end through the C ABI: the same steps from the seeded fields, every timed step with the state
    # host -> device (pinned), the step, device -> host
    hbuf = torch.empty(9 * N, dtype=torch.float64).pin_memory()
    dbuf = torch.empty(9 * N, dtype=torch.float64, device='cuda')
    fv.fv_state_reset(h['st'], h['init'])
    for _ in range(args.warmup):
        fv.fv_time_step(h['st'], h['V'], h['P'], 1, **opts)
    fv.fv_state_get(h['st'], dbuf)
    hbuf.copy_(dbuf)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    e0.record(stream)
    for _ in range(args.steps):
        dbuf.copy_(hbuf, non_blocking=True)
        fv.fv_state_set(h['st'], dbuf)
        fv.fv_time_step(h['st'], h['V'], h['P'], 1, **opts)
        fv.fv_state_get(h['st'], dbuf)
        hbuf.copy_(dbuf, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1) / args.steps
    if ws > 1:
        ms_e2e = max_over_ranks(ms_e2e, 'cuda')
    e2e_same = bool(np.array_equal(hbuf.numpy(), x_head))

    # roofline of the dominant kernel category (measured live over the timed region)
    peaks = json.load(open(os.path.join(ROOT, 'MEASURED_PEAKS.json'))) if os.path.exists(
        os.path.join(ROOT, 'MEASURED_PEAKS.json')) else {}
    hbm = peaks.get('hbm_gbs', 6800.0)
    ranked = sorted((v['ms_total'], k) for k, v in kern.items() if not k.startswith('phase'))

    def roof_of(top):
        per_launch_ms = kern[top]['ms_total'] / kern[top]['launches']
        tr = TRAFFIC.get(top) if not args.ns else None
        common = {'kernel': top, 'ms_per_launch': round(per_launch_ms, 4), 'traffic': tr[0] if tr else None,
                  'traffic_source': tr[1] if tr else None,
                  'share_of_step': round(kern[top]['ms_total'] / (ms_prof * args.steps), 3),
                  'top_kernel': ranked[-1][1]}
        if top.startswith('net_fwd'):
            flops = network_flops(c)
            ach = flops / (per_launch_ms * 1e-3) / 1e12
            pk = peaks.get('bf16_tflops_sustained', 1700.0)
            return dict(common, bound='tensor', achieved=round(ach, 2), peak=pk, unit='TFLOP/s',
                        frac=round(ach / pk, 4), flops_per_launch=flops,
                        peak_source='MEASURED_PEAKS.json bf16_tflops_sustained (of measured; kernel inside a long step)')
        bytes_per = algorithmic_bytes(top, c, N, 8)
        if not bytes_per:
            return None
        bwd = top.replace('ras_fwd', 'ras_bwd')
        if top.startswith('ras_fwd') and bwd not in kern:  # sweeps fused into one launch: both counted
            bytes_per += algorithmic_bytes(bwd, c, N, 8)
        ach = bytes_per / (per_launch_ms * 1e-3) / 1e9
        return dict(common, bound='hbm', achieved=round(ach, 1), peak=hbm, unit='GB/s', frac=round(ach / hbm, 4),
                    bytes_per_launch=bytes_per, peak_source='MEASURED_PEAKS.json hbm_gbs (of measured)')

    roof, roof_hbm = None, None
    for _, top in reversed(ranked):  # the dominant category with an algorithmic figure
        roof = roof or roof_of(top)
        if not top.startswith('net_fwd') and roof_of(top) and roof_hbm is None:
            roof_hbm = roof_of(top)
        if roof and roof_hbm:
            break
    if roof is not roof_hbm and roof_hbm is not None and roof is not None and roof['kernel'] != roof_hbm['kernel']:
        roof['next_hbm_bound'] = roof_hbm
    stencil = {k: roof_of(k) for k in ('apply_vtbe_fp32', 'apply_ppbe_fp32', 'apply_vtbe', 'apply_ppbe')
               if k in kern}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, cpu = oracle_step_time(c, args.steps)
        cpu['value'] = round(v, 1)

    if rank == 0:
        print(json.dumps({
            'metric': METRIC, 'value': round(ms, 3), 'unit': 'ms/step', 'n_gpus': ws, 'steps': args.steps,
            'warmup': args.warmup, 'ms_per_step': round(ms, 3), 'higher_is_better': False, 'scaling': 'weak',
            'vs_baseline': None,
            'dtype': {'fp64': 'f64', 'mixed': 'f32 inner / f64 outer', 'bf16': 'f32 inner (bf16 factors) / f64 outer',
                      'learned': 'f32 inner / f64 outer, bf16 network'}[head],
            'data': 'synthetic',
            'precision': head,
            'arms': others,
            'learned': ({k: (round(v, 4) if isinstance(v, float) else v) for k, v in info.items()} if info else None),
            'config': {'workload': workload_name(c),
                       'cells': 6 * c['Ns'] ** 2 * c['Nr'], 'subdomains': 6 * c['p'][0] * c['p'][1] * c['p'][2],
                       'overlap': c['overlap'], 'ppbe_levels': c['levels'], 'rtol': c['rtol'],
                       'restart': c['restart'], 'dt': dt, 'cfl_alfven_initial': round(cfl_unit * dt, 4),
                       'l2': 'working set > L2 (no flush needed)',
                       'parallelism': 'replicas' if ws > 1 else 'single GPU'},
            'iterations': {'vtbe': [i[0] for i in iters], 'ppbe': [i[1] for i in iters],
                           'vtbe_inner': [i[2] for i in iters], 'ppbe_inner': [i[3] for i in iters]},
            'diag': diag, 'error_vs_fp64': err,
            'setup_s': round(t_setup, 2), 'clocks': clocks,
            'e2e': {'value': round(ms_e2e, 3), 'unit': 'ms/step', 'h2d_bytes_per_step': 9 * N * 8,
                    'd2h_bytes_per_step': 9 * N * 8, 'same_fields_as_timed_pass': e2e_same},
            'gpu_launches': int(sum(v['launches'] for k, v in kern.items() if not k.startswith('phase'))),
            'kernels_note': 'per-category CUDA-event times of a profiled pass over the same steps (eager launches, '
                            '%.1f ms/step with timing on)' % ms_prof,
            'kernels': kern, 'roofline': roof, 'stencil': stencil, 'cpu_baseline': cpu}))
    free_arm(fv, h)
    if ws > 1:
        dist.destroy_process_group()


def _split(n, parts):
    return [n // parts + (1 if q < n % parts else 0) for q in range(parts)]


def box_cells(Ns, Nr, p, delta):
    """Cells of all overlapping subdomain boxes (panel boxes extended by delta, radially clipped)."""
    tot = 0
    ks = _split(Nr, p[2])
    k0 = 0
    for kz in ks:
        nz = min(Nr, k0 + kz + delta) - max(0, k0 - delta)
        for sx in _split(Ns, p[0]):
            for sy in _split(Ns, p[1]):
                tot += (sx + 2 * delta) * (sy + 2 * delta) * nz
        k0 += kz
    return 6 * tot


def network_flops(c):
    """Algorithmic FLOPs of one forward pass of the learned correction (one sample): 2 * 27 * ci * co per cell
    of each convolution's level, logical channel counts."""
    learn = c.get('learn', LEARN)
    C, L = learn['C'], learn['levels']
    ns, nr = c['Ns'] // 2, c['Nr'] // 2
    cells = [6 * (ns >> l) ** 2 * (nr >> l) for l in range(L + 1)]
    f = 0
    for l in range(L + 1):
        f += 2 * 27 * (2 if l == 0 else C) * C * cells[l] + 2 * 27 * C * C * cells[l]
    for l in range(L):
        f += 2 * 27 * 2 * C * C * cells[l]
    return f + 2 * 27 * C * 2 * cells[0]


def workload_name(c):
    """Description of the time-step workload c (a CONFIGS entry, possibly resized)."""
    cells = 6 * c['Ns'] ** 2 * c['Nr']
    nsub = 6 * c['p'][0] * c['p'][1] * c['p'][2]
    lv = {1: 'one-level', 2: 'two-level', 3: 'three-level'}.get(c['levels'], '%d-level' % c['levels'])
    return ('shell 6x%d^2x%d (%.2fM cells), time step: VTBE one-level RAS + PPBE %s RAS, %d subdomains overlap %d, '
            'FGMRES(%d) to 1e-8 relative FP64 residual; mixed precision = FP32 inner FGMRES (operator, ILU(0) sweeps, '
            'coarse levels; one Gram-Schmidt pass) inside FP64 outer FGMRES (two passes); learned = mixed with the '
            'PPBE coarse solve replaced by a BF16 cubed-sphere U-Net followed by a few coarse FGMRES iterations'
            % (c['Ns'], c['Nr'], cells / 1e6, lv, nsub, c['overlap'], c['restart'])
            + ('; coarse boxes %d x %d x %d a panel' % tuple(c['coarse_p']) if c.get('coarse_p') else ''))


def config_of(args):
    """The workload of the command line: --config, optionally resized to 6 x ns^2 x ns by --ns."""
    c = dict(CONFIGS[args.config], name=args.config, learn=LEARN_BY_CONFIG.get(args.config, LEARN))
    if args.ns:
        c['Ns'] = c['Nr'] = args.ns
    if args.levels:
        c['levels'] = args.levels
    if args.coarse_its:
        c['coarse_its'] = args.coarse_its
    if args.ppbe_inner:
        c['ppbe_inner'] = args.ppbe_inner
    if args.vtbe_inner:
        c['vtbe_inner'] = args.vtbe_inner
    if args.coarse_p:
        c['coarse_p'] = tuple(int(v) for v in args.coarse_p.split(','))
    if args.learned_its:
        c['learn'] = dict(c['learn'], coarse_its=args.learned_its)
    if args.learn_guess:
        c['learn'] = dict(c['learn'], guess=True)
    return c


def algorithmic_bytes(cat, c, N, es):
    """Algorithmic HBM bytes of one launch of a timing category: what it must read and write.

    apply: read x, write y (d values per cell).  RAS forward sweep (gather fused): per box cell
    read r and the cell map (8 bytes), read the L factors (5 d off-diagonal + d(d-1)/2
    diagonal-block entries), write the local vector; backward sweep (scatter fused): per box
    cell read the local vector, the cell map and owner flag (9 bytes) and the U factors
    (5 d + d(d+1)/2), and write z once per grid cell (d values)."""
    es = 4 if cat.endswith('_fp32') else 8
    base = cat.replace('_fp32', '')
    coarse = base.endswith('_coarse')
    base = base.replace('_coarse', '')
    ncell = N // 8 if coarse else N
    if base in ('apply_vtbe', 'apply_ppbe'):
        d = 7 if base == 'apply_vtbe' else 2
        return 2 * d * ncell * es
    if base.startswith('ras_'):
        d = 7 if base.endswith('vtbe') else 2
        if coarse:
            cp = tuple(min(a or b, m) for a, b, m in zip(c.get('coarse_p', (0, 0, 0)), c['p'],
                                                          (c['Ns'] // 2, c['Ns'] // 2, c['Nr'] // 2)))
            cells = box_cells(c['Ns'] // 2, c['Nr'] // 2, cp, c['overlap_coarse'])
        else:
            cells = box_cells(c['Ns'], c['Nr'], c['p'], c['overlap'])
        fwd = cells * (es * (2 * d + 5 * d + d * (d - 1) // 2) + 8)
        bwd = cells * (es * (d + 5 * d + d * (d + 1) // 2) + 9) + ncell * d * es
        return fwd if base.startswith('ras_fwd') else bwd
    return None


if __name__ == '__main__':
    main()
