"""Thin ctypes binding of libfv.so (the C ABI of include/fv.h and include/fv_net.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
Vectors are torch CUDA float64 tensors (contiguous, component-major
[comp][panel][k][j][i]); their device pointers are passed to the library
together with torch's current CUDA stream.  There is no CPU fallback: if
libfv.so is missing the import of this module raises.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, 'libfv.so')

FV_VTBE, FV_PPBE = 0, 1
FV_PREC_FP64, FV_PREC_FP32, FV_PREC_BF16 = 0, 1, 2
ERRORS = {-1: 'FV_EINVAL', -2: 'FV_ENOMEM', -3: 'FV_ECUDA', -4: 'FV_ENOCONV', -5: 'FV_EBREAKDOWN', -6: 'FV_ENAN'}


class FvError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__('%s: %s' % (ERRORS.get(code, code), msg))
        self.code = code


class fv_grid_desc(ctypes.Structure):
    _fields_ = [('Ns', ctypes.c_int), ('Nr', ctypes.c_int), ('ri', ctypes.c_double), ('ro', ctypes.c_double)]


class fv_phys(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ('E', 'Ra', 'Pr', 'Pm', 'dt')]


class fv_pc_desc(ctypes.Structure):
    _fields_ = [('p1', ctypes.c_int), ('p2', ctypes.c_int), ('p3', ctypes.c_int), ('overlap', ctypes.c_int),
                ('levels', ctypes.c_int), ('overlap_coarse', ctypes.c_int), ('coarse_rtol', ctypes.c_double),
                ('coarse_restart', ctypes.c_int), ('coarse_maxit', ctypes.c_int), ('precision', ctypes.c_int),
                ('inner_rtol', ctypes.c_double), ('inner_restart', ctypes.c_int), ('inner_maxit', ctypes.c_int),
                ('nboxes', ctypes.c_int), ('boxes', ctypes.POINTER(ctypes.c_int)), ('inner_gs_passes', ctypes.c_int),
                ('cp1', ctypes.c_int), ('cp2', ctypes.c_int), ('cp3', ctypes.c_int)]


class fv_gmres_opts(ctypes.Structure):
    _fields_ = [('restart', ctypes.c_int), ('max_it', ctypes.c_int), ('atol', ctypes.c_double),
                ('rtol', ctypes.c_double)]


class fv_solve_stats(ctypes.Structure):
    _fields_ = [('iters', ctypes.c_int), ('inner_iters', ctypes.c_int), ('converged', ctypes.c_int),
                ('r0', ctypes.c_double), ('rfinal', ctypes.c_double), ('time_ms', ctypes.c_double),
                ('fallback', ctypes.c_int)]


class fv_diag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ('E_kin', 'E_mag', 'cfl_alfven', 'divB_face', 'divB_rhs', 'divU_face',
                                               'divU_rhs', 'divB_cell', 'divU_cell')] + [('steps', ctypes.c_longlong)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class fv_net_desc(ctypes.Structure):
    _fields_ = [('C', ctypes.c_int), ('levels', ctypes.c_int), ('Ns', ctypes.c_int), ('Nr', ctypes.c_int),
                ('max_batch', ctypes.c_int)]


class fv_adam_opts(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ('lr', 'beta1', 'beta2', 'eps')]


class fv_train_opts(ctypes.Structure):
    _fields_ = [('epochs', ctypes.c_int), ('batch', ctypes.c_int), ('seed', ctypes.c_ulonglong),
                ('adam', fv_adam_opts)]


# (name, argtypes) of every symbol include/fv.h declares
_P, _VP, _DP = ctypes.POINTER, ctypes.c_void_p, ctypes.c_void_p
SIGNATURES = {
    'fv_build_grid': [_P(fv_grid_desc), _P(_VP)],
    'fv_free_grid': [_VP],
    'fv_grid_cells': [_VP, _P(ctypes.c_longlong)],
    'fv_assemble_system': [_VP, ctypes.c_int, _P(fv_phys), _P(fv_pc_desc), _P(_VP)],
    'fv_free_system': [_VP],
    'fv_system_size': [_VP, _P(ctypes.c_longlong)],
    'fv_apply_op': [_VP, _DP, _DP, _VP],
    'fv_apply_op_noalloc': [_VP, _DP, _DP, _VP],
    'fv_apply_op_fp32': [_VP, _DP, _DP, _VP],
    'fv_precond_apply': [_VP, _DP, _DP, _VP],
    'fv_gmres_solve': [_VP, _DP, _DP, _P(fv_gmres_opts), _P(fv_solve_stats), _VP],
    'fv_gmres_solve_batch': [_VP, ctypes.c_int, _DP, _DP, _P(fv_gmres_opts), _P(fv_solve_stats), _VP],
    'fv_state_create': [_VP, _P(fv_phys), _DP, _P(_VP)],
    'fv_free_state': [_VP],
    'fv_state_get': [_VP, _DP, _VP],
    'fv_state_set': [_VP, _DP, _VP],
    'fv_state_reset': [_VP, _DP, _VP],
    'fv_state_diagnostics': [_VP, _VP, _P(fv_diag), _VP],
    'fv_time_step': [_VP, _VP, _VP, _P(fv_gmres_opts), ctypes.c_int, _P(fv_solve_stats), _VP],
    'fv_time_step_opts': [_VP, _VP, _VP, _P(fv_gmres_opts), _P(fv_gmres_opts), ctypes.c_int, _P(fv_solve_stats), _VP],
    'fv_profile_enable': [ctypes.c_int],
    'fv_profile_read': [ctypes.c_int, _P(ctypes.c_longlong), _P(ctypes.c_double)],
    'fv_last_error': [],
    # include/fv_net.h
    'fv_net_create': [_P(fv_net_desc), _P(_VP)],
    'fv_net_free': [_VP],
    'fv_net_param_count': [_VP, _P(ctypes.c_longlong)],
    'fv_net_set_params': [_VP, _VP],
    'fv_net_get_params': [_VP, _VP],
    'fv_net_init': [_VP, ctypes.c_ulonglong],
    'fv_net_forward': [_VP, ctypes.c_int, _DP, _DP, _VP],
    'fv_net_loss_grad': [_VP, ctypes.c_int, _DP, _DP, _P(ctypes.c_double), _VP, _VP],
    'fv_net_adam_step': [_VP, _VP, _P(fv_adam_opts)],
    'fv_net_train': [_VP, ctypes.c_int, _DP, _DP, _P(fv_train_opts), _VP, _VP],
    'fv_coarse_system': [_VP, _P(_VP)],
    'fv_restrict_coarse': [_VP, _DP, _DP, _VP],
    'fv_prolong_coarse': [_VP, _DP, _DP, _VP],
    'fv_pc_set_learned': [_VP, _VP, ctypes.c_int, ctypes.c_int],
}
FV_LEARN_GUESS = 1


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError('libfv.so is not built (run __graft_entry__.build()); there is no CPU fallback')
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == 'fv_last_error' else ctypes.c_int
    return lib


lib = _load()


def _check(rc):
    if rc != 0:
        raise FvError(rc, lib.fv_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, n=None):
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError('expected a contiguous CUDA float64 tensor')
    if n is not None and t.numel() != n:
        raise ValueError('expected %d values, got %d' % (n, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- C ABI, same names
def fv_build_grid(Ns, Nr, ri=7.0 / 13.0, ro=20.0 / 13.0):
    h = ctypes.c_void_p()
    _check(lib.fv_build_grid(ctypes.byref(fv_grid_desc(Ns, Nr, ri, ro)), ctypes.byref(h)))
    return h


def fv_assemble_system(grid, kind, E, Ra, Pr, Pm, dt, p=(1, 1, 1), overlap=1, levels=1, overlap_coarse=1,
                       coarse_rtol=0.1, coarse_restart=30, coarse_maxit=30, precision=FV_PREC_FP64, inner_rtol=1e-3,
                       inner_restart=30, inner_maxit=30, boxes=None, inner_gs_passes=2, coarse_p=(0, 0, 0)):
    h = ctypes.c_void_p()
    nb, bp = 0, None
    if boxes is not None:
        flat = (ctypes.c_int * (7 * len(boxes)))(*[int(v) for bx in boxes for v in bx])
        nb, bp = len(boxes), ctypes.cast(flat, ctypes.POINTER(ctypes.c_int))
    pc = fv_pc_desc(p[0], p[1], p[2], overlap, levels, overlap_coarse, coarse_rtol, coarse_restart, coarse_maxit,
                    precision, inner_rtol, inner_restart, inner_maxit, nb, bp, inner_gs_passes, *coarse_p)
    _check(lib.fv_assemble_system(grid, kind, ctypes.byref(fv_phys(E, Ra, Pr, Pm, dt)), ctypes.byref(pc),
                                  ctypes.byref(h)))
    return h


def fv_system_size(system):
    n = ctypes.c_longlong()
    _check(lib.fv_system_size(system, ctypes.byref(n)))
    return n.value


def fv_apply_op(system, x, y):
    n = fv_system_size(system)
    _check(lib.fv_apply_op(system, _ptr(x, n), _ptr(y, n), _stream()))
    return y


def _ptr32(t, n):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == n):
        raise ValueError('expected a contiguous CUDA float32 tensor of %d values' % n)
    return ctypes.c_void_p(t.data_ptr())


def fv_apply_op_fp32(system, x, y):
    """y = A x in FP32 (float32 CUDA tensors) for a system assembled with FV_PREC_FP32."""
    n = fv_system_size(system)
    _check(lib.fv_apply_op_fp32(system, _ptr32(x, n), _ptr32(y, n), _stream()))
    return y


def fv_apply_op_noalloc(system, x, y):
    """y = A x with the ghost layer in the library's static device array (no allocation)."""
    n = fv_system_size(system)
    _check(lib.fv_apply_op_noalloc(system, _ptr(x, n), _ptr(y, n), _stream()))
    return y


def fv_precond_apply(system, r, z):
    n = fv_system_size(system)
    _check(lib.fv_precond_apply(system, _ptr(r, n), _ptr(z, n), _stream()))
    return z


def fv_gmres_solve(system, b, x, restart=30, max_it=3000, atol=0.0, rtol=1e-8, raise_on_noconv=True):
    n = fv_system_size(system)
    st = fv_solve_stats()
    rc = lib.fv_gmres_solve(system, _ptr(b, n), _ptr(x, n), ctypes.byref(fv_gmres_opts(restart, max_it, atol, rtol)),
                            ctypes.byref(st), _stream())
    if rc != 0 and (raise_on_noconv or rc != -4):
        _check(rc)
    return st


def fv_gmres_solve_batch(system, B, X, restart=30, max_it=3000, atol=0.0, rtol=1e-8, raise_on_noconv=True):
    """Solve A x_r = b_r for the rows of B (nrhs x n CUDA float64) into X (in: x0)."""
    n = fv_system_size(system)
    if B.dim() != 2 or B.shape[1] != n or X.shape != B.shape:
        raise ValueError('B and X must be (nrhs, n)')
    nrhs = B.shape[0]
    stats = (fv_solve_stats * nrhs)()
    rc = lib.fv_gmres_solve_batch(system, nrhs, _ptr(B), _ptr(X), ctypes.byref(fv_gmres_opts(restart, max_it, atol, rtol)),
                                  stats, _stream())
    if rc != 0 and (raise_on_noconv or rc != -4):
        _check(rc)
    return list(stats)


def fv_state_create(grid, init, E, Ra, Pr, Pm, dt):
    h = ctypes.c_void_p()
    ncell = ctypes.c_longlong()
    _check(lib.fv_grid_cells(grid, ctypes.byref(ncell)))
    _check(lib.fv_state_create(grid, ctypes.byref(fv_phys(E, Ra, Pr, Pm, dt)), _ptr(init, 9 * ncell.value),
                               ctypes.byref(h)))
    return h


def fv_state_get(state, out):
    _check(lib.fv_state_get(state, _ptr(out), _stream()))
    return out


def fv_state_set(state, src):
    _check(lib.fv_state_set(state, _ptr(src), _stream()))


def fv_state_reset(state, src):
    """Fields from src and a fresh history: the next step is a first step, as after fv_state_create."""
    _check(lib.fv_state_reset(state, _ptr(src), _stream()))


def fv_state_diagnostics(state, ppbe=None):
    """Energies, Alfven CFL number and divergence norms of the state (fv_diag as a dict)."""
    d = fv_diag()
    _check(lib.fv_state_diagnostics(state, ppbe, ctypes.byref(d), _stream()))
    return d.as_dict()


def fv_time_step(state, vtbe, ppbe, nsteps=1, restart=30, max_it=3000, atol=0.0, rtol=1e-8):
    stats = (fv_solve_stats * (2 * nsteps))()
    _check(lib.fv_time_step(state, vtbe, ppbe, ctypes.byref(fv_gmres_opts(restart, max_it, atol, rtol)), nsteps,
                            stats, _stream()))
    return list(stats)


def fv_time_step_opts(state, vtbe, ppbe, nsteps=1, vtbe_opts=None, ppbe_opts=None):
    """Time steps with separate FGMRES options per system: dicts of restart, max_it, atol, rtol."""
    def mk(o):
        o = dict(dict(restart=30, max_it=3000, atol=0.0, rtol=1e-8), **(o or {}))
        return fv_gmres_opts(o['restart'], o['max_it'], o['atol'], o['rtol'])
    stats = (fv_solve_stats * (2 * nsteps))()
    _check(lib.fv_time_step_opts(state, vtbe, ppbe, ctypes.byref(mk(vtbe_opts)), ctypes.byref(mk(ppbe_opts)), nsteps,
                                 stats, _stream()))
    return list(stats)


def fv_free_grid(h):
    _check(lib.fv_free_grid(h))


def fv_free_system(h):
    _check(lib.fv_free_system(h))


def fv_free_state(h):
    _check(lib.fv_free_state(h))


K_NAMES = {0: 'ghost', 1: 'apply_vtbe', 2: 'apply_ppbe', 3: 'ras_fwd_vtbe', 4: 'ras_bwd_vtbe', 5: 'cgs', 6: 'vec',
           7: 'glue', 8: 'transfer', 9: 'phase_pc_c', 10: 'phase_pc_f', 11: 'phase_pc_i', 12: 'ras_fwd_ppbe',
           13: 'ras_bwd_ppbe', 14: 'net_fwd', 15: 'net_train'}
K_NAMES_INV = {v: k for k, v in K_NAMES.items()}
K_COARSE, K_FP32, K_COUNT = 16, 32, 64


def category_name(c):
    return K_NAMES[c % 16] + ('_coarse' if c & K_COARSE else '') + ('_fp32' if c & K_FP32 else '')


def fv_profile_enable(on=True):
    _check(lib.fv_profile_enable(1 if on else 0))


def fv_profile_read(category):
    n, t = ctypes.c_longlong(), ctypes.c_double()
    _check(lib.fv_profile_read(category, ctypes.byref(n), ctypes.byref(t)))
    return n.value, t.value


def fv_last_error():
    return lib.fv_last_error().decode()


# ---------------------------------------------------------------- learned coarse correction (include/fv_net.h)
def _fptr(a, n):
    """Host float32 numpy array of n values -> pointer."""
    import numpy as np
    if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous and a.size == n):
        raise ValueError('expected a contiguous float32 numpy array of %d values' % n)
    return ctypes.c_void_p(a.ctypes.data)


def fv_net_create(C, Ns, Nr, levels=3, max_batch=1):
    h = ctypes.c_void_p()
    _check(lib.fv_net_create(ctypes.byref(fv_net_desc(C, levels, Ns, Nr, max_batch)), ctypes.byref(h)))
    return h


def fv_net_free(net):
    _check(lib.fv_net_free(net))


def fv_net_param_count(net):
    n = ctypes.c_longlong()
    _check(lib.fv_net_param_count(net, ctypes.byref(n)))
    return n.value


def fv_net_set_params(net, params):
    _check(lib.fv_net_set_params(net, _fptr(params, fv_net_param_count(net))))


def fv_net_init(net, seed=0):
    _check(lib.fv_net_init(net, seed))


def fv_net_get_params(net):
    import numpy as np
    out = np.empty(fv_net_param_count(net), dtype=np.float32)
    _check(lib.fv_net_get_params(net, ctypes.c_void_p(out.ctypes.data)))
    return out


def fv_net_forward(net, nb, r, e):
    _check(lib.fv_net_forward(net, nb, _ptr(r), _ptr(e), _stream()))
    return e


def fv_net_loss_grad(net, nb, r, e, want_grads=True):
    """(mean squared error, FP32 numpy gradient or None)."""
    import numpy as np
    loss = ctypes.c_double()
    g = np.empty(fv_net_param_count(net), dtype=np.float32) if want_grads else None
    _check(lib.fv_net_loss_grad(net, nb, _ptr(r), _ptr(e), ctypes.byref(loss),
                                ctypes.c_void_p(g.ctypes.data) if want_grads else None, _stream()))
    return loss.value, g


def fv_net_adam_step(net, grads, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(lib.fv_net_adam_step(net, _fptr(grads, fv_net_param_count(net)),
                                ctypes.byref(fv_adam_opts(lr, beta1, beta2, eps))))


def fv_net_train(net, R, E, epochs=1, batch=1, seed=0, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """Train on the rows of R, E (npairs x 2*6*Ns^2*Nr CUDA float64); returns the mean loss of each epoch."""
    import numpy as np
    if R.dim() != 2 or E.shape != R.shape:
        raise ValueError('R and E must be (npairs, coarse n)')
    losses = np.zeros(max(epochs, 1), dtype=np.float64)
    o = fv_train_opts(epochs, batch, seed, fv_adam_opts(lr, beta1, beta2, eps))
    _check(lib.fv_net_train(net, R.shape[0], _ptr(R), _ptr(E), ctypes.byref(o),
                            ctypes.c_void_p(losses.ctypes.data), _stream()))
    return losses[:epochs]


def fv_coarse_system(system):
    h = ctypes.c_void_p()
    _check(lib.fv_coarse_system(system, ctypes.byref(h)))
    return h


def fv_restrict_coarse(system, x, xc):
    _check(lib.fv_restrict_coarse(system, _ptr(x), _ptr(xc), _stream()))
    return xc


def fv_prolong_coarse(system, xc, x):
    """x = the piecewise-constant prolongation of coarse vector xc (the two-level preconditioner's I_c^f)."""
    _check(lib.fv_prolong_coarse(system, _ptr(xc), _ptr(x), _stream()))
    return x


def fv_pc_set_learned(system, net, coarse_its=0, flags=0):
    _check(lib.fv_pc_set_learned(system, net, coarse_its, flags))
