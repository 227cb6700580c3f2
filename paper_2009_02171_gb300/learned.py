"""Training the learned coarse correction of a two-level PPBE system (include/fv_net.h).

Orchestration of C-ABI calls only: the coarse operator, the restriction, the
batched coarse solves that produce the targets, the network's forward and
backward passes and Adam all run in libfv's kernels.  PyTorch holds the device
buffers and repeats a coarse field onto the fine grid (each coarse cell's value
on its 8 children) so that the library's own restriction forms the coarse
right-hand side exactly as the preconditioner does.

Training right-hand sides (seeded, synthetic): multiscale fields on the coarse
grid (inputs.multiscale_fields) and, for every second sample, the coarse
operator applied to such a field; targets are the plain coarse solver's
solutions (FGMRES with the coarse one-level RAS to `target_rtol`).
"""
import time

import torch

from . import fv
from .inputs import multiscale_fields


def coarse_training_pairs(system, Ns, Nr, npairs, seed=5, target_rtol=1e-6, chunk=32):
    """(R, E, info): npairs coarse right-hand sides of `system` (fine grid 6 x Ns^2 x Nr) and the plain
    coarse solver's solutions, as rows of CUDA float64 tensors."""
    c = fv.fv_coarse_system(system)
    nc, n = fv.fv_system_size(c), fv.fv_system_size(system)
    ns, nr = Ns // 2, Nr // 2
    if nc != 12 * ns * ns * nr or n != 8 * nc:
        raise ValueError('system is not a two-level PPBE system on a 6 x %d^2 x %d grid' % (Ns, Nr))
    t0 = time.perf_counter()
    F = multiscale_fields(ns, nr, npairs, seed=seed)
    R = torch.empty(npairs, nc, dtype=torch.float64, device='cuda')
    tmp = torch.empty(nc, dtype=torch.float64, device='cuda')
    fine = torch.empty(n, dtype=torch.float64, device='cuda')
    for i in range(npairs):
        f = torch.tensor(F[i], device='cuda')
        if i % 2:
            fv.fv_apply_op(c, f, tmp)
            f = tmp
        # the coarse right-hand side the preconditioner would form from the prolonged field
        fv.fv_prolong_coarse(system, f, fine)
        fv.fv_restrict_coarse(system, fine, R[i])
    E = torch.zeros_like(R)
    its = []
    for i in range(0, npairs, chunk):
        st = fv.fv_gmres_solve_batch(c, R[i:i + chunk].contiguous(), E[i:i + chunk], rtol=target_rtol)
        its += [x.iters for x in st]
    torch.cuda.synchronize()
    return R, E, {'pairs': npairs, 'target_rtol': target_rtol, 'target_iters_mean': sum(its) / len(its),
                  'data_seconds': time.perf_counter() - t0}


def train_learned_correction(system, Ns, Nr, C=16, levels=3, npairs=256, epochs=40, batch=8, lr=3e-4,
                             data_seed=5, init_seed=9, train_seed=3, coarse_its=6, attach=True, flags=0):
    """Train a network for the coarse grid of `system` (fine grid Ns x Ns x Nr) and attach it.

    Returns (net, info).  The caller frees the network (after detaching it) with fv_net_free."""
    R, E, info = coarse_training_pairs(system, Ns, Nr, npairs, seed=data_seed)
    net = fv.fv_net_create(C, Ns // 2, Nr // 2, levels=levels, max_batch=batch)
    fv.fv_net_init(net, init_seed)
    t0 = time.perf_counter()
    losses = fv.fv_net_train(net, R, E, epochs=epochs, batch=batch, seed=train_seed, lr=lr)
    torch.cuda.synchronize()
    info.update({'C': C, 'levels': levels, 'params': fv.fv_net_param_count(net), 'epochs': epochs, 'batch': batch,
                 'lr': lr, 'train_seconds': time.perf_counter() - t0, 'loss_first_epoch': float(losses[0]),
                 'loss_last_epoch': float(losses[-1]), 'coarse_its': coarse_its})
    del R, E
    if attach:
        fv.fv_pc_set_learned(system, net, coarse_its=coarse_its, flags=flags)
    return net, info
