/* fv_net.h -- learned coarse correction of the two-level preconditioner (libfv.so).
 *
 * Not in the paper.  The two-level restricted additive Schwarz preconditioner
 * of Sec. 3.3 (eqn:twolevel) spends most of its time in the coarse solve
 * A_c e_c = r_c (eqn:coarsesolve), an inner GMRES on the coarse grid.  These
 * calls build, train and attach a small network N that predicts e_c from r_c
 * instead (optionally followed by a few coarse GMRES iterations started from
 * N(r_c)), and that predicts a correction of the initial guess.  The plain
 * coarse GMRES stays the fallback: a solve whose learned preconditioner fails
 * to converge is finished with the plain one.
 *
 * Network: a U-Net with `levels` poolings and width C on the cubed sphere.
 * Before every 3x3x3 convolution each panel is padded by one cell in (eta, xi)
 * with the neighbouring panel's cells across each edge (the cell sharing the
 * edge face; zero at the ring corners) and by zeros radially.
 *   s = RMS of r_c over the whole coarse vector (N(a r) = a N(r) for a > 0)
 *   level l = 0..L: input r_c/s (l = 0) or the 2x2x2 mean pooling of E_{l-1};
 *                   A_l = relu(conv(input)), E_l = relu(conv(A_l))
 *   D_L = E_L; l = L-1..0: D_l = relu(conv([E_l, upsample(D_{l+1})]))
 *   e_c = s conv(D_0; C -> 2)
 * conv = 3x3x3 cross-correlation plus a bias over the panel's (k, j, i) =
 * (radial, eta, xi) cells (input channels: 2 for the first, 2C for the
 * decoder, else C).  Parameters are FP32 masters, flat, layer by layer (e0a,
 * e0b, ..., eLa, eLb, d(L-1), ..., d0, out): W[co][ci][dz][dy][dx] then b[co]
 * (C = 32, L = 3: 363,234 parameters).  Activations, weights and gradients are
 * stored as BF16; products accumulate in FP32 on the tensor cores.  Training
 * minimises the mean squared error of N(r)/s against e/s with Adam (Kingma &
 * Ba, 2015) on FP32 masters.
 *
 * Vectors follow fv.h: caller-owned device FP64, a coarse PPBE vector is
 * [comp = P, P_b][panel][k][j][i] on the coarse grid (2 * 6 Ns^2 Nr values);
 * a batch of nb samples stores sample b at offset b * 2 * 6 Ns^2 Nr.
 */
#ifndef FV_NET_H
#define FV_NET_H

#include "fv.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fv_net fv_net;

/* Network on a grid of 6 panels x Ns x Ns x Nr cells (the coarse grid of the
 * system it serves).  C in {16, 32}; levels in [0, 4]; Ns, Nr >= 1 and
 * divisible by 2^levels; max_batch >= 1 samples per forward / training step
 * (activation memory scales with it: about 600 bytes per cell and sample at
 * C = 32, twice that while training).  Weights start at zero: set them with
 * fv_net_set_params. */
typedef struct {
  int C, levels, Ns, Nr, max_batch;
} fv_net_desc;

fv_status fv_net_create(const fv_net_desc* desc, fv_net** out);
fv_status fv_net_free(fv_net* net);
fv_status fv_net_param_count(const fv_net* net, long long* n);
/* params: HOST FP32 array of fv_net_param_count values, layout above. */
fv_status fv_net_set_params(fv_net* net, const float* params);
fv_status fv_net_get_params(const fv_net* net, float* params);
/* He initialisation: every weight of a layer with ci input channels drawn from
 * N(0, 2 / (27 ci)) (Box-Muller on 53-bit uniforms of the splitmix64 stream
 * started at `seed`, layer by layer in parameter order), biases zero; resets
 * Adam's state like fv_net_set_params. */
fv_status fv_net_init(fv_net* net, unsigned long long seed);

/* e = N(r) for nb <= max_batch samples.  r, e: device FP64 (layout above);
 * a sample with r = 0 gives e = 0. */
fv_status fv_net_forward(fv_net* net, int nb, const double* r, double* e, void* stream);

/* Mean squared error L = mean over all nb * 2 * 6 Ns^2 Nr entries of
 * (N(r)/s - e/s)^2 (s the RMS of each sample's r) and its gradient with respect to the
 * parameters.  loss: host, may be NULL; grads: HOST FP32 array of
 * fv_net_param_count values, may be NULL.  Synchronizes the stream. */
fv_status fv_net_loss_grad(fv_net* net, int nb, const double* r, const double* e, double* loss, float* grads,
                           void* stream);

typedef struct {
  double lr, beta1, beta2, eps;
} fv_adam_opts;

/* One Adam step of the FP32 masters with the given HOST FP32 gradient
 * (step counter, first and second moments kept in the network). */
fv_status fv_net_adam_step(fv_net* net, const float* grads, const fv_adam_opts* opts);

/* Train on npairs samples (R, E: device FP64, npairs * 2 * 6 Ns^2 Nr values
 * each, sample b at offset b * 2 * 6 Ns^2 Nr): `epochs` passes, each over a
 * permutation of the samples drawn from `seed` (splitmix64, Fisher-Yates), in
 * batches of `batch` <= max_batch samples, one Adam step per batch.
 * epoch_loss: host, `epochs` values (mean batch loss of each epoch), or NULL. */
typedef struct {
  int epochs, batch;
  unsigned long long seed;
  fv_adam_opts adam;
} fv_train_opts;
fv_status fv_net_train(fv_net* net, int npairs, const double* R, const double* E, const fv_train_opts* opts,
                       double* epoch_loss, void* stream);

/* The coarse-level system of a two-level system (borrowed, freed with it):
 * what its preconditioner solves with inner GMRES.  Used to generate training
 * targets with fv_gmres_solve / fv_gmres_solve_batch. */
fv_status fv_coarse_system(const fv_system* s, const fv_system** coarse);

/* r_c = the coarse right-hand side the two-level preconditioner of s forms
 * from a fine vector x (cell-volume mean restriction; for PPBE the pressure
 * component's volume-weighted mean removed).  x: n values, xc: coarse n. */
fv_status fv_restrict_coarse(const fv_system* s, const double* x, double* xc, void* stream);

/* x = I_c^f xc, the piecewise-constant prolongation of the two-level
 * preconditioner of s (eqn:coarsesolve: every fine cell takes the value of
 * the coarse cell that contains it).  xc: coarse n values, x: n values
 * (device, component-major; not aliased).  FV_EINVAL for a one-level
 * system or null pointers. */
fv_status fv_prolong_coarse(const fv_system* s, const double* xc, double* x, void* stream);

/* Attach (net != NULL) or detach (net == NULL) a learned coarse correction to
 * a two-level PPBE system whose coarse grid matches the network.  The coarse
 * solve of every preconditioner application becomes e_c = N(r_c) followed by
 * coarse_its in [0, 31] coarse FGMRES iterations started from it (FP32
 * fixed-iteration inner solve under mixed precision).  flags: FV_LEARN_GUESS
 * also corrects the initial guess of each top-level solve,
 * x0 <- x0 + I_c^f N(r_c(b - A x0)).  The system borrows the network: keep
 * it alive while attached.  A top-level solve that has not converged within
 * one restart cycle (opts->restart iterations) under the learned
 * preconditioner, or meets a NaN, continues with the plain coarse GMRES for
 * the remaining iterations (stats->fallback = 1). */
#define FV_LEARN_GUESS 1
fv_status fv_pc_set_learned(fv_system* s, fv_net* net, int coarse_its, int flags);

#ifdef __cplusplus
}
#endif
#endif /* FV_NET_H */
