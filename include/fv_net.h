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
 * Network (per cubed-sphere panel; panels never exchange data inside it):
 *   s  = ||r_c||_2 over the whole coarse vector (N(a r) = a N(r))
 *   a1 = relu(conv(r_c/s; 2 -> C))      a2 = relu(conv(a1; C -> C))
 *   p  = 2x2x2 mean pooling of a2
 *   a3 = relu(conv(p; C -> 2C))         a4 = relu(conv(a3; 2C -> 2C))
 *   a5 = relu(conv([a2, upsample(a4)]; 3C -> C))   (nearest upsampling, concat)
 *   e_c = s conv(a5; C -> 2)
 * conv = 3x3x3 cross-correlation with zero padding 1 inside each panel plus a
 * bias, over the panel's (k, j, i) = (radial, eta, xi) cells.  Parameters are
 * FP32 masters, flat, layer by layer: W[co][ci][dz][dy][dx] then b[co]
 * (~71k parameters for C = 16, ~284k for C = 32).  Activations, weights and
 * gradients are stored as BF16; products accumulate in FP32 on the tensor
 * cores.  Training minimises the mean squared error of N(r)/s against e/s
 * with Adam (Kingma & Ba, 2015) on FP32 masters.
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
 * system it serves).  C in {16, 32}; Ns, Nr even and >= 2; max_batch >= 1
 * samples per forward / training step (activation memory scales with it:
 * about 700 bytes per cell and sample at C = 32).  Weights start at zero:
 * set them with fv_net_set_params. */
typedef struct {
  int C, Ns, Nr, max_batch;
} fv_net_desc;

fv_status fv_net_create(const fv_net_desc* desc, fv_net** out);
fv_status fv_net_free(fv_net* net);
fv_status fv_net_param_count(const fv_net* net, long long* n);
/* params: HOST FP32 array of fv_net_param_count values, layout above. */
fv_status fv_net_set_params(fv_net* net, const float* params);
fv_status fv_net_get_params(const fv_net* net, float* params);

/* e = N(r) for nb <= max_batch samples.  r, e: device FP64 (layout above);
 * a sample with r = 0 gives e = 0. */
fv_status fv_net_forward(fv_net* net, int nb, const double* r, double* e, void* stream);

/* Mean squared error L = mean over all nb * 2 * 6 Ns^2 Nr entries of
 * (N(r)/s - e/s)^2 (s per sample) and its gradient with respect to the
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

/* Attach (net != NULL) or detach (net == NULL) a learned coarse correction to
 * a two-level PPBE system whose coarse grid matches the network.  The coarse
 * solve of every preconditioner application becomes e_c = N(r_c) followed by
 * coarse_its in [0, 31] coarse FGMRES iterations started from it (FP32
 * fixed-iteration inner solve under mixed precision).  flags: FV_LEARN_GUESS
 * also corrects the initial guess of each top-level solve,
 * x0 <- x0 + I_c^f N(r_c(b - A x0)).  The system borrows the network: keep
 * it alive while attached.  A top-level solve that ends without convergence
 * (FV_ENOCONV or FV_ENAN) under the learned preconditioner continues with the
 * plain coarse GMRES for the remaining iterations (stats->fallback = 1). */
#define FV_LEARN_GUESS 1
fv_status fv_pc_set_learned(fv_system* s, fv_net* net, int coarse_its, int flags);

#ifdef __cplusplus
}
#endif
#endif /* FV_NET_H */
