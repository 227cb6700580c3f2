/* fv.h -- C ABI of the GB300 shell dynamo solve path (libfv.so).
 *
 * Method: Yin, Yang, Ma, Cai, Zhang, "Parallel finite volume simulation of the
 * spherical shell dynamo with pseudo-vacuum magnetic boundary conditions"
 * (arXiv 2009.02171).  The library solves the two linear systems of the
 * paper's approximate-factorization time step (Sec. 3.1): VTBE
 * (eqn:tsvelocity, eqn:tstemperature, eqn:tsmag; unknowns u, Theta, B) and
 * PPBE (eqn:tsp, eqn:tspb; unknowns P, P_b), discretized by the collocated
 * finite-volume scheme on the equiangular cubed-sphere shell (Sec. 3.2), with
 * restarted right-preconditioned (flexible) GMRES and one- or two-level
 * restricted additive Schwarz preconditioning (Sec. 3.3).
 *
 * Conventions for every call:
 * - Every function returns fv_status: FV_OK (0) or a negative error code.  No
 *   function aborts or throws; fv_last_error() returns a thread-local message
 *   describing the last failure of the calling thread.
 * - Handles (fv_grid, fv_system, fv_state) are opaque and owned by the
 *   library; release each with its fv_free_* call.  A system or state keeps a
 *   reference to its grid: free it before the grid.
 * - Vectors are CALLER-OWNED DEVICE pointers (e.g. torch.Tensor.data_ptr() of
 *   a CUDA float64 tensor on the current device) holding FP64 values, laid out
 *   component-major [comp][panel][k][j][i] with i fastest (N = 6 Ns^2 Nr cells
 *   per component).  VTBE comps: u_x, u_y, u_z, Theta, B_x, B_y, B_z (Cartesian
 *   components, 7N values); PPBE comps: P, P_b (2N values).  The library never
 *   frees, reallocates or retains them beyond the call.
 * - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls enqueue
 *   their kernels on it; calls that return statistics synchronize it.
 * - Internal scratch (ghost layers, Krylov bases, factors) is device memory
 *   allocated by the library at fv_assemble_system / fv_state_create.
 */
#ifndef FV_H
#define FV_H

#ifdef __cplusplus
extern "C" {
#endif

typedef int fv_status;
#define FV_OK 0
#define FV_EINVAL (-1)      /* bad argument (null handle, bad size, odd grid for two levels) */
#define FV_ENOMEM (-2)      /* device allocation failed */
#define FV_ECUDA (-3)       /* a CUDA call failed; the message names it */
#define FV_ENOCONV (-4)     /* GMRES hit max_it before the tolerance; x holds the last iterate */
#define FV_EBREAKDOWN (-5)  /* zero pivot in ILU(0) */
#define FV_ENAN (-6)        /* NaN/Inf residual; x holds the last finite iterate */

typedef struct fv_grid fv_grid;
typedef struct fv_system fv_system;
typedef struct fv_state fv_state;

/* Grid of 6 panels x Ns x Ns x Nr cells (paper Sec. 3.2, cell centres
 * xi_i = -pi/4 + (i+1/2) h_s, r_k = r_i + (k+1/2) h_r).  Ns >= 4, Nr >= 2.
 * ri < ro are the shell radii (the paper uses 7/13 and 20/13). */
typedef struct {
  int Ns, Nr;
  double ri, ro;
} fv_grid_desc;

fv_status fv_build_grid(const fv_grid_desc* desc, fv_grid** out);
fv_status fv_free_grid(fv_grid* g);
/* number of cells N = 6 Ns^2 Nr */
fv_status fv_grid_cells(const fv_grid* g, long long* n_cells);

/* Non-dimensional parameters (paper Sec. 2, eqn:velocity ..) and time step. */
typedef struct {
  double E, Ra, Pr, Pm, dt;
} fv_phys;

#define FV_VTBE 0
#define FV_PPBE 1

/* Preconditioner (paper Sec. 3.3).  Each panel is split into p1 x p2 x p3
 * boxes (xi, eta, r), overlap `overlap` cells (extended across panel edges);
 * ILU(0) subdomain solves.  levels = 1: one-level RAS (eqn:onelevel);
 * levels = 2: hybrid two-level RAS (eqn:twolevel) with a coarse mesh of
 * (Ns/2, Nr/2), coarse overlap `overlap_coarse`, coarse system solved by inner
 * FGMRES(coarse_restart) to relative tolerance coarse_rtol (at most
 * coarse_maxit iterations) preconditioned by one-level RAS on the coarse mesh
 * (eqn:coarsepreconditioner).  levels = L > 2 (up to 6): the multilevel hybrid
 * RAS of Sec. 3.3 -- the coarse system's preconditioner is itself the
 * (L-1)-level construction on the next 1:2 mesh, with the same coarse_rtol,
 * coarse_restart, coarse_maxit and overlap_coarse on every coarse level.
 * Every mesh that is coarsened needs even Ns >= 8 and even Nr >= 4.  Every box,
 * overlap included, must be smaller than 1024 cells in each dimension, and
 * its sweep tables must fit in the device's shared memory (FV_EINVAL
 * otherwise). */
typedef struct {
  int p1, p2, p3;
  int overlap;
  int levels;
  int overlap_coarse;
  double coarse_rtol;
  int coarse_restart;
  int coarse_maxit;
  /* Mixed precision (not in the paper).  precision = FV_PREC_FP64: everything
   * above runs in FP64.  precision = FV_PREC_FP32: the preconditioner M^{-1}
   * of the FP64 outer FGMRES is an FP32 inner FGMRES of exactly inner_maxit
   * iterations (1..31; FP32 operator applies, FP32 ILU(0) factors and sweeps)
   * whose own preconditioner is the RAS above in FP32, with a coarse solve of
   * exactly coarse_maxit iterations for levels = 2.  These inner solves run
   * on the device without host synchronisation (replayed as one CUDA graph);
   * inner_rtol, inner_restart and coarse_rtol are not used by them.  The
   * outer residual, its Arnoldi dot products and norms and the Hessenberg
   * least squares stay FP64, so the final residual is a true FP64 residual. */
  int precision;
  double inner_rtol;
  int inner_restart;
  int inner_maxit;
  /* Uneven decompositions (not in the paper; p1, p2, p3 are then ignored):
   * nboxes > 0 owned boxes given as 7 ints each in host memory,
   * (panel, i0, i1, j0, j1, k0, k1) with half-open ranges, that must tile the
   * shell exactly (FV_EINVAL otherwise).  With levels = 2 every bound must be
   * even; the coarse level uses the halved boxes.  Read during the call only. */
  int nboxes;
  const int* boxes;
  /* Gram-Schmidt passes of the FP32 fixed-iteration inner solves (mixed
   * precision only): 2 (classical Gram-Schmidt twice, the default; 0 means 2)
   * or 1 (once).  The FP64 outer FGMRES always uses two passes. */
  int inner_gs_passes;
  /* Box split of the coarse levels (not in the paper): cp1 x cp2 x cp3 boxes
   * a panel on every coarse mesh, each capped by that mesh's size; 0 (the
   * default) takes p1, p2, p3, so a coarse box covers the coarse cells of one
   * fine box.  Ignored with nboxes > 0 (the coarse level halves the boxes). */
  int cp1, cp2, cp3;
} fv_pc_desc;
#define FV_PREC_FP64 0
#define FV_PREC_FP32 1
/* FV_PREC_BF16: FV_PREC_FP32 with the ILU(0) factors of every level stored in
 * BF16 (rounded from the FP64 factorization; the sweeps convert them and
 * compute in FP32), halving the factor bytes the sweeps read.  The outer
 * residual stays FP64.  fv_gmres_solve_batch rejects such systems. */
#define FV_PREC_BF16 2

/* Builds the system `kind` (FV_VTBE: A = I - dt/2 [L1 R1; R2 L2; L3];
 * FV_PPBE: A = dt/2 D G for (P Neumann, P_b Dirichlet)), its subdomain
 * matrices and their ILU(0) factors on the GPU (setup, once per grid and dt). */
fv_status fv_assemble_system(const fv_grid* g, int kind, const fv_phys* phys, const fv_pc_desc* pc,
                             fv_system** out);
fv_status fv_free_system(fv_system* s);
/* number of unknowns n = d N (d = 7 for VTBE, 2 for PPBE) */
fv_status fv_system_size(const fv_system* s, long long* n);

/* y = A x  (matrix-free, paper eqn:divdiscretization for every operator).
 * x, y: device FP64, n values each, must not overlap. */
fv_status fv_apply_op(const fv_system* s, const double* x, double* y, void* stream);

/* y = A x in FP32: the operator of the mixed-precision inner solves (FP32
 * coefficient tables and arithmetic, paper eqn:divdiscretization).  s must
 * have been assembled with precision = FV_PREC_FP32 (FV_EINVAL otherwise).
 * x, y: device FP32, n values each, must not overlap. */
fv_status fv_apply_op_fp32(const fv_system* s, const float* x, float* y, void* stream);

/* y = A x like fv_apply_op, for callers that must not allocate device memory
 * while they run -- for instance code whose device memory is owned by a
 * framework's pool allocator (a cudaMalloc behind its back would bypass the
 * pool and its accounting), or a solver loop that cannot afford the implicit
 * device synchronisation that cudaMalloc/cudaFree may cause.  This call
 * allocates nothing: its scratch (the panel-edge ghost layer, d x 24 x Nr x
 * (Ns + 2) doubles) lives in one file-scope static device array of
 * FV_STATIC_GHOST_DOUBLES doubles (8 MiB) that every GPU loading the library
 * holds until the process exits.  Systems whose ghost layer is larger (e.g.
 * VTBE beyond Ns = Nr = 64, PPBE beyond Ns = Nr = 128) are rejected with
 * FV_EINVAL.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, once per device and
 * process (concurrent first calls from several host threads are safe); make
 * that first call before any stream capture.  The address is not looked up
 * again: after cudaDeviceReset, do not call this on that device again.  All calls share the array: calls whose kernels
 * overlap on the GPU (e.g. on two streams at once) race on it; serialise them.
 * The array keeps the last call's contents, and each call overwrites every
 * slot it reads.  The paper has no counterpart: this is a deployment
 * variant of the operator apply above. */
#define FV_STATIC_GHOST_DOUBLES (1 << 20)
fv_status fv_apply_op_noalloc(const fv_system* s, const double* x, double* y, void* stream);

/* z = M^{-1} r (eqn:onelevel or eqn:twolevel per the system's pc).
 * r, z: device FP64, n values each, must not overlap. */
fv_status fv_precond_apply(const fv_system* s, const double* r, double* z, void* stream);

/* Restarted right-preconditioned flexible GMRES(restart) (paper Sec. 3.3):
 * stops when ||b - A x|| <= max(atol, rtol ||b - A x0||) or after max_it
 * iterations.  x: in = x0, out = solution.  stats may be NULL. */
typedef struct {
  int restart, max_it;
  double atol, rtol;
} fv_gmres_opts;

typedef struct {
  int iters;             /* outer (F)GMRES iterations */
  int inner_iters;       /* coarse-level inner iterations (two-level only) */
  int converged;
  double r0, rfinal;     /* ||b - A x0||, ||b - A x|| (true residuals) */
  double time_ms;        /* wall time of the call */
  int fallback;          /* 1: a learned coarse correction (fv_net.h) failed and the
                            plain coarse solve finished the call */
} fv_solve_stats;

fv_status fv_gmres_solve(const fv_system* s, const double* b, double* x, const fv_gmres_opts* opts,
                         fv_solve_stats* stats, void* stream);

/* Many right-hand sides of one system solved together (not in the paper): the
 * FGMRES above in lock-step for nrhs right-hand sides, each with its own
 * Hessenberg matrix, tolerance and convergence flag.  B, X: device FP64,
 * nrhs * n values, right-hand side r at offset r * n (X: in = x0, out = x).
 * The preconditioner is the system's one-level RAS (levels = 1 only), with
 * FP32 subdomain solves when the system was assembled with FV_PREC_FP32;
 * every factor the batched sweeps load is applied to a group of right-hand
 * sides (the group size is tuned by timing on the first call for a given
 * nrhs), in one persistent launch that takes subdomains largest first.
 * stats: NULL or nrhs entries. */
fv_status fv_gmres_solve_batch(const fv_system* s, int nrhs, const double* B, double* X, const fv_gmres_opts* opts,
                               fv_solve_stats* stats, void* stream);

/* Time-stepping state (paper Sec. 3.1): u, Theta, B, P, P_b at step n, the
 * nonlinear terms at n-1 (Adams-Bashforth) and the previous VTBE solution.
 * init: device FP64, 9N values (u_x, u_y, u_z, Theta, B_x, B_y, B_z, P, P_b),
 * copied into the state. */
fv_status fv_state_create(const fv_grid* g, const fv_phys* phys, const double* init, fv_state** out);
fv_status fv_free_state(fv_state* st);
/* copy the current 9N fields of the state into `out` (device FP64) */
fv_status fv_state_get(const fv_state* st, double* out, void* stream);
/* overwrite the 9N fields of the state from `in` (device FP64); the
 * Adams-Bashforth history (f^{n-1}) and the previous solutions used as initial
 * guesses are kept, so the next step continues the trajectory those fields
 * came from (e.g. fields read with fv_state_get and written back). */
fv_status fv_state_set(fv_state* st, const double* in, void* stream);
/* overwrite the 9N fields from `in` and drop the history: the next
 * fv_time_step is a first step (f^{1/2} = f^0, u^0 = u^0, B^0 = B^0,
 * Sec. 3.1; initial guesses from the fields), exactly as after
 * fv_state_create with the same `in`. */
fv_status fv_state_reset(fv_state* st, const double* in, void* stream);

/* Advance nsteps steps of the predictor-corrector scheme (Steps 1-3 of
 * Sec. 3.1): VTBE solve, PPBE solve, projection.  stats: NULL or 2*nsteps
 * entries (VTBE, PPBE per step). */
fv_status fv_time_step(fv_state* st, const fv_system* vtbe, const fv_system* ppbe, const fv_gmres_opts* opts,
                       int nsteps, fv_solve_stats* stats, void* stream);
/* fv_time_step with separate stopping rules for the two systems: vopts for
 * VTBE, popts for PPBE (the paper's presets of Sec. 4 are eps_a/eps_r =
 * 1e-10/1e-8 for VTBE and 1e-8/1e-6 for PPBE). */
fv_status fv_time_step_opts(fv_state* st, const fv_system* vtbe, const fv_system* ppbe, const fv_gmres_opts* vopts,
                            const fv_gmres_opts* popts, int nsteps, fv_solve_stats* stats, void* stream);

/* Diagnostics of the state after its last step (paper Sec. 4.2 and the
 * divergence constraint eqn:divtime).  Norms are Euclidean over cells.
 * - E_kin = Pm^2/2 sum V |u|^2, E_mag = Pm/(2E) sum V |B|^2 (Sec. 4.2);
 * - cfl_alfven: dt max(|v^1|/h_s + |v^2|/h_s + |v^3|/h_r), v = B/sqrt(E Pm) in
 *   contravariant components (Sec. 4.2, tab:gridlevels);
 * - divB_face: ||D_f B^{n+1}|| of the projected face fluxes
 *   F_f(B~) - dt/2 (G_f P_b).S_f, which equals the P_b block of the last PPBE
 *   residual and so is bounded by that solve's rfinal; divB_rhs = ||D(B~)||,
 *   its right-hand side.  divU_face, divU_rhs: the same for u and P;
 * - divB_cell, divU_cell: ||D B^{n+1}||, ||D u^{n+1}|| of the cell-centred
 *   fields of eqn:ubtilde (discretization error, O(h^2)).
 * ppbe: the PPBE system of the last step, or NULL (face values -1, as before
 * the first step).  Synchronizes `stream`. */
typedef struct {
  double E_kin, E_mag;
  double cfl_alfven;
  double divB_face, divB_rhs, divU_face, divU_rhs;
  double divB_cell, divU_cell;
  long long steps;             /* steps since fv_state_create / fv_state_reset */
} fv_diag;
fv_status fv_state_diagnostics(fv_state* st, const fv_system* ppbe, fv_diag* out, void* stream);

/* Kernel timing (optional).  While enabled, the library brackets each launch of
 * the categories below with CUDA events on the launching stream (a few
 * microseconds of host time per launch, no device work) and runs the
 * mixed-precision inner solves eagerly instead of replaying their CUDA graph;
 * fv_profile_read synchronizes the device and returns the launch count and
 * summed device time of one category since the last enable.  A category is a
 * base value plus FV_K_COARSE for launches on the coarse level of a two-level
 * preconditioner, plus FV_K_FP32 for FP32 launches of mixed precision.  The
 * phases PC-C (coarse solve), PC-F (fine one-level RAS) and PC-I
 * (restriction, prolongation and residual) follow the paper's breakdown of
 * the two-level preconditioner (Sec. 4.3). */
#define FV_K_GHOST 0
#define FV_K_APPLY_VTBE 1
#define FV_K_APPLY_PPBE 2
#define FV_K_RAS_FWD_VTBE 3
#define FV_K_RAS_BWD_VTBE 4
#define FV_K_CGS 5
#define FV_K_VEC 6
#define FV_K_GLUE 7
#define FV_K_TRANSFER 8
#define FV_K_PHASE_PC_C 9
#define FV_K_PHASE_PC_F 10
#define FV_K_PHASE_PC_I 11
#define FV_K_RAS_FWD_PPBE 12
#define FV_K_RAS_BWD_PPBE 13
#define FV_K_NET_FWD 14     /* learned coarse correction: inference (fv_net.h) */
#define FV_K_NET_TRAIN 15   /* learned coarse correction: loss, backward pass, Adam */
#define FV_K_COARSE 16
#define FV_K_FP32 32
#define FV_K_COUNT 64
fv_status fv_profile_enable(int on);
fv_status fv_profile_read(int category, long long* launches, double* total_ms);

/* Message of the calling thread's last failure ("" if none). */
const char* fv_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FV_H */
