// Time-stepping state and the predictor-corrector step (paper Sec. 3.1).
//
// Crank-Nicolson on the linear terms, Adams-Bashforth f^{n+1/2} = 3/2 f^n -
// 1/2 f^{n-1} (f^{1/2} = f^0) on the nonlinear terms;
//   Step 1: u^ = u - dt/2 G P^n, B^ = B - dt/2 G P_b^n (u^0 = u^0, B^0 = B^0 on
//           the first step); solve VTBE A_V x~ = 2 x^ - A_V x^ + dt f^{n+1/2}
//           (A_V = I - dt/2 M, so this is x^ + dt/2 M x^ + dt f) for
//           x~ = (u~, Theta^{n+1}, B~);
//   Step 2: solve PPBE dt/2 D G (P, P_b) = (D u~, D B~); the Neumann pressure
//           right-hand side and solution are kept at zero volume-weighted mean;
//   Step 3: u = u~ - dt/2 G P, B = B~ - dt/2 G P_b.
// Initial guesses: the previous step's solutions (the current state on the
// first step).
#include <chrono>
#include <cstring>

#include "fv_internal.h"

using namespace fv;

extern "C" {

fv_status fv_state_create(const fv_grid* g, const fv_phys* ph, const double* init, fv_state** out) {
  if (!g || !ph || !init || !out) return set_error("fv_state_create: null argument"), FV_EINVAL;
  fv_state* s = new fv_state();
  s->grid = g, s->phys = *ph, s->N = g->h.N;
  const size_t N = (size_t)s->N;
  struct {
    double** p;
    size_t n;
  } bufs[] = {{&s->X, 9 * N},   {&s->fprev, 7 * N}, {&s->fcur, 7 * N}, {&s->fh, 7 * N},
              {&s->xhat, 7 * N}, {&s->bV, 7 * N},    {&s->tmp, 7 * N},  {&s->xV, 7 * N},
              {&s->bP, 2 * N},   {&s->xP, 2 * N},    {&s->grad, 6 * N},
              {&s->gh, (size_t)7 * 6 * 4 * g->h.Nr * (g->h.Ns + 2)},
              {&s->part, 32 * 304}, {&s->sums, 32}};
  for (auto& b : bufs) {
    if (cudaMalloc((void**)b.p, b.n * sizeof(double)) != cudaSuccess) {
      for (void* p : s->allocs) cudaFree(p);
      delete s;
      return set_error("fv_state_create: device allocation failed"), FV_ENOMEM;
    }
    s->allocs.push_back(*b.p);
  }
  FV_CUDA(cudaMemcpy(s->X, init, 9 * N * sizeof(double), cudaMemcpyDeviceToDevice));
  *out = s;
  return FV_OK;
}

fv_status fv_free_state(fv_state* s) {
  if (!s) return FV_OK;
  for (void* p : s->allocs) cudaFree(p);
  delete s;
  return FV_OK;
}

fv_status fv_state_get(const fv_state* s, double* out, void* stream) {
  if (!s || !out) return set_error("fv_state_get: null argument"), FV_EINVAL;
  FV_CUDA(cudaMemcpyAsync(out, s->X, 9 * (size_t)s->N * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return FV_OK;
}

fv_status fv_state_set(fv_state* s, const double* in, void* stream) {
  if (!s || !in) return set_error("fv_state_set: null argument"), FV_EINVAL;
  FV_CUDA(cudaMemcpyAsync(s->X, in, 9 * (size_t)s->N * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return FV_OK;
}

// fields from `in` and a fresh history: the next step is a first step (f^{1/2} = f^0, u^ = u, B^ = B,
// initial guesses from the state), exactly as after fv_state_create
fv_status fv_state_reset(fv_state* s, const double* in, void* stream) {
  if (!s || !in) return set_error("fv_state_reset: null argument"), FV_EINVAL;
  FV_CUDA(cudaMemcpyAsync(s->X, in, 9 * (size_t)s->N * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  s->first = true;
  s->steps = 0;
  return FV_OK;
}

fv_status fv_time_step(fv_state* s, const fv_system* vtbe, const fv_system* ppbe, const fv_gmres_opts* opts,
                       int nsteps, fv_solve_stats* stats, void* stream) {
  return fv_time_step_opts(s, vtbe, ppbe, opts, opts, nsteps, stats, stream);
}

fv_status fv_time_step_opts(fv_state* s, const fv_system* vtbe, const fv_system* ppbe, const fv_gmres_opts* opts,
                            const fv_gmres_opts* popts, int nsteps, fv_solve_stats* stats, void* stream) {
  if (!s || !vtbe || !ppbe || !opts || !popts || nsteps < 0 || vtbe->kind != FV_VTBE || ppbe->kind != FV_PPBE ||
      vtbe->grid != s->grid || ppbe->grid != s->grid)
    return set_error("fv_time_step: bad argument (systems must be VTBE and PPBE of the state's grid)"), FV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const fv_grid* g = s->grid;
  const long long N = s->N;
  const double dt = s->phys.dt;
  fv_status rc;
  for (int step = 0; step < nsteps; ++step) {
    double* u = s->X;
    double* P = s->X + 7 * N;
    // nonlinear terms f^n and their Adams-Bashforth extrapolation
    if ((rc = ghost_fill(g->geo, u, s->gh, 7, st)) || (rc = nonlinear_terms(g, s->phys, u, s->fcur, s->gh, st))) return rc;
    if (s->first) rc = axpby(7 * N, 1.0, s->fcur, 0.0, nullptr, s->fh, st);
    else rc = axpby(7 * N, 1.5, s->fcur, -0.5, s->fprev, s->fh, st);
    if (rc) return rc;
    // x^ = (u - dt/2 G P, Theta, B - dt/2 G P_b)
    FV_CUDA(cudaMemcpyAsync(s->xhat, u, 7 * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (!s->first) {
      if ((rc = ghost_fill(g->geo, P, s->gh, 2, st)) ||
          (rc = cell_gradient(g, P, 0, 1.0 / s->phys.E, s->grad, s->gh, st)) ||
          (rc = axpby(3 * N, 1.0, u, -0.5 * dt, s->grad, s->xhat, st)) ||
          (rc = axpby(3 * N, 1.0, u + 4 * N, -0.5 * dt, s->grad + 3 * N, s->xhat + 4 * N, st)))
        return rc;
    }
    // b_V = 2 x^ - A_V x^ + dt f^{n+1/2}
    if ((rc = apply_op(vtbe, s->xhat, s->tmp, st)) || (rc = axpby(7 * N, 2.0, s->xhat, -1.0, s->tmp, s->bV, st)) ||
        (rc = axpby(7 * N, 1.0, s->bV, dt, s->fh, s->bV, st)))
      return rc;
    if (s->first) FV_CUDA(cudaMemcpyAsync(s->xV, u, 7 * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    fv_solve_stats sv{}, sp{};
    rc = gmres(vtbe, s->bV, s->xV, opts, &sv, st, false);
    if (rc) return rc;
    // PPBE right-hand side (D u~, D B~), zero-mean pressure part
    if ((rc = ghost_fill(g->geo, s->xV, s->gh, 7, st)) || (rc = face_divergence_uB(g, s->xV, s->bP, s->gh, st)) ||
        (rc = weighted_mean_remove(g, s->bP, st, s->part, s->sums)))
      return rc;
    FV_CUDA(cudaMemcpyAsync(s->xP, P, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    rc = gmres(ppbe, s->bP, s->xP, popts, &sp, st, false);
    if (rc) return rc;
    if ((rc = weighted_mean_remove(g, s->xP, st, s->part, s->sums))) return rc;
    // projection: u = u~ - dt/2 G P, B = B~ - dt/2 G P_b
    if ((rc = ghost_fill(g->geo, s->xP, s->gh, 2, st)) ||
        (rc = cell_gradient(g, s->xP, 0, 1.0 / s->phys.E, s->grad, s->gh, st)) ||
        (rc = axpby(3 * N, 1.0, s->xV, -0.5 * dt, s->grad, u, st)) ||
        (rc = axpby(3 * N, 1.0, s->xV + 4 * N, -0.5 * dt, s->grad + 3 * N, u + 4 * N, st)))
      return rc;
    FV_CUDA(cudaMemcpyAsync(u + 3 * N, s->xV + 3 * N, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    FV_CUDA(cudaMemcpyAsync(P, s->xP, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    std::swap(s->fprev, s->fcur);
    s->first = false;
    ++s->steps;
    if (stats) stats[2 * step] = sv, stats[2 * step + 1] = sp;
  }
  FV_CUDA(cudaStreamSynchronize(st));
  return FV_OK;
}

}  // extern "C"
