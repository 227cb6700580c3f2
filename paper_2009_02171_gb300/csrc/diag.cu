// Diagnostics of a time-stepping state (fv_state_diagnostics).
//
// Paper Sec. 4.2: kinetic energy E_kin = Pm^2/2 int |u|^2 dV, magnetic energy
// E_mag = Pm/(2E) int |B|^2 dV, and the Alfven CFL number
// CFL_A = dt max(|v^1|/h_s + |v^2|/h_s + |v^3|/h_r) with v = B / sqrt(E Pm) in
// contravariant components (v^1 = v . grad xi, v^2 = v . grad eta,
// v^3 = v . rhat).
//
// Divergence constraint eqn:divtime (D u^{n+1} = D B^{n+1} = 0), two readings:
// * face: the fluxes of the projected fields through every face,
//   F_f(B^{n+1}) = F_f(B~) - dt/2 (G_f P_b) . S_f with the compact face
//   gradient of the PPBE operator, give per cell
//   D_f B^{n+1} = D(B~) - dt/2 D_f G_f P_b, which is the P_b block of the PPBE
//   residual b - A x of the last solve: it stays at the solver tolerance.
// * cell: D applied to the cell-centred B^{n+1} = B~ - dt/2 G_c P_b of
//   eqn:ubtilde (face means of cell values); the mismatch between D G_c and
//   D_f G_f leaves it at the discretization error, O(h^2).
// The same two numbers are reported for u (P block).  All sums are per-block
// partials in FP64 added on the host in a fixed order (deterministic).
#include <cmath>
#include <vector>

#include "stencil.cuh"

namespace fv {

enum { Q_EKIN = 0, Q_EMAG, Q_DIVB_F, Q_DIVB_RHS, Q_DIVU_F, Q_DIVU_RHS, Q_DIVB_C, Q_DIVU_C, Q_COUNT };
constexpr int DIAG_BLOCKS = 304;
constexpr int DIAG_THREADS = 256;

__device__ __forceinline__ double dwarp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double dwarp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// part[q * gridDim.x + block] for the Q_COUNT sums, part[Q_COUNT * gridDim.x + block] for the CFL maximum
// (per unit dt).  bP / AxP null: no PPBE solve yet, the face entries stay 0.
__global__ void __launch_bounds__(DIAG_THREADS) diag_kernel(Geo G, const double* __restrict__ cb,
                                                            const double* __restrict__ X,
                                                            const double* __restrict__ bP,
                                                            const double* __restrict__ AxP,
                                                            const double* __restrict__ divc, double vA,
                                                            double* __restrict__ part) {
  const long long N = G.N;
  const int Ns = G.Ns, Nr = G.Nr;
  double acc[Q_COUNT];
#pragma unroll
  for (int q = 0; q < Q_COUNT; ++q) acc[q] = 0.0;
  double mx = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % Ns);
    long long r = e / Ns;
    const int j = (int)(r % Ns);
    r /= Ns;
    const int k = (int)(r % Nr);
    const int p = (int)(r / Nr);
    const int ji = j * Ns + i;
    const double V = 1.0 / (G.invsig[ji] * G.invr2[k]);
    const double u[3] = {X[e], X[N + e], X[2 * N + e]};
    const double b[3] = {X[4 * N + e], X[5 * N + e], X[6 * N + e]};
    acc[Q_EKIN] += V * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    acc[Q_EMAG] += V * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    double g1[3], g2[3], rh[3];
    rotate(p, cb + 6 * ji, g1);
    rotate(p, cb + 6 * ji + 3, g2);
    rotate(p, G.xhat + 3 * ji, rh);
    const double rk = G.rc[k];
    const double v1 = (b[0] * g1[0] + b[1] * g1[1] + b[2] * g1[2]) / rk;
    const double v2 = (b[0] * g2[0] + b[1] * g2[1] + b[2] * g2[2]) / rk;
    const double v3 = b[0] * rh[0] + b[1] * rh[1] + b[2] * rh[2];
    mx = fmax(mx, vA * ((fabs(v1) + fabs(v2)) / G.hs + fabs(v3) / G.hr));
    if (bP) {
      const double rB = bP[N + e] - AxP[N + e], rU = bP[e] - AxP[e];
      acc[Q_DIVB_F] += rB * rB;
      acc[Q_DIVB_RHS] += bP[N + e] * bP[N + e];
      acc[Q_DIVU_F] += rU * rU;
      acc[Q_DIVU_RHS] += bP[e] * bP[e];
    }
    acc[Q_DIVU_C] += divc[e] * divc[e];
    acc[Q_DIVB_C] += divc[N + e] * divc[N + e];
  }
  __shared__ double sm[DIAG_THREADS / 32][Q_COUNT + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < Q_COUNT; ++q) {
    const double t = dwarp_sum(acc[q]);
    if (lane == 0) sm[wid][q] = t;
  }
  mx = dwarp_max(mx);
  if (lane == 0) sm[wid][Q_COUNT] = mx;
  __syncthreads();
  if (threadIdx.x <= Q_COUNT) {
    double t = 0.0;  // sums, or the maximum of non-negative values
    for (int w = 0; w < DIAG_THREADS / 32; ++w)
      t = threadIdx.x == Q_COUNT ? fmax(t, sm[w][Q_COUNT]) : t + sm[w][threadIdx.x];
    part[threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
}

}  // namespace fv

using namespace fv;

extern "C" fv_status fv_state_diagnostics(fv_state* s, const fv_system* ppbe, fv_diag* out, void* stream) {
  if (!s || !out) return set_error("fv_state_diagnostics: null argument"), FV_EINVAL;
  if (ppbe && (ppbe->kind != FV_PPBE || ppbe->grid != s->grid))
    return set_error("fv_state_diagnostics: ppbe must be the PPBE system of the state's grid"), FV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const fv_grid* g = s->grid;
  const bool face = ppbe && s->steps > 0;
  fv_status rc;
  // A x_P of the last PPBE solve into tmp (7N >= 2N values); D(u), D(B) of the current fields into grad
  if (face && (rc = apply_op(ppbe, s->xP, s->tmp, st))) return rc;
  if ((rc = ghost_fill(g->geo, s->X, s->gh, 7, st)) || (rc = face_divergence_uB(g, s->X, s->grad, s->gh, st)))
    return rc;
  const double vA = 1.0 / std::sqrt(s->phys.E * s->phys.Pm);
  diag_kernel<<<DIAG_BLOCKS, DIAG_THREADS, 0, st>>>(g->geo, g->cbasis, s->X, face ? s->bP : nullptr,
                                                    face ? s->tmp : nullptr, s->grad, vA, s->part);
  FV_CUDA(cudaGetLastError());
  std::vector<double> h((size_t)(Q_COUNT + 1) * DIAG_BLOCKS);
  FV_CUDA(cudaMemcpyAsync(h.data(), s->part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  FV_CUDA(cudaStreamSynchronize(st));
  double sum[Q_COUNT] = {}, mx = 0.0;
  for (int q = 0; q < Q_COUNT; ++q)
    for (int b = 0; b < DIAG_BLOCKS; ++b) sum[q] += h[(size_t)q * DIAG_BLOCKS + b];
  for (int b = 0; b < DIAG_BLOCKS; ++b) mx = std::fmax(mx, h[(size_t)Q_COUNT * DIAG_BLOCKS + b]);
  const fv_phys& ph = s->phys;
  out->E_kin = 0.5 * ph.Pm * ph.Pm * sum[Q_EKIN];
  out->E_mag = 0.5 * ph.Pm / ph.E * sum[Q_EMAG];
  out->cfl_alfven = mx * ph.dt;
  out->divB_face = face ? std::sqrt(sum[Q_DIVB_F]) : -1.0;
  out->divB_rhs = face ? std::sqrt(sum[Q_DIVB_RHS]) : -1.0;
  out->divU_face = face ? std::sqrt(sum[Q_DIVU_F]) : -1.0;
  out->divU_rhs = face ? std::sqrt(sum[Q_DIVU_RHS]) : -1.0;
  out->divB_cell = std::sqrt(sum[Q_DIVB_C]);
  out->divU_cell = std::sqrt(sum[Q_DIVU_C]);
  out->steps = s->steps;
  return FV_OK;
}
