// Restarted right-preconditioned flexible GMRES on the GPU (paper Sec. 3.3).
//
// Right preconditioning A M^{-1} (M x) = b (eqn:newlinear): the residual of
// the preconditioned system is the true residual b - A x; stop when
// ||b - A x|| <= max(eps_a, eps_r ||b - A x_0||).  The flexible form stores
// Z_j = M^{-1} v_j and updates x = x_0 + Z y, which allows the variable
// two-level preconditioner (inner GMRES on the coarse mesh).  Arnoldi uses
// classical Gram-Schmidt applied twice (CGS2): each pass is one fused sweep
// over the basis (multi-dot, then update-and-dot, then update-and-norm), with
// deterministic two-stage reductions (per-block partials summed in a fixed
// order).  Hessenberg, Givens rotations and the small least-squares solve
// run on the host in FP64; vectors never leave the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "fv_internal.h"

namespace fv {

constexpr int KMAX = 32;     // max basis vectors in one fused pass
constexpr int RBLOCKS = 304; // reduction blocks (2 per SM)
constexpr int RTHREADS = 256;

struct Krylov {
  int m = 0;
  long long n = 0;
  double *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr;
  double* part = nullptr;  // [KMAX][RBLOCKS]
  double* h = nullptr;     // [3][KMAX]: h1, h2, nrm2
  double* hhost = nullptr; // pinned [3][KMAX]
};

void free_krylov(Krylov* k) {
  if (!k) return;
  cudaFree(k->V), cudaFree(k->Z), cudaFree(k->w), cudaFree(k->r), cudaFree(k->part), cudaFree(k->h);
  cudaFreeHost(k->hhost);
  delete k;
}

static fv_status ensure_krylov(const fv_system* s, int m) {
  Krylov* k = s->kry;
  if (k && k->m >= m && k->n == s->n) return FV_OK;
  free_krylov(k);
  k = new Krylov();
  const_cast<fv_system*>(s)->kry = k;
  k->m = m, k->n = s->n;
  const size_t n = (size_t)s->n;
  if (cudaMalloc(&k->V, (m + 1) * n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&k->Z, m * n * sizeof(double)) != cudaSuccess || cudaMalloc(&k->w, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&k->r, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&k->part, KMAX * RBLOCKS * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&k->h, 3 * KMAX * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&k->hhost, 3 * KMAX * sizeof(double)) != cudaSuccess) {
    free_krylov(k);
    const_cast<fv_system*>(s)->kry = nullptr;
    return set_error("fv_gmres_solve: device allocation of the Krylov basis failed"), FV_ENOMEM;
  }
  return FV_OK;
}

// ------------------------------------------------------------------ vector kernels
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-reduce acc[0..nv) into part[v * gridDim.x + blockIdx.x]
__device__ __forceinline__ void block_store(double (&acc)[KMAX], int nv, double* part) {
  __shared__ double sm[RTHREADS / 32][KMAX];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < KMAX; ++v) {
    if (v < nv) {
      double t = warp_sum(acc[v]);
      if (lane == 0) sm[wid][v] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double t = 0.0;
    for (int q = 0; q < RTHREADS / 32; ++q) t += sm[q][threadIdx.x];
    part[threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
}

// mode 0: part = V^T w
// mode 1: w -= V h; part = V^T w
// mode 2: w -= V h; part[0] = w^T w
__global__ void __launch_bounds__(RTHREADS) cgs_kernel(long long n, const double* __restrict__ V, int nv,
                                                       const double* __restrict__ h, double* __restrict__ w,
                                                       double* __restrict__ part, int mode) {
  double acc[KMAX];
  double hv[KMAX];
#pragma unroll
  for (int v = 0; v < KMAX; ++v) {
    acc[v] = 0.0;
    hv[v] = (mode > 0 && v < nv) ? h[v] : 0.0;
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double we = w[e];
    if (mode > 0) {
#pragma unroll
      for (int v = 0; v < KMAX; ++v)
        if (v < nv) we -= hv[v] * V[v * n + e];
      w[e] = we;
    }
    if (mode < 2) {
#pragma unroll
      for (int v = 0; v < KMAX; ++v)
        if (v < nv) acc[v] += V[v * n + e] * we;
    } else {
      acc[0] += we * we;
    }
  }
  block_store(acc, mode < 2 ? nv : 1, part);
}

// out[v] = sum_b part[v * nb + b] (fixed order); if add: out[v] += previous value in `prev`
__global__ void reduce_kernel(const double* __restrict__ part, int nb, int nv, double* __restrict__ out,
                              const double* __restrict__ prev) {
  __shared__ double sm[RTHREADS];
  for (int v = 0; v < nv; ++v) {
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) t += part[v * nb + b];
    sm[threadIdx.x] = t;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[v] = sm[0] + (prev ? prev[v] : 0.0);
    __syncthreads();
  }
}

__global__ void axpby_kernel(long long n, double a, const double* __restrict__ x, double b, const double* y,
                             double* out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = a * x[e] + (b == 0.0 ? 0.0 : b * y[e]);
}

struct Coef {
  double c[KMAX];
};

// x += sum_v y_v Z_v
__global__ void update_kernel(long long n, const double* __restrict__ Z, int nv, Coef y, double* __restrict__ x) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double s = x[e];
#pragma unroll
    for (int v = 0; v < KMAX; ++v)
      if (v < nv) s += y.c[v] * Z[v * n + e];
    x[e] = s;
  }
}

static int vblocks(long long n) { return (int)std::min<long long>(std::max<long long>((n + 255) / 256, 1), 152LL * 16); }

fv_status axpby(long long n, double a, const double* x, double b, const double* y, double* out, cudaStream_t st) {
  ProfScope ps(FV_K_VEC, st);
  axpby_kernel<<<vblocks(n), 256, 0, st>>>(n, a, x, b, y, out);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

static fv_status norm2(Krylov* k, long long n, const double* x, cudaStream_t st, double* out) {
  cgs_kernel<<<RBLOCKS, RTHREADS, 0, st>>>(n, x, 0, nullptr, const_cast<double*>(x), k->part, 2);
  reduce_kernel<<<1, RTHREADS, 0, st>>>(k->part, RBLOCKS, 1, k->h + 2 * KMAX, nullptr);
  FV_CUDA(cudaGetLastError());
  FV_CUDA(cudaMemcpyAsync(k->hhost, k->h + 2 * KMAX, sizeof(double), cudaMemcpyDeviceToHost, st));
  FV_CUDA(cudaStreamSynchronize(st));
  *out = std::sqrt(k->hhost[0]);
  return FV_OK;
}

// ------------------------------------------------------------------ FGMRES
fv_status gmres(const fv_system* s, const double* b, double* x, const fv_gmres_opts* o, fv_solve_stats* stats,
                cudaStream_t st, bool inner) {
  auto t0 = std::chrono::steady_clock::now();
  const int m = o->restart;
  if (m < 1 || m > KMAX - 1 || o->max_it < 0) return set_error("fv_gmres_solve: restart must be in [1, 31]"), FV_EINVAL;
  fv_status rc = ensure_krylov(s, m);
  if (rc) return rc;
  Krylov* k = s->kry;
  const long long n = s->n;
  if (!inner) s->last_inner = 0;
  // r = b - A x
  if ((rc = apply_op(s, x, k->r, st))) return rc;
  if ((rc = axpby(n, 1.0, b, -1.0, k->r, k->r, st))) return rc;
  double beta;
  if ((rc = norm2(k, n, k->r, st, &beta))) return rc;
  const double r0 = beta, target = std::max(o->atol, o->rtol * r0);
  int its = 0;
  bool nan = !std::isfinite(beta);
  std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  while (!nan && beta > target && its < o->max_it) {
    if ((rc = axpby(n, 1.0 / beta, k->r, 0.0, nullptr, k->V, st))) return rc;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    bool breakdown = false;
    for (; j < m; ++j) {
      double* vj = k->V + (size_t)j * n;
      double* zj = k->Z + (size_t)j * n;
      if ((rc = precond_apply(s, vj, zj, st))) return rc;
      if ((rc = apply_op(s, zj, k->w, st))) return rc;
      const int nv = j + 1;
      {
      ProfScope ps(FV_K_CGS + FV_K_COARSE * s->level, st);
      cgs_kernel<<<RBLOCKS, RTHREADS, 0, st>>>(n, k->V, nv, nullptr, k->w, k->part, 0);
      reduce_kernel<<<1, RTHREADS, 0, st>>>(k->part, RBLOCKS, nv, k->h, nullptr);
      cgs_kernel<<<RBLOCKS, RTHREADS, 0, st>>>(n, k->V, nv, k->h, k->w, k->part, 1);
      reduce_kernel<<<1, RTHREADS, 0, st>>>(k->part, RBLOCKS, nv, k->h + KMAX, nullptr);
      cgs_kernel<<<RBLOCKS, RTHREADS, 0, st>>>(n, k->V, nv, k->h + KMAX, k->w, k->part, 2);
      reduce_kernel<<<1, RTHREADS, 0, st>>>(k->part, RBLOCKS, 1, k->h + 2 * KMAX, nullptr);
      }
      FV_CUDA(cudaGetLastError());
      FV_CUDA(cudaMemcpyAsync(k->hhost, k->h, 3 * KMAX * sizeof(double), cudaMemcpyDeviceToHost, st));
      FV_CUDA(cudaStreamSynchronize(st));
      double* hc = &H[0];
      std::vector<double> col(j + 2);
      for (int i = 0; i <= j; ++i) col[i] = k->hhost[i] + k->hhost[KMAX + i];  // CGS2: h = h1 + h2
      const double hn = std::sqrt(k->hhost[2 * KMAX]);
      col[j + 1] = hn;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
      }
      const double den = std::hypot(col[j], col[j + 1]);
      cs[j] = col[j] / den, sn[j] = col[j + 1] / den;
      col[j] = den, col[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) hc[i * m + j] = col[i];
      ++its;
      if (!std::isfinite(hn) || !std::isfinite(g[j + 1])) {
        nan = true;
        ++j;
        break;
      }
      if (hn == 0.0) breakdown = true;
      if (std::fabs(g[j + 1]) <= target || its >= o->max_it || breakdown) {
        ++j;
        break;
      }
      if ((rc = axpby(n, 1.0 / hn, k->w, 0.0, nullptr, k->V + (size_t)(j + 1) * n, st))) return rc;
    }
    const int kk = std::min(j, m);
    if (!nan) {
      for (int i = kk - 1; i >= 0; --i) {
        double sacc = g[i];
        for (int q = i + 1; q < kk; ++q) sacc -= H[i * m + q] * y[q];
        y[i] = sacc / H[i * m + i];
      }
      Coef c{};
      for (int i = 0; i < kk; ++i) c.c[i] = y[i];
      ProfScope ps(FV_K_VEC, st);
      update_kernel<<<vblocks(n), 256, 0, st>>>(n, k->Z, kk, c, x);
      FV_CUDA(cudaGetLastError());
    }
    if ((rc = apply_op(s, x, k->r, st))) return rc;
    if ((rc = axpby(n, 1.0, b, -1.0, k->r, k->r, st))) return rc;
    if ((rc = norm2(k, n, k->r, st, &beta))) return rc;
    if (!std::isfinite(beta)) nan = true;
    if (breakdown) break;
  }
  const bool conv = !nan && beta <= target;
  if (stats) {
    stats->iters = its;
    stats->inner_iters = s->last_inner;
    stats->converged = conv ? 1 : 0;
    stats->r0 = r0;
    stats->rfinal = beta;
    stats->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  if (nan) return set_error("fv_gmres_solve: NaN or Inf residual"), FV_ENAN;
  if (!conv) return set_error("fv_gmres_solve: max_it reached before the tolerance"), FV_ENOCONV;
  return FV_OK;
}

// volume-weighted mean removal of the first component (Neumann pressure gauge)
__global__ void wsum_kernel(long long N, int Ns, int Nr, const double* __restrict__ invsig, const double* __restrict__ invr2,
                            const double* __restrict__ x, double* __restrict__ part) {
  double acc[KMAX];
  acc[0] = 0.0, acc[1] = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    const int ij = (int)(e % ((long long)Ns * Ns));
    const int k = (int)((e / ((long long)Ns * Ns)) % Nr);
    const double V = 1.0 / (invsig[ij] * invr2[k]);
    acc[0] += V * x[e];
    acc[1] += V;
  }
  block_store(acc, 2, part);
}

__global__ void shift_kernel(long long N, const double* __restrict__ sums, double* __restrict__ x) {
  const double mean = sums[0] / sums[1];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x)
    x[e] -= mean;
}

fv_status weighted_mean_remove(const fv_grid* g, double* x, cudaStream_t st, double* part, double* sums) {
  const Geo& G = g->geo;
  wsum_kernel<<<RBLOCKS, RTHREADS, 0, st>>>(G.N, G.Ns, G.Nr, G.invsig, G.invr2, x, part);
  reduce_kernel<<<1, RTHREADS, 0, st>>>(part, RBLOCKS, 2, sums, nullptr);
  shift_kernel<<<vblocks(G.N), 256, 0, st>>>(G.N, sums, x);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

}  // namespace fv
