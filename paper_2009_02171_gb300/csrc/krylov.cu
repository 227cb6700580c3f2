// Restarted right-preconditioned flexible GMRES on the GPU (paper Sec. 3.3).
//
// Right preconditioning A M^{-1} (M x) = b (eqn:newlinear): the residual of
// the preconditioned system is the true residual b - A x; stop when
// ||b - A x|| <= max(eps_a, eps_r ||b - A x_0||).  The flexible form stores
// Z_j = M^{-1} v_j and updates x = x_0 + Z y, which allows the variable
// two-level preconditioner (inner GMRES on the coarse mesh) and, in mixed
// precision, an FP32 inner solve as preconditioner of the FP64 outer solve.
// Arnoldi uses classical Gram-Schmidt applied twice (CGS2): each pass is one
// fused sweep over the basis (multi-dot, then update-and-dot, then
// update-and-norm), with deterministic two-stage reductions (per-block
// partials in FP64 summed in a fixed order).  Hessenberg, Givens rotations and
// the small least-squares solve run on the host in FP64.
//
// The vector type T is double (FP64 path, outer solve of mixed precision) or
// float (inner solves of mixed precision).  For float vectors each thread sums
// at most 32 products in FP32 before adding them into its FP64 accumulators;
// block and grid reductions are FP64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <utility>
#include <vector>

#include "../../include/fv_net.h"
#include "fv_internal.h"

namespace fv {

constexpr int KMAX = 32;     // max basis vectors in one fused pass
constexpr int RBLOCKS = 304; // reduction blocks of the weighted sums (2 per SM)
constexpr int CGS_BMAX = 608; // reduction blocks of a basis pass at most (4 per SM)
constexpr int RTHREADS = 256;

// Arnoldi bookkeeping of a device-driven solve (no host synchronisation)
struct ArnoldiDev {
  double H[KMAX * KMAX];  // upper Hessenberg after rotations, column-major H[j * KMAX + i]
  double cs[KMAX], sn[KMAX], g[KMAX + 1], y[KMAX];
  double scale;           // 1 / norm of the newest basis vector (0 after a breakdown)
  int k_eff;              // number of usable columns (first breakdown)
};

template <class T>
struct KrylovT {
  int m = 0;
  long long n = 0;
  T *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr;
  double* part = nullptr;   // [KMAX][CGS_BMAX]
  double* h = nullptr;      // [3][KMAX]: h1, h2, nrm2
  double* hhost = nullptr;  // pinned [3][KMAX]
  ArnoldiDev* ad = nullptr; // device-driven solves
  unsigned* ticket = nullptr; // last-block counter of the fused reductions (returns to 0 after each use)
};

struct Krylov {
  KrylovT<double> d;
  KrylovT<float> f;
};

template <class T>
static void free_kt(KrylovT<T>& k) {
  cudaFree(k.V), cudaFree(k.Z), cudaFree(k.w), cudaFree(k.r), cudaFree(k.part), cudaFree(k.h), cudaFree(k.ad), cudaFree(k.ticket);
  cudaFreeHost(k.hhost);
  k = KrylovT<T>();
}

void free_krylov(Krylov* k) {
  if (!k) return;
  free_kt(k->d);
  free_kt(k->f);
  delete k;
}

template <class T>
static KrylovT<T>& kt(Krylov* k);
template <>
KrylovT<double>& kt<double>(Krylov* k) { return k->d; }
template <>
KrylovT<float>& kt<float>(Krylov* k) { return k->f; }

template <class T>
static fv_status ensure_krylov(const fv_system* s, int m) {
  fv_system* sm = const_cast<fv_system*>(s);
  if (!sm->kry) sm->kry = new Krylov();
  KrylovT<T>& k = kt<T>(sm->kry);
  if (k.m >= m && k.n == s->n) return FV_OK;
  free_kt(k);
  k.m = m, k.n = s->n;
  const size_t n = (size_t)s->n;
  if (cudaMalloc(&k.V, (m + 1) * n * sizeof(T)) != cudaSuccess || cudaMalloc(&k.Z, m * n * sizeof(T)) != cudaSuccess ||
      cudaMalloc(&k.w, n * sizeof(T)) != cudaSuccess || cudaMalloc(&k.r, n * sizeof(T)) != cudaSuccess ||
      cudaMalloc(&k.part, KMAX * CGS_BMAX * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&k.h, 3 * KMAX * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&k.ad, sizeof(ArnoldiDev)) != cudaSuccess || cudaMalloc(&k.ticket, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(k.ticket, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMallocHost(&k.hhost, 3 * KMAX * sizeof(double)) != cudaSuccess) {
    free_kt(k);
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

// block-reduce acc[0..nv) (nv <= NA) into part[v * gridDim.x + blockIdx.x]
template <int NA>
__device__ __forceinline__ void block_store_n(double (&acc)[NA], int nv, double* part) {
  __shared__ double sm[RTHREADS / 32][NA];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < NA; ++v) {
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

// Givens update of column j of the device-driven Arnoldi (thread 0 of one block):
// h = h1 + h2 (CGS2), h_{j+1,j} = sqrt(nrm2); previous rotations, new rotation,
// right-hand side update; scale = 1 / h_{j+1,j}
__device__ void givens_update(int j, const double* __restrict__ h, double nrm2, ArnoldiDev* ad) {
  double col[KMAX + 1];
  for (int i = 0; i <= j; ++i) col[i] = h[i] + h[KMAX + i];
  const double hn = sqrt(nrm2);
  col[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = ad->cs[i] * col[i] + ad->sn[i] * col[i + 1];
    col[i + 1] = -ad->sn[i] * col[i] + ad->cs[i] * col[i + 1];
    col[i] = a;
  }
  const double den = hypot(col[j], col[j + 1]);
  const double c = den > 0.0 ? col[j] / den : 1.0, s = den > 0.0 ? col[j + 1] / den : 0.0;
  ad->cs[j] = c, ad->sn[j] = s;
  col[j] = den;
  ad->g[j + 1] = -s * ad->g[j];
  ad->g[j] = c * ad->g[j];
  for (int i = 0; i <= j; ++i) ad->H[j * KMAX + i] = col[i];
  if (!(den > 0.0) && ad->k_eff > j) ad->k_eff = j;              // no usable column j
  else if (!(hn > 0.0) && ad->k_eff > j + 1) ad->k_eff = j + 1;  // lucky breakdown after column j
  ad->scale = hn > 0.0 ? 1.0 / hn : 0.0;
}

// sum of the nb partials p[0..nb) by one warp in a fixed order; the loads of a lane are issued
// together (L2, written by other blocks of this launch) before they are added
__device__ __forceinline__ double last_block_sum(const double* p, int nb, int lane) {
  double t = 0.0;
  for (int b0 = 0; b0 < nb; b0 += 32 * 8) {
    double q[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int b = b0 + u * 32 + lane;
      q[u] = b < nb ? __ldcg(p + b) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) t += q[u];
  }
  return warp_sum(t);
}

// 16-byte vector of T: four floats or two doubles
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
  static constexpr int L = 4;
  __device__ static void load(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
  }
  __device__ static void ldg(const float* p, float (&v)[4]) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
  }
  __device__ static void store(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Vec16<double> {
  static constexpr int L = 2;
  __device__ static void load(const double* p, double (&v)[2]) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x, v[1] = q.y;
  }
  __device__ static void ldg(const double* p, double (&v)[2]) {
    const double2 q = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = q.x, v[1] = q.y;
  }
  __device__ static void store(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};

// mode 0: part = V^T w
// mode 1: w -= V h; part = V^T w
// mode 2: w -= V h; part[0] = w^T w
// NV (the number of basis vectors) is a template parameter so the loops over
// the basis unroll exactly; h is staged in shared memory.  With `vec` (n a
// multiple of the 16-byte width and 16-byte aligned bases) a thread moves 16
// bytes of every vector per iteration, which keeps enough loads in flight to
// stream the basis at HBM rate; otherwise one element at a time.  FP32
// products are summed in FP32 for up to 32 elements of a thread, then in FP64;
// FP64 products go straight into the FP64 accumulators.  With `out`, the last
// block to finish sums the per-block partials in a fixed order into
// out[0..nv) (and, for mode 2 with `ad`, applies the Givens update of column
// gj), so no separate reduction launch is needed.
template <int NV, class T>
__global__ void __launch_bounds__(RTHREADS, (NV > (sizeof(T) == 8 ? 18 : 14) ? 1 : 2)) cgs_kernel(long long n, int vec, const T* __restrict__ V,
                                                          const double* __restrict__ h, T* __restrict__ w,
                                                          double* __restrict__ part, int mode, double* out,
                                                          unsigned* ticket, ArnoldiDev* ad, int gj,
                                                          const double* __restrict__ hg) {
  constexpr int NA = NV > 0 ? NV : 1;
  constexpr int L = Vec16<T>::L;
  constexpr bool F32 = sizeof(T) == 4;
  __shared__ T hs[NA];
  if (mode > 0)
    for (int v = threadIdx.x; v < NV; v += blockDim.x) hs[v] = (T)h[v];
  __syncthreads();
  double acc[NA];
  T cur[NA];
#pragma unroll
  for (int v = 0; v < NA; ++v) acc[v] = 0.0, cur[v] = T(0);
  double accn = 0.0;
  T curn = T(0);
  int cnt = 0;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  const long long ng = vec ? n / L : 0;
  for (long long g = tid; g < ng; g += stride) {
    const long long e = g * L;
    T we[L];
    Vec16<T>::load(w + e, we);
    if (mode > 0 && NV > 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T vv[L];
        Vec16<T>::ldg(V + v * n + e, vv);
        const T hv = hs[v];
#pragma unroll
        for (int l = 0; l < L; ++l) we[l] -= hv * vv[l];
      }
      Vec16<T>::store(w + e, we);
    }
    if (mode < 2) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T vv[L];
        Vec16<T>::ldg(V + v * n + e, vv);
#pragma unroll
        for (int l = 0; l < L; ++l) {
          if constexpr (F32) cur[v] += vv[l] * we[l];
          else acc[v] += vv[l] * we[l];
        }
      }
    } else {
#pragma unroll
      for (int l = 0; l < L; ++l) {
        if constexpr (F32) curn += we[l] * we[l];
        else accn += we[l] * we[l];
      }
    }
    if constexpr (F32) {  // FP32 partial sums go into the FP64 accumulators every 32 elements
      cnt += L;
      if (cnt >= 32) {
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += (double)cur[v], cur[v] = T(0);
        accn += (double)curn, curn = T(0);
        cnt = 0;
      }
    }
  }
  for (long long e = ng * L + tid; e < n; e += stride) {
    T we = w[e];
    if (mode > 0 && NV > 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) we -= hs[v] * V[v * n + e];
      w[e] = we;
    }
    if (mode < 2) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if constexpr (F32) cur[v] += V[v * n + e] * we;
        else acc[v] += V[v * n + e] * we;
      }
    } else {
      if constexpr (F32) curn += we * we;
      else accn += we * we;
    }
    if constexpr (F32) {  // FP32 partial sums go into the FP64 accumulators every 32 elements
      cnt += 1;
      if (cnt >= 32) {
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += (double)cur[v], cur[v] = T(0);
        accn += (double)curn, curn = T(0);
        cnt = 0;
      }
    }
  }
  if constexpr (F32) {
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] += (double)cur[v];
    accn += (double)curn;
  }
  if (mode == 2) acc[0] = accn;
  const int nvv = mode < 2 ? NV : 1;
  block_store_n<NA>(acc, nvv, part);
  if (!out) return;
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int v = wid; v < nvv; v += nw) out[v] = last_block_sum(part + v * gridDim.x, (int)gridDim.x, lane);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (mode == 2 && ad) givens_update(gj, hg, out[0], ad);
    *ticket = 0u;
  }
}

// reduction blocks of a basis pass over n elements: about four 16-byte groups (or elements) a
// thread, at most CGS_BMAX blocks (short vectors: fewer partials for the final sum); consumers of
// the partials take the same count
template <class T>
static int cgs_blocks(long long n, bool vec) {
  const long long g = vec ? n / Vec16<T>::L : n;
  return (int)std::min<long long>(std::max<long long>((g + 4 * RTHREADS - 1) / (4 * RTHREADS), 1), CGS_BMAX);
}

template <class T>
static bool cgs_vec(long long n, const T* V, const T* w) {
  return n % Vec16<T>::L == 0 && (reinterpret_cast<uintptr_t>(V) & 15) == 0 && (reinterpret_cast<uintptr_t>(w) & 15) == 0;
}

struct CgsFuse {
  double* out = nullptr;       // fused final reduction target (null: partials only)
  unsigned* ticket = nullptr;
  ArnoldiDev* ad = nullptr;    // mode 2: Givens update of column gj in the last block
  int gj = 0;
  const double* hg = nullptr;  // CGS2 coefficients h1 [0, KMAX), h2 [KMAX, 2 KMAX) of that column
};

template <int NV, class T>
static void cgs_launch_t(long long n, const T* V, const double* h, T* w, double* part, int mode, CgsFuse f,
                         cudaStream_t st) {
  const bool vec = cgs_vec<T>(n, V, w);
  cgs_kernel<NV, T><<<cgs_blocks<T>(n, vec), RTHREADS, 0, st>>>(n, vec ? 1 : 0, V, h, w, part, mode, f.out, f.ticket,
                                                                 f.ad, f.gj, f.hg);
}

template <class T, int... I>
static void cgs_dispatch(int nv, long long n, const T* V, const double* h, T* w, double* part, int mode, CgsFuse f,
                         cudaStream_t st, std::integer_sequence<int, I...>) {
  using F = void (*)(long long, const T*, const double*, T*, double*, int, CgsFuse, cudaStream_t);
  static const F table[] = {&cgs_launch_t<I, T>...};
  table[nv](n, V, h, w, part, mode, f, st);
}

template <class T>
static void cgs_launch(int nv, long long n, const T* V, const double* h, T* w, double* part, int mode,
                       cudaStream_t st, CgsFuse f = CgsFuse()) {
  cgs_dispatch<T>(nv, n, V, h, w, part, mode, f, st, std::make_integer_sequence<int, KMAX>{});
}

// out[v] = sum_b part[v * nb + b]: one warp per vector, fixed summation order
__global__ void reduce_kernel(const double* __restrict__ part, int nb, int nv, double* __restrict__ out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int v = wid; v < nv; v += nw) {
    double t = 0.0;
    for (int b = lane; b < nb; b += 32) t += part[v * nb + b];
    t = warp_sum(t);
    if (lane == 0) out[v] = t;
  }
}

template <class T, class U>
__global__ void axpby_kernel(long long n, double a, const U* __restrict__ x, double b, const T* y, T* out) {
  const T at = (T)a, bt = (T)b;
  const bool has_y = b != 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = at * (T)x[e] + (has_y ? bt * y[e] : T(0));
}

template <class T>
struct Coef {
  T c[KMAX];
};

// x += sum_v y_v Z_v
template <int NV, class T>
__global__ void update_kernel(long long n, const T* __restrict__ Z, Coef<T> y, T* __restrict__ x) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    T s = x[e];
#pragma unroll
    for (int v = 0; v < NV; ++v) s += y.c[v] * Z[v * n + e];
    x[e] = s;
  }
}

template <int NV, class T>
static void update_launch_t(int blocks, long long n, const T* Z, const Coef<T>& y, T* x, cudaStream_t st) {
  update_kernel<NV, T><<<blocks, 256, 0, st>>>(n, Z, y, x);
}

template <class T, int... I>
static void update_dispatch(int nv, int blocks, long long n, const T* Z, const Coef<T>& y, T* x, cudaStream_t st,
                            std::integer_sequence<int, I...>) {
  using F = void (*)(int, long long, const T*, const Coef<T>&, T*, cudaStream_t);
  static const F table[] = {&update_launch_t<I, T>...};
  table[nv](blocks, n, Z, y, x, st);
}

static int vblocks(long long n) { return (int)std::min<long long>(std::max<long long>((n + 255) / 256, 1), 152LL * 16); }

fv_status axpby(long long n, double a, const double* x, double b, const double* y, double* out, cudaStream_t st) {
  ProfScope ps(FV_K_VEC, st);
  axpby_kernel<double, double><<<vblocks(n), 256, 0, st>>>(n, a, x, b, y, out);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

fv_status axpby32(long long n, double a, const float* x, double b, const float* y, float* out, cudaStream_t st) {
  ProfScope ps(FV_K_VEC, st);
  axpby_kernel<float, float><<<vblocks(n), 256, 0, st>>>(n, a, x, b, y, out);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

fv_status to_fp32(long long n, const double* x, float* out, cudaStream_t st) {
  ProfScope ps(FV_K_VEC, st);
  axpby_kernel<float, double><<<vblocks(n), 256, 0, st>>>(n, 1.0, x, 0.0, nullptr, out);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

fv_status to_fp64(long long n, const float* x, double* out, cudaStream_t st) {
  ProfScope ps(FV_K_VEC, st);
  axpby_kernel<double, float><<<vblocks(n), 256, 0, st>>>(n, 1.0, x, 0.0, nullptr, out);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

template <class T>
static fv_status axpby_t(long long n, double a, const T* x, double b, const T* y, T* out, cudaStream_t st) {
  ProfScope ps(FV_K_VEC, st);
  axpby_kernel<T, T><<<vblocks(n), 256, 0, st>>>(n, a, x, b, y, out);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

template <class T>
static fv_status norm2(KrylovT<T>& k, long long n, const T* x, cudaStream_t st, double* out) {
  cgs_launch<T>(0, n, x, nullptr, const_cast<T*>(x), k.part, 2, st);
  reduce_kernel<<<1, RTHREADS, 0, st>>>(k.part, cgs_blocks<T>(n, cgs_vec<T>(n, x, x)), 1, k.h + 2 * KMAX);
  FV_CUDA(cudaGetLastError());
  FV_CUDA(cudaMemcpyAsync(k.hhost, k.h + 2 * KMAX, sizeof(double), cudaMemcpyDeviceToHost, st));
  FV_CUDA(cudaStreamSynchronize(st));
  *out = std::sqrt(k.hhost[0]);
  return FV_OK;
}

template <class T>
static fv_status apply_t(const fv_system* s, const T* x, T* y, cudaStream_t st);
template <>
fv_status apply_t<double>(const fv_system* s, const double* x, double* y, cudaStream_t st) {
  return apply_op(s, x, y, st);
}
template <>
fv_status apply_t<float>(const fv_system* s, const float* x, float* y, cudaStream_t st) {
  return apply_op32(s, x, y, st);
}

template <class T>
static fv_status precond_t(const fv_system* s, const T* r, T* z, cudaStream_t st);
template <>
fv_status precond_t<double>(const fv_system* s, const double* r, double* z, cudaStream_t st) {
  return precond_apply(s, r, z, st);
}
template <>
fv_status precond_t<float>(const fv_system* s, const float* r, float* z, cudaStream_t st) {
  return precond_apply32(s, r, z, st);
}

// ------------------------------------------------------------------ device-driven FGMRES
// beta = ||r|| from the norm partials; g = (beta, 0, ...); scale = 1/beta
__global__ void start_kernel(const double* __restrict__ part, int nb, ArnoldiDev* ad) {
  const int lane = threadIdx.x;
  double t = 0.0;
  for (int b = lane; b < nb; b += 32) t += part[b];
  t = warp_sum(t);
  if (lane == 0) {
    const double beta = sqrt(t);
    for (int i = 0; i <= KMAX; ++i) ad->g[i] = 0.0;
    ad->g[0] = beta;
    ad->scale = beta > 0.0 ? 1.0 / beta : 0.0;
    ad->k_eff = beta > 0.0 ? KMAX : 0;
  }
}

// y = H^{-1} g on the first min(m, k_eff) columns (back substitution), zero beyond
__global__ void lsq_kernel(int m, ArnoldiDev* ad) {
  if (threadIdx.x != 0) return;
  const int kk = m < ad->k_eff ? m : ad->k_eff;
  for (int i = KMAX - 1; i >= 0; --i) ad->y[i] = 0.0;
  for (int i = kk - 1; i >= 0; --i) {
    double s = ad->g[i];
    for (int q = i + 1; q < kk; ++q) s -= ad->H[q * KMAX + i] * ad->y[q];
    ad->y[i] = s / ad->H[i * KMAX + i];
  }
}

template <class T>
__global__ void dscale_kernel(long long n, const T* __restrict__ x, const double* __restrict__ scale, T* __restrict__ out) {
  const T a = (T)*scale;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = a * x[e];
}

// x = sum_v y_v Z_v with y in device memory
template <int NV, class T>
__global__ void dupdate_kernel(long long n, const T* __restrict__ Z, const double* __restrict__ y, T* __restrict__ x) {
  T c[NV > 0 ? NV : 1];
#pragma unroll
  for (int v = 0; v < NV; ++v) c[v] = (T)y[v];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    T s = T(0);
#pragma unroll
    for (int v = 0; v < NV; ++v) s += c[v] * Z[v * n + e];
    x[e] = s;
  }
}

template <int NV, class T>
static void dupdate_launch_t(int blocks, long long n, const T* Z, const double* y, T* x, cudaStream_t st) {
  dupdate_kernel<NV, T><<<blocks, 256, 0, st>>>(n, Z, y, x);
}

template <class T, int... I>
static void dupdate_dispatch(int nv, int blocks, long long n, const T* Z, const double* y, T* x, cudaStream_t st,
                             std::integer_sequence<int, I...>) {
  using F = void (*)(int, long long, const T*, const double*, T*, cudaStream_t);
  static const F table[] = {&dupdate_launch_t<I, T>...};
  table[nv](blocks, n, Z, y, x, st);
}

// Exactly m FGMRES iterations from x0 = 0, driven entirely on the device (no host
// synchronisation, so the call can be captured in a CUDA graph).  A flexible outer
// solve accepts this as a (variable) preconditioner.
template <class T>
static fv_status gmres_fixed_t(const fv_system* s, const T* b, T* x, int m, cudaStream_t st) {
  if (m < 1 || m > KMAX - 1) return set_error("fixed-iteration FGMRES: iterations must be in [1, 31]"), FV_EINVAL;
  fv_status rc = ensure_krylov<T>(s, m);
  if (rc) return rc;
  KrylovT<T>& k = kt<T>(s->kry);
  const long long n = s->n;
  const int lvl = FV_K_COARSE * s->level + (sizeof(T) == 4 ? FV_K_FP32 : 0);
  const bool once = s->pc.inner_gs_passes == 1;
  {
    ProfScope ps(FV_K_CGS + lvl, st);
    if (once) FV_CUDA(cudaMemsetAsync(k.h + KMAX, 0, KMAX * sizeof(double), st));
    cgs_launch<T>(0, n, b, nullptr, const_cast<T*>(b), k.part, 2, st);
    start_kernel<<<1, 32, 0, st>>>(k.part, cgs_blocks<T>(n, cgs_vec<T>(n, b, b)), k.ad);
    dscale_kernel<T><<<vblocks(n), 256, 0, st>>>(n, b, &k.ad->scale, k.V);
  }
  for (int j = 0; j < m; ++j) {
    T* vj = k.V + (size_t)j * n;
    T* zj = k.Z + (size_t)j * n;
    if ((rc = precond_t<T>(s, vj, zj, st))) return rc;
    if ((rc = apply_t<T>(s, zj, k.w, st))) return rc;
    const int nv = j + 1;
    ProfScope ps(FV_K_CGS + lvl, st);
    CgsFuse f;
    f.ticket = k.ticket;
    f.out = k.h;
    cgs_launch<T>(nv, n, k.V, nullptr, k.w, k.part, 0, st, f);
    if (once) {  // one pass: w -= V h1 with the norm; the second coefficients stay zero
      f.out = k.h + 2 * KMAX, f.ad = k.ad, f.gj = j, f.hg = k.h;
      cgs_launch<T>(nv, n, k.V, k.h, k.w, k.part, 2, st, f);
    } else {
      f.out = k.h + KMAX;
      cgs_launch<T>(nv, n, k.V, k.h, k.w, k.part, 1, st, f);
      f.out = k.h + 2 * KMAX, f.ad = k.ad, f.gj = j, f.hg = k.h;
      cgs_launch<T>(nv, n, k.V, k.h + KMAX, k.w, k.part, 2, st, f);
    }
    if (j + 1 < m) dscale_kernel<T><<<vblocks(n), 256, 0, st>>>(n, k.w, &k.ad->scale, k.V + (size_t)(j + 1) * n);
  }
  ProfScope ps(FV_K_VEC, st);
  lsq_kernel<<<1, 32, 0, st>>>(m, k.ad);
  dupdate_dispatch<T>(m, vblocks(n), n, k.Z, k.ad->y, x, st, std::make_integer_sequence<int, KMAX>{});
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

fv_status gmres_fixed32(const fv_system* s, const float* b, float* x, int m, cudaStream_t st) {
  return gmres_fixed_t<float>(s, b, x, m, st);
}

// ------------------------------------------------------------------ FGMRES
template <class T>
static fv_status gmres_t(const fv_system* s, const T* b, T* x, const fv_gmres_opts* o, fv_solve_stats* stats,
                         cudaStream_t st, bool inner) {
  auto t0 = std::chrono::steady_clock::now();
  const int m = o->restart;
  if (m < 1 || m > KMAX - 1 || o->max_it < 0) return set_error("fv_gmres_solve: restart must be in [1, 31]"), FV_EINVAL;
  fv_status rc = ensure_krylov<T>(s, m);
  if (rc) return rc;
  KrylovT<T>& k = kt<T>(s->kry);
  const long long n = s->n;
  const int lvl = FV_K_COARSE * s->level + (sizeof(T) == 4 ? FV_K_FP32 : 0);
  if (!inner) s->last_inner = 0;
  // r = b - A x
  if ((rc = apply_t<T>(s, x, k.r, st))) return rc;
  if ((rc = axpby_t<T>(n, 1.0, b, -1.0, k.r, k.r, st))) return rc;
  double beta;
  if ((rc = norm2<T>(k, n, k.r, st, &beta))) return rc;
  const double r0 = beta, target = std::max(o->atol, o->rtol * r0);
  int its = 0;
  bool nan = !std::isfinite(beta);
  std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  while (!nan && beta > target && its < o->max_it) {
    if ((rc = axpby_t<T>(n, 1.0 / beta, k.r, 0.0, nullptr, k.V, st))) return rc;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    bool breakdown = false;
    for (; j < m; ++j) {
      T* vj = k.V + (size_t)j * n;
      T* zj = k.Z + (size_t)j * n;
      if ((rc = precond_t<T>(s, vj, zj, st))) return rc;
      if ((rc = apply_t<T>(s, zj, k.w, st))) return rc;
      const int nv = j + 1;
      {
        ProfScope ps(FV_K_CGS + lvl, st);
        CgsFuse f;
        f.ticket = k.ticket;
        f.out = k.h;
        cgs_launch<T>(nv, n, k.V, nullptr, k.w, k.part, 0, st, f);
        f.out = k.h + KMAX;
        cgs_launch<T>(nv, n, k.V, k.h, k.w, k.part, 1, st, f);
        f.out = k.h + 2 * KMAX;
        cgs_launch<T>(nv, n, k.V, k.h + KMAX, k.w, k.part, 2, st, f);
      }
      FV_CUDA(cudaGetLastError());
      FV_CUDA(cudaMemcpyAsync(k.hhost, k.h, 3 * KMAX * sizeof(double), cudaMemcpyDeviceToHost, st));
      FV_CUDA(cudaStreamSynchronize(st));
      std::vector<double> col(j + 2);
      for (int i = 0; i <= j; ++i) col[i] = k.hhost[i] + k.hhost[KMAX + i];  // CGS2: h = h1 + h2
      const double hn = std::sqrt(k.hhost[2 * KMAX]);
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
      for (int i = 0; i <= j; ++i) H[i * m + j] = col[i];
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
      if ((rc = axpby_t<T>(n, 1.0 / hn, k.w, 0.0, nullptr, k.V + (size_t)(j + 1) * n, st))) return rc;
    }
    const int kk = std::min(j, m);
    if (!nan) {
      for (int i = kk - 1; i >= 0; --i) {
        double sacc = g[i];
        for (int q = i + 1; q < kk; ++q) sacc -= H[i * m + q] * y[q];
        y[i] = sacc / H[i * m + i];
      }
      Coef<T> c{};
      for (int i = 0; i < kk; ++i) c.c[i] = (T)y[i];
      ProfScope ps(FV_K_VEC, st);
      update_dispatch<T>(kk, vblocks(n), n, k.Z, c, x, st, std::make_integer_sequence<int, KMAX>{});
      FV_CUDA(cudaGetLastError());
    }
    if ((rc = apply_t<T>(s, x, k.r, st))) return rc;
    if ((rc = axpby_t<T>(n, 1.0, b, -1.0, k.r, k.r, st))) return rc;
    if ((rc = norm2<T>(k, n, k.r, st, &beta))) return rc;
    if (!std::isfinite(beta)) nan = true;
    if (breakdown) break;
  }
  const bool conv = !nan && beta <= target;
  if (stats) {
    stats->iters = its;
    stats->fallback = 0;
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

// Top-level solves of a system with a learned coarse correction: optional
// learned initial guess, then FGMRES for at most one restart cycle; if that
// ends without convergence, the plain coarse solve finishes from the last
// finite iterate with the original absolute target max(atol, rtol ||b - A x0||)
// and the iterations left.
static fv_status gmres_learned(const fv_system* s, const double* b, double* x, const fv_gmres_opts* o,
                               fv_solve_stats* stats, cudaStream_t st) {
  fv_system* sm = const_cast<fv_system*>(s);
  const size_t bytes = (size_t)s->n * sizeof(double);
  FV_CUDA(cudaMemcpyAsync(s->xbak, x, bytes, cudaMemcpyDeviceToDevice, st));
  fv_solve_stats s1{};
  fv_status rc = FV_OK;
  double r0 = -1.0;
  if (s->learned_flags & FV_LEARN_GUESS) {
    // the tolerance stays relative to the caller's x0
    const fv_gmres_opts o0{o->restart, 0, o->atol, o->rtol};
    fv_status rr = gmres_t<double>(s, b, x, &o0, &s1, st, false);
    if (rr && rr != FV_ENOCONV && rr != FV_ENAN) return rr;
    r0 = s1.r0;
    if ((rc = learned_guess(s, b, x, st))) return rc;
  }
  fv_gmres_opts o1 = *o;
  if (r0 >= 0.0) o1.atol = std::max(o->atol, o->rtol * r0), o1.rtol = 0.0;
  // the learned preconditioner gets one restart cycle; a solve it has not finished by then
  // (a stall, or a network that does not fit this problem) goes on with the plain one
  o1.max_it = std::min(o->max_it, o->restart);
  rc = gmres_t<double>(s, b, x, &o1, &s1, st, false);
  int inner = s->last_inner;
  if (r0 >= 0.0) s1.r0 = r0;
  if (rc == FV_ENOCONV || rc == FV_ENAN) {
    if (rc == FV_ENAN) FV_CUDA(cudaMemcpyAsync(x, s->xbak, bytes, cudaMemcpyDeviceToDevice, st));
    fv_gmres_opts o2 = *o;
    o2.max_it = std::max(0, o->max_it - s1.iters);
    o2.atol = std::max(o->atol, o->rtol * s1.r0), o2.rtol = 0.0;
    fv_solve_stats s2{};
    set_learned_active(sm, 0);
    rc = gmres_t<double>(s, b, x, &o2, &s2, st, false);
    set_learned_active(sm, 1);
    inner += s->last_inner;
    s1.iters += s2.iters, s1.converged = s2.converged, s1.rfinal = s2.rfinal, s1.time_ms += s2.time_ms;
    s1.fallback = 1;
  }
  s->last_inner = inner;
  s1.inner_iters = inner;
  if (stats) *stats = s1;
  return rc;
}

fv_status gmres(const fv_system* s, const double* b, double* x, const fv_gmres_opts* o, fv_solve_stats* stats,
                cudaStream_t st, bool inner) {
  if (!inner && s->net) return gmres_learned(s, b, x, o, stats, st);
  return gmres_t<double>(s, b, x, o, stats, st, inner);
}

fv_status gmres32(const fv_system* s, const float* b, float* x, const fv_gmres_opts* o, fv_solve_stats* stats,
                  cudaStream_t st) {
  return gmres_t<float>(s, b, x, o, stats, st, true);
}

// volume-weighted mean removal of the first component (Neumann pressure gauge)
// I: the index type, 32-bit whenever N allows (32-bit divisions in the index decomposition)
template <class T, class I>
__global__ void wsum_kernel(long long N, int Ns, int Nr, const double* __restrict__ invsig,
                            const double* __restrict__ invr2, const T* __restrict__ x, double* __restrict__ part) {
  double acc[KMAX];
  acc[0] = 0.0, acc[1] = 0.0;
  const I ns2 = (I)Ns * Ns;
  for (I e = blockIdx.x * (I)blockDim.x + threadIdx.x; e < (I)N; e += (I)gridDim.x * blockDim.x) {
    const int ij = (int)(e % ns2);
    const int k = (int)((e / ns2) % Nr);
    const double V = 1.0 / (invsig[ij] * invr2[k]);
    acc[0] += V * (double)x[e];
    acc[1] += V;
  }
  block_store(acc, 2, part);
}

template <class T>
__global__ void shift_kernel(long long N, const double* __restrict__ sums, T* __restrict__ x) {
  const T mean = (T)(sums[0] / sums[1]);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x)
    x[e] -= mean;
}

template <class T>
static fv_status wmr(const fv_grid* g, T* x, cudaStream_t st, double* part, double* sums) {
  const Geo& G = g->geo;
  ProfScope ps(FV_K_VEC, st);
  if (G.N < (1LL << 31) - (1LL << 24))
    wsum_kernel<T, int><<<RBLOCKS, RTHREADS, 0, st>>>(G.N, G.Ns, G.Nr, G.invsig, G.invr2, x, part);
  else
    wsum_kernel<T, long long><<<RBLOCKS, RTHREADS, 0, st>>>(G.N, G.Ns, G.Nr, G.invsig, G.invr2, x, part);
  reduce_kernel<<<1, RTHREADS, 0, st>>>(part, RBLOCKS, 2, sums);
  shift_kernel<T><<<vblocks(G.N), 256, 0, st>>>(G.N, sums, x);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

fv_status weighted_mean_remove(const fv_grid* g, double* x, cudaStream_t st, double* part, double* sums) {
  return wmr<double>(g, x, st, part, sums);
}

fv_status weighted_mean_remove32(const fv_grid* g, float* x, cudaStream_t st, double* part, double* sums) {
  return wmr<float>(g, x, st, part, sums);
}

}  // namespace fv
