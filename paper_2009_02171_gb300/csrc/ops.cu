// Operator kernels: panel-edge ghost layer, matrix-free VTBE / PPBE apply,
// and extraction of the structured subdomain matrices for ILU(0).
#include <cstdio>
#include <mutex>
#include <string>

#include "stencil.cuh"

namespace fv {

// ---------------------------------------------------------------- ghost layer
// Ghost centre beyond `side` of panel p at tangential index t: quadratic
// Lagrange interpolation along the neighbour's first grid line (paper
// Sec. 3.3 overlap across block interfaces; one ghost layer).  Corner ghosts
// (t = -1 or Ns on the xi sides): phi(-1,-1) = phi(-1,0) + phi(0,-1) - phi(0,0).
template <class T, class GT>
__global__ void ghost_kernel(GT G, const T* __restrict__ x, T* __restrict__ gh, int d) {
  using R = typename GT::real;
  const int Ns = G.Ns, Nr = G.Nr;
  const long long total = (long long)d * 6 * 4 * Nr * (Ns + 2);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e;
    const int tp = (int)(r % (Ns + 2));
    r /= (Ns + 2);
    const int k = (int)(r % Nr);
    r /= Nr;
    const int side = (int)(r % 4);
    r /= 4;
    const int p = (int)(r % 6);
    const int comp = (int)(r / 6);
    const int t = tp - 1;
    R v = R(0);
    if (t >= 0 && t < Ns) {
      v = interp_ghost(G, x, comp, p, side, k, t);
    } else if (side == XI_MIN || side == XI_MAX) {
      const int jin = t < 0 ? 0 : Ns - 1;
      const int iin = side == XI_MIN ? 0 : Ns - 1;
      v = interp_ghost(G, x, comp, p, side, k, jin) + interp_ghost(G, x, comp, p, t < 0 ? ETA_MIN : ETA_MAX, k, iin) -
          (R)x[comp * G.N + cidx(G, p, k, jin, iin)];
    }
    gh[e] = (T)v;
  }
}

static int grid_blocks(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return (int)(b < 152LL * 32 ? (b < 1 ? 1 : b) : 152LL * 32);
}

fv_status ghost_fill(const Geo& G, const double* x, double* gh, int d, cudaStream_t st) {
  const long long total = (long long)d * 6 * 4 * G.Nr * (G.Ns + 2);
  ghost_kernel<double, Geo><<<grid_blocks(total, 256), 256, 0, st>>>(G, x, gh, d);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

// ---------------------------------------------------------------- apply (term visitor)
// The row-visitor apply of fv_apply_op_noalloc (fv_apply_op and the FP32 inner solves use the tiled
// kernels of apply.cu).  One launch covers every row: the first blocks map threads onto the (Ns-2)^2 interior of
// each panel layer (no warp touches a panel edge, so none diverges into the out-of-line edge
// path), the remaining blocks onto the 4 (Ns-1) cells of each layer's boundary ring, so the
// edge rows run beside the interior ones.  grid.y = k, grid.z = comp * 6 + panel; 32-bit index math.
constexpr int APPLY_THREADS = 256;

template <int KIND, class T, class GT>
__global__ void __launch_bounds__(APPLY_THREADS) apply_kernel(GT G, Coefs<typename GT::real> cf,
                                                              const T* __restrict__ x, const T* __restrict__ gh,
                                                              T* __restrict__ y) {
  const int Ns = G.Ns, ni = Ns - 2;
  const int nib = (ni * ni + APPLY_THREADS - 1) / APPLY_THREADS;  // interior blocks
  int i, j;
  if ((int)blockIdx.x < nib) {
    const int q = blockIdx.x * APPLY_THREADS + threadIdx.x;
    if (q >= ni * ni) return;
    i = 1 + q % ni, j = 1 + q / ni;
  } else {  // walk the boundary ring: j = 0 row, i = Ns-1 column, j = Ns-1 row, i = 0 column
    const int q = (blockIdx.x - nib) * APPLY_THREADS + threadIdx.x;
    if (q >= 4 * (Ns - 1)) return;
    const int s = q / (Ns - 1), t = q % (Ns - 1);
    if (s == 0) i = t, j = 0;
    else if (s == 1) i = Ns - 1, j = t;
    else if (s == 2) i = Ns - 1 - t, j = Ns - 1;
    else i = 0, j = Ns - 1 - t;
  }
  const int k = blockIdx.y, a = blockIdx.z / 6, p = blockIdx.z - 6 * a;
  ApplyAcc<T, typename GT::real> acc(G, x, gh);
  if (KIND == FV_VTBE) vtbe_row(G, cf, acc, p, k, j, i, a);
  else ppbe_row(G, cf, acc, p, k, j, i, a);
  y[(long long)a * G.N + ((long long)(p * G.Nr + k) * G.Ns + j) * G.Ns + i] = (T)acc.sum;
}

template <int KIND, class T, class GT>
static void launch_apply(const GT& G, const Coefs<typename GT::real>& cf, int d, const T* x, const T* gh, T* y,
                         cudaStream_t st) {
  const int ni = G.Ns - 2;
  const int blocks = (ni * ni + APPLY_THREADS - 1) / APPLY_THREADS + (4 * (G.Ns - 1) + APPLY_THREADS - 1) / APPLY_THREADS;
  apply_kernel<KIND, T, GT><<<dim3(blocks, G.Nr, 6 * d), APPLY_THREADS, 0, st>>>(G, cf, x, gh, y);
}

// ---------------------------------------------------------------- apply without allocation
// Ghost layer of fv_apply_op_noalloc: one static array per device, shared by all calls.
static __device__ __align__(256) double g_static_ghost[FV_STATIC_GHOST_DOUBLES];

static const int kMaxDevices = 64;
// device address of the array per device, looked up once per device (std::call_once makes concurrent first
// calls from several host threads safe); a device reset invalidates it (documented in fv.h)
static double* g_static_ghost_addr[kMaxDevices] = {};
static cudaError_t g_static_ghost_err[kMaxDevices] = {};
static std::once_flag g_static_ghost_once[kMaxDevices];

static fv_status static_ghost_address(double** out) {
  int dev = 0;
  FV_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error("fv_apply_op_noalloc: device ordinal out of range"), FV_EINVAL;
  std::call_once(g_static_ghost_once[dev], [dev] {
    void* p = nullptr;
    g_static_ghost_err[dev] = cudaGetSymbolAddress(&p, g_static_ghost);
    g_static_ghost_addr[dev] = static_cast<double*>(p);
  });
  FV_CUDA(g_static_ghost_err[dev]);
  *out = g_static_ghost_addr[dev];
  return FV_OK;
}

fv_status apply_op_noalloc(const fv_system* s, const double* x, double* y, cudaStream_t st) {
  const Geo& G = s->grid->geo;
  const long long total = (long long)s->d * 6 * 4 * G.Nr * (G.Ns + 2);
  if (total > FV_STATIC_GHOST_DOUBLES)
    return set_error("fv_apply_op_noalloc: ghost layer of this system (" + std::to_string(total) +
                     " doubles) exceeds FV_STATIC_GHOST_DOUBLES"),
           FV_EINVAL;
  double* gh = nullptr;
  fv_status rc = static_ghost_address(&gh);
  if (rc) return rc;
  ghost_kernel<double, Geo><<<grid_blocks(total, 256), 256, 0, st>>>(G, x, gh, s->d);
  FV_CUDA(cudaGetLastError());
  const Coefs<double> cf = make_coefs<double>(Phys{s->phys.E, s->phys.Ra, s->phys.Pr, s->phys.Pm, s->phys.dt},
                                               s->grid->h.ri, s->grid->h.ro);
  if (s->kind == FV_VTBE) launch_apply<FV_VTBE>(G, cf, s->d, x, (const double*)gh, y, st);
  else launch_apply<FV_PPBE>(G, cf, s->d, x, (const double*)gh, y, st);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

// ---------------------------------------------------------------- assembly
// Structured slots (di, dj, dk) in ascending natural order of the neighbour;
// slot 5 is the cell itself (dense d x d block), others are component-diagonal.
__device__ __constant__ static const signed char kOff[11][3] = {
    {0, 0, -1}, {-1, -1, 0}, {0, -1, 0}, {1, -1, 0}, {-1, 0, 0}, {0, 0, 0},
    {1, 0, 0},  {-1, 1, 0},  {0, 1, 0},  {1, 1, 0},  {0, 0, 1}};

struct AssembleAcc {
  const Geo* G;
  int row_comp;
  long long col[11];  // global cell of each slot, -1 if absent
  double off[11];
  double diag[8];
  __device__ __noinline__ void cell(double c, int p, int k, int j, int i, int comp) {
    const long long g = cidx(*G, p, k, j, i);
    if (g == col[5]) {
      diag[comp] += c;
      return;
    }
    if (comp != row_comp) return;
    for (int s = 0; s < 11; ++s)
      if (s != 5 && col[s] == g) {
        off[s] += c;
        return;
      }
  }
  __device__ __noinline__ void interp(double c, int p, int side, int k, int t, int comp) {
    const int Ns = G->Ns;
    const int id = (p * 4 + side) * Ns + t;
    const int q = G->gq[id];
    for (int m = 0; m < 3; ++m) {
      const int src = G->gsrc[3 * id + m];
      cell(c * G->gw[3 * id + m], q, k, src / Ns, src % Ns, comp);
    }
  }
  __device__ __noinline__ void ghost(double c, int p, int side, int k, int t, int comp) {
    const int Ns = G->Ns;
    if (t >= 0 && t < Ns) {
      interp(c, p, side, k, t, comp);
    } else {
      const int jin = t < 0 ? 0 : Ns - 1;
      const int iin = side == XI_MIN ? 0 : Ns - 1;
      interp(c, p, side, k, jin, comp);
      interp(c, p, t < 0 ? ETA_MIN : ETA_MAX, k, iin, comp);
      cell(-c, p, k, jin, iin, comp);
    }
  }
};

__global__ void assemble_kernel(Geo G, Coefs<double> cf, int kind, int d, int count, const long long* __restrict__ cell_off,
                                const int* __restrict__ dims, const long long* __restrict__ gmap,
                                double* __restrict__ off, double* __restrict__ diag) {
  const long long total = cell_off[count];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total * d;
       e += (long long)gridDim.x * blockDim.x) {
    const long long cell = e / d;
    const int a = (int)(e - cell * d);
    // find the subdomain (binary search over offsets)
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) / 2;
      if (cell_off[mid] <= cell) lo = mid;
      else hi = mid - 1;
    }
    const int nx = dims[3 * lo], ny = dims[3 * lo + 1], nz = dims[3 * lo + 2];
    const long long base = cell_off[lo];
    const int loc = (int)(cell - base);
    const int li = loc % nx, lj = (loc / nx) % ny, lk = loc / (nx * ny);
    AssembleAcc acc;
    acc.G = G.self;
    acc.row_comp = a;
    for (int s = 0; s < 11; ++s) {
      const int ni = li + kOff[s][0], nj = lj + kOff[s][1], nk = lk + kOff[s][2];
      acc.col[s] = (ni >= 0 && ni < nx && nj >= 0 && nj < ny && nk >= 0 && nk < nz)
                       ? gmap[base + (nk * ny + nj) * nx + ni]
                       : -1;
      acc.off[s] = 0.0;
    }
    for (int b = 0; b < 8; ++b) acc.diag[b] = 0.0;
    const long long g = acc.col[5];
    if (g >= 0) {
      long long c = g;
      const int i = (int)(c % G.Ns);
      c /= G.Ns;
      const int j = (int)(c % G.Ns);
      c /= G.Ns;
      const int k = (int)(c % G.Nr);
      const int p = (int)(c / G.Nr);
      if (kind == FV_VTBE) vtbe_row(G, cf, acc, p, k, j, i, a);
      else ppbe_row(G, cf, acc, p, k, j, i, a);
      for (int s = 0; s < 11; ++s)
        if (acc.col[s] < 0) acc.off[s] = 0.0;
    } else {
      acc.diag[a] = 1.0;  // position past a cube corner: identity row
    }
    for (int s = 0; s < 11; ++s) off[(cell * 11 + s) * d + a] = acc.off[s];
    for (int b = 0; b < d; ++b) diag[(cell * d + a) * d + b] = acc.diag[b];
  }
}

fv_status assemble_subdomains(fv_system* s) {
  const Geo& G = s->grid->geo;
  const Coefs<double> cf = make_coefs<double>(Phys{s->phys.E, s->phys.Ra, s->phys.Pr, s->phys.Pm, s->phys.dt},
                                               s->grid->h.ri, s->grid->h.ro);
  const long long work = s->subs.total_cells * s->d;
  assemble_kernel<<<grid_blocks(work, 128), 128>>>(G, cf, s->kind, s->d, s->subs.count, s->subs.cell_off,
                                                   s->subs.dims, s->subs.gmap, s->subs.off, s->subs.diag);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

}  // namespace fv
