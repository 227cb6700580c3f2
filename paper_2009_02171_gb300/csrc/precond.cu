// Restricted additive Schwarz preconditioning on the GPU (paper Sec. 3.3).
//
// * Subdomains: each panel split into p1 x p2 x p3 boxes; each box extended by
//   `overlap` cells in its panel's extended index space (cells across a panel
//   edge are the neighbour panel's cells through the edge correspondence;
//   radial overlap stops at the walls; box positions past a cube corner hold
//   no cell and are identity rows).
// * A_i^delta on the structured pattern: 11 neighbours (i+-1, j+-1,
//   (i+-1, j+-1), k+-1), dense d x d diagonal block, component-diagonal
//   off-diagonal blocks; other couplings of A are dropped.
// * ILU(0) (the paper's "ILU with no fill-in") in natural box order (k, j, i),
//   components innermost.  Factorization and both triangular sweeps run one
//   CTA per subdomain over wavefronts: cell (i, j, k) depends only on cells of
//   smaller level i + 2 j + k, so each level is one parallel step.
// * RAS (eqn:onelevel): gather R_i^delta r inside the forward sweep, scatter
//   the owned cells (R_i^0)^T inside the backward sweep; owned cells
//   partition the grid, so no atomics.
// * Two-level hybrid (eqn:twolevel, eqn:coarsesolve, eqn:finesolve): coarse
//   value = mean of the 8 children, piecewise-constant prolongation; the
//   restricted Neumann-pressure right-hand side is projected to zero coarse
//   volume-weighted mean so the singular coarse system is consistent.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "fv_internal.h"

namespace fv {

__device__ __constant__ static const signed char kSlot[11][3] = {
    {0, 0, -1}, {-1, -1, 0}, {0, -1, 0}, {1, -1, 0}, {-1, 0, 0}, {0, 0, 0},
    {1, 0, 0},  {-1, 1, 0},  {0, 1, 0},  {1, 1, 0},  {0, 0, 1}};

// ------------------------------------------------------------------ host setup
static std::vector<int> split(int n, int parts) {
  std::vector<int> o(parts + 1, 0);
  for (int b = 0; b < parts; ++b) o[b + 1] = o[b] + n / parts + (b < n % parts ? 1 : 0);
  return o;
}

// global cell at (k, j, i) of panel p's extended index space, -1 past a cube corner
static long long ext_cell(const GridHost& h, int p, int k, int j, int i) {
  const int Ns = h.Ns;
  const bool in_i = i >= 0 && i < Ns, in_j = j >= 0 && j < Ns;
  auto cell = [&](int q, int jj, int ii) { return ((long long)(q * h.Nr + k) * Ns + jj) * Ns + ii; };
  if (in_i && in_j) return cell(p, j, i);
  if (!in_i && !in_j) return -1;
  int side, m, t;
  if (i < 0) side = XI_MIN, m = -1 - i, t = j;
  else if (i >= Ns) side = XI_MAX, m = i - Ns, t = j;
  else if (j < 0) side = ETA_MIN, m = -1 - j, t = i;
  else side = ETA_MAX, m = j - Ns, t = i;
  const int ps = p * 4 + side;
  const int q = h.pq[ps], sq = h.psq[ps], tq = h.ptmap[ps * Ns + t];
  switch (sq) {
    case XI_MIN: return cell(q, tq, m);
    case XI_MAX: return cell(q, tq, Ns - 1 - m);
    case ETA_MIN: return cell(q, m, tq);
    default: return cell(q, Ns - 1 - m, tq);
  }
}

template <class T>
static T* dalloc(fv_system* s, size_t n) {
  void* d = nullptr;
  if (cudaMalloc(&d, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return nullptr;
  s->allocs.push_back(d);
  return static_cast<T*>(d);
}

fv_status build_subdomains(fv_system* s, const fv_grid* g) {
  const GridHost& h = g->h;
  const fv_pc_desc& pc = s->pc;
  const int delta = pc.overlap;
  if (pc.p1 < 1 || pc.p2 < 1 || pc.p3 < 1 || pc.p1 > h.Ns || pc.p2 > h.Ns || pc.p3 > h.Nr || delta < 0 ||
      delta > h.Ns / 2)
    return set_error("fv_assemble_system: bad decomposition (p1, p2, p3, overlap)"), FV_EINVAL;
  const int d = s->d;
  auto bi = split(h.Ns, pc.p1), bj = split(h.Ns, pc.p2), bk = split(h.Nr, pc.p3);
  std::vector<long long> cell_off{0}, gmap;
  std::vector<int> dims;
  std::vector<unsigned char> owned;
  std::vector<std::vector<int>> orders;
  int max_levels = 0;
  for (int p = 0; p < 6; ++p)
    for (int c = 0; c < pc.p3; ++c)
      for (int b = 0; b < pc.p2; ++b)
        for (int a = 0; a < pc.p1; ++a) {
          const int i0 = bi[a], i1 = bi[a + 1], j0 = bj[b], j1 = bj[b + 1], k0 = bk[c], k1 = bk[c + 1];
          const int lo_i = i0 - delta, lo_j = j0 - delta, lo_k = std::max(0, k0 - delta);
          const int nx = i1 - i0 + 2 * delta, ny = j1 - j0 + 2 * delta, nz = std::min(h.Nr, k1 + delta) - lo_k;
          dims.insert(dims.end(), {nx, ny, nz});
          const int levels = (nx - 1) + 2 * (ny - 1) + (nz - 1) + 1;
          max_levels = std::max(max_levels, levels);
          std::vector<int> cnt(levels + 1, 0), ord(nx * ny * nz);
          for (int lk = 0; lk < nz; ++lk)
            for (int lj = 0; lj < ny; ++lj)
              for (int li = 0; li < nx; ++li) {
                const int i = lo_i + li, j = lo_j + lj, k = lo_k + lk;
                gmap.push_back(ext_cell(h, p, k, j, i));
                owned.push_back(i >= i0 && i < i1 && j >= j0 && j < j1 && k >= k0 && k < k1);
                cnt[li + 2 * lj + lk + 1]++;
              }
          for (int L = 0; L < levels; ++L) cnt[L + 1] += cnt[L];
          std::vector<int> pos(cnt.begin(), cnt.end() - 1);
          for (int lk = 0; lk < nz; ++lk)
            for (int lj = 0; lj < ny; ++lj)
              for (int li = 0; li < nx; ++li) ord[pos[li + 2 * lj + lk]++] = (lk * ny + lj) * nx + li;
          orders.push_back(ord);
          cell_off.push_back(cell_off.back() + (long long)nx * ny * nz);
        }
  const int count = (int)dims.size() / 3;
  // level offsets per subdomain, padded to max_levels + 1
  std::vector<int> level_off((size_t)count * (max_levels + 1), 0), order;
  order.reserve(gmap.size());
  for (int sd = 0; sd < count; ++sd) {
    const int nx = dims[3 * sd], ny = dims[3 * sd + 1], nz = dims[3 * sd + 2];
    const int levels = (nx - 1) + 2 * (ny - 1) + (nz - 1) + 1;
    std::vector<int> cnt(levels + 1, 0);
    for (int lk = 0; lk < nz; ++lk)
      for (int lj = 0; lj < ny; ++lj)
        for (int li = 0; li < nx; ++li) cnt[li + 2 * lj + lk + 1]++;
    for (int L = 0; L < levels; ++L) cnt[L + 1] += cnt[L];
    for (int L = 0; L <= max_levels; ++L) level_off[(size_t)sd * (max_levels + 1) + L] = cnt[std::min(L, levels)];
    order.insert(order.end(), orders[sd].begin(), orders[sd].end());
  }
  std::vector<int> lpt(count);
  std::iota(lpt.begin(), lpt.end(), 0);
  std::stable_sort(lpt.begin(), lpt.end(),
                   [&](int a, int b) { return cell_off[a + 1] - cell_off[a] > cell_off[b + 1] - cell_off[b]; });

  Subdomains& S = s->subs;
  S.count = count, S.d = d, S.total_cells = cell_off.back(), S.max_levels = max_levels;
  const long long T = S.total_cells;
  S.cell_off = dalloc<long long>(s, count + 1);
  S.dims = dalloc<int>(s, dims.size());
  S.gmap = dalloc<long long>(s, T);
  S.owned = dalloc<unsigned char>(s, T);
  S.level_off = dalloc<int>(s, level_off.size());
  S.order = dalloc<int>(s, T);
  S.off = dalloc<double>(s, (size_t)T * 11 * d);
  S.diag = dalloc<double>(s, (size_t)T * d * d);
  S.work = dalloc<double>(s, (size_t)T * d);
  S.status = dalloc<int>(s, 1);
  S.lpt = dalloc<int>(s, count);
  if (!S.cell_off || !S.dims || !S.gmap || !S.owned || !S.level_off || !S.order || !S.off || !S.diag || !S.work ||
      !S.status || !S.lpt)
    return set_error("fv_assemble_system: device allocation of subdomain data failed"), FV_ENOMEM;
  FV_CUDA(cudaMemcpy(S.cell_off, cell_off.data(), cell_off.size() * sizeof(long long), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(S.dims, dims.data(), dims.size() * sizeof(int), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(S.gmap, gmap.data(), gmap.size() * sizeof(long long), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(S.owned, owned.data(), owned.size(), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(S.level_off, level_off.data(), level_off.size() * sizeof(int), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(S.order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(S.lpt, lpt.data(), lpt.size() * sizeof(int), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemset(S.status, 0, sizeof(int)));
  return FV_OK;
}

// ------------------------------------------------------------------ ILU(0)
struct Box {
  int nx, ny, nz;
  __device__ __forceinline__ bool in(int i, int j, int k) const {
    return i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz;
  }
};

__device__ __forceinline__ int slot_delta(const Box& b, int s) {
  return (kSlot[s][2] * b.ny + kSlot[s][1]) * b.nx + kSlot[s][0];
}

__global__ void ilu_factor_kernel(int d, const long long* __restrict__ cell_off, const int* __restrict__ dims,
                                  const int* __restrict__ level_off, int max_levels, const int* __restrict__ order,
                                  const int* __restrict__ lpt, double* __restrict__ off, double* __restrict__ diag,
                                  int* __restrict__ status) {
  const int sd = lpt[blockIdx.x];
  const long long base = cell_off[sd];
  const Box b{dims[3 * sd], dims[3 * sd + 1], dims[3 * sd + 2]};
  const int* lo = level_off + (size_t)sd * (max_levels + 1);
  const int levels = (b.nx - 1) + 2 * (b.ny - 1) + (b.nz - 1) + 1;
  for (int L = 0; L < levels; ++L) {
    for (int idx = lo[L] + threadIdx.x; idx < lo[L + 1]; idx += blockDim.x) {
      const int c = order[base + idx];
      const int li = c % b.nx, lj = (c / b.nx) % b.ny, lk = c / (b.nx * b.ny);
      const long long C = base + c;
      double* dc = diag + C * d * d;
      for (int a = 0; a < d; ++a) {
        // lower-neighbour pivots, ascending column order
        for (int s = 0; s < 5; ++s) {
          if (!b.in(li + kSlot[s][0], lj + kSlot[s][1], lk + kSlot[s][2])) continue;
          const long long Q = C + slot_delta(b, s);
          const double l = off[(C * 11 + s) * d + a] / diag[(Q * d + a) * d + a];
          off[(C * 11 + s) * d + a] = l;
          for (int u = 6; u < 11; ++u) {
            const int ti = kSlot[s][0] + kSlot[u][0], tj = kSlot[s][1] + kSlot[u][1], tk = kSlot[s][2] + kSlot[u][2];
            int t = -1;
            for (int z = 0; z < 11; ++z)
              if (kSlot[z][0] == ti && kSlot[z][1] == tj && kSlot[z][2] == tk) t = z;
            if (t < 0 || !b.in(li + ti, lj + tj, lk + tk)) continue;
            const double val = off[(Q * 11 + u) * d + a];
            if (t == 5) dc[a * d + a] -= l * val;
            else off[(C * 11 + t) * d + a] -= l * val;
          }
        }
        // pivots inside the diagonal block
        for (int bb = 0; bb < a; ++bb) {
          const double l = dc[a * d + bb] / dc[bb * d + bb];
          dc[a * d + bb] = l;
          for (int cc = bb + 1; cc < d; ++cc) dc[a * d + cc] -= l * dc[bb * d + cc];
        }
        if (dc[a * d + a] == 0.0) atomicCAS(status, 0, 1 + (int)C);
      }
    }
    __syncthreads();
  }
}

fv_status ilu_factor(fv_system* s) {
  Subdomains& S = s->subs;
  ilu_factor_kernel<<<S.count, 256>>>(S.d, S.cell_off, S.dims, S.level_off, S.max_levels, S.order, S.lpt, S.off,
                                      S.diag, S.status);
  FV_CUDA(cudaGetLastError());
  int st = 0;
  FV_CUDA(cudaMemcpy(&st, S.status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) return set_error("fv_assemble_system: zero pivot in ILU(0)"), FV_EBREAKDOWN;
  return FV_OK;
}

// ------------------------------------------------------------------ RAS apply
__global__ void ras_forward_kernel(int d, long long N, const long long* __restrict__ cell_off,
                                   const int* __restrict__ dims, const int* __restrict__ level_off, int max_levels,
                                   const int* __restrict__ order, const int* __restrict__ lpt,
                                   const long long* __restrict__ gmap, const double* __restrict__ off,
                                   const double* __restrict__ diag, const double* __restrict__ r,
                                   double* __restrict__ work) {
  const int sd = lpt[blockIdx.x];
  const long long base = cell_off[sd];
  const Box b{dims[3 * sd], dims[3 * sd + 1], dims[3 * sd + 2]};
  const int* lo = level_off + (size_t)sd * (max_levels + 1);
  const int levels = (b.nx - 1) + 2 * (b.ny - 1) + (b.nz - 1) + 1;
  for (int L = 0; L < levels; ++L) {
    for (int idx = lo[L] + threadIdx.x; idx < lo[L + 1]; idx += blockDim.x) {
      const int c = order[base + idx];
      const int li = c % b.nx, lj = (c / b.nx) % b.ny, lk = c / (b.nx * b.ny);
      const long long C = base + c;
      const long long g = gmap[C];
      for (int a = 0; a < d; ++a) {
        double y = g >= 0 ? r[a * N + g] : 0.0;
        for (int s = 0; s < 5; ++s) {
          if (!b.in(li + kSlot[s][0], lj + kSlot[s][1], lk + kSlot[s][2])) continue;
          y -= off[(C * 11 + s) * d + a] * work[(C + slot_delta(b, s)) * d + a];
        }
        for (int bb = 0; bb < a; ++bb) y -= diag[(C * d + a) * d + bb] * work[C * d + bb];
        work[C * d + a] = y;
      }
    }
    __syncthreads();
  }
}

__global__ void ras_backward_kernel(int d, long long N, const long long* __restrict__ cell_off,
                                    const int* __restrict__ dims, const int* __restrict__ level_off, int max_levels,
                                    const int* __restrict__ order, const int* __restrict__ lpt,
                                    const long long* __restrict__ gmap, const unsigned char* __restrict__ owned,
                                    const double* __restrict__ off, const double* __restrict__ diag,
                                    double* __restrict__ work, double* __restrict__ z) {
  const int sd = lpt[blockIdx.x];
  const long long base = cell_off[sd];
  const Box b{dims[3 * sd], dims[3 * sd + 1], dims[3 * sd + 2]};
  const int* lo = level_off + (size_t)sd * (max_levels + 1);
  const int levels = (b.nx - 1) + 2 * (b.ny - 1) + (b.nz - 1) + 1;
  for (int L = levels - 1; L >= 0; --L) {
    for (int idx = lo[L] + threadIdx.x; idx < lo[L + 1]; idx += blockDim.x) {
      const int c = order[base + idx];
      const int li = c % b.nx, lj = (c / b.nx) % b.ny, lk = c / (b.nx * b.ny);
      const long long C = base + c;
      const bool own = owned[C];
      const long long g = gmap[C];
      for (int a = d - 1; a >= 0; --a) {
        double x = work[C * d + a];
        for (int bb = a + 1; bb < d; ++bb) x -= diag[(C * d + a) * d + bb] * work[C * d + bb];
        for (int s = 6; s < 11; ++s) {
          if (!b.in(li + kSlot[s][0], lj + kSlot[s][1], lk + kSlot[s][2])) continue;
          x -= off[(C * 11 + s) * d + a] * work[(C + slot_delta(b, s)) * d + a];
        }
        x /= diag[(C * d + a) * d + a];
        work[C * d + a] = x;
        if (own) z[a * N + g] = x;
      }
    }
    __syncthreads();
  }
}

fv_status ras_apply(const fv_system* s, const double* r, double* z, cudaStream_t st) {
  const Subdomains& S = s->subs;
  const long long N = s->grid->geo.N;
  {
  ProfScope ps(FV_K_RAS_FWD + FV_K_COARSE * s->level, st);
  ras_forward_kernel<<<S.count, 256, 0, st>>>(S.d, N, S.cell_off, S.dims, S.level_off, S.max_levels, S.order, S.lpt,
                                               S.gmap, S.off, S.diag, r, S.work);
  }
  FV_CUDA(cudaGetLastError());
  ProfScope ps(FV_K_RAS_BWD + FV_K_COARSE * s->level, st);
  ras_backward_kernel<<<S.count, 256, 0, st>>>(S.d, N, S.cell_off, S.dims, S.level_off, S.max_levels, S.order,
                                                S.lpt, S.gmap, S.owned, S.off, S.diag, S.work, z);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

// ------------------------------------------------------------------ two levels
__global__ void restrict_kernel(int d, int Ns, int Nr, const double* __restrict__ x, double* __restrict__ xc) {
  const int nc = Ns / 2, mc = Nr / 2;
  const long long Nc = 6LL * nc * nc * mc, N = 6LL * Ns * Ns * Nr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < d * Nc;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e;
    const int i = (int)(r % nc);
    r /= nc;
    const int j = (int)(r % nc);
    r /= nc;
    const int k = (int)(r % mc);
    r /= mc;
    const int p = (int)(r % 6);
    const int a = (int)(r / 6);
    const double* xa = x + a * N;
    double sum = 0.0;
    for (int dk = 0; dk < 2; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di)
          sum += xa[((long long)(p * Nr + 2 * k + dk) * Ns + 2 * j + dj) * Ns + 2 * i + di];
    xc[e] = sum * 0.125;
  }
}

__global__ void prolong_kernel(int d, int Ns, int Nr, const double* __restrict__ xc, double* __restrict__ x) {
  const int nc = Ns / 2, mc = Nr / 2;
  const long long N = 6LL * Ns * Ns * Nr, Nc = 6LL * nc * nc * mc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < d * N;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e;
    const int i = (int)(r % Ns);
    r /= Ns;
    const int j = (int)(r % Ns);
    r /= Ns;
    const int k = (int)(r % Nr);
    r /= Nr;
    const int p = (int)(r % 6);
    const int a = (int)(r / 6);
    x[e] = xc[a * Nc + ((long long)(p * mc + k / 2) * nc + j / 2) * nc + i / 2];
  }
}

static int nblocks(long long n) {
  long long b = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(b, 1), 152LL * 32);
}

fv_status restrict_mean(const fv_grid* g, int d, const double* x, double* xc, cudaStream_t st) {
  ProfScope ps(FV_K_TRANSFER, st);
  restrict_kernel<<<nblocks(d * g->h.N / 8), 256, 0, st>>>(d, g->h.Ns, g->h.Nr, x, xc);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

fv_status prolong_inject(const fv_grid* g, int d, const double* xc, double* x, cudaStream_t st) {
  ProfScope ps(FV_K_TRANSFER, st);
  prolong_kernel<<<nblocks(d * g->h.N), 256, 0, st>>>(d, g->h.Ns, g->h.Nr, xc, x);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

fv_status precond_apply(const fv_system* s, const double* r, double* z, cudaStream_t st) {
  if (s->pc.levels < 2) return ras_apply(s, r, z, st);
  // w = I_c^f A_c^{-1} I_f^c r   (eqn:coarsesolve), inner FGMRES to coarse_rtol
  const fv_system* c = s->coarse;
  fv_status rc;
  {
    ProfScope ph(FV_K_PHASE_PC_I, st);
    if ((rc = restrict_mean(s->grid, s->d, r, s->xc, st))) return rc;
    // The coarse Neumann-pressure matrix is singular with the coarse cell volumes as
    // left null vector: project the restricted P right-hand side onto its range.
    if (s->kind == FV_PPBE && (rc = weighted_mean_remove(c->grid, s->xc, st, s->red, s->red + 32 * 304))) return rc;
    FV_CUDA(cudaMemsetAsync(s->ec, 0, c->n * sizeof(double), st));
  }
  {
    ProfScope ph(FV_K_PHASE_PC_C, st);
    fv_gmres_opts o{s->pc.coarse_restart, s->pc.coarse_maxit, 0.0, s->pc.coarse_rtol};
    fv_solve_stats cs{};
    rc = gmres(c, s->xc, s->ec, &o, &cs, st, true);
    if (rc && rc != FV_ENOCONV) return rc;
    s->last_inner += cs.iters;
  }
  {
    ProfScope ph(FV_K_PHASE_PC_I, st);
    if ((rc = prolong_inject(s->grid, s->d, s->ec, s->w, st))) return rc;
    // y = w + M_one^{-1} (r - A_f w)   (eqn:finesolve)
    if ((rc = apply_op(s, s->w, s->t, st))) return rc;
    if ((rc = axpby(s->n, 1.0, r, -1.0, s->t, s->t, st))) return rc;
  }
  {
    ProfScope ph(FV_K_PHASE_PC_F, st);
    if ((rc = ras_apply(s, s->t, z, st))) return rc;
  }
  ProfScope ph(FV_K_PHASE_PC_I, st);
  return axpby(s->n, 1.0, z, 1.0, s->w, z, st);
}

}  // namespace fv
