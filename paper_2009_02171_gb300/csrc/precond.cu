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
#include <array>
#include <cstring>
#include <numeric>
#include <vector>

#include <cuda_bf16.h>

#include "fv_internal.h"

namespace fv {

// factor storage (FP64, FP32, or BF16 for the FP32 sweeps of FV_PREC_BF16) to the sweep arithmetic type
__device__ __forceinline__ float fcvt(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float fcvt(float v) { return v; }
__device__ __forceinline__ double fcvt(double v) { return v; }
template <class FT>
__device__ __forceinline__ FT to_factor(double v) { return (FT)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_factor<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

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
  if ((pc.nboxes <= 0 && (pc.p1 < 1 || pc.p2 < 1 || pc.p3 < 1 || pc.p1 > h.Ns || pc.p2 > h.Ns || pc.p3 > h.Nr)) ||
      delta < 0 || delta > h.Ns / 2)
    return set_error("fv_assemble_system: bad decomposition (p1, p2, p3, overlap)"), FV_EINVAL;
  const int d = s->d;
  // owned boxes: the structured p1 x p2 x p3 split of each panel, or an explicit list
  std::vector<std::array<int, 7>> own;
  if (pc.nboxes > 0) {
    if (!pc.boxes) return set_error("fv_assemble_system: nboxes > 0 with a null box list"), FV_EINVAL;
    std::vector<unsigned char> cover((size_t)h.N, 0);
    for (int q = 0; q < pc.nboxes; ++q) {
      std::array<int, 7> bx;
      for (int t = 0; t < 7; ++t) bx[t] = pc.boxes[7 * q + t];
      const int p = bx[0];
      if (p < 0 || p > 5 || bx[1] < 0 || bx[2] > h.Ns || bx[1] >= bx[2] || bx[3] < 0 || bx[4] > h.Ns || bx[3] >= bx[4] ||
          bx[5] < 0 || bx[6] > h.Nr || bx[5] >= bx[6])
        return set_error("fv_assemble_system: box outside the grid or empty"), FV_EINVAL;
      for (int k = bx[5]; k < bx[6]; ++k)
        for (int j = bx[3]; j < bx[4]; ++j)
          for (int i = bx[1]; i < bx[2]; ++i) {
            unsigned char& c = cover[((size_t)(p * h.Nr + k) * h.Ns + j) * h.Ns + i];
            if (c) return set_error("fv_assemble_system: boxes overlap"), FV_EINVAL;
            c = 1;
          }
      own.push_back(bx);
    }
    for (unsigned char c : cover)
      if (!c) return set_error("fv_assemble_system: boxes do not cover the grid"), FV_EINVAL;
  } else {
    auto bi = split(h.Ns, pc.p1), bj = split(h.Ns, pc.p2), bk = split(h.Nr, pc.p3);
    for (int p = 0; p < 6; ++p)
      for (int c = 0; c < pc.p3; ++c)
        for (int b = 0; b < pc.p2; ++b)
          for (int a = 0; a < pc.p1; ++a) own.push_back({p, bi[a], bi[a + 1], bj[b], bj[b + 1], bk[c], bk[c + 1]});
  }
  std::vector<long long> cell_off{0}, gmap;
  std::vector<int> dims;
  std::vector<unsigned char> owned;
  std::vector<std::vector<int>> orders, perms;
  int max_levels = 0, max_cols = 0;
  for (const auto& bx : own) {
          const int p = bx[0], i0 = bx[1], i1 = bx[2], j0 = bx[3], j1 = bx[4], k0 = bx[5], k1 = bx[6];
          const int lo_i = i0 - delta, lo_j = j0 - delta, lo_k = std::max(0, k0 - delta);
          const int nx = i1 - i0 + 2 * delta, ny = j1 - j0 + 2 * delta, nz = std::min(h.Nr, k1 + delta) - lo_k;
          dims.insert(dims.end(), {nx, ny, nz});
          max_cols = std::max(max_cols, nx * ny);
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
          // wavefront order for the sweeps: level, then j, then i
          std::vector<int> pp(nx * ny * nz);
          int pos_ = 0;
          for (int L = 0; L < levels; ++L)
            for (int lj = 0; lj < ny; ++lj) {
              const int lo_ = std::max(0, L - 2 * lj - (nz - 1)), hi_ = std::min(nx - 1, L - 2 * lj);
              for (int li = lo_; li <= hi_; ++li) pp[((L - li - 2 * lj) * ny + lj) * nx + li] = pos_++;
            }
          perms.push_back(pp);
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
  std::vector<int> perm;
  std::vector<long long> gmap_p(gmap.size());
  std::vector<unsigned char> owned_p(owned.size());
  perm.reserve(gmap.size());
  for (int sd = 0; sd < count; ++sd) {
    perm.insert(perm.end(), perms[sd].begin(), perms[sd].end());
    for (size_t c = 0; c < perms[sd].size(); ++c) {
      gmap_p[cell_off[sd] + perms[sd][c]] = gmap[cell_off[sd] + c];
      owned_p[cell_off[sd] + perms[sd][c]] = owned[cell_off[sd] + c];
    }
  }
  std::vector<int> lpt(count);
  std::iota(lpt.begin(), lpt.end(), 0);
  std::stable_sort(lpt.begin(), lpt.end(),
                   [&](int a, int b) { return cell_off[a + 1] - cell_off[a] > cell_off[b + 1] - cell_off[b]; });

  Subdomains& S = s->subs;
  S.count = count, S.d = d, S.total_cells = cell_off.back(), S.max_levels = max_levels, S.max_cols = max_cols;
  const long long T = S.total_cells;
  S.cell_off = dalloc<long long>(s, count + 1);
  S.dims = dalloc<int>(s, dims.size());
  S.gmap = dalloc<long long>(s, T);
  S.owned = dalloc<unsigned char>(s, T);
  S.level_off = dalloc<int>(s, level_off.size());
  S.order = dalloc<int>(s, T);
  S.off = dalloc<double>(s, (size_t)T * 11 * d);
  S.diag = dalloc<double>(s, (size_t)T * d * d);
  S.status = dalloc<int>(s, 1);
  S.lpt = dalloc<int>(s, count);
  S.perm = dalloc<int>(s, T);
  S.gmap_p = dalloc<long long>(s, T);
  S.owned_p = dalloc<unsigned char>(s, T);
  if (!S.cell_off || !S.dims || !S.gmap || !S.owned || !S.level_off || !S.order || !S.off || !S.diag ||
      !S.status || !S.lpt || !S.perm || !S.gmap_p || !S.owned_p)
    return set_error("fv_assemble_system: device allocation of subdomain data failed"), FV_ENOMEM;
  FV_CUDA(cudaMemcpy(S.cell_off, cell_off.data(), cell_off.size() * sizeof(long long), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(S.dims, dims.data(), dims.size() * sizeof(int), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(S.gmap, gmap.data(), gmap.size() * sizeof(long long), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(S.owned, owned.data(), owned.size(), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(S.level_off, level_off.data(), level_off.size() * sizeof(int), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(S.order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(S.lpt, lpt.data(), lpt.size() * sizeof(int), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(S.perm, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(S.gmap_p, gmap_p.data(), gmap_p.size() * sizeof(long long), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(S.owned_p, owned_p.data(), owned_p.size(), cudaMemcpyHostToDevice));
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

// ------------------------------------------------------------------ sweep layout
static void release(fv_system* s, void* ptr) {
  for (auto it = s->allocs.begin(); it != s->allocs.end(); ++it)
    if (*it == ptr) {
      cudaFree(ptr);
      s->allocs.erase(it);
      return;
    }
}

__device__ __forceinline__ int find_subdomain(const long long* cell_off, int count, long long cell) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (cell_off[mid] <= cell) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// factors: natural layout off[C][11][d], diag[C][d][d]  ->  packed SoA in wavefront order:
// q = s d + a (lower slots 0..4), 5 d + a d + b (diagonal block: L strictly below, U above, 1 / U_aa on the
// diagonal), 5 d + d^2 + (s-6) d + a (upper slots)
template <class T>
__global__ void repack_kernel(int d, int count, const long long* __restrict__ cell_off, const int* __restrict__ perm,
                              const double* __restrict__ off, const double* __restrict__ diag, T* __restrict__ F) {
  const long long total = cell_off[count];
  const int Q = 10 * d + d * d;
  for (long long C = blockIdx.x * (long long)blockDim.x + threadIdx.x; C < total;
       C += (long long)gridDim.x * blockDim.x) {
    const int sd = find_subdomain(cell_off, count, C);
    const long long base = cell_off[sd];
    const long long nc = cell_off[sd + 1] - base;
    T* Fs = F + base * Q + perm[C];
    for (int s = 0; s < 11; ++s) {
      if (s == 5) continue;
      for (int a = 0; a < d; ++a) {
        const int q = s < 5 ? s * d + a : 5 * d + d * d + (s - 6) * d + a;
        Fs[q * nc] = to_factor<T>(off[(C * 11 + s) * d + a]);
      }
    }
    // U's diagonal entries are stored as their reciprocals (computed in FP64), so the backward sweeps
    // multiply instead of dividing on their critical path
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        const double v = diag[(C * d + a) * d + b];
        Fs[(5 * d + a * d + b) * nc] = to_factor<T>(a == b ? 1.0 / v : v);
      }
  }
}

// Per-cell operand blocks of the staged d = 2 sweeps (packed position order, 16-byte multiples so a
// thread stages its cell's block with 16-byte copies).  Forward: the 5 d lower off-diagonal slots
// (slot s, component a at s d + a), then L's strictly lower diagonal-block entry (1, 0), then the packed
// (i, j, k).  Backward: the 5 d upper slots, then U's diagonal block 1 / (0,0), (0,1), 1 / (1,1), the packed
// (i, j, k) and the scatter target (grid cell of an owned cell, else -1).
template <class T>
struct alignas(16) FwdBlk {
  T f[11];
  int ijk;
};
template <class T>
struct alignas(16) BwdBlk {
  T f[13];
  int ijk;
  long long go;
};
static_assert(sizeof(FwdBlk<float>) == 48 && sizeof(BwdBlk<float>) == 64, "block layout");
static_assert(sizeof(FwdBlk<double>) == 96 && sizeof(BwdBlk<double>) == 128, "block layout");
static_assert(sizeof(FwdBlk<__nv_bfloat16>) == 32 && sizeof(BwdBlk<__nv_bfloat16>) == 48, "block layout");

template <class T>
__global__ void stage_pack_kernel(int count, const long long* __restrict__ cell_off, const T* __restrict__ F,
                                  const int* __restrict__ ijk, const long long* __restrict__ gmap_p,
                                  const unsigned char* __restrict__ owned_p, FwdBlk<T>* __restrict__ bf,
                                  BwdBlk<T>* __restrict__ bb) {
  constexpr int D = 2, Q = 10 * D + D * D, U = 5 * D + D * D;
  const long long total = cell_off[count];
  for (long long C = blockIdx.x * (long long)blockDim.x + threadIdx.x; C < total;
       C += (long long)gridDim.x * blockDim.x) {
    const int sd = find_subdomain(cell_off, count, C);
    const long long base = cell_off[sd], nc = cell_off[sd + 1] - base;
    const T* Fs = F + base * Q + (C - base);
    FwdBlk<T> f{};
    BwdBlk<T> g{};
    for (int q = 0; q < 5 * D; ++q) f.f[q] = Fs[q * nc], g.f[q] = Fs[(U + q) * nc];
    f.f[5 * D] = Fs[(5 * D + 1 * D + 0) * nc];
    g.f[5 * D + 0] = Fs[(5 * D + 0 * D + 0) * nc];
    g.f[5 * D + 1] = Fs[(5 * D + 0 * D + 1) * nc];
    g.f[5 * D + 2] = Fs[(5 * D + 1 * D + 1) * nc];
    f.ijk = g.ijk = ijk[C];
    g.go = owned_p[C] ? gmap_p[C] : -1;
    bf[C] = f;
    bb[C] = g;
  }
}

constexpr int DENSE_THREADS = 384;  // CTA size bound of the generic sweeps (170 registers per thread)

static size_t table_bytes(int levels, int ny) { return (size_t)(levels + 1 + levels * ny) * sizeof(int); }

// prec: 0 FP64 factors and sweeps, 1 FP32, 2 FP32 sweeps reading BF16 factors
fv_status prepare_sweeps(fv_system* s, int prec) {
  Subdomains& S = s->subs;
  const int d = S.d, Q = 10 * d + d * d;
  const int fp32 = prec != 0;
  const size_t es = fp32 ? sizeof(float) : sizeof(double);  // the sweep vectors and rings
  S.fp32 = fp32;
  S.bf16 = prec == 2;
  S.F = S.bf16 ? (void*)dalloc<__nv_bfloat16>(s, (size_t)S.total_cells * Q)
        : fp32 ? (void*)dalloc<float>(s, (size_t)S.total_cells * Q)
               : (void*)dalloc<double>(s, (size_t)S.total_cells * Q);
  S.loc = fp32 ? (void*)dalloc<float>(s, (size_t)S.total_cells * d) : (void*)dalloc<double>(s, (size_t)S.total_cells * d);
  if (!S.F || !S.loc) return set_error("fv_assemble_system: allocation of sweep data failed"), FV_ENOMEM;
  const int blocks = (int)std::min<long long>((S.total_cells + 255) / 256, 152LL * 32);
  if (S.bf16)
    repack_kernel<__nv_bfloat16><<<blocks, 256>>>(d, S.count, S.cell_off, S.perm, S.off, S.diag, (__nv_bfloat16*)S.F);
  else if (fp32)
    repack_kernel<float><<<blocks, 256>>>(d, S.count, S.cell_off, S.perm, S.off, S.diag, (float*)S.F);
  else
    repack_kernel<double><<<blocks, 256>>>(d, S.count, S.cell_off, S.perm, S.off, S.diag, (double*)S.F);
  FV_CUDA(cudaGetLastError());
  FV_CUDA(cudaDeviceSynchronize());
  release(s, S.off), release(s, S.diag), release(s, S.perm);
  S.off = S.diag = nullptr;
  S.perm = nullptr;
  // the widest box's level table and wavefront step; the 4-plane ring in shared memory when it fits
  std::vector<int> dims(3 * S.count);
  FV_CUDA(cudaMemcpy(dims.data(), S.dims, dims.size() * sizeof(int), cudaMemcpyDeviceToHost));
  size_t tab = 0;
  int widest = 1;  // most cells in one wavefront step of any box
  for (int sd = 0; sd < S.count; ++sd) {
    const int nx = dims[3 * sd], ny = dims[3 * sd + 1], nz = dims[3 * sd + 2];
    const int levels = (nx - 1) + 2 * (ny - 1) + (nz - 1) + 1;
    tab = std::max(tab, table_bytes(levels, ny));
    for (int L = 0; L < levels; ++L) {
      int cnt = 0;
      for (int j = 0; j < ny; ++j) cnt += std::max(0, std::min(nx - 1, L - 2 * j) - std::max(0, L - 2 * j - (nz - 1)) + 1);
      widest = std::max(widest, cnt);
    }
  }
  S.dense_threads = std::min(DENSE_THREADS, (widest + 31) / 32 * 32);
  S.dense_single = widest <= S.dense_threads;  // one cell per thread and step: the pipelined sweeps
  // (i, j, k) of every packed position (wavefront order: step, then j, then i), so the pipelined
  // sweeps load a cell's coordinates with its factors instead of searching the step's rows
  {
    std::vector<long long> off(S.count + 1);
    FV_CUDA(cudaMemcpy(off.data(), S.cell_off, off.size() * sizeof(long long), cudaMemcpyDeviceToHost));
    std::vector<int> ijk(S.total_cells);
    for (int sd = 0; sd < S.count; ++sd) {
      const int nx = dims[3 * sd], ny = dims[3 * sd + 1], nz = dims[3 * sd + 2];
      if (nx >= 1024 || ny >= 1024 || nz >= 1024) return set_error("fv_assemble_system: subdomain too large"), FV_EINVAL;
      long long pos = off[sd];
      for (int L = 0; L < nx - 1 + 2 * (ny - 1) + nz; ++L)
        for (int j = 0; j < ny; ++j)
          for (int i = std::max(0, L - 2 * j - (nz - 1)); i <= std::min(nx - 1, L - 2 * j); ++i)
            ijk[pos++] = i | j << 10 | (L - i - 2 * j) << 20;
    }
    S.ijk = dalloc<int>(s, S.total_cells);
    if (!S.ijk) return set_error("fv_assemble_system: allocation of the sweep cell table failed"), FV_ENOMEM;
    FV_CUDA(cudaMemcpy(S.ijk, ijk.data(), ijk.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  const size_t ring = 4 * (size_t)S.max_cols * d * es;
  const size_t ring_al = (ring + 15) / 16 * 16;
  S.ring_in_smem = ring_al + tab <= 200 * 1024;
  S.smem = (S.ring_in_smem ? ring_al : 0) + tab;
  if (!S.ring_in_smem) {
    S.ring = fp32 ? (void*)dalloc<float>(s, (size_t)S.count * 4 * S.max_cols * d)
                  : (void*)dalloc<double>(s, (size_t)S.count * 4 * S.max_cols * d);
    if (!S.ring) return set_error("fv_assemble_system: allocation of the sweep ring failed"), FV_ENOMEM;
  }
  // d = 2 boxes whose steps fit the CTA: the shared-memory staged sweeps, 8, 6 or 4 steps deep when
  // the stage ring fits beside the 4-plane ring and the tables (per thread and slot: the forward's block,
  // d right-hand side values and an 8-byte cell map entry, or the backward's block and d values)
  S.stage = 0;
  if (d == 2 && S.dense_single && S.ring_in_smem) {
    const size_t fwd = (S.bf16 ? sizeof(FwdBlk<__nv_bfloat16>) : fp32 ? sizeof(FwdBlk<float>) : sizeof(FwdBlk<double>)) +
                       d * es + 8;
    const size_t bwd = (S.bf16 ? sizeof(BwdBlk<__nv_bfloat16>) : fp32 ? sizeof(BwdBlk<float>) : sizeof(BwdBlk<double>)) +
                       d * es;
    const size_t per = (size_t)S.dense_threads * std::max(fwd, bwd);
    int max_nx = 0;
    for (int sd = 0; sd < S.count; ++sd) max_nx = std::max(max_nx, dims[3 * sd]);
    S.stage_pad = (max_nx + 1) * d;  // the ring's zero padding on each side (elements)
    const size_t sring = ((4 * (size_t)S.max_cols * d + 2 * S.stage_pad) * es + 15) / 16 * 16;
    const size_t off = (sring + tab + 15) / 16 * 16;
    // at most 200 KB a CTA: a 6-deep ring of 221 KB on the 36 x 36 x 20 fine PPBE boxes ran the forward sweep
    // 29 % slower than the 4-deep one (too little L1 left beside it)
    for (int sg : {8, 6, 4})
      if (off + sg * per <= 200 * 1024) {
        S.stage = sg, S.stage_off = off, S.stage_smem = off + sg * per;
        break;
      }
    if (S.stage) {
      if (S.bf16) {
        using B = __nv_bfloat16;
        S.blk_f = dalloc<FwdBlk<B>>(s, S.total_cells), S.blk_b = dalloc<BwdBlk<B>>(s, S.total_cells);
        if (S.blk_f && S.blk_b)
          stage_pack_kernel<B><<<blocks, 256>>>(S.count, S.cell_off, (const B*)S.F, S.ijk, S.gmap_p, S.owned_p,
                                                (FwdBlk<B>*)S.blk_f, (BwdBlk<B>*)S.blk_b);
      } else if (fp32) {
        S.blk_f = dalloc<FwdBlk<float>>(s, S.total_cells), S.blk_b = dalloc<BwdBlk<float>>(s, S.total_cells);
        if (S.blk_f && S.blk_b)
          stage_pack_kernel<float><<<blocks, 256>>>(S.count, S.cell_off, (const float*)S.F, S.ijk, S.gmap_p,
                                                    S.owned_p, (FwdBlk<float>*)S.blk_f, (BwdBlk<float>*)S.blk_b);
      } else {
        S.blk_f = dalloc<FwdBlk<double>>(s, S.total_cells), S.blk_b = dalloc<BwdBlk<double>>(s, S.total_cells);
        if (S.blk_f && S.blk_b)
          stage_pack_kernel<double><<<blocks, 256>>>(S.count, S.cell_off, (const double*)S.F, S.ijk, S.gmap_p,
                                                     S.owned_p, (FwdBlk<double>*)S.blk_f, (BwdBlk<double>*)S.blk_b);
      }
      if (!S.blk_f || !S.blk_b) return set_error("fv_assemble_system: allocation of the sweep blocks failed"), FV_ENOMEM;
      FV_CUDA(cudaGetLastError());
      FV_CUDA(cudaDeviceSynchronize());
    }
  }
  return FV_OK;
}

// ------------------------------------------------------------------ RAS apply
// Wavefront sweeps: step L updates the box cells with i + 2j + k = L.  A cell's in-plane
// neighbours and its own column's previous cell are read from a ring of 4 planes indexed by
// k mod 4 (a neighbour of level L-1..L-3 is never overwritten before it is read).
struct SweepBox {
  int nx, ny, nz, levels, ncols;
  long long base, nc;
};

__device__ __forceinline__ SweepBox sweep_box(const long long* cell_off, const int* dims, int sd) {
  SweepBox b;
  b.nx = dims[3 * sd], b.ny = dims[3 * sd + 1], b.nz = dims[3 * sd + 2];
  b.levels = (b.nx - 1) + 2 * (b.ny - 1) + (b.nz - 1) + 1;
  b.ncols = b.nx * b.ny;
  b.base = cell_off[sd];
  b.nc = cell_off[sd + 1] - b.base;
  return b;
}

// level start offsets and per-(level, row) offsets of the wavefront order (rowoff == nullptr: levels only)
__device__ __forceinline__ void build_tables(const SweepBox& b, int* lvl, int* rowoff) {
  for (int L = threadIdx.x; L < b.levels; L += blockDim.x) {
    int cnt = 0;
    for (int j = 0; j < b.ny; ++j) {
      if (rowoff) rowoff[L * b.ny + j] = cnt;
      const int lo = max(0, L - 2 * j - (b.nz - 1)), hi = min(b.nx - 1, L - 2 * j);
      if (hi >= lo) cnt += hi - lo + 1;
    }
    lvl[L + 1] = cnt;
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // prefix sum of the step sizes by warp 0, each lane over a contiguous chunk
    const int lane = threadIdx.x, per = (b.levels + 31) / 32;
    const int lo = min(b.levels, lane * per), hi = min(b.levels, lo + per);
    int sum = 0;
    for (int L = lo; L < hi; ++L) sum += lvl[L + 1];
    int inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    int run = inc - sum;
    for (int L = lo; L < hi; ++L) lvl[L + 1] = run += lvl[L + 1];
    if (lane == 0) lvl[0] = 0;
  }
  __syncthreads();
}

// Generic sweeps (d = 7, and d = 2 boxes too wide for the column-prefetching kernels below):
// at wavefront step L the thread with local index t takes the t-th cell of the level in
// wavefront order (row j by binary search in the level's row offsets), so every active
// lane does work; at most DENSE_THREADS threads leave each thread enough registers to
// keep all of a cell's factor loads in flight at once.  The forward sweep gathers
// R_i^delta r itself; the backward sweep scatters the owned cells, (R_i^0)^T.
__device__ __forceinline__ void level_cell(const SweepBox& b, const int* rowoff, int L, int t, int& i, int& j,
                                           int& k) {
  const int* ro = rowoff + L * b.ny;
  int lo = 0, hi = b.ny - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ro[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  j = lo;
  i = t - ro[j] + max(0, L - 2 * j - (b.nz - 1));
  k = L - i - 2 * j;
}

template <class T, int D, class V, class FT = T>
__global__ void __launch_bounds__(DENSE_THREADS, 1) ras_fwd_kernel(const long long* __restrict__ cell_off,
                                                                 const int* __restrict__ dims, const int* __restrict__ lpt,
                                                                 const FT* __restrict__ F, T* __restrict__ loc, T* ring_g,
                                                                 int ring_in_smem, int max_cols, long long N,
                                                                 const long long* __restrict__ gmap_p,
                                                                 const V* __restrict__ r) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int sd = lpt[blockIdx.x];
  const SweepBox b = sweep_box(cell_off, dims, sd);
  const size_t ring_bytes = ring_in_smem ? ((4 * (size_t)max_cols * D * sizeof(T) + 15) / 16 * 16) : 0;
  T* ring = ring_in_smem ? (T*)smem : ring_g + (size_t)blockIdx.x * 4 * max_cols * D;
  int* lvl = (int*)(smem + ring_bytes);
  int* rowoff = lvl + b.levels + 1;
  build_tables(b, lvl, rowoff);
  constexpr int Q = 10 * D + D * D;
  const FT* Fb = F + b.base * Q;
  T* Lb = loc + b.base * D;
  const long long* gm = gmap_p + b.base;
  const long long nc = b.nc;
  // the cell map entry of each thread's first cell of the next step is loaded before the
  // barrier, so a step issues its right-hand-side and factor loads together
  long long gnext = threadIdx.x < lvl[1] ? gm[threadIdx.x] : -1;
  for (int L = 0; L < b.levels; ++L) {
    const int cnt = lvl[L + 1] - lvl[L];
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      int i, j, k;
      level_cell(b, rowoff, L, t, i, j, k);
      const int col = j * b.nx + i;
      const long long pos = lvl[L] + t;
      const int pk = k & 3;
      T* rp = ring + (size_t)(pk * b.ncols) * D;
      const T* r0 = ring + (size_t)(((k - 1) & 3) * b.ncols + col) * D;
      const long long g = t == threadIdx.x ? gnext : gm[pos];
      T y[D];
#pragma unroll
      for (int a = 0; a < D; ++a) y[a] = g >= 0 ? (T)r[a * N + g] : T(0);
      if constexpr (sizeof(T) == 4 || D < 7) {
        // every factor slot exists (zero where the neighbour is outside the box): load them all
        // unconditionally so they are in flight together; only the neighbour reads are guarded
        T fl[5 * D], fd[D * D];
#pragma unroll
        for (int q = 0; q < 5 * D; ++q) fl[q] = fcvt(Fb[q * nc + pos]);
#pragma unroll
        for (int a = 1; a < D; ++a)
#pragma unroll
          for (int c = 0; c < a; ++c) fd[a * D + c] = fcvt(Fb[(5 * D + a * D + c) * nc + pos]);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          if (k > 0) y[a] -= fl[0 * D + a] * r0[a];
          if (i > 0 && j > 0) y[a] -= fl[1 * D + a] * rp[(col - b.nx - 1) * D + a];
          if (j > 0) y[a] -= fl[2 * D + a] * rp[(col - b.nx) * D + a];
          if (j > 0 && i + 1 < b.nx) y[a] -= fl[3 * D + a] * rp[(col - b.nx + 1) * D + a];
          if (i > 0) y[a] -= fl[4 * D + a] * rp[(col - 1) * D + a];
#pragma unroll
          for (int c = 0; c < a; ++c) y[a] -= fd[a * D + c] * y[c];
        }
      } else {  // FP64 7x7 blocks: too many registers to batch; FP64 arithmetic bounds this path
#pragma unroll
        for (int a = 0; a < D; ++a) {
          if (k > 0) y[a] -= fcvt(Fb[(0 * D + a) * nc + pos]) * r0[a];
          if (i > 0 && j > 0) y[a] -= fcvt(Fb[(1 * D + a) * nc + pos]) * rp[(col - b.nx - 1) * D + a];
          if (j > 0) y[a] -= fcvt(Fb[(2 * D + a) * nc + pos]) * rp[(col - b.nx) * D + a];
          if (j > 0 && i + 1 < b.nx) y[a] -= fcvt(Fb[(3 * D + a) * nc + pos]) * rp[(col - b.nx + 1) * D + a];
          if (i > 0) y[a] -= fcvt(Fb[(4 * D + a) * nc + pos]) * rp[(col - 1) * D + a];
#pragma unroll
          for (int c = 0; c < a; ++c) y[a] -= fcvt(Fb[(5 * D + a * D + c) * nc + pos]) * y[c];
        }
      }
#pragma unroll
      for (int a = 0; a < D; ++a) {
        rp[col * D + a] = y[a];
        Lb[a * nc + pos] = y[a];
      }
    }
    if (L + 1 < b.levels && threadIdx.x < lvl[L + 2] - lvl[L + 1]) gnext = gm[lvl[L + 1] + threadIdx.x];
    __syncthreads();
  }
}

template <class T, int D, class V, class FT = T>
__global__ void __launch_bounds__(DENSE_THREADS, 1) ras_bwd_kernel(const long long* __restrict__ cell_off,
                                                                 const int* __restrict__ dims, const int* __restrict__ lpt,
                                                                 const FT* __restrict__ F, const T* __restrict__ loc,
                                                                 T* ring_g, int ring_in_smem, int max_cols, long long N,
                                                                 const long long* __restrict__ gmap_p,
                                                                 const unsigned char* __restrict__ owned_p,
                                                                 V* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int sd = lpt[blockIdx.x];
  const SweepBox b = sweep_box(cell_off, dims, sd);
  const size_t ring_bytes = ring_in_smem ? ((4 * (size_t)max_cols * D * sizeof(T) + 15) / 16 * 16) : 0;
  T* ring = ring_in_smem ? (T*)smem : ring_g + (size_t)blockIdx.x * 4 * max_cols * D;
  int* lvl = (int*)(smem + ring_bytes);
  int* rowoff = lvl + b.levels + 1;
  build_tables(b, lvl, rowoff);
  constexpr int Q = 10 * D + D * D;
  const FT* Fb = F + b.base * Q;
  const T* Lb = loc + b.base * D;
  const long long* gm = gmap_p + b.base;
  const unsigned char* ow = owned_p + b.base;
  const long long nc = b.nc;
  for (int L = b.levels - 1; L >= 0; --L) {
    const int cnt = lvl[L + 1] - lvl[L];
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      int i, j, k;
      level_cell(b, rowoff, L, t, i, j, k);
      const int col = j * b.nx + i;
      const long long pos = lvl[L] + t;
      T* rp = ring + (size_t)((k & 3) * b.ncols) * D;
      const T* r1 = ring + (size_t)(((k + 1) & 3) * b.ncols + col) * D;
      constexpr int U = 5 * D + D * D;
      T x[D];
#pragma unroll
      for (int a = 0; a < D; ++a) x[a] = Lb[a * nc + pos];
      if constexpr (sizeof(T) == 4 || D < 7) {
        T fu[5 * D], fd[D * D];
#pragma unroll
        for (int q = 0; q < 5 * D; ++q) fu[q] = fcvt(Fb[(U + q) * nc + pos]);
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int c = a; c < D; ++c) fd[a * D + c] = fcvt(Fb[(5 * D + a * D + c) * nc + pos]);
#pragma unroll
        for (int a = D - 1; a >= 0; --a) {
#pragma unroll
          for (int c = a + 1; c < D; ++c) x[a] -= fd[a * D + c] * x[c];
          if (i + 1 < b.nx) x[a] -= fu[0 * D + a] * rp[(col + 1) * D + a];
          if (i > 0 && j + 1 < b.ny) x[a] -= fu[1 * D + a] * rp[(col + b.nx - 1) * D + a];
          if (j + 1 < b.ny) x[a] -= fu[2 * D + a] * rp[(col + b.nx) * D + a];
          if (i + 1 < b.nx && j + 1 < b.ny) x[a] -= fu[3 * D + a] * rp[(col + b.nx + 1) * D + a];
          if (k + 1 < b.nz) x[a] -= fu[4 * D + a] * r1[a];
          x[a] *= fd[a * D + a];  // 1 / U_aa
        }
      } else {
#pragma unroll
        for (int a = D - 1; a >= 0; --a) {
#pragma unroll
          for (int c = a + 1; c < D; ++c) x[a] -= fcvt(Fb[(5 * D + a * D + c) * nc + pos]) * x[c];
          if (i + 1 < b.nx) x[a] -= fcvt(Fb[(U + 0 * D + a) * nc + pos]) * rp[(col + 1) * D + a];
          if (i > 0 && j + 1 < b.ny) x[a] -= fcvt(Fb[(U + 1 * D + a) * nc + pos]) * rp[(col + b.nx - 1) * D + a];
          if (j + 1 < b.ny) x[a] -= fcvt(Fb[(U + 2 * D + a) * nc + pos]) * rp[(col + b.nx) * D + a];
          if (i + 1 < b.nx && j + 1 < b.ny)
            x[a] -= fcvt(Fb[(U + 3 * D + a) * nc + pos]) * rp[(col + b.nx + 1) * D + a];
          if (k + 1 < b.nz) x[a] -= fcvt(Fb[(U + 4 * D + a) * nc + pos]) * r1[a];
          x[a] *= fcvt(Fb[(5 * D + a * D + a) * nc + pos]);  // 1 / U_aa
        }
      }
#pragma unroll
      for (int a = 0; a < D; ++a) rp[col * D + a] = x[a];
      if (ow[pos]) {
        const long long g = gm[pos];
#pragma unroll
        for (int a = 0; a < D; ++a) z[a * N + g] = (V)x[a];
      }
    }
    __syncthreads();
  }
}


// Level-mapped sweeps with every thread holding at most one cell a step (the widest step fits the
// CTA): the next step's factors and right-hand side are loaded into registers before the barrier
// (they do not depend on this step's results) and the cell map two steps ahead, so a step's
// critical path is the barrier, shared-memory ring reads and arithmetic.
template <class T, int D, class V, class FT = T>
__global__ void __launch_bounds__(DENSE_THREADS, 1) ras_fwd_pipe_kernel(const long long* __restrict__ cell_off,
                                                                      const int* __restrict__ dims,
                                                                      const int* __restrict__ lpt,
                                                                      const FT* __restrict__ F, T* __restrict__ loc,
                                                                      T* ring_g, int ring_in_smem, int max_cols,
                                                                      long long N, const long long* __restrict__ gmap_p,
                                                                      const int* __restrict__ ijk,
                                                                      const V* __restrict__ r) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int sd = lpt[blockIdx.x];
  const SweepBox b = sweep_box(cell_off, dims, sd);
  const size_t ring_bytes = ring_in_smem ? ((4 * (size_t)max_cols * D * sizeof(T) + 15) / 16 * 16) : 0;
  T* ring = ring_in_smem ? (T*)smem : ring_g + (size_t)blockIdx.x * 4 * max_cols * D;
  int* lvl = (int*)(smem + ring_bytes);
  build_tables(b, lvl, nullptr);
  constexpr int Q = 10 * D + D * D;
  const FT* Fb = F + b.base * Q;
  T* Lb = loc + b.base * D;
  const long long* gm = gmap_p + b.base;
  const long long nc = b.nc;
  const int t = threadIdx.x;
  auto cnt_of = [&](int L) { return L < b.levels ? lvl[L + 1] - lvl[L] : 0; };
  long long gn = t < cnt_of(0) ? gm[t] : -1;  // cell map entry of the next fetch
  T y0[D], fl[5 * D], fd[D * D];
  int ci = 0, cj = 0, ck = 0;
  long long cp = -1;
  const int* cells = ijk + b.base;
  auto fetch = [&](int L) {
    cp = -1;
    if (t >= cnt_of(L)) return;
    cp = lvl[L] + t;
    const int c = cells[cp];
    ci = c & 1023, cj = (c >> 10) & 1023, ck = c >> 20;
    const long long g = gn;
#pragma unroll
    for (int a = 0; a < D; ++a) y0[a] = g >= 0 ? (T)r[a * N + g] : T(0);
#pragma unroll
    for (int q = 0; q < 5 * D; ++q) fl[q] = fcvt(Fb[q * nc + cp]);
#pragma unroll
    for (int a = 1; a < D; ++a)
#pragma unroll
      for (int c = 0; c < a; ++c) fd[a * D + c] = fcvt(Fb[(5 * D + a * D + c) * nc + cp]);
  };
  fetch(0);
  gn = t < cnt_of(1) ? gm[lvl[1] + t] : -1;
  for (int L = 0; L < b.levels; ++L) {
    if (cp >= 0) {
      const int i = ci, j = cj, k = ck, col = j * b.nx + i;
      T* rp = ring + (size_t)((k & 3) * b.ncols) * D;
      const T* r0 = ring + (size_t)(((k - 1) & 3) * b.ncols + col) * D;
      T y[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        y[a] = y0[a];
        if (k > 0) y[a] -= fl[0 * D + a] * r0[a];
        if (i > 0 && j > 0) y[a] -= fl[1 * D + a] * rp[(col - b.nx - 1) * D + a];
        if (j > 0) y[a] -= fl[2 * D + a] * rp[(col - b.nx) * D + a];
        if (j > 0 && i + 1 < b.nx) y[a] -= fl[3 * D + a] * rp[(col - b.nx + 1) * D + a];
        if (i > 0) y[a] -= fl[4 * D + a] * rp[(col - 1) * D + a];
#pragma unroll
        for (int c = 0; c < a; ++c) y[a] -= fd[a * D + c] * y[c];
      }
#pragma unroll
      for (int a = 0; a < D; ++a) {
        rp[col * D + a] = y[a];
        Lb[a * nc + cp] = y[a];
      }
    }
    fetch(L + 1);
    if (L + 2 < b.levels) gn = t < cnt_of(L + 2) ? gm[lvl[L + 2] + t] : -1;
    __syncthreads();
  }
}

template <class T, int D, class V, class FT = T>
__global__ void __launch_bounds__(DENSE_THREADS, 1) ras_bwd_pipe_kernel(const long long* __restrict__ cell_off,
                                                                      const int* __restrict__ dims,
                                                                      const int* __restrict__ lpt,
                                                                      const FT* __restrict__ F, const T* __restrict__ loc,
                                                                      T* ring_g, int ring_in_smem, int max_cols,
                                                                      long long N, const long long* __restrict__ gmap_p,
                                                                      const unsigned char* __restrict__ owned_p,
                                                                      const int* __restrict__ ijk,
                                                                      V* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int sd = lpt[blockIdx.x];
  const SweepBox b = sweep_box(cell_off, dims, sd);
  const size_t ring_bytes = ring_in_smem ? ((4 * (size_t)max_cols * D * sizeof(T) + 15) / 16 * 16) : 0;
  T* ring = ring_in_smem ? (T*)smem : ring_g + (size_t)blockIdx.x * 4 * max_cols * D;
  int* lvl = (int*)(smem + ring_bytes);
  build_tables(b, lvl, nullptr);
  constexpr int Q = 10 * D + D * D, U = 5 * D + D * D;
  const int* cells = ijk + b.base;
  const FT* Fb = F + b.base * Q;
  const T* Lb = loc + b.base * D;
  const long long* gm = gmap_p + b.base;
  const unsigned char* ow = owned_p + b.base;
  const long long nc = b.nc;
  const int t = threadIdx.x;
  T x0[D], fu[5 * D], fd[D * D];
  int ci = 0, cj = 0, ck = 0;
  long long cp = -1, go = -1;  // go: cell map entry of an owned cell, else -1
  auto fetch = [&](int L) {
    cp = -1;
    if (L < 0 || t >= lvl[L + 1] - lvl[L]) return;
    cp = lvl[L] + t;
    const int c = cells[cp];
    ci = c & 1023, cj = (c >> 10) & 1023, ck = c >> 20;
#pragma unroll
    for (int a = 0; a < D; ++a) x0[a] = Lb[a * nc + cp];
#pragma unroll
    for (int q = 0; q < 5 * D; ++q) fu[q] = fcvt(Fb[(U + q) * nc + cp]);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int c = a; c < D; ++c) fd[a * D + c] = fcvt(Fb[(5 * D + a * D + c) * nc + cp]);
    const long long g = gm[cp];
    go = ow[cp] ? g : -1;
  };
  fetch(b.levels - 1);
  for (int L = b.levels - 1; L >= 0; --L) {
    if (cp >= 0) {
      const int i = ci, j = cj, k = ck, col = j * b.nx + i;
      T* rp = ring + (size_t)((k & 3) * b.ncols) * D;
      const T* r1 = ring + (size_t)(((k + 1) & 3) * b.ncols + col) * D;
      T x[D];
#pragma unroll
      for (int a = 0; a < D; ++a) x[a] = x0[a];
#pragma unroll
      for (int a = D - 1; a >= 0; --a) {
#pragma unroll
        for (int c = a + 1; c < D; ++c) x[a] -= fd[a * D + c] * x[c];
        if (i + 1 < b.nx) x[a] -= fu[0 * D + a] * rp[(col + 1) * D + a];
        if (i > 0 && j + 1 < b.ny) x[a] -= fu[1 * D + a] * rp[(col + b.nx - 1) * D + a];
        if (j + 1 < b.ny) x[a] -= fu[2 * D + a] * rp[(col + b.nx) * D + a];
        if (i + 1 < b.nx && j + 1 < b.ny) x[a] -= fu[3 * D + a] * rp[(col + b.nx + 1) * D + a];
        if (k + 1 < b.nz) x[a] -= fu[4 * D + a] * r1[a];
        x[a] *= fd[a * D + a];  // 1 / U_aa
      }
#pragma unroll
      for (int a = 0; a < D; ++a) rp[col * D + a] = x[a];
      if (go >= 0) {
#pragma unroll
        for (int a = 0; a < D; ++a) z[a * N + go] = (V)x[a];
      }
    }
    fetch(L - 1);
    __syncthreads();
  }
}

// Shared-memory staged sweeps (d = 2 boxes whose widest step fits the CTA): every thread copies its
// own cell's operand block (FwdBlk / BwdBlk) and vector values for the step SG - 1 ahead into a slot
// of an SG-deep ring with cp.async (one commit group a step) and reads them back after waiting for
// that step's group, so SG - 1 steps of load latency overlap the step in progress at no register
// cost, with a few 16-byte copies a cell.  A thread reads only what it copied itself: the wait orders
// it, and the step keeps one barrier (for the 4-plane ring).  Chunk c of thread t's block in slot s
// sits at 16-byte element (s * nchunks + c) * blockDim + t (no bank conflicts); the forward result
// is kept per cell, [cell][d], so the backward sweep stages it with one copy.  The ring is zeroed
// at launch and padded by `pad` >= (nx + 1) d elements on each side, so every neighbour is read
// unconditionally: the factor slot of a neighbour outside the box is exactly zero (assembly writes
// zero there and the factorization never updates it), and the ring holds only finite values.
template <int B>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const size_t g = __cvta_generic_to_global(src);
  if constexpr (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(g) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(g), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <class Blk>
union StagedBlk {
  Blk b;
  uint4 u[sizeof(Blk) / 16];
};

template <class T, class V, int SG, class FT = T>
__global__ void __launch_bounds__(DENSE_THREADS, 1) ras_fwd_stage_kernel(const long long* __restrict__ cell_off,
                                                                       const int* __restrict__ dims,
                                                                       const int* __restrict__ lpt,
                                                                       const FwdBlk<FT>* __restrict__ blk,
                                                                       T* __restrict__ loc, int max_cols, int pad,
                                                                       long long N,
                                                                       const long long* __restrict__ gmap_p,
                                                                       const V* __restrict__ r, int stage_off) {
  constexpr int D = 2, NC = sizeof(FwdBlk<FT>) / 16;
  extern __shared__ __align__(16) unsigned char smem[];
  const int sd = lpt[blockIdx.x];
  const SweepBox b = sweep_box(cell_off, dims, sd);
  const int ring_bytes = ((4 * max_cols * D + 2 * pad) * (int)sizeof(T) + 15) / 16 * 16;
  T* ring = (T*)smem + pad;  // the padded 4-plane ring: the staged sweeps run only where it fits
  int* lvl = (int*)(smem + ring_bytes);
  for (int e = threadIdx.x; e < 4 * b.ncols * D + 2 * pad; e += blockDim.x) ((T*)smem)[e] = T(0);
  build_tables(b, lvl, nullptr);  // its barriers also order the zeroing
  const int Tn = blockDim.x, t = threadIdx.x;
  uint4* sB = (uint4*)(smem + stage_off);                 // [SG][NC][Tn] operand blocks
  V* sY = (V*)(sB + (size_t)SG * NC * Tn);                // [SG][D][Tn] gathered right-hand side
  long long* sG = (long long*)(sY + (size_t)SG * D * Tn); // [SG][Tn] cell map entry SG - 1 steps later
  const FwdBlk<FT>* Bb = blk + b.base;
  T* Lb = loc + b.base * D;
  const long long* gm = gmap_p + b.base;
  auto cnt_of = [&](int L) { return L < b.levels ? lvl[L + 1] - lvl[L] : 0; };
  // step g into slot g % SG (gg: this thread's cell map entry in step g), and the cell map entry of
  // step g + SG - 1, which the copies of that step need for the gather
  auto issue = [&](int g, long long gg) {
    const int s = g % SG;
    if (t < cnt_of(g)) {
      const uint4* src = reinterpret_cast<const uint4*>(Bb + lvl[g] + t);
#pragma unroll
      for (int c = 0; c < NC; ++c) cp_async<16>(sB + (s * NC + c) * Tn + t, src + c);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        if (gg >= 0) cp_async<sizeof(V)>(sY + (s * D + a) * Tn + t, r + a * N + gg);
        else sY[(s * D + a) * Tn + t] = V(0);
      }
    }
    const int h = g + SG - 1;
    if (t < cnt_of(h)) cp_async<8>(sG + s * Tn + t, gm + lvl[h] + t);
    cp_commit();
  };
  {  // the first SG - 1 steps' cell map entries, loaded together before any copy is issued
    long long g0[SG - 1];
#pragma unroll
    for (int g = 0; g < SG - 1; ++g) g0[g] = t < cnt_of(g) ? gm[lvl[g] + t] : -1;
#pragma unroll
    for (int g = 0; g < SG - 1; ++g) issue(g, g0[g]);
  }
  for (int L = 0; L < b.levels; ++L) {
    cp_wait<SG - 2>();  // step L's group has landed (the SG - 2 later ones may be in flight)
    const int s = L % SG;
    issue(L + SG - 1, t < cnt_of(L + SG - 1) ? sG[s * Tn + t] : -1);  // into the slot step L - 1 used
    if (t < cnt_of(L)) {
      StagedBlk<FwdBlk<FT>> q;
#pragma unroll
      for (int c = 0; c < NC; ++c) q.u[c] = sB[(s * NC + c) * Tn + t];
      const FT* f = q.b.f;
      const int i = q.b.ijk & 1023, j = (q.b.ijk >> 10) & 1023, k = q.b.ijk >> 20, col = j * b.nx + i;
      T* rp = ring + ((k & 3) * b.ncols) * D;
      const T* r0 = ring + (((k - 1) & 3) * b.ncols + col) * D;
      T y[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        y[a] = (T)sY[(s * D + a) * Tn + t];
        y[a] -= fcvt(f[0 * D + a]) * r0[a];
        y[a] -= fcvt(f[1 * D + a]) * rp[(col - b.nx - 1) * D + a];
        y[a] -= fcvt(f[2 * D + a]) * rp[(col - b.nx) * D + a];
        y[a] -= fcvt(f[3 * D + a]) * rp[(col - b.nx + 1) * D + a];
        y[a] -= fcvt(f[4 * D + a]) * rp[(col - 1) * D + a];
      }
      y[1] -= fcvt(f[5 * D]) * y[0];
      const long long cp = lvl[L] + t;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        rp[col * D + a] = y[a];
        Lb[cp * D + a] = y[a];
      }
    }
    __syncthreads();
  }
  cp_wait<0>();
}

// Backward sweep of the staged pair: steps in reverse; each thread's block and its cell's forward
// result are copied SG - 1 steps ahead.  Nothing a copy needs depends on a staged value, so a step's
// copies are issued before it waits.
template <class T, class V, int SG, class FT = T>
__global__ void __launch_bounds__(DENSE_THREADS, 1) ras_bwd_stage_kernel(const long long* __restrict__ cell_off,
                                                                       const int* __restrict__ dims,
                                                                       const int* __restrict__ lpt,
                                                                       const BwdBlk<FT>* __restrict__ blk,
                                                                       const T* __restrict__ loc, int max_cols,
                                                                       int pad, long long N,
                                                                       V* __restrict__ z, int stage_off) {
  constexpr int D = 2, NC = sizeof(BwdBlk<FT>) / 16;
  extern __shared__ __align__(16) unsigned char smem[];
  const int sd = lpt[blockIdx.x];
  const SweepBox b = sweep_box(cell_off, dims, sd);
  const int ring_bytes = ((4 * max_cols * D + 2 * pad) * (int)sizeof(T) + 15) / 16 * 16;
  T* ring = (T*)smem + pad;  // the padded 4-plane ring: the staged sweeps run only where it fits
  int* lvl = (int*)(smem + ring_bytes);
  for (int e = threadIdx.x; e < 4 * b.ncols * D + 2 * pad; e += blockDim.x) ((T*)smem)[e] = T(0);
  build_tables(b, lvl, nullptr);  // its barriers also order the zeroing
  const int Tn = blockDim.x, t = threadIdx.x;
  uint4* sB = (uint4*)(smem + stage_off);  // [SG][NC][Tn] operand blocks
  T* sX = (T*)(sB + (size_t)SG * NC * Tn); // [SG][Tn][D] forward result
  const BwdBlk<FT>* Bb = blk + b.base;
  const T* Lb = loc + b.base * D;
  auto issue = [&](int n) {  // n-th step of the backward order (level levels - 1 - n) into slot n % SG
    const int L = b.levels - 1 - n, s = n % SG;
    if (L >= 0 && t < lvl[L + 1] - lvl[L]) {
      const long long cp = lvl[L] + t;
      const uint4* src = reinterpret_cast<const uint4*>(Bb + cp);
#pragma unroll
      for (int c = 0; c < NC; ++c) cp_async<16>(sB + (s * NC + c) * Tn + t, src + c);
      cp_async<D * sizeof(T)>(sX + ((size_t)s * Tn + t) * D, Lb + cp * D);
    }
    cp_commit();
  };
  for (int n = 0; n < SG - 1; ++n) issue(n);
  for (int n = 0; n < b.levels; ++n) {
    issue(n + SG - 1);  // into the slot step n - 1 used
    cp_wait<SG - 1>();  // step n's group has landed
    const int L = b.levels - 1 - n, s = n % SG;
    if (t < lvl[L + 1] - lvl[L]) {
      StagedBlk<BwdBlk<FT>> q;
#pragma unroll
      for (int c = 0; c < NC; ++c) q.u[c] = sB[(s * NC + c) * Tn + t];
      const FT* f = q.b.f;
      const int i = q.b.ijk & 1023, j = (q.b.ijk >> 10) & 1023, k = q.b.ijk >> 20, col = j * b.nx + i;
      T* rp = ring + ((k & 3) * b.ncols) * D;
      const T* r1 = ring + (((k + 1) & 3) * b.ncols + col) * D;
      T x[D];
#pragma unroll
      for (int a = 0; a < D; ++a) x[a] = sX[((size_t)s * Tn + t) * D + a];
      // U's diagonal block at f[5 d + 0, 1, 2] = 1 / (0,0), (0,1), 1 / (1,1)
#pragma unroll
      for (int a = D - 1; a >= 0; --a) {
        if (a == 0) x[0] -= fcvt(f[5 * D + 1]) * x[1];
        x[a] -= fcvt(f[0 * D + a]) * rp[(col + 1) * D + a];
        x[a] -= fcvt(f[1 * D + a]) * rp[(col + b.nx - 1) * D + a];
        x[a] -= fcvt(f[2 * D + a]) * rp[(col + b.nx) * D + a];
        x[a] -= fcvt(f[3 * D + a]) * rp[(col + b.nx + 1) * D + a];
        x[a] -= fcvt(f[4 * D + a]) * r1[a];
        x[a] *= fcvt(f[a == 0 ? 5 * D : 5 * D + 2]);  // 1 / U_aa
      }
#pragma unroll
      for (int a = 0; a < D; ++a) rp[col * D + a] = x[a];
      if (q.b.go >= 0) {
#pragma unroll
        for (int a = 0; a < D; ++a) z[a * N + q.b.go] = (V)x[a];
      }
    }
    __syncthreads();
  }
  cp_wait<0>();
}

template <class T, int D, class V, class FT = T>
static fv_status ras_apply_t(const fv_system* s, const V* r, V* z, cudaStream_t st) {
  const Subdomains& S = s->subs;
  const long long N = s->grid->geo.N;
  T* loc = (T*)S.loc;
  const int pf = (s->kind == FV_VTBE ? FV_K_RAS_FWD_VTBE : FV_K_RAS_FWD_PPBE) + FV_K_COARSE * s->level +
                 FV_K_FP32 * S.fp32;
  const int pb = (s->kind == FV_VTBE ? FV_K_RAS_BWD_VTBE : FV_K_RAS_BWD_PPBE) + FV_K_COARSE * s->level +
                 FV_K_FP32 * S.fp32;
  {
    ProfScope ps(pf, st);
    {
      bool piped = false;
      if constexpr (D == 2) {
        const int so = (int)S.stage_off;
        const FwdBlk<FT>* bf = (const FwdBlk<FT>*)S.blk_f;
        if (S.stage == 8)
          ras_fwd_stage_kernel<T, V, 8, FT><<<S.count, S.dense_threads, S.stage_smem, st>>>(
              S.cell_off, S.dims, S.lpt, bf, loc, S.max_cols, S.stage_pad, N, S.gmap_p, r, so);
        else if (S.stage == 6)
          ras_fwd_stage_kernel<T, V, 6, FT><<<S.count, S.dense_threads, S.stage_smem, st>>>(
              S.cell_off, S.dims, S.lpt, bf, loc, S.max_cols, S.stage_pad, N, S.gmap_p, r, so);
        else if (S.stage == 4)
          ras_fwd_stage_kernel<T, V, 4, FT><<<S.count, S.dense_threads, S.stage_smem, st>>>(
              S.cell_off, S.dims, S.lpt, bf, loc, S.max_cols, S.stage_pad, N, S.gmap_p, r, so);
        piped = S.stage != 0;
      }
      if constexpr (sizeof(T) == 4 || D < 7) {
        if (S.dense_single && !piped) {
          ras_fwd_pipe_kernel<T, D, V, FT><<<S.count, S.dense_threads, S.smem, st>>>(
              S.cell_off, S.dims, S.lpt, (const FT*)S.F, loc, (T*)S.ring, S.ring_in_smem, S.max_cols, N, S.gmap_p,
              S.ijk, r);
          piped = true;
        }
      }
      if (!piped)
        ras_fwd_kernel<T, D, V, FT><<<S.count, S.dense_threads, S.smem, st>>>(
            S.cell_off, S.dims, S.lpt, (const FT*)S.F, loc, (T*)S.ring, S.ring_in_smem, S.max_cols, N, S.gmap_p, r);
    }
  }
  FV_CUDA(cudaGetLastError());
  {
    ProfScope ps(pb, st);
    {
      bool piped = false;
      if constexpr (D == 2) {
        const int so = (int)S.stage_off;
        const BwdBlk<FT>* bb = (const BwdBlk<FT>*)S.blk_b;
        if (S.stage == 8)
          ras_bwd_stage_kernel<T, V, 8, FT><<<S.count, S.dense_threads, S.stage_smem, st>>>(
              S.cell_off, S.dims, S.lpt, bb, loc, S.max_cols, S.stage_pad, N, z, so);
        else if (S.stage == 6)
          ras_bwd_stage_kernel<T, V, 6, FT><<<S.count, S.dense_threads, S.stage_smem, st>>>(
              S.cell_off, S.dims, S.lpt, bb, loc, S.max_cols, S.stage_pad, N, z, so);
        else if (S.stage == 4)
          ras_bwd_stage_kernel<T, V, 4, FT><<<S.count, S.dense_threads, S.stage_smem, st>>>(
              S.cell_off, S.dims, S.lpt, bb, loc, S.max_cols, S.stage_pad, N, z, so);
        piped = S.stage != 0;
      }
      if constexpr (sizeof(T) == 4 || D < 7) {
        if (S.dense_single && !piped) {
          ras_bwd_pipe_kernel<T, D, V, FT><<<S.count, S.dense_threads, S.smem, st>>>(
              S.cell_off, S.dims, S.lpt, (const FT*)S.F, loc, (T*)S.ring, S.ring_in_smem, S.max_cols, N, S.gmap_p,
              S.owned_p, S.ijk, z);
          piped = true;
        }
      }
      if (!piped)
        ras_bwd_kernel<T, D, V, FT><<<S.count, S.dense_threads, S.smem, st>>>(
            S.cell_off, S.dims, S.lpt, (const FT*)S.F, loc, (T*)S.ring, S.ring_in_smem, S.max_cols, N, S.gmap_p,
            S.owned_p, z);
    }
  }
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

// The limit is a property of the kernel function, shared by every system that launches it:
// raise it to the device's opt-in maximum (never lower it for a smaller system).
template <class T, int D, class FT = T>
static fv_status set_smem_attr(int limit) {
  FV_CUDA(cudaFuncSetAttribute(ras_fwd_kernel<T, D, T, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
  FV_CUDA(cudaFuncSetAttribute(ras_bwd_kernel<T, D, T, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
  if constexpr (sizeof(T) == 4 || D < 7) {
    FV_CUDA(cudaFuncSetAttribute(ras_fwd_pipe_kernel<T, D, T, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    FV_CUDA(cudaFuncSetAttribute(ras_bwd_pipe_kernel<T, D, T, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
  }
  if constexpr (D == 2) {
    FV_CUDA(cudaFuncSetAttribute(ras_fwd_stage_kernel<T, T, 8, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    FV_CUDA(cudaFuncSetAttribute(ras_bwd_stage_kernel<T, T, 8, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    FV_CUDA(cudaFuncSetAttribute(ras_fwd_stage_kernel<T, T, 6, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    FV_CUDA(cudaFuncSetAttribute(ras_bwd_stage_kernel<T, T, 6, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    FV_CUDA(cudaFuncSetAttribute(ras_fwd_stage_kernel<T, T, 4, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    FV_CUDA(cudaFuncSetAttribute(ras_bwd_stage_kernel<T, T, 4, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
  }
  return FV_OK;
}

fv_status sweeps_smem_attr(const fv_system* s) {
  const Subdomains& S = s->subs;
  int dev = 0, limit = 0;
  FV_CUDA(cudaGetDevice(&dev));
  FV_CUDA(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (S.smem > (size_t)limit || S.stage_smem > (size_t)limit)
    return set_error("fv_assemble_system: sweep tables exceed shared memory"), FV_EINVAL;
  if (S.bf16) return S.d == 2 ? set_smem_attr<float, 2, __nv_bfloat16>(limit) : set_smem_attr<float, 7, __nv_bfloat16>(limit);
  if (S.d == 2) return S.fp32 ? set_smem_attr<float, 2>(limit) : set_smem_attr<double, 2>(limit);
  return S.fp32 ? set_smem_attr<float, 7>(limit) : set_smem_attr<double, 7>(limit);
}

fv_status ras_apply(const fv_system* s, const double* r, double* z, cudaStream_t st) {
  const Subdomains& S = s->subs;
  if (S.fp32) return set_error("ras_apply: FP32 factors need FP32 vectors"), FV_EINVAL;
  if (S.d == 2) return ras_apply_t<double, 2, double>(s, r, z, st);
  return ras_apply_t<double, 7, double>(s, r, z, st);
}

static fv_status ras_apply32(const fv_system* s, const float* r, float* z, cudaStream_t st) {
  const Subdomains& S = s->subs;
  if (!S.fp32) return set_error("ras_apply32: FP64 factors need FP64 vectors"), FV_EINVAL;
  if (S.bf16)
    return S.d == 2 ? ras_apply_t<float, 2, float, __nv_bfloat16>(s, r, z, st)
                    : ras_apply_t<float, 7, float, __nv_bfloat16>(s, r, z, st);
  if (S.d == 2) return ras_apply_t<float, 2, float>(s, r, z, st);
  return ras_apply_t<float, 7, float>(s, r, z, st);
}

// ------------------------------------------------------------------ two levels
// The index type I is 32-bit whenever d N fits (every shell here): the index decomposition then uses
// 32-bit divisions by the grid sizes instead of 64-bit ones.
template <class T, class I>
__global__ void restrict_kernel(int d, int Ns, int Nr, const T* __restrict__ x, T* __restrict__ xc) {
  const I nc = Ns / 2, mc = Nr / 2;
  const I Nc = (I)6 * nc * nc * mc, N = (I)6 * Ns * Ns * Nr;
  for (I e = blockIdx.x * (I)blockDim.x + threadIdx.x; e < (I)d * Nc; e += (I)gridDim.x * blockDim.x) {
    I r = e;
    const I i = r % nc;
    r /= nc;
    const I j = r % nc;
    r /= nc;
    const I k = r % mc;
    r /= mc;
    const I p = r % 6;
    const I a = r / 6;
    const T* xa = x + (long long)a * N;
    T sum = T(0);
    for (int dk = 0; dk < 2; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di)
          sum += xa[((long long)(p * Nr + 2 * k + dk) * Ns + 2 * j + dj) * Ns + 2 * i + di];
    xc[e] = sum * T(0.125);
  }
}

template <class T, class I>
__global__ void prolong_kernel(int d, int Ns, int Nr, const T* __restrict__ xc, T* __restrict__ x) {
  const I nc = Ns / 2, mc = Nr / 2;
  const I N = (I)6 * Ns * Ns * Nr, Nc = (I)6 * nc * nc * mc;
  for (I e = blockIdx.x * (I)blockDim.x + threadIdx.x; e < (I)d * N; e += (I)gridDim.x * blockDim.x) {
    I r = e;
    const I i = r % Ns;
    r /= Ns;
    const I j = r % Ns;
    r /= Ns;
    const I k = r % Nr;
    r /= Nr;
    const I p = r % 6;
    const I a = r / 6;
    x[e] = xc[(long long)a * Nc + ((long long)(p * mc + k / 2) * nc + j / 2) * nc + i / 2];
  }
}

// 32-bit indexing of the transfer kernels: the element count plus one grid stride (at most 152 x 32 x 256)
// stays below 2^31
constexpr long long kIndex32 = (1LL << 31) - (1LL << 24);

static int nblocks(long long n) {
  long long b = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(b, 1), 152LL * 32);
}

template <class T>
static fv_status restrict_t(const fv_grid* g, int d, const T* x, T* xc, cudaStream_t st) {
  ProfScope ps(FV_K_TRANSFER, st);
  if ((long long)d * g->h.N < kIndex32)
    restrict_kernel<T, int><<<nblocks(d * g->h.N / 8), 256, 0, st>>>(d, g->h.Ns, g->h.Nr, x, xc);
  else
    restrict_kernel<T, long long><<<nblocks(d * g->h.N / 8), 256, 0, st>>>(d, g->h.Ns, g->h.Nr, x, xc);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

template <class T>
static fv_status prolong_t(const fv_grid* g, int d, const T* xc, T* x, cudaStream_t st) {
  ProfScope ps(FV_K_TRANSFER, st);
  if ((long long)d * g->h.N < kIndex32)
    prolong_kernel<T, int><<<nblocks(d * g->h.N), 256, 0, st>>>(d, g->h.Ns, g->h.Nr, xc, x);
  else
    prolong_kernel<T, long long><<<nblocks(d * g->h.N), 256, 0, st>>>(d, g->h.Ns, g->h.Nr, xc, x);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

fv_status restrict_mean(const fv_grid* g, int d, const double* x, double* xc, cudaStream_t st) {
  return restrict_t<double>(g, d, x, xc, st);
}

fv_status prolong_inject(const fv_grid* g, int d, const double* xc, double* x, cudaStream_t st) {
  return prolong_t<double>(g, d, xc, x, st);
}

// Mixed precision: M^{-1} r of the FP64 outer solve is an FP32 inner FGMRES of exactly
// inner_maxit iterations (its two-level preconditioner's coarse solve: exactly
// coarse_maxit iterations), driven on the device.  The sequence r32 -> x32 has fixed
// buffers and no host synchronisation: it is captured once into a CUDA graph and
// replayed (kernel timing, when enabled, runs it eagerly instead).
static fv_status inner_sequence(const fv_system* s, cudaStream_t st) {
  return gmres_fixed32(s, s->r32, s->x32, s->pc.inner_maxit, st);
}

static fv_status inner_solve(const fv_system* s, const double* r, double* z, cudaStream_t st) {
  fv_status rc;
  if ((rc = to_fp32(s->n, r, s->r32, st))) return rc;
  if (prof_enabled()) {
    if ((rc = inner_sequence(s, st))) return rc;
  } else {
    fv_system* sm = const_cast<fv_system*>(s);
    if (!sm->inner_warm) {
      // first call: run eagerly so every lazily allocated workspace exists before capture
      if ((rc = inner_sequence(s, st))) return rc;
      sm->inner_warm = 1;
    } else if (!sm->inner_graph) {
      cudaStream_t cs;
      FV_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaGraph_t graph;
      FV_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      rc = inner_sequence(s, cs);
      cudaError_t ce = cudaStreamEndCapture(cs, &graph);
      cudaStreamDestroy(cs);
      if (rc) return rc;
      FV_CUDA(ce);
      ce = cudaGraphInstantiate(&sm->inner_graph, graph, 0);
      cudaGraphDestroy(graph);
      FV_CUDA(ce);
    }
    if (sm->inner_graph) FV_CUDA(cudaGraphLaunch(s->inner_graph, st));
  }
  s->last_inner += s->pc.inner_maxit;
  return to_fp64(s->n, s->x32, z, st);
}

fv_status precond_apply(const fv_system* s, const double* r, double* z, cudaStream_t st) {
  if (s->prec32) return inner_solve(s, r, z, st);
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
    int its = s->pc.coarse_maxit;
    if (s->net && s->learned_on) {  // learned e_c = N(r_c), then learned_its iterations from it
      if ((rc = net_forward64(s->net, s->xc, s->ec, st))) return rc;
      its = s->learned_its;
    }
    if (its > 0) {
      fv_gmres_opts o{s->pc.coarse_restart, its, 0.0, s->pc.coarse_rtol};
      fv_solve_stats cs{};
      rc = gmres(c, s->xc, s->ec, &o, &cs, st, true);
      if (rc && rc != FV_ENOCONV) return rc;
      s->last_inner += cs.iters;
    }
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

// The same preconditioners on FP32 vectors (inner solves of mixed precision)
fv_status precond_apply32(const fv_system* s, const float* r, float* z, cudaStream_t st) {
  if (s->pc.levels < 2) return ras_apply32(s, r, z, st);
  const fv_system* c = s->coarse;
  fv_status rc;
  {
    ProfScope ph(FV_K_PHASE_PC_I, st);
    if ((rc = restrict_t<float>(s->grid, s->d, r, s->xc32, st))) return rc;
    if (s->kind == FV_PPBE && (rc = weighted_mean_remove32(c->grid, s->xc32, st, s->red, s->red + 32 * 304)))
      return rc;
  }
  {
    ProfScope ph(FV_K_PHASE_PC_C, st);
    if (s->net && s->learned_on) {
      // learned e_c = N(r_c), then learned_its iterations on the residual r_c - A_c e_c
      if ((rc = net_forward32(s->net, s->xc32, s->ec32, st))) return rc;
      if (s->learned_its > 0) {
        if ((rc = apply_op32(c, s->ec32, s->tc32, st)) || (rc = axpby32(c->n, 1.0, s->xc32, -1.0, s->tc32, s->tc32, st)) ||
            (rc = gmres_fixed32(c, s->tc32, s->dc32, s->learned_its, st)) ||
            (rc = axpby32(c->n, 1.0, s->ec32, 1.0, s->dc32, s->ec32, st)))
          return rc;
      }
    } else if ((rc = gmres_fixed32(c, s->xc32, s->ec32, s->pc.coarse_maxit, st))) {
      return rc;
    }
  }
  {
    ProfScope ph(FV_K_PHASE_PC_I, st);
    if ((rc = prolong_t<float>(s->grid, s->d, s->ec32, s->w32, st))) return rc;
    if ((rc = apply_op32(s, s->w32, s->t32, st))) return rc;
    if ((rc = axpby32(s->n, 1.0, r, -1.0, s->t32, s->t32, st))) return rc;
  }
  {
    ProfScope ph(FV_K_PHASE_PC_F, st);
    if ((rc = ras_apply32(s, s->t32, z, st))) return rc;
  }
  ProfScope ph(FV_K_PHASE_PC_I, st);
  return axpby32(s->n, 1.0, z, 1.0, s->w32, z, st);
}

// the coarse right-hand side of the two-level preconditioner (restriction and,
// for the Neumann pressure, the volume-weighted mean removal)
fv_status restrict_coarse(const fv_system* s, const double* x, double* xc, cudaStream_t st) {
  fv_status rc = restrict_mean(s->grid, s->d, x, xc, st);
  if (rc) return rc;
  if (s->kind == FV_PPBE) return weighted_mean_remove(s->coarse->grid, xc, st, s->red, s->red + 32 * 304);
  return FV_OK;
}

// switch the learned coarse correction on or off; the captured inner solve of
// mixed precision contains the coarse solve, so it is captured again
void set_learned_active(fv_system* s, int on) {
  if (s->learned_on == on) return;
  s->learned_on = on;
  if (s->inner_graph) cudaGraphExecDestroy(s->inner_graph);
  s->inner_graph = nullptr;
  s->inner_warm = 0;
}

// x <- x + I_c^f N(r_c(b - A x)): the learned initial-guess correction
fv_status learned_guess(const fv_system* s, const double* b, double* x, cudaStream_t st) {
  fv_status rc;
  if ((rc = apply_op(s, x, s->t, st)) || (rc = axpby(s->n, 1.0, b, -1.0, s->t, s->t, st)) ||
      (rc = restrict_coarse(s, s->t, s->xc, st)) || (rc = net_forward64(s->net, s->xc, s->ec, st)) ||
      (rc = prolong_inject(s->grid, s->d, s->ec, s->w, st)))
    return rc;
  return axpby(s->n, 1.0, x, 1.0, s->w, x, st);
}

}  // namespace fv
