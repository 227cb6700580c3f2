// Tiled matrix-free operator apply y = A x for VTBE and PPBE (paper eqn:divdiscretization with the
// operators of eqn:tsvelocity, eqn:tstemperature, eqn:tsmag, eqn:tsp, eqn:tspb).
//
// Per cell and component the Laplacian is (1/V) sum_faces F.  The horizontal faces give a 9-point stencil
// whose weights depend only on (j, i): the angular metric is the same on every panel and level, and h_r is
// folded in.  A face on a panel edge carries the mean of the two panels' one-sided fluxes (reading R3); with
// the panel-edge ghosts expanded into their interpolation sources that flux is a fixed linear combination
// of cell values of the same level on two or three panels, tabulated once per grid (build_edge_table).
// The radial faces give a 3-point stencil r_f^2 sigma h_s^2 / h_r (x_{k+1} - x_k) with the wall ghost rules.
//
// One launch, one CTA per (coupled component group, panel, TJ x 32 tile of (j, i), chunk of levels k).
// Groups: VTBE {u_x, u_y, u_z, Theta} (Coriolis, buoyancy and r . u couple them at a cell) and
// {B_x, B_y, B_z} (the pseudo-vacuum wall rule couples them); PPBE {P}, {P_b}.  The CTA marches k with a
// ring of three (TJ + 2) x 34 planes of its components in shared memory (halo cells across a panel edge are
// the quadratic ghost interpolants), prefetching the plane two levels ahead into registers while it
// computes; each thread owns RJ rows of one column.  Every x value is read from HBM once (plus the planes at
// chunk boundaries) and every y value is written once: the algorithmic 2 d values per cell.
#include <mutex>
#include <type_traits>
#include <vector>

#include "stencil.cuh"

namespace fv {

constexpr int TILE_I = 32;    // tile width in i: one warp per row set
constexpr int TILE_WARPS = 4;
constexpr int EDGE_TERMS = 40;  // bound on the terms of one panel-edge face flux (checked when tabulated)
constexpr int RING = 8;         // planes of the tile ring: levels k - 1 .. k + 3 in use, a power of two

template <class T>
struct TileShape {
  static constexpr int RJ = 4;  // rows per thread
  static constexpr int TJ = TILE_WARPS * RJ;
  static constexpr int PW = TILE_I + 2, PH = TJ + 2, PLANE = PW * PH;
  static constexpr int HALO = 2 * PH + 2 * TILE_I;  // halo cells of one plane
};

template <class R>
struct EdgeTab {
  const int* cnt;
  const int* off;
  const R* w;
};

// ------------------------------------------------------------------ panel-edge face table
// Records the terms of a face flux as (cell offset within a level, weight), ghosts expanded into their
// interpolation sources (cube-corner ghosts: phi(-1,-1) = phi(-1,0) + phi(0,-1) - phi(0,0)).
struct RecordAcc {
  const Geo* G;
  int n;
  int bad;
  int off[EDGE_TERMS];
  double w[EDGE_TERMS];
  __device__ void cell(double c, int p, int, int j, int i, int) {
    const int o = (p * G->Nr * G->Ns + j) * G->Ns + i;
    for (int m = 0; m < n; ++m)
      if (off[m] == o) {
        w[m] += c;
        return;
      }
    if (n == EDGE_TERMS) {
      bad = 1;
      return;
    }
    off[n] = o, w[n] = c, ++n;
  }
  __device__ void interp(double c, int p, int side, int t) {
    const int Ns = G->Ns, id = (p * 4 + side) * Ns + t, q = G->gq[id];
    for (int m = 0; m < 3; ++m) {
      const int src = G->gsrc[3 * id + m];
      cell(c * G->gw[3 * id + m], q, 0, src / Ns, src % Ns, 0);
    }
  }
  __device__ void ghost(double c, int p, int side, int, int t, int) {
    const int Ns = G->Ns;
    if (t >= 0 && t < Ns) {
      interp(c, p, side, t);
    } else {
      const int jin = t < 0 ? 0 : Ns - 1, iin = side == XI_MIN ? 0 : Ns - 1;
      interp(c, p, side, jin);
      interp(c, p, t < 0 ? ETA_MIN : ETA_MAX, iin);
      cell(-c, p, 0, jin, iin, 0);
    }
  }
};

// one thread per panel-edge face f = (p, side, t): cnt[f], then the terms in term-major slots
// (off[m * nf + f], wt[m * nf + f]), so that neighbouring faces read neighbouring slots
__global__ void edge_table_kernel(Geo G, int* __restrict__ cnt, int* __restrict__ off, double* __restrict__ wt,
                                  int* __restrict__ status) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int nf = 24 * G.Ns;
  if (e >= nf) return;
  const int ps = e / G.Ns, t = e % G.Ns;
  RecordAcc acc;
  acc.G = G.self, acc.n = 0, acc.bad = 0;
  edge_flux(*G.self, acc, 1.0, ps / 4, ps % 4, 0, t, 0);
  if (acc.bad) atomicExch(status, 1);
  int n = 0;
  for (int m = 0; m < acc.n; ++m)  // drop terms that cancelled exactly
    if (acc.w[m] != 0.0) off[n * nf + e] = acc.off[m], wt[n * nf + e] = acc.w[m], ++n;
  cnt[e] = n;
}

__global__ void to_float_kernel(const double* __restrict__ a, float* __restrict__ b, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) b[e] = (float)a[e];
}

fv_status build_edge_table(fv_grid* g) {
  const int nf = 24 * g->h.Ns;
  int *cnt = nullptr, *off = nullptr, *status = nullptr;
  double* wt = nullptr;
  float* wtf = nullptr;
  FV_CUDA(cudaMalloc(&cnt, nf * sizeof(int)));
  g->allocs.push_back(cnt);
  FV_CUDA(cudaMalloc(&off, (size_t)nf * EDGE_TERMS * sizeof(int)));
  g->allocs.push_back(off);
  FV_CUDA(cudaMalloc(&wt, (size_t)nf * EDGE_TERMS * sizeof(double)));
  g->allocs.push_back(wt);
  FV_CUDA(cudaMalloc(&wtf, (size_t)nf * EDGE_TERMS * sizeof(float)));
  g->allocs.push_back(wtf);
  FV_CUDA(cudaMalloc(&status, sizeof(int)));
  FV_CUDA(cudaMemset(status, 0, sizeof(int)));
  edge_table_kernel<<<(nf + 63) / 64, 64>>>(g->geo, cnt, off, wt, status);
  FV_CUDA(cudaGetLastError());
  to_float_kernel<<<(nf * EDGE_TERMS + 255) / 256, 256>>>(wt, wtf, nf * EDGE_TERMS);
  FV_CUDA(cudaGetLastError());
  int bad = 0;
  FV_CUDA(cudaMemcpy(&bad, status, sizeof(int), cudaMemcpyDeviceToHost));
  cudaFree(status);
  if (bad) return set_error("fv_build_grid: a panel-edge face flux has more terms than the table holds"), FV_EINVAL;
  g->edge_cnt = cnt, g->edge_off = off, g->edge_w = wt, g->edge_wf = wtf;
  return FV_OK;
}

// ------------------------------------------------------------------ tiled apply

// E[(c Nr + k) 24 Ns + f] = flux through panel-edge face f = (p, side, t) at level k, component c, measured
// along p's coordinate: one thread per (level, face); each term's slot is read once for all components
template <int D, class T, class R>
__global__ void __launch_bounds__(256) edge_flux_kernel(int Ns, int Nr, EdgeTab<R> et, const T* __restrict__ x,
                                                        T* __restrict__ E) {
  const int nf = 24 * Ns, N = 6 * Nr * Ns * Ns;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nf * Nr) return;
  const int f = e % nf, k = e / nf;
  const int n = et.cnt[f];
  const T* xk = x + k * Ns * Ns;
  R acc[D];
#pragma unroll
  for (int c = 0; c < D; ++c) acc[c] = R(0);
  // four terms at a time: their table slots, then all their cell values, are in flight together
  for (int m0 = 0; m0 < n; m0 += 4) {
    int o[4];
    R w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool on = m0 + u < n;
      o[u] = on ? et.off[(m0 + u) * nf + f] : 0;
      w[u] = on ? et.w[(m0 + u) * nf + f] : R(0);
    }
    T xv[4][D];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < D; ++c) xv[u][c] = m0 + u < n ? xk[c * N + o[u]] : T(0);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < D; ++c) acc[c] += w[u] * (R)xv[u][c];
  }
#pragma unroll
  for (int c = 0; c < D; ++c) E[(c * Nr + k) * nf + f] = (T)acc[c];
}

// value of component c at (p, k, j, i) for a tile's halo: a cell, a panel-edge ghost (one index beyond the
// panel), or 0 where no stencil of a computed cell reads it (cube corners, positions past the ghosts)
template <class T, class GT>
__device__ __forceinline__ T halo_value(const GT& G, const T* __restrict__ x, int c, int p, int k, int j, int i) {
  const int Ns = G.Ns;
  const bool in_i = i >= 0 && i < Ns, in_j = j >= 0 && j < Ns;
  if (in_i && in_j) return x[(c * 6 + p) * (G.Nr * Ns * Ns) + (k * Ns + j) * Ns + i];
  if (in_j && (i == -1 || i == Ns)) return (T)interp_ghost(G, x, c, p, i < 0 ? XI_MIN : XI_MAX, k, j);
  if (in_i && (j == -1 || j == Ns)) return (T)interp_ghost(G, x, c, p, j < 0 ? ETA_MIN : ETA_MAX, k, i);
  return T(0);
}

// one component c of one tile and level chunk (blockIdx.x = tile * D + c, so the D components of a tile run
// side by side and the couplings below read each other's values from L2; y = level chunk, z = panel)
template <int KIND, class T, class GT>
__global__ void __launch_bounds__(TILE_I* TILE_WARPS, sizeof(T) == 8 ? 3 : (KIND == FV_VTBE ? 4 : 5)) tile_apply_kernel(
    GT G, Coefs<typename GT::real> cf, const T* __restrict__ x, T* __restrict__ y, int kchunk,
    const T* __restrict__ E) {
  using R = typename GT::real;
  using S = TileShape<T>;
  constexpr int D = KIND == FV_VTBE ? 7 : 2;
  constexpr int RJ = S::RJ, TJ = S::TJ, PW = S::PW, PLANE = S::PLANE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* const sh = reinterpret_cast<T*>(smem_raw);  // ring of RING planes, slot = level & (RING - 1)
  const int Ns = G.Ns, Nr = G.Nr, Ns2 = Ns * Ns;
  const int NP = Nr * Ns2;  // cells of one panel
  const int N = 6 * NP;
  const int c = blockIdx.x % D, tile = blockIdx.x / D;
  const int nti = (Ns + TILE_I - 1) / TILE_I;
  const int i0 = (tile % nti) * TILE_I, j0 = (tile / nti) * TJ;
  const int p = blockIdx.z;
  const int kb = blockIdx.y * kchunk, ke = min(Nr, kb + kchunk);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TILE_I + tx;
  const int i = i0 + tx, jb = j0 + ty * RJ;
  const T* const xc = x + c * N;
  T* const yc = y + c * N;

  // per-cell constants, loaded once for all levels
  R w[RJ][9], crf[RJ], isg[RJ], rh[RJ][3];
  int nown = 0;  // own rows (a ragged tile has fewer)
#pragma unroll
  for (int r = 0; r < RJ; ++r) {
    const int j = jb + r;
    const bool o = i < Ns && j < Ns;
    nown += o;
    const int ji = o ? j * Ns + i : 0;
#pragma unroll
    for (int m = 0; m < 9; ++m) w[r][m] = G.w9[9 * ji + m];
    crf[r] = G.crf[ji];
    isg[r] = G.invsig[ji];
    R xl[3] = {G.xhat[3 * ji], G.xhat[3 * ji + 1], G.xhat[3 * ji + 2]};
    rotate(p, xl, rh[r]);
  }
  const bool full = nown == RJ && i < Ns;  // every row of this thread is a cell of the panel
  // panel-edge faces of the own cells: bit 0 xi-min, 1 xi-max, 2 eta-min, 3 eta-max (4 bits a row)
  int edges = 0;
#pragma unroll
  for (int r = 0; r < RJ; ++r)
    if (i < Ns && jb + r < Ns)
      edges |= ((i == 0) | ((i == Ns - 1) << 1) | ((jb + r == 0) << 2) | ((jb + r == Ns - 1) << 3)) << (4 * r);
  // wall rule of this component: 0 odd (-x), 1 even (+x), 2 pseudo-vacuum B
  const int wall = KIND == FV_VTBE ? (c >= 4 ? 2 : 0) : (c == 0 ? 1 : 0);
  // the Cartesian direction of this component (u_a, B_a: a; selected, not indexed, to stay in registers)
  const int ca = c >= 4 ? c - 4 : c;
  R rhc[RJ];
#pragma unroll
  for (int r = 0; r < RJ; ++r) rhc[r] = ca == 0 ? rh[r][0] : (ca == 1 ? rh[r][1] : rh[r][2]);

  // halo cell of this thread (tid < HALO), resolved once: value at level k = sum_m hw[m] xc[ho[m] + k Ns^2]
  // (a cell: one term; a panel-edge ghost: its three interpolation sources; else nothing)
  int hpos = 0, ho[3] = {0, 0, 0};
  R hw[3] = {R(0), R(0), R(0)};
  if (tid < S::HALO) {
    int hj, hi;
    if (tid < S::PH) hj = tid, hi = 0;
    else if (tid < 2 * S::PH) hj = tid - S::PH, hi = PW - 1;
    else if (tid < 2 * S::PH + TILE_I) hj = 0, hi = 1 + tid - 2 * S::PH;
    else hj = S::PH - 1, hi = 1 + tid - 2 * S::PH - TILE_I;
    hpos = hj * PW + hi;
    const int j = j0 - 1 + hj, ii = i0 - 1 + hi;
    const bool in_i = ii >= 0 && ii < Ns, in_j = j >= 0 && j < Ns;
    int side = -1, t = 0;
    if (in_i && in_j) ho[0] = p * NP + j * Ns + ii, hw[0] = R(1);
    else if (in_j && (ii == -1 || ii == Ns)) side = ii < 0 ? XI_MIN : XI_MAX, t = j;
    else if (in_i && (j == -1 || j == Ns)) side = j < 0 ? ETA_MIN : ETA_MAX, t = ii;
    if (side >= 0) {
      const int id = (p * 4 + side) * Ns + t, q = G.gq[id];
#pragma unroll
      for (int m = 0; m < 3; ++m) ho[m] = q * NP + G.gsrc[3 * id + m], hw[m] = G.gw[3 * id + m];
    }
  }
  const int own0 = p * NP + jb * Ns + i;     // own cell of row 0 at level 0 (+ k Ns^2 + r Ns)
  const int pos0 = (1 + ty * RJ) * PW + 1 + tx;  // its plane position (+ r PW)
  const int vpos0 = ty * RJ * PW + tx;           // top-left of its 3 x (RJ + 2) neighbourhood
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(sh);

  // the outer wall's ghost plane (level Nr) at the mirror radius: odd -x, even +x, B: -B + fac (B.rhat) rhat;
  // the inner wall's (level -1) likewise from level 0
  auto wall_plane = [&](int k, T* pl) {
    const int kw = k < 0 ? 0 : Nr - 1;
    const R fac = k < 0 ? G.wall_in : G.wall_out;
#pragma unroll
    for (int r = 0; r < RJ; ++r) {
      if (i >= Ns || jb + r >= Ns) continue;
      const int e = own0 + kw * Ns2 + r * Ns;
      const R v0 = (R)xc[e];
      R g = wall == 1 ? v0 : -v0;
      if (wall == 2)
        g += fac * rhc[r] * (rh[r][0] * (R)x[4 * N + e] + rh[r][1] * (R)x[5 * N + e] + rh[r][2] * (R)x[6 * N + e]);
      pl[pos0 + r * PW] = (T)g;
    }
  };
  // planes kb - 1 .. kb + 2 (up to the chunk's last plane ke), then the halo of kb + 3 into registers
  R hnext = R(0);
  for (int k = kb - 1; k <= kb + 2 && k <= ke; ++k) {
    T* pl = sh + (k & (RING - 1)) * PLANE;
    if (k < 0 || k >= Nr) {
      wall_plane(k, pl);
    } else {
      if (tid < S::HALO) {
        const T* xk = xc + k * Ns2;
        pl[hpos] = (T)(hw[0] * (R)xk[ho[0]] + hw[1] * (R)xk[ho[1]] + hw[2] * (R)xk[ho[2]]);
      }
#pragma unroll
      for (int r = 0; r < RJ; ++r) {
        if (i < Ns && jb + r < Ns)
          pl[pos0 + r * PW] = xc[own0 + k * Ns2 + r * Ns];
        else
          pl[pos0 + r * PW] = halo_value(G, x, c, p, k, jb + r, i);
      }
    }
  }
  if (kb + 3 < Nr && kb + 3 <= ke && tid < S::HALO) {
    const T* xk = xc + (kb + 3) * Ns2;
    hnext = hw[0] * (R)xk[ho[0]] + hw[1] * (R)xk[ho[1]] + hw[2] * (R)xk[ho[2]];
  }
  // the other components a VTBE row of (u, Theta) couples with at one cell (Coriolis, buoyancy, r . u),
  // loaded one level ahead: c = 3 reads u_x, u_y, u_z; c < 3 reads Theta and (c = 0, 1) u_y or u_x
  constexpr bool CPL = KIND == FV_VTBE;
  constexpr bool CPL_AHEAD = CPL && sizeof(T) == 4;  // FP64 (bound by its pipe) loads them at their own level
  const bool cpl_on = CPL && c <= 3;
  const int cc0 = c == 3 ? 0 : 3, cc1 = c == 3 ? 1 : (c == 0 ? 1 : 0), cc2 = 2;
  const int ncc = c == 3 ? 3 : (c == 2 ? 1 : 2);
  R cv[RJ][3];
  auto load_cpl = [&](int k) {
#pragma unroll
    for (int r = 0; r < RJ; ++r) {
      cv[r][0] = cv[r][1] = cv[r][2] = R(0);
      if (!cpl_on || k >= Nr || i >= Ns || jb + r >= Ns) continue;
      const int e = own0 + k * Ns2 + r * Ns;
      cv[r][0] = (R)x[cc0 * N + e];
      if (ncc > 1) cv[r][1] = (R)x[cc1 * N + e];
      if (ncc > 2) cv[r][2] = (R)x[cc2 * N + e];
    }
  };
  if (CPL_AHEAD) load_cpl(kb);
  __syncthreads();

  const R cdiag = KIND == FV_PPBE ? cf.pp : (c < 3 ? cf.h : (c == 3 ? cf.hpr : cf.hpm));
  for (int k = kb; k < ke; ++k) {
    const int s0 = (k & (RING - 1)) * PLANE, sm = ((k - 1) & (RING - 1)) * PLANE, sp = ((k + 1) & (RING - 1)) * PLANE;
    // level k + 3 into the slot of level k - 5 (no thread reads it after the last barrier); the own cells by
    // asynchronous copies that land while levels k and k + 1 are computed (one commit group a level)
    if (k + 3 <= ke && k + 3 < Nr) {
      const int s3 = ((k + 3) & (RING - 1)) * PLANE;
      if (tid < S::HALO) sh[s3 + hpos] = (T)hnext;
      if (full) {
        const T* src = xc + own0 + (k + 3) * Ns2;
#pragma unroll
        for (int r = 0; r < RJ; ++r)
          asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sbase + (unsigned)((s3 + pos0 + r * PW) * sizeof(T))),
                       "l"(src + r * Ns), "n"(sizeof(T)));
      } else {
#pragma unroll
        for (int r = 0; r < RJ; ++r)
          sh[s3 + pos0 + r * PW] = (i < Ns && jb + r < Ns) ? xc[own0 + (k + 3) * Ns2 + r * Ns]
                                                           : halo_value(G, x, c, p, k + 3, jb + r, i);
      }
      if (k + 4 < Nr && k + 4 <= ke && tid < S::HALO) {
        const T* xk = xc + (k + 4) * Ns2;
        hnext = hw[0] * (R)xk[ho[0]] + hw[1] * (R)xk[ho[1]] + hw[2] * (R)xk[ho[2]];
      }
    } else if (k + 3 == Nr && k + 3 <= ke) {  // the outer wall's ghost plane
      wall_plane(Nr, sh + ((k + 3) & (RING - 1)) * PLANE);
    }
    asm volatile("cp.async.commit_group;\n" ::);
    const R q = G.invr2[k], rb = G.rf2[k], rt = G.rf2[k + 1], rk = G.rc[k];
    const int ek = own0 + k * Ns2;
    // couplings of a VTBE row with other components of the same cell, from the values loaded a level ago
    if (CPL && !CPL_AHEAD) load_cpl(k);
    R cpl[RJ];
#pragma unroll
    for (int r = 0; r < RJ; ++r) cpl[r] = R(0);
    if (CPL && c <= 3) {
      const R b1 = cf.r1 * rk, b2 = cf.r2 / (rk * rk);
#pragma unroll
      for (int r = 0; r < RJ; ++r) {
        if (c == 3) {
          cpl[r] = b2 * (rh[r][0] * cv[r][0] + rh[r][1] * cv[r][1] + rh[r][2] * cv[r][2]);
        } else {
          cpl[r] = b1 * rhc[r] * cv[r][0];
          if (c == 0) cpl[r] += cf.cor * cv[r][1];
          if (c == 1) cpl[r] -= cf.cor * cv[r][1];
        }
      }
    }
    if (CPL_AHEAD && k + 1 < ke) load_cpl(k + 1);
    R v[RJ + 2][3];
#pragma unroll
    for (int rr = 0; rr < RJ + 2; ++rr)
#pragma unroll
      for (int di = 0; di < 3; ++di) v[rr][di] = (R)sh[s0 + vpos0 + rr * PW + di];
#pragma unroll
    for (int r = 0; r < RJ; ++r) {
      R h = R(0);
#pragma unroll
      for (int dj = 0; dj < 3; ++dj)
#pragma unroll
        for (int di = 0; di < 3; ++di) h = fma(w[r][dj * 3 + di], v[r + dj][di], h);
      const int eb = (edges >> (4 * r)) & 15;
      if (eb) {  // panel-edge faces: + flux at the max sides, - at the min sides
        const T* Ec = E + (c * Nr + k) * 24 * Ns + p * 4 * Ns;
        const int j = jb + r;
        if (eb & 1) h -= (R)Ec[XI_MIN * Ns + j];
        if (eb & 2) h += (R)Ec[XI_MAX * Ns + j];
        if (eb & 4) h -= (R)Ec[ETA_MIN * Ns + i];
        if (eb & 8) h += (R)Ec[ETA_MAX * Ns + i];
      }
      const R x0 = v[r + 1][1];
      const R below = x0 - (R)sh[sm + pos0 + r * PW], above = (R)sh[sp + pos0 + r * PW] - x0;
      const R lap = (h + crf[r] * (rt * above - rb * below)) * (isg[r] * q);
      const R out = KIND == FV_PPBE ? cdiag * lap : x0 + cdiag * lap + cpl[r];
      if (i < Ns && jb + r < Ns) yc[ek + r * Ns] = (T)out;
    }
    // level k + 1 reads plane k + 2, whose copies were issued a level ago: all but the newest group landed
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <int KIND, class T, class GT>
static fv_status launch_tiled(const GT& G, const Coefs<typename GT::real>& cf, const EdgeTab<typename GT::real>& et,
                              const T* x, T* E, T* y, cudaStream_t st, int cat) {
  using S = TileShape<T>;
  const int D = KIND == FV_VTBE ? 7 : 2;
  const size_t smem = (size_t)RING * S::PLANE * sizeof(T);
  static std::once_flag once[64];
  static cudaError_t attr_err[64];
  int dev = 0;
  FV_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error("apply: device ordinal out of range"), FV_EINVAL;
  std::call_once(once[dev], [&] {
    attr_err[dev] = cudaFuncSetAttribute(tile_apply_kernel<KIND, T, GT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  FV_CUDA(attr_err[dev]);
  const int tiles = ((G.Ns + TILE_I - 1) / TILE_I) * ((G.Ns + S::TJ - 1) / S::TJ);
  // about eight CTAs per SM of the 152, chunks of at least 4 levels
  const int per_chunk = tiles * D * 6;
  const int kmax = G.Nr / 4 > 0 ? G.Nr / 4 : 1;
  int nchunk = (152 * 8 + per_chunk - 1) / per_chunk;
  nchunk = nchunk < 1 ? 1 : (nchunk > kmax ? kmax : nchunk);
  const int kchunk = (G.Nr + nchunk - 1) / nchunk;
  nchunk = (G.Nr + kchunk - 1) / kchunk;
  {
    ProfScope ps(FV_K_GHOST + (cat & ~15), st);
    const int ne = 24 * G.Ns * G.Nr;
    edge_flux_kernel<D, T, typename GT::real><<<(ne + 255) / 256, 256, 0, st>>>(G.Ns, G.Nr, et,
                                                                                                     x, E);
  }
  FV_CUDA(cudaGetLastError());
  {
    ProfScope ps(cat, st);
    tile_apply_kernel<KIND, T, GT><<<dim3(tiles * D, nchunk, 6), dim3(TILE_I, TILE_WARPS), smem, st>>>(G, cf, x, y,
                                                                                                      kchunk, E);
  }
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

fv_status apply_op(const fv_system* s, const double* x, double* y, cudaStream_t st) {
  const fv_grid* g = s->grid;
  const Coefs<double> cf = make_coefs<double>(Phys{s->phys.E, s->phys.Ra, s->phys.Pr, s->phys.Pm, s->phys.dt},
                                               g->h.ri, g->h.ro);
  const EdgeTab<double> et{g->edge_cnt, g->edge_off, g->edge_w};
  const int cat = (s->kind == FV_VTBE ? FV_K_APPLY_VTBE : FV_K_APPLY_PPBE) + FV_K_COARSE * s->level;
  if (s->kind == FV_VTBE) return launch_tiled<FV_VTBE>(g->geo, cf, et, x, s->ghost, y, st, cat);
  return launch_tiled<FV_PPBE>(g->geo, cf, et, x, s->ghost, y, st, cat);
}

// FP32 operator (mixed-precision inner solves): FP32 tables, FP32 arithmetic
fv_status apply_op32(const fv_system* s, const float* x, float* y, cudaStream_t st) {
  const fv_grid* g = s->grid;
  const Coefs<float> cf = make_coefs<float>(Phys{s->phys.E, s->phys.Ra, s->phys.Pr, s->phys.Pm, s->phys.dt},
                                             g->h.ri, g->h.ro);
  const EdgeTab<float> et{g->edge_cnt, g->edge_off, g->edge_wf};
  const int cat = (s->kind == FV_VTBE ? FV_K_APPLY_VTBE : FV_K_APPLY_PPBE) + FV_K_COARSE * s->level + FV_K_FP32;
  if (s->kind == FV_VTBE) return launch_tiled<FV_VTBE>(g->geof, cf, et, x, s->ghost32, y, st, cat);
  return launch_tiled<FV_PPBE>(g->geof, cf, et, x, s->ghost32, y, st, cat);
}

}  // namespace fv

extern "C" fv_status fv_apply_op_fp32(const fv_system* s, const float* x, float* y, void* stream) {
  if (!s || !x || !y) return fv::set_error("fv_apply_op_fp32: null argument"), FV_EINVAL;
  if (!s->prec32) return fv::set_error("fv_apply_op_fp32: the system was not assembled with FV_PREC_FP32"), FV_EINVAL;
  return fv::apply_op32(s, x, y, (cudaStream_t)stream);
}
