// Discrete operators of the shell dynamo as term visitors (device code).
//
// Each operator row is written once, as a sequence of (coefficient, value)
// terms; an accumulator decides what a term does:
//   ApplyAcc    -- y_row += coef * x[value]   (matrix-free apply; ghosts read
//                  from the ghost layer filled beforehand)
//   AssembleAcc -- adds coef into the structured subdomain-matrix slot of the
//                  referenced cell (ILU(0) setup), expanding ghosts into their
//                  interpolation sources.
//
// Finite-volume divergence by the Gauss theorem (paper eqn:divdiscretization):
//   lap(phi)_c = (1/V_c) sum_faces +-F,  V = sqrt(g) h_s^2 h_r,
//   F_xi  = h_r [a11 (phi_R - phi_L) + a12/4 (phi_{L,j+1} - phi_{L,j-1} + phi_{R,j+1} - phi_{R,j-1})]
//   F_eta likewise with a22 and the xi-differences,
//   F_r   = sigma h_s^2 r_f^2 (phi_{k} - phi_{k-1}) / h_r.
// A face on a panel edge carries the mean of the two panels' one-sided fluxes
// (each computed with that panel's own ghosts), so fluxes telescope.
// Walls: ghost at the mirror radius; odd = -cell (u, Theta, P_b), even = +cell
// (P), B: -B + (1 + (r_c/r_g)^2)(B.rhat) rhat (pseudo-vacuum, eqn:pvc).
#pragma once
#include "fv_internal.h"

namespace fv {

// panel rotation: Cartesian = M_p * local(1, X, Y), entries in {-1, 0, 1}
__device__ __constant__ static const signed char kPM[6][9] = {
    {1, 0, 0, 0, 1, 0, 0, 0, 1},  {0, -1, 0, 1, 0, 0, 0, 0, 1}, {-1, 0, 0, 0, -1, 0, 0, 0, 1},
    {0, 1, 0, -1, 0, 0, 0, 0, 1}, {0, 0, -1, 0, 1, 0, 1, 0, 0}, {0, 0, 1, 0, 1, 0, -1, 0, 0},
};

template <class R>
__device__ __forceinline__ void rotate(int p, const R* l, R* v) {
#pragma unroll
  for (int a = 0; a < 3; ++a) v[a] = kPM[p][3 * a] * l[0] + kPM[p][3 * a + 1] * l[1] + kPM[p][3 * a + 2] * l[2];
}

template <class GT>
__device__ __forceinline__ long long cidx(const GT& G, int p, int k, int j, int i) {
  return (long long)(((p * G.Nr + k) * G.Ns + j) * G.Ns + i);
}

// ghost layer: [comp][p][side][k][t+1], t in [-1, Ns] (corners stored on xi sides)
template <class GT>
__device__ __forceinline__ long long gidx(const GT& G, int comp, int p, int side, int k, int t) {
  return ((((long long)comp * 6 + p) * 4 + side) * G.Nr + k) * (G.Ns + 2) + (t + 1);
}

// value at extended horizontal position (j, i in [-1, Ns]) of panel p, level k
template <class GT, class Acc>
__device__ inline void emit_h(const GT& G, Acc& acc, typename GT::real c, int p, int k, int j, int i, int comp) {
  const int Ns = G.Ns;
  if (i >= 0 && i < Ns) {
    if (j >= 0 && j < Ns)
      acc.cell(c, p, k, j, i, comp);
    else
      acc.ghost(c, p, j < 0 ? ETA_MIN : ETA_MAX, k, i, comp);
  } else {
    acc.ghost(c, p, i < 0 ? XI_MIN : XI_MAX, k, j, comp);
  }
}

// one-sided flux through the xi face f (between cells f-1 and f) of row j
template <class GT, class Acc>
__device__ inline void xi_flux(const GT& G, Acc& acc, typename GT::real s, int p, int k, int j, int f, int comp) {
  const int id = j * (G.Ns + 1) + f;
  const typename GT::real a = G.ax11[id] * s, b = G.ax12[id] * s;
  emit_h(G, acc, a, p, k, j, f, comp);
  emit_h(G, acc, -a, p, k, j, f - 1, comp);
  emit_h(G, acc, b, p, k, j + 1, f - 1, comp);
  emit_h(G, acc, -b, p, k, j - 1, f - 1, comp);
  emit_h(G, acc, b, p, k, j + 1, f, comp);
  emit_h(G, acc, -b, p, k, j - 1, f, comp);
}

// one-sided flux through the eta face f (between rows f-1 and f) of column i
template <class GT, class Acc>
__device__ inline void eta_flux(const GT& G, Acc& acc, typename GT::real s, int p, int k, int f, int i, int comp) {
  const int id = f * G.Ns + i;
  const typename GT::real a = G.ay22[id] * s, b = G.ay12[id] * s;
  emit_h(G, acc, a, p, k, f, i, comp);
  emit_h(G, acc, -a, p, k, f - 1, i, comp);
  emit_h(G, acc, b, p, k, f - 1, i + 1, comp);
  emit_h(G, acc, -b, p, k, f - 1, i - 1, comp);
  emit_h(G, acc, b, p, k, f, i + 1, comp);
  emit_h(G, acc, -b, p, k, f, i - 1, comp);
}

template <class GT, class Acc>
__device__ __noinline__ void own_side_flux(const GT& G, Acc& acc, typename GT::real s, int p, int side, int k, int t,
                                              int comp) {
  const int Ns = G.Ns;
  switch (side) {
    case XI_MIN: xi_flux(G, acc, s, p, k, t, 0, comp); break;
    case XI_MAX: xi_flux(G, acc, s, p, k, t, Ns, comp); break;
    case ETA_MIN: eta_flux(G, acc, s, p, k, 0, t, comp); break;
    default: eta_flux(G, acc, s, p, k, Ns, t, comp); break;
  }
}

// panel-edge face: mean of the two panels' one-sided fluxes (measured along p's coordinate)
template <class GT, class Acc>
__device__ __noinline__ void edge_flux(const GT& G, Acc& acc, typename GT::real s, int p, int side, int k, int t, int comp) {
  const int ps = p * 4 + side;
  using R = typename GT::real;
  own_side_flux(*G.self, acc, R(0.5) * s, p, side, k, t, comp);
  own_side_flux(*G.self, acc, R(0.5) * s * R(G.psgn[ps]), G.pq[ps], G.psq[ps], k, G.ptmap[ps * G.Ns + t], comp);
}

// wall ghost of component `comp` at the cell (kc, j, i) next to a wall
template <class GT, class Acc>
__device__ __forceinline__ void wall_ghost(const GT& G, Acc& acc, typename GT::real c, int p, int kc, int j, int i, int comp,
                                           int wall, int bbase, typename GT::real fac) {
  if (wall == WALL_ODD) {
    acc.cell(-c, p, kc, j, i, comp);
  } else if (wall == WALL_EVEN) {
    acc.cell(c, p, kc, j, i, comp);
  } else {
    typename GT::real rh[3];
    rotate(p, G.xhat + 3 * (j * G.Ns + i), rh);
    const int a = comp - bbase;
    acc.cell(-c, p, kc, j, i, comp);
#pragma unroll
    for (int b = 0; b < 3; ++b) acc.cell(c * fac * rh[a] * rh[b], p, kc, j, i, bbase + b);
  }
}

// radial flux through face kf (between k = kf-1 and kf) of column (j, i)
template <class GT, class Acc>
__device__ __forceinline__ void r_flux(const GT& G, Acc& acc, typename GT::real s, int p, int kf, int j, int i, int comp,
                                       int wall, int bbase) {
  const typename GT::real c = G.crf[j * G.Ns + i] * G.rf2[kf] * s;
  if (kf > 0 && kf < G.Nr) {
    acc.cell(c, p, kf, j, i, comp);
    acc.cell(-c, p, kf - 1, j, i, comp);
  } else if (kf == 0) {
    acc.cell(c, p, 0, j, i, comp);
    wall_ghost(G, acc, -c, p, 0, j, i, comp, wall, bbase, G.wall_in);
  } else {
    wall_ghost(G, acc, c, p, G.Nr - 1, j, i, comp, wall, bbase, G.wall_out);
    acc.cell(-c, p, G.Nr - 1, j, i, comp);
  }
}

// interior xi / eta fluxes: every value is a cell of panel p (1 <= i, j <= Ns-2)
template <class GT, class Acc>
__device__ __forceinline__ void xi_flux_in(const GT& G, Acc& acc, typename GT::real s, int p, int k, int j, int f, int comp) {
  const int id = j * (G.Ns + 1) + f;
  const typename GT::real a = G.ax11[id] * s, b = G.ax12[id] * s;
  acc.cell(a, p, k, j, f, comp);
  acc.cell(-a, p, k, j, f - 1, comp);
  acc.cell(b, p, k, j + 1, f - 1, comp);
  acc.cell(-b, p, k, j - 1, f - 1, comp);
  acc.cell(b, p, k, j + 1, f, comp);
  acc.cell(-b, p, k, j - 1, f, comp);
}

template <class GT, class Acc>
__device__ __forceinline__ void eta_flux_in(const GT& G, Acc& acc, typename GT::real s, int p, int k, int f, int i, int comp) {
  const int id = f * G.Ns + i;
  const typename GT::real a = G.ay22[id] * s, b = G.ay12[id] * s;
  acc.cell(a, p, k, f, i, comp);
  acc.cell(-a, p, k, f - 1, i, comp);
  acc.cell(b, p, k, f - 1, i + 1, comp);
  acc.cell(-b, p, k, f - 1, i - 1, comp);
  acc.cell(b, p, k, f, i + 1, comp);
  acc.cell(-b, p, k, f, i - 1, comp);
}

// horizontal part of s * lap at a cell on a panel edge (i or j in {0, Ns-1})
template <class GT, class Acc>
__device__ __noinline__ void lap_h_edge(const GT& G, Acc& acc, typename GT::real sv, int p, int k, int j, int i, int comp) {
  const int Ns = G.Ns;
  if (i + 1 == Ns) edge_flux(G, acc, sv, p, XI_MAX, k, j, comp);
  else xi_flux(G, acc, sv, p, k, j, i + 1, comp);
  if (i == 0) edge_flux(G, acc, -sv, p, XI_MIN, k, j, comp);
  else xi_flux(G, acc, -sv, p, k, j, i, comp);
  if (j + 1 == Ns) edge_flux(G, acc, sv, p, ETA_MAX, k, i, comp);
  else eta_flux(G, acc, sv, p, k, j + 1, i, comp);
  if (j == 0) edge_flux(G, acc, -sv, p, ETA_MIN, k, i, comp);
  else eta_flux(G, acc, -sv, p, k, j, i, comp);
}

// s * lap(phi_comp) at cell (p, k, j, i)
template <class GT, class Acc>
__device__ __forceinline__ void lap_row(const GT& G, Acc& acc, typename GT::real s, int p, int k, int j, int i, int comp,
                                        int wall, int bbase) {
  const int Ns = G.Ns;
  const typename GT::real sv = s * G.invsig[j * Ns + i] * G.invr2[k];
  if (i > 0 && j > 0 && i + 1 < Ns && j + 1 < Ns) {
    xi_flux_in(G, acc, sv, p, k, j, i + 1, comp);
    xi_flux_in(G, acc, -sv, p, k, j, i, comp);
    eta_flux_in(G, acc, sv, p, k, j + 1, i, comp);
    eta_flux_in(G, acc, -sv, p, k, j, i, comp);
  } else {
    Acc tmp = acc;  // only the copy's address escapes into the out-of-line edge path
    lap_h_edge(*G.self, tmp, sv, p, k, j, i, comp);
    acc = tmp;
  }
  r_flux(G, acc, sv, p, k + 1, j, i, comp, wall, bbase);
  r_flux(G, acc, -sv, p, k, j, i, comp, wall, bbase);
}

struct Phys {
  double E, Ra, Pr, Pm, dt;
};

// Physics coefficients of the VTBE / PPBE rows, computed once on the host in
// the coefficient type R (no division or FP64 arithmetic per row).
template <class R>
struct Coefs {
  R one;    // 1
  R h;      // -dt/2
  R cor;    // -dt/2 * 2/E        (Coriolis, u_y in the u_x row; negated in the u_y row)
  R r1;     // -dt/2 * Ra/(E r_o) (buoyancy, times r_k xhat_a)
  R r2;     // -dt/2 * r_i r_o    (times xhat_c / r^2)
  R hpr;    // -dt/2 / Pr
  R hpm;    // -dt/2 / Pm
  R pp;     // dt/(2E)            (PPBE)
};

template <class R>
inline Coefs<R> make_coefs(const Phys& ph, double ri, double ro) {
  const double h = -0.5 * ph.dt;
  Coefs<R> c;
  c.one = R(1), c.h = R(h), c.cor = R(h * 2.0 / ph.E), c.r1 = R(h * ph.Ra / (ph.E * ro)), c.r2 = R(h * ri * ro);
  c.hpr = R(h / ph.Pr), c.hpm = R(h / ph.Pm), c.pp = R(0.5 * ph.dt / ph.E);
  return c;
}

// Row `a` of the VTBE matrix A = I - dt/2 M (eqn:tsvelocity, eqn:tstemperature, eqn:tsmag):
//   u_a:   u - dt/2 [lap u - (2/E) z x u + Ra/(E r_o) Theta r]_a
//   Theta: Theta - dt/2 [lap Theta / Pr + r_i r_o / r^3 (u . r)]
//   B_a:   B - dt/2 [lap B / Pm]_a
template <class GT, class Acc>
__device__ __forceinline__ void vtbe_row(const GT& G, const Coefs<typename GT::real>& cf, Acc& acc, int p, int k,
                                         int j, int i, int a) {
  using R = typename GT::real;
  acc.cell(cf.one, p, k, j, i, a);
  if (a < 3) {
    lap_row(G, acc, cf.h, p, k, j, i, a, WALL_ODD, 0);
    if (a == 0) acc.cell(cf.cor, p, k, j, i, 1);
    if (a == 1) acc.cell(-cf.cor, p, k, j, i, 0);
    R xl[3], x[3];
    for (int c = 0; c < 3; ++c) xl[c] = G.xhat[3 * (j * G.Ns + i) + c];
    rotate(p, xl, x);
    acc.cell(cf.r1 * G.rc[k] * x[a], p, k, j, i, 3);
  } else if (a == 3) {
    lap_row(G, acc, cf.hpr, p, k, j, i, 3, WALL_ODD, 0);
    R xl[3], x[3];
    for (int c = 0; c < 3; ++c) xl[c] = G.xhat[3 * (j * G.Ns + i) + c];
    rotate(p, xl, x);
    const R r = G.rc[k];
    const R w = cf.r2 / (r * r);
    for (int c = 0; c < 3; ++c) acc.cell(w * x[c], p, k, j, i, c);
  } else {
    lap_row(G, acc, cf.hpm, p, k, j, i, a, WALL_B, 4);
  }
}

// Row `a` of the PPBE matrix dt/2 D G = dt/(2E) lap (eqn:tsp, eqn:tspb): P even walls, P_b odd walls
template <class GT, class Acc>
__device__ __forceinline__ void ppbe_row(const GT& G, const Coefs<typename GT::real>& cf, Acc& acc, int p, int k,
                                         int j, int i, int a) {
  lap_row(G, acc, cf.pp, p, k, j, i, a, a == 0 ? WALL_EVEN : WALL_ODD, 0);
}

// T: element type of x and the ghost layer; R: accumulation type (FP64 for the
// FP64 path, FP32 for the inner solves of mixed precision)
template <class T, class R = double>
struct ApplyAcc {
  long long N;
  int Ns, Nr;
  const T* x;
  const T* gh;
  R sum;
  template <class GT>
  __device__ __forceinline__ ApplyAcc(const GT& G, const T* x_, const T* gh_)
      : N(G.N), Ns(G.Ns), Nr(G.Nr), x(x_), gh(gh_), sum(R(0)) {}
  __device__ __forceinline__ void cell(R c, int p, int k, int j, int i, int comp) {
    sum += c * (R)x[(long long)comp * N + (long long)(((p * Nr + k) * Ns + j) * Ns + i)];
  }
  __device__ __forceinline__ void ghost(R c, int p, int side, int k, int t, int comp) {
    sum += c * (R)gh[((((long long)comp * 6 + p) * 4 + side) * Nr + k) * (Ns + 2) + (t + 1)];
  }
};

// Ghost centre beyond `side` of panel p at tangential index t (t in [0, Ns)): quadratic
// Lagrange interpolation along the neighbour's first grid line.
template <class T, class GT>
__device__ __forceinline__ typename GT::real interp_ghost(const GT& G, const T* x, int comp, int p, int side, int k,
                                                          int t) {
  using R = typename GT::real;
  const int id = (p * 4 + side) * G.Ns + t;
  const int q = G.gq[id];
  const T* base = x + comp * G.N + ((long long)(q * G.Nr + k) * G.Ns) * G.Ns;
  return G.gw[3 * id] * (R)base[G.gsrc[3 * id]] + G.gw[3 * id + 1] * (R)base[G.gsrc[3 * id + 1]] +
         G.gw[3 * id + 2] * (R)base[G.gsrc[3 * id + 2]];
}

}  // namespace fv
