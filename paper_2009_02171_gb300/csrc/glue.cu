// Face-flux kernels of the time step (paper Sec. 3.1 and 3.2):
//   NL   -- nonlinear terms in conservative form (eqn:nonlinearoperator,
//           eqn:nonlinearint) with Cartesian components:
//           f1_k = -div(u u_k) + div(B B_k)/(E Pm), f2 = -div(u Theta),
//           f3_k = div(B u_k) - div(u B_k); face flux (a_f . S_f) b_f.
//   DIV  -- face divergence D(v) = (1/V) sum_faces v_f . S_f of u~ and B~
//           (right-hand side of eqn:tsp, eqn:tspb).
//   GRAD -- cell Gauss gradient G(phi) = (1/E)(1/V) sum_faces phi_f S_f of P
//           and P_b (eqn:ubhat, eqn:ubtilde).
// Face values are means of the two adjacent values (ghosts across panel edges
// and walls); S_f is the contravariant face area vector (sqrt(g) g^i) h h in
// Cartesian components.  A panel-edge face carries the mean of the two
// panels' one-sided fluxes.
#include "stencil.cuh"

namespace fv {

enum { MODE_NL = 0, MODE_DIV = 1, MODE_GRAD = 2 };

struct Field {
  const double* x;
  const double* gh;
  int wall[7];
  int bbase;
};

// one-sided face mean of component c on panel p.  type 0: xi face f = i
// (cells i-1, i of row j); type 1: eta face f = j (rows j-1, j of column i);
// type 2: radial face kf = k (levels k-1, k).  General form: either cell may be a
// panel-edge ghost or a wall ghost.
__device__ __noinline__ double face_val_any(const Geo& G, const Field& F, int c, int p, int type, int k, int j, int i) {
  ApplyAcc<double> acc(G, F.x, F.gh);
  if (type == 0) {
    emit_h(G, acc, 0.5, p, k, j, i - 1, c);
    emit_h(G, acc, 0.5, p, k, j, i, c);
  } else if (type == 1) {
    emit_h(G, acc, 0.5, p, k, j - 1, i, c);
    emit_h(G, acc, 0.5, p, k, j, i, c);
  } else if (k > 0 && k < G.Nr) {
    acc.cell(0.5, p, k - 1, j, i, c);
    acc.cell(0.5, p, k, j, i, c);
  } else {
    const int kc = k == 0 ? 0 : G.Nr - 1;
    acc.cell(0.5, p, kc, j, i, c);
    wall_ghost(G, acc, 0.5, p, kc, j, i, c, F.wall[c], F.bbase, k == 0 ? G.wall_in : G.wall_out);
  }
  return acc.sum;
}

// The same mean when both cells are interior cells of panel p (the common case): two loads,
// the same arithmetic as the general form (0.5 x1, then fma with 0.5 x2).
__device__ __forceinline__ double face_val(const Geo& G, const Field& F, int c, int p, int type, int k, int j, int i) {
  const int Ns = G.Ns;
  long long d = -1;
  if (type == 0 && i > 0 && i < Ns) d = 1;
  else if (type == 1 && j > 0 && j < Ns) d = Ns;
  else if (type == 2 && k > 0 && k < G.Nr) d = (long long)Ns * Ns;
  if (d < 0) return face_val_any(G, F, c, p, type, k, j, i);
  const double* xc = F.x + (long long)c * G.N + ((long long)(p * G.Nr + k) * Ns + j) * Ns + i;
  return fma(0.5, xc[0], 0.5 * xc[-d]);
}

// face area vector S_f (Cartesian) of face (type, k, j, i) of panel p: the panel's tabulated vector times
// the radius factor of the level (r_k for horizontal faces, r_f^2 for radial ones)
__device__ __forceinline__ void face_area(const Geo& G, int p, int type, int k, int j, int i, double S[3]) {
  const double* l;
  double sc;
  const int Ns = G.Ns;
  if (type == 0) l = G.sxp + 3 * (((long long)p * Ns + j) * (Ns + 1) + i), sc = G.rc[k];
  else if (type == 1) l = G.syp + 3 * (((long long)p * (Ns + 1) + j) * Ns + i), sc = G.rc[k];
  else l = G.srp + 3 * (((long long)p * Ns + j) * Ns + i), sc = G.rf2[k];
  S[0] = l[0] * sc, S[1] = l[1] * sc, S[2] = l[2] * sc;
}

template <int MODE>
__device__ __forceinline__ void face_flux(const Geo& G, const Field& F, double cL, int p, int type, int k, int j, int i,
                                       double* out) {
  double S[3];
  face_area(G, p, type, k, j, i, S);
  if (MODE == MODE_NL) {
    double v[7];
    for (int c = 0; c < 7; ++c) v[c] = face_val(G, F, c, p, type, k, j, i);
    const double un = v[0] * S[0] + v[1] * S[1] + v[2] * S[2];
    const double bn = v[4] * S[0] + v[5] * S[1] + v[6] * S[2];
    for (int c = 0; c < 3; ++c) {
      out[c] = -un * v[c] + cL * bn * v[4 + c];
      out[4 + c] = bn * v[c] - un * v[4 + c];
    }
    out[3] = -un * v[3];
  } else if (MODE == MODE_DIV) {
    double u[3], b[3];
    for (int c = 0; c < 3; ++c) u[c] = face_val(G, F, c, p, type, k, j, i), b[c] = face_val(G, F, 4 + c, p, type, k, j, i);
    out[0] = u[0] * S[0] + u[1] * S[1] + u[2] * S[2];
    out[1] = b[0] * S[0] + b[1] * S[1] + b[2] * S[2];
  } else {
    const double P = face_val(G, F, 0, p, type, k, j, i), Pb = face_val(G, F, 1, p, type, k, j, i);
    for (int c = 0; c < 3; ++c) out[c] = P * S[c], out[3 + c] = Pb * S[c];
  }
}

template <int MODE>
__device__ __forceinline__ void side_face_flux(const Geo& G, const Field& F, double cL, int p, int side, int k, int t,
                                               double* out) {
  const int Ns = G.Ns;
  switch (side) {
    case XI_MIN: face_flux<MODE>(G, F, cL, p, 0, k, t, 0, out); break;
    case XI_MAX: face_flux<MODE>(G, F, cL, p, 0, k, t, Ns, out); break;
    case ETA_MIN: face_flux<MODE>(G, F, cL, p, 1, k, 0, t, out); break;
    default: face_flux<MODE>(G, F, cL, p, 1, k, Ns, t, out); break;
  }
}

template <int MODE, int NO>
__device__ __noinline__ void edge_face_flux(const Geo& G, const Field& F, double cL, int p, int side, int k, int t,
                                            double* out) {
  const int ps = p * 4 + side;
  double a[7], b[7];
  side_face_flux<MODE>(G, F, cL, p, side, k, t, a);
  side_face_flux<MODE>(G, F, cL, G.pq[ps], G.psq[ps], k, G.ptmap[ps * G.Ns + t], b);
  const double sg = G.psgn[ps];
  for (int m = 0; m < NO; ++m) out[m] = 0.5 * (a[m] + sg * b[m]);
}

// Interior and radial faces of every cell (panel-edge faces contribute zero here and are added by
// edge_face_kernel, so no warp of this kernel waits on the ghost interpolation of an edge cell).
// grid: x = tiles of the (j, i) plane, y = k, z = panel
template <int MODE, int NO>
__global__ void face_kernel(Geo G, Field F, double cL, double scale, double* __restrict__ out) {
  const int Ns = G.Ns;
  const int ij = blockIdx.x * blockDim.x + threadIdx.x;
  if (ij < Ns * Ns) {
    const int i = ij % Ns, j = ij / Ns, k = blockIdx.y, p = blockIdx.z;
    const long long e = ((long long)(p * G.Nr + k) * Ns + j) * Ns + i;
    double acc[NO], fl[7];
    for (int m = 0; m < NO; ++m) acc[m] = 0.0;
    // xi faces
    if (i + 1 < Ns) {
      face_flux<MODE>(G, F, cL, p, 0, k, j, i + 1, fl);
      for (int m = 0; m < NO; ++m) acc[m] += fl[m];
    }
    if (i > 0) {
      face_flux<MODE>(G, F, cL, p, 0, k, j, i, fl);
      for (int m = 0; m < NO; ++m) acc[m] -= fl[m];
    }
    // eta faces
    if (j + 1 < Ns) {
      face_flux<MODE>(G, F, cL, p, 1, k, j + 1, i, fl);
      for (int m = 0; m < NO; ++m) acc[m] += fl[m];
    }
    if (j > 0) {
      face_flux<MODE>(G, F, cL, p, 1, k, j, i, fl);
      for (int m = 0; m < NO; ++m) acc[m] -= fl[m];
    }
    // radial faces
    face_flux<MODE>(G, F, cL, p, 2, k + 1, j, i, fl);
    for (int m = 0; m < NO; ++m) acc[m] += fl[m];
    face_flux<MODE>(G, F, cL, p, 2, k, j, i, fl);
    for (int m = 0; m < NO; ++m) acc[m] -= fl[m];
    const double iv = scale * G.invsig[j * Ns + i] * G.invr2[k];
    for (int m = 0; m < NO; ++m) out[m * G.N + e] = acc[m] * iv;
  }
}

// Panel-edge faces (the mean of the two panels' one-sided fluxes), added to the cells that own
// them after face_kernel: one thread per cell of a panel's perimeter, which takes its one or two
// edge faces in turn (no two threads write one cell).
// grid: x = perimeter cells 4 (Ns - 1) of a (panel, k) plane, y = k, z = panel
template <int MODE, int NO>
__global__ void edge_face_kernel(Geo G, Field F, double cL, double scale, double* __restrict__ out) {
  const int Ns = G.Ns;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * (Ns - 1)) return;
  const int k = blockIdx.y, p = blockIdx.z;
  // the perimeter walked as four runs of Ns - 1 cells: row j = 0, column i = Ns - 1, row j = Ns - 1,
  // column i = 0 (each run starts at a corner)
  const int run = t / (Ns - 1), q = t - run * (Ns - 1);
  int i, j;
  if (run == 0) j = 0, i = q;
  else if (run == 1) i = Ns - 1, j = q;
  else if (run == 2) j = Ns - 1, i = Ns - 1 - q;
  else i = 0, j = Ns - 1 - q;
  double acc[NO], fl[7];
  for (int m = 0; m < NO; ++m) acc[m] = 0.0;
  if (i + 1 == Ns) {
    edge_face_flux<MODE, NO>(G, F, cL, p, XI_MAX, k, j, fl);
    for (int m = 0; m < NO; ++m) acc[m] += fl[m];
  }
  if (i == 0) {
    edge_face_flux<MODE, NO>(G, F, cL, p, XI_MIN, k, j, fl);
    for (int m = 0; m < NO; ++m) acc[m] -= fl[m];
  }
  if (j + 1 == Ns) {
    edge_face_flux<MODE, NO>(G, F, cL, p, ETA_MAX, k, i, fl);
    for (int m = 0; m < NO; ++m) acc[m] += fl[m];
  }
  if (j == 0) {
    edge_face_flux<MODE, NO>(G, F, cL, p, ETA_MIN, k, i, fl);
    for (int m = 0; m < NO; ++m) acc[m] -= fl[m];
  }
  const long long e = ((long long)(p * G.Nr + k) * Ns + j) * Ns + i;
  const double iv = scale * G.invsig[j * Ns + i] * G.invr2[k];
  for (int m = 0; m < NO; ++m) out[m * G.N + e] += acc[m] * iv;
}

template <int MODE, int NO>
static fv_status face_launch(const Geo& G, const Field& F, double cL, double scale, double* out, cudaStream_t st) {
  face_kernel<MODE, NO><<<dim3((G.Ns * G.Ns + 127) / 128, G.Nr, 6), 128, 0, st>>>(G, F, cL, scale, out);
  edge_face_kernel<MODE, NO><<<dim3((4 * (G.Ns - 1) + 127) / 128, G.Nr, 6), 128, 0, st>>>(G, F, cL, scale, out);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

// 7-component field (u, Theta, B): odd walls for u and Theta, pseudo-vacuum for B
static Field field7(const double* x, const double* gh) {
  Field F{x, gh, {WALL_ODD, WALL_ODD, WALL_ODD, WALL_ODD, WALL_B, WALL_B, WALL_B}, 4};
  return F;
}

fv_status nonlinear_terms(const fv_grid* g, const fv_phys& ph, const double* x7, double* f, double* gh7,
                          cudaStream_t st) {
  ProfScope ps(FV_K_GLUE, st);
  return face_launch<MODE_NL, 7>(g->geo, field7(x7, gh7), 1.0 / (ph.E * ph.Pm), 1.0, f, st);
}

fv_status face_divergence_uB(const fv_grid* g, const double* x7, double* bP, double* gh7, cudaStream_t st) {
  ProfScope ps(FV_K_GLUE, st);
  return face_launch<MODE_DIV, 2>(g->geo, field7(x7, gh7), 0.0, 1.0, bP, st);
}

// gradient of (P, P_b) (2N values, P even walls, P_b odd walls) -> out6 = (G P, G P_b), times `scale`
fv_status cell_gradient(const fv_grid* g, const double* x2, int /*wall*/, double scale, double* out6, double* gh2,
                        cudaStream_t st) {
  Field F{x2, gh2, {WALL_EVEN, WALL_ODD, 0, 0, 0, 0, 0}, 0};
  ProfScope ps(FV_K_GLUE, st);
  return face_launch<MODE_GRAD, 6>(g->geo, F, 0.0, scale, out6, st);
}

}  // namespace fv
