// Grid setup: geometry tables of the equiangular cubed-sphere shell (host, FP64).
//
// Paper Sec. 3.2: six panels with local (xi, eta, r), xi, eta in [-pi/4, pi/4];
// cell centres xi_i = -pi/4 + (i + 1/2) h_s, h_s = pi / (2 Ns),
// r_k = r_i + (k + 1/2) h_r, h_r = (r_o - r_i) / Nr;
// sqrt(g) = r^2 sec^2(xi) sec^2(eta) / (1 + tan^2 xi + tan^2 eta)^{3/2}.
// With X = tan xi, Y = tan eta, delta = 1 + X^2 + Y^2 the inverse metric of the
// gnomonic map gives sqrt(g) g^11 = (1+Y^2)/sqrt(delta), sqrt(g) g^22 =
// (1+X^2)/sqrt(delta), sqrt(g) g^12 = X Y / sqrt(delta), g^33 = 1 (no r
// dependence in the angular face coefficients).
// Panel orientation: panels 0..3 equatorial, centred on +x, +y, -x, -y (eta
// north), panel 4 = +z, panel 5 = -z; unit vector = M_p (1, X, Y) / sqrt(delta).
// Panel-edge ghosts: one layer, quadratic Lagrange interpolation along the
// neighbour panel's first grid line parallel to the edge at the ghost's
// exact tangential position (the ghost centre lies on that line).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fv_internal.h"

namespace fv {

// M_p as rows: Cartesian = M_p * (1, X, Y)
static const int kPanelM[6][3][3] = {
    {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},    // ( 1,  X,  Y)
    {{0, -1, 0}, {1, 0, 0}, {0, 0, 1}},   // (-X,  1,  Y)
    {{-1, 0, 0}, {0, -1, 0}, {0, 0, 1}},  // (-1, -X,  Y)
    {{0, 1, 0}, {-1, 0, 0}, {0, 0, 1}},   // ( X, -1,  Y)
    {{0, 0, -1}, {0, 1, 0}, {1, 0, 0}},   // (-Y,  X,  1)
    {{0, 0, 1}, {0, 1, 0}, {-1, 0, 0}},   // ( Y,  X, -1)
};

static void to_cart(int p, double xi, double eta, double v[3]) {
  double X = std::tan(xi), Y = std::tan(eta), n = std::sqrt(1 + X * X + Y * Y);
  double l[3] = {1.0 / n, X / n, Y / n};
  for (int a = 0; a < 3; ++a) v[a] = kPanelM[p][a][0] * l[0] + kPanelM[p][a][1] * l[1] + kPanelM[p][a][2] * l[2];
}

// local frame components (1, X, Y) direction of v on panel p: M_p^T v
static void to_local(int p, const double v[3], double w[3]) {
  for (int b = 0; b < 3; ++b) w[b] = kPanelM[p][0][b] * v[0] + kPanelM[p][1][b] * v[1] + kPanelM[p][2][b] * v[2];
}

static int which_panel(const double v[3]) {
  int best = 0;
  double bv = -1e300;
  for (int p = 0; p < 6; ++p) {
    double w[3];
    to_local(p, v, w);
    if (w[0] > bv) bv = w[0], best = p;
  }
  return best;
}

static void side_point(int side, double tang, double edge, double* xi, double* eta) {
  switch (side) {
    case XI_MIN: *xi = -edge, *eta = tang; break;
    case XI_MAX: *xi = edge, *eta = tang; break;
    case ETA_MIN: *xi = tang, *eta = -edge; break;
    default: *xi = tang, *eta = edge; break;
  }
}

void set_error(const std::string& msg);

template <class T>
static T* upload(fv_grid* g, const std::vector<T>& h) {
  void* d = nullptr;
  if (cudaMalloc(&d, h.size() * sizeof(T)) != cudaSuccess) return nullptr;
  if (cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return nullptr;
  }
  g->allocs.push_back(d);
  return static_cast<T*>(d);
}

fv_status build_grid(const fv_grid_desc* desc, fv_grid** out) {
  if (!desc || !out) return set_error("fv_build_grid: null argument"), FV_EINVAL;
  const int Ns = desc->Ns, Nr = desc->Nr;
  if (Ns < 4 || Nr < 2 || !(desc->ro > desc->ri) || !(desc->ri > 0))
    return set_error("fv_build_grid: need Ns >= 4, Nr >= 2, 0 < ri < ro"), FV_EINVAL;
  fv_grid* g = new fv_grid();
  GridHost& h = g->h;
  h.Ns = Ns, h.Nr = Nr, h.ri = desc->ri, h.ro = desc->ro;
  h.hs = M_PI / (2.0 * Ns);
  h.hr = (h.ro - h.ri) / Nr;
  h.N = 6LL * Ns * Ns * Nr;
  const double hs = h.hs, hr = h.hr;
  auto xc = [&](int i) { return -M_PI / 4 + (i + 0.5) * hs; };
  auto xf = [&](int i) { return -M_PI / 4 + i * hs; };

  // angular metric pieces at (xi, eta)
  struct Ang {
    double sigma, a11, a22, a12, e1[3], e2[3], xh[3];
  };
  auto ang = [](double xi, double eta) {
    Ang a;
    double X = std::tan(xi), Y = std::tan(eta), d = 1 + X * X + Y * Y, sd = std::sqrt(d);
    a.sigma = (1 + X * X) * (1 + Y * Y) / (d * sd);
    a.a11 = (1 + Y * Y) / sd;
    a.a22 = (1 + X * X) / sd;
    a.a12 = X * Y / sd;
    double c1 = (1 + X * X) / (d * sd), c2 = (1 + Y * Y) / (d * sd);
    a.e1[0] = -X * c1, a.e1[1] = (1 + Y * Y) * c1, a.e1[2] = -X * Y * c1;
    a.e2[0] = -Y * c2, a.e2[1] = -X * Y * c2, a.e2[2] = (1 + X * X) * c2;
    a.xh[0] = 1 / sd, a.xh[1] = X / sd, a.xh[2] = Y / sd;
    return a;
  };

  std::vector<double> ax11(Ns * (Ns + 1)), ax12(Ns * (Ns + 1)), ay22((Ns + 1) * Ns), ay12((Ns + 1) * Ns);
  std::vector<double> sx(3 * Ns * (Ns + 1)), sy(3 * (Ns + 1) * Ns), sr(3 * Ns * Ns), xhat(3 * Ns * Ns);
  std::vector<double> crf(Ns * Ns), invsig(Ns * Ns), rf2(Nr + 1), invr2(Nr), rc(Nr), cbasis(6 * Ns * Ns);
  for (int j = 0; j < Ns; ++j)
    for (int f = 0; f <= Ns; ++f) {
      Ang a = ang(xf(f), xc(j));
      int id = j * (Ns + 1) + f;
      ax11[id] = a.a11 * hr;
      ax12[id] = a.a12 * hr / 4;
      for (int c = 0; c < 3; ++c) sx[3 * id + c] = (a.a11 * a.e1[c] + a.a12 * a.e2[c]) * hs * hr;
    }
  for (int f = 0; f <= Ns; ++f)
    for (int i = 0; i < Ns; ++i) {
      Ang a = ang(xc(i), xf(f));
      int id = f * Ns + i;
      ay22[id] = a.a22 * hr;
      ay12[id] = a.a12 * hr / 4;
      for (int c = 0; c < 3; ++c) sy[3 * id + c] = (a.a12 * a.e1[c] + a.a22 * a.e2[c]) * hs * hr;
    }
  for (int j = 0; j < Ns; ++j)
    for (int i = 0; i < Ns; ++i) {
      Ang a = ang(xc(i), xc(j));
      int id = j * Ns + i;
      crf[id] = a.sigma * hs * hs / hr;
      invsig[id] = 1.0 / a.sigma;
      for (int c = 0; c < 3; ++c) {
        xhat[3 * id + c] = a.xh[c];
        sr[3 * id + c] = a.sigma * hs * hs * a.xh[c];
        // contravariant basis r grad(xi), r grad(eta) = (sqrt(g) g^{1b} e_b) / sigma on the unit sphere
        cbasis[6 * id + c] = (a.a11 * a.e1[c] + a.a12 * a.e2[c]) / a.sigma;
        cbasis[6 * id + 3 + c] = (a.a12 * a.e1[c] + a.a22 * a.e2[c]) / a.sigma;
      }
    }
  for (int k = 0; k <= Nr; ++k) {
    double r = h.ri + k * hr;
    rf2[k] = r * r;
  }
  for (int k = 0; k < Nr; ++k) {
    rc[k] = h.ri + (k + 0.5) * hr;
    invr2[k] = 1.0 / (rc[k] * rc[k] * hs * hs * hr);
  }

  // 9-point horizontal weights of F(j, i+1) - F(j, i) + G(j+1, i) - G(j, i) (face fluxes of the Laplacian
  // with F(j, f) = ax11 (x[j][f] - x[j][f-1]) + ax12 (x[j+1][f-1] - x[j-1][f-1] + x[j+1][f] - x[j-1][f]) and
  // G likewise with ay22, ay12 and the roles of i and j exchanged).  A face on a panel edge is left out: its
  // flux is the mean of the two panels' one-sided fluxes, added separately.
  std::vector<double> w9(9 * Ns * Ns, 0.0);
  for (int j = 0; j < Ns; ++j)
    for (int i = 0; i < Ns; ++i) {
      double* w = &w9[9 * (j * Ns + i)];
      auto W = [&](int dj, int di) -> double& { return w[(dj + 1) * 3 + (di + 1)]; };
      if (i + 1 < Ns) {  // + F(j, i+1)
        const double a = ax11[j * (Ns + 1) + i + 1], b = ax12[j * (Ns + 1) + i + 1];
        W(0, 1) += a, W(0, 0) -= a, W(1, 0) += b, W(-1, 0) -= b, W(1, 1) += b, W(-1, 1) -= b;
      }
      if (i > 0) {  // - F(j, i)
        const double a = ax11[j * (Ns + 1) + i], b = ax12[j * (Ns + 1) + i];
        W(0, 0) -= a, W(0, -1) += a, W(1, -1) -= b, W(-1, -1) += b, W(1, 0) -= b, W(-1, 0) += b;
      }
      if (j + 1 < Ns) {  // + G(j+1, i)
        const double c = ay22[(j + 1) * Ns + i], e = ay12[(j + 1) * Ns + i];
        W(1, 0) += c, W(0, 0) -= c, W(0, 1) += e, W(0, -1) -= e, W(1, 1) += e, W(1, -1) -= e;
      }
      if (j > 0) {  // - G(j, i)
        const double c = ay22[j * Ns + i], e = ay12[j * Ns + i];
        W(0, 0) -= c, W(-1, 0) += c, W(-1, 1) -= e, W(-1, -1) += e, W(0, 1) -= e, W(0, -1) += e;
      }
    }

  // panel-edge ghost interpolation and face pairing, from the geometry
  h.gq.assign(6 * 4 * Ns, 0);
  h.gsrc.assign(6 * 4 * Ns * 3, 0);
  h.gw.assign(6 * 4 * Ns * 3, 0.0);
  h.pq.assign(24, 0), h.psq.assign(24, 0), h.psgn.assign(24, 0);
  h.ptmap.assign(6 * 4 * Ns, 0);
  const double lim = M_PI / 4 - hs / 2;
  for (int p = 0; p < 6; ++p)
    for (int side = 0; side < 4; ++side) {
      int q_prev = -1, sq_prev = -1;
      for (int t = 0; t < Ns; ++t) {
        double xi, eta, v[3], w[3];
        side_point(side, xc(t), M_PI / 4 + hs / 2, &xi, &eta);
        to_cart(p, xi, eta, v);
        int q = which_panel(v);
        to_local(q, v, w);
        double xq = std::atan(w[1] / w[0]), yq = std::atan(w[2] / w[0]);
        int sq;
        double tau;
        if (std::fabs(xq + lim) < 1e-9) sq = XI_MIN, tau = yq;
        else if (std::fabs(xq - lim) < 1e-9) sq = XI_MAX, tau = yq;
        else if (std::fabs(yq + lim) < 1e-9) sq = ETA_MIN, tau = xq;
        else if (std::fabs(yq - lim) < 1e-9) sq = ETA_MAX, tau = xq;
        else {
          delete g;
          return set_error("fv_build_grid: ghost centre off the neighbour grid line"), FV_EINVAL;
        }
        if (q == p || (q_prev >= 0 && (q != q_prev || sq != sq_prev))) {
          delete g;
          return set_error("fv_build_grid: inconsistent panel-edge pairing"), FV_EINVAL;
        }
        q_prev = q, sq_prev = sq;
        double frac = (tau + M_PI / 4) / hs - 0.5;
        int c = (int)std::lround(frac);
        c = c < 1 ? 1 : (c > Ns - 2 ? Ns - 2 : c);
        double s = frac - c;
        double wts[3] = {0.5 * s * (s - 1.0), 1.0 - s * s, 0.5 * s * (s + 1.0)};
        int n0 = (sq == XI_MIN || sq == ETA_MIN) ? 0 : Ns - 1;
        int id = (p * 4 + side) * Ns + t;
        h.gq[id] = q;
        for (int m = 0; m < 3; ++m) {
          int a = c + m - 1;
          int jj = (sq == XI_MIN || sq == XI_MAX) ? a : n0;
          int ii = (sq == XI_MIN || sq == XI_MAX) ? n0 : a;
          h.gsrc[3 * id + m] = jj * Ns + ii;
          h.gw[3 * id + m] = wts[m];
        }
        // the face centre on the edge: its tangential index on q
        side_point(side, xc(t), M_PI / 4, &xi, &eta);
        to_cart(p, xi, eta, v);
        to_local(q, v, w);
        double ft = (sq == XI_MIN || sq == XI_MAX) ? std::atan(w[2] / w[0]) : std::atan(w[1] / w[0]);
        double tf = (ft + M_PI / 4) / hs - 0.5;
        h.ptmap[id] = (int)std::lround(tf);
      }
      int sp = (side == XI_MAX || side == ETA_MAX) ? 1 : -1;
      int sqq = (sq_prev == XI_MAX || sq_prev == ETA_MAX) ? 1 : -1;
      h.pq[p * 4 + side] = q_prev, h.psq[p * 4 + side] = sq_prev, h.psgn[p * 4 + side] = -sp * sqq;
    }

  // the face area vectors of every panel in Cartesian components (the panel rotations have entries in
  // {-1, 0, 1}, so these are the local components permuted and signed, exactly), for the FP64 face kernels
  static const int kRot[6][9] = {
      {1, 0, 0, 0, 1, 0, 0, 0, 1},  {0, -1, 0, 1, 0, 0, 0, 0, 1}, {-1, 0, 0, 0, -1, 0, 0, 0, 1},
      {0, 1, 0, -1, 0, 0, 0, 0, 1}, {0, 0, -1, 0, 1, 0, 1, 0, 0}, {0, 0, 1, 0, 1, 0, -1, 0, 0},
  };
  auto per_panel = [&](const std::vector<double>& l) {
    const size_t n = l.size() / 3;
    std::vector<double> out(6 * l.size());
    for (int p = 0; p < 6; ++p)
      for (size_t e = 0; e < n; ++e)
        for (int a = 0; a < 3; ++a) {
          double v = 0.0;
          for (int b = 0; b < 3; ++b)
            if (kRot[p][3 * a + b]) v = kRot[p][3 * a + b] > 0 ? l[3 * e + b] : -l[3 * e + b];
          out[(p * n + e) * 3 + a] = v;
        }
    return out;
  };
  const std::vector<double> sxp = per_panel(sx), syp = per_panel(sy), srp = per_panel(sr);

  Geo& G = g->geo;
  G.Ns = Ns, G.Nr = Nr, G.N = h.N, G.hs = hs, G.hr = hr, G.ri = h.ri, G.ro = h.ro;
  double rci = h.ri + 0.5 * hr, rgi = h.ri - 0.5 * hr, rco = h.ro - 0.5 * hr, rgo = h.ro + 0.5 * hr;
  G.wall_in = 1.0 + (rci / rgi) * (rci / rgi);
  G.wall_out = 1.0 + (rco / rgo) * (rco / rgo);
  bool ok = (G.ax11 = upload(g, ax11)) && (G.ax12 = upload(g, ax12)) && (G.ay22 = upload(g, ay22)) &&
            (G.ay12 = upload(g, ay12)) && (G.crf = upload(g, crf)) && (G.rf2 = upload(g, rf2)) &&
            (G.invsig = upload(g, invsig)) && (G.invr2 = upload(g, invr2)) && (G.rc = upload(g, rc)) &&
            (G.xhat = upload(g, xhat)) && (G.sx = upload(g, sx)) && (G.sy = upload(g, sy)) &&
            (G.sr = upload(g, sr)) && (G.sxp = upload(g, sxp)) && (G.syp = upload(g, syp)) &&
            (G.srp = upload(g, srp)) && (G.gq = upload(g, h.gq)) && (G.gsrc = upload(g, h.gsrc)) &&
            (G.gw = upload(g, h.gw)) && (G.pq = upload(g, h.pq)) && (G.psq = upload(g, h.psq)) &&
            (G.psgn = upload(g, h.psgn)) && (G.ptmap = upload(g, h.ptmap)) && (g->cbasis = upload(g, cbasis)) &&
            (G.w9 = upload(g, w9));
  if (ok) {
    Geo* dself = nullptr;
    if (cudaMalloc(&dself, sizeof(Geo)) != cudaSuccess) ok = false;
    else {
      g->allocs.push_back(dself);
      G.self = dself;
      ok = cudaMemcpy(dself, &G, sizeof(Geo), cudaMemcpyHostToDevice) == cudaSuccess;
    }
  }
  // FP32 copy of the tables for the mixed-precision inner solves
  auto f32 = [](const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); };
  GeoF& F = g->geof;
  F.Ns = Ns, F.Nr = Nr, F.N = h.N, F.hs = (float)hs, F.hr = (float)hr, F.ri = (float)h.ri, F.ro = (float)h.ro;
  F.wall_in = (float)G.wall_in, F.wall_out = (float)G.wall_out;
  F.gq = G.gq, F.gsrc = G.gsrc, F.pq = G.pq, F.psq = G.psq, F.psgn = G.psgn, F.ptmap = G.ptmap;
  ok = ok && (F.ax11 = upload(g, f32(ax11))) && (F.ax12 = upload(g, f32(ax12))) && (F.ay22 = upload(g, f32(ay22))) &&
       (F.ay12 = upload(g, f32(ay12))) && (F.crf = upload(g, f32(crf))) && (F.rf2 = upload(g, f32(rf2))) &&
       (F.invsig = upload(g, f32(invsig))) && (F.invr2 = upload(g, f32(invr2))) && (F.rc = upload(g, f32(rc))) &&
       (F.xhat = upload(g, f32(xhat))) && (F.sx = upload(g, f32(sx))) && (F.sy = upload(g, f32(sy))) &&
       (F.sr = upload(g, f32(sr))) && (F.gw = upload(g, f32(h.gw))) && (F.w9 = upload(g, f32(w9)));
  if (ok) {
    GeoF* dself = nullptr;
    if (cudaMalloc(&dself, sizeof(GeoF)) != cudaSuccess) ok = false;
    else {
      g->allocs.push_back(dself);
      F.self = dself;
      ok = cudaMemcpy(dself, &F, sizeof(GeoF), cudaMemcpyHostToDevice) == cudaSuccess;
    }
  }
  if (!ok) {
    free_grid(g);
    return set_error("fv_build_grid: device allocation of geometry tables failed"), FV_ENOMEM;
  }
  if (fv_status rc = build_edge_table(g)) {
    free_grid(g);
    return rc;
  }
  *out = g;
  return FV_OK;
}

void free_grid(fv_grid* g) {
  if (!g) return;
  if (g->coarse) free_grid(g->coarse);
  for (void* p : g->allocs) cudaFree(p);
  delete g;
}

}  // namespace fv
