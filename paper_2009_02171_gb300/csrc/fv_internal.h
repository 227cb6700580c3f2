// Internal types of libfv: device geometry tables, systems, error plumbing.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/fv.h"

namespace fv {

// panel sides: 0 = xi-min, 1 = xi-max, 2 = eta-min, 3 = eta-max
enum { XI_MIN = 0, XI_MAX = 1, ETA_MIN = 2, ETA_MAX = 3 };
// wall rules of the ghost at the mirror radius (radial direction)
enum { WALL_ODD = 0, WALL_EVEN = 1, WALL_B = 2 };

// Device-side geometry of one grid level, passed by value to kernels.
// Angular tables are shared by the 6 panels (identical local coordinates);
// Cartesian vectors are stored in the panel-local frame (1, X, Y) and rotated
// by the panel's signed-permutation matrix in the kernels.  R is the type of
// the coefficient tables and of the coefficient arithmetic: double for the
// FP64 path, float for the FP32 inner solves of mixed precision.
template <class R>
struct GeoT {
  using real = R;
  int Ns, Nr;
  long long N;                 // 6 Ns^2 Nr
  R hs, hr, ri, ro;
  R wall_in, wall_out;         // 1 + (r_c/r_g)^2 at the inner / outer wall
  const R* ax11;               // [j][if]  a11 * h_r            (xi faces, Ns x (Ns+1))
  const R* ax12;               // [j][if]  a12 * h_r / 4
  const R* ay22;               // [jf][i]  a22 * h_r            (eta faces, (Ns+1) x Ns)
  const R* ay12;               // [jf][i]  a12 * h_r / 4
  const R* crf;                // [j][i]   sigma h_s^2 / h_r    (radial faces, times r_f^2)
  const R* rf2;                // [kf]     r_f^2
  const R* invsig;             // [j][i]   1 / sigma
  const R* invr2;              // [k]      1 / (r_k^2 h_s^2 h_r)
  const R* rc;                 // [k]      r_k
  const R* xhat;               // [j][i][3] unit position vector, local frame
  const R* sx;                 // [j][if][3] (a11 e1 + a12 e2) h_s h_r, local frame (times r_k)
  const R* sy;                 // [jf][i][3] (a12 e1 + a22 e2) h_s h_r
  const R* sr;                 // [j][i][3]  sigma h_s^2 xhat     (times r_f^2)
  const R* sxp;                // [p][j][if][3] sx in Cartesian components of panel p (FP64 tables only)
  const R* syp;                // [p][jf][i][3]
  const R* srp;                // [p][j][i][3]
  const int* gq;               // [p][side][t]      panel holding the ghost's source line
  const int* gsrc;             // [p][side][t][3]   source cells (j*Ns + i) on that panel
  const R* gw;                 // [p][side][t][3]   quadratic Lagrange weights
  const int* pq;               // [p][side]  neighbour panel across the side
  const int* psq;              // [p][side]  its side
  const int* psgn;             // [p][side]  F_p = psgn F_q for the shared face
  const int* ptmap;            // [p][side][t] tangential index on the neighbour side
  const R* w9;                 // [j][i][9] horizontal 9-point weights of sum_faces F (panel-edge faces left out),
                               // index (dj + 1) * 3 + (di + 1)
  const GeoT* self;            // device copy of this struct (out-of-line device code reads it
                               // through this pointer so kernels never take a parameter's address)
};
using Geo = GeoT<double>;
using GeoF = GeoT<float>;

struct GridHost {
  int Ns, Nr;
  double ri, ro, hs, hr;
  long long N;
  // host copies of the tables needed by host setup code
  std::vector<int> gq, gsrc, pq, psq, psgn, ptmap;
  std::vector<double> gw;
};

struct Krylov;
struct BatchWork;

}  // namespace fv

struct fv_net;

struct fv_grid {
  fv::GridHost h;
  fv::Geo geo;                 // device pointers (FP64 tables)
  fv::GeoF geof;               // the same tables in FP32 (mixed-precision inner solves)
  std::vector<void*> allocs;   // device allocations owned by the grid
  fv_grid* coarse = nullptr;   // (Ns/2, Nr/2) grid, built on demand
  double* cbasis = nullptr;    // [j][i][6] r grad(xi), r grad(eta) at cell centres, local frame (diagnostics)
  // panel-edge face fluxes as linear combinations of cell values of one level (apply.cu), per face
  // (p, side, t): term count, then (cell offset within the level, weight) slots
  int* edge_cnt = nullptr;
  int* edge_off = nullptr;
  double* edge_w = nullptr;
  float* edge_wf = nullptr;
};

namespace fv {

// structured ILU(0) subdomain set of one system on one grid level
struct Subdomains {
  int count = 0;
  int d = 0;
  long long total_cells = 0;      // sum of box cells
  int max_levels = 0;
  // device arrays
  long long* cell_off = nullptr;  // [count+1] offsets into the packed per-cell arrays
  int* dims = nullptr;            // [count][3] nx, ny, nz
  long long* gmap = nullptr;      // [total_cells] global cell or -1 (hole)
  unsigned char* owned = nullptr; // [total_cells]
  int* level_off = nullptr;       // [count][max_levels+1] offsets into `order` (relative to cell_off)
  int* order = nullptr;           // [total_cells] local cells sorted by level (i + 2 j + k)
  double* off = nullptr;          // [total_cells][11][d] structured coefficients (slot 5 unused)
  double* diag = nullptr;         // [total_cells][d][d] diagonal blocks (LU in place)
  int* status = nullptr;          // [1] 0 ok, else 1 + first zero-pivot cell
  int* lpt = nullptr;             // [count] subdomains in decreasing size (processing order)
  // sweep layout (built after factorization): per subdomain, cells in wavefront
  // order (level i + 2j + k, then j, then i), structure of arrays
  int* perm = nullptr;            // [total_cells] natural local index -> packed position (setup only)
  long long* gmap_p = nullptr;    // [total_cells] packed: global cell or -1
  int* ijk = nullptr;             // [total_cells] packed: box cell (i | j << 10 | k << 20)
  unsigned char* owned_p = nullptr;
  void* F = nullptr;              // [cell_off * Q + q * ncell + pos], Q = 10 d + d^2, element type per `fp32`
  void* loc = nullptr;            // [cell_off * d + a * ncell + pos] sweep vector
  void* ring = nullptr;           // global 4-plane ring per CTA when it does not fit in shared memory
  int fp32 = 0;                   // 1: sweeps in FP32 (factors FP32, or BF16 when bf16)
  int bf16 = 0;                   // 1: factors stored in BF16 (FV_PREC_BF16)
  int max_cols = 0;               // max nx * ny
  int dense_threads = 0;          // CTA size of the level-mapped generic sweeps
  int dense_single = 0;           // 1: no step is wider than the CTA (the pipelined sweeps apply)
  size_t smem = 0;                // dynamic shared memory of the sweeps
  int ring_in_smem = 0;
  int stage = 0;                  // d = 2: depth of the shared-memory staged sweeps (8 or 4), 0 = not used
  size_t stage_off = 0;           // offset of the stage ring in dynamic shared memory
  int stage_pad = 0;              // zero padding (elements) on each side of the staged sweeps' 4-plane ring
  size_t stage_smem = 0;          // dynamic shared memory of the staged sweeps
  void* blk_f = nullptr;          // [total_cells] staged sweeps: forward operand block per packed position
  void* blk_b = nullptr;          // [total_cells] staged sweeps: backward operand block per packed position
};

}  // namespace fv

// time-stepping state of fv_state_create / fv_time_step (timestep.cu, diag.cu)
struct fv_state {
  const fv_grid* grid = nullptr;
  fv_phys phys{};
  long long N = 0;
  bool first = true;                    // next step is a first step (no history)
  long long steps = 0;                  // steps since create / reset
  double *X = nullptr;                  // [9N] u, Theta, B, P, P_b
  double *fprev = nullptr, *fcur = nullptr, *fh = nullptr, *xhat = nullptr, *bV = nullptr, *tmp = nullptr;
  double *xV = nullptr;                 // [7N] last VTBE solution (u~, Theta, B~)
  double *bP = nullptr, *xP = nullptr;  // [2N] last PPBE right-hand side (D u~, D B~) and solution
  double *grad = nullptr;
  double *gh = nullptr;                 // 7-component ghost layer
  double *part = nullptr, *sums = nullptr;
  std::vector<void*> allocs;
};

struct fv_system {
  const fv_grid* grid = nullptr;
  int kind = 0, d = 0;
  long long n = 0;
  fv_phys phys{};
  fv_pc_desc pc{};
  double* ghost = nullptr;     // [d][6][4][Nr][Ns+2] ghost layer scratch
  fv::Subdomains subs;
  // two-level data
  fv_system* coarse = nullptr;
  double* xc = nullptr;        // coarse rhs
  double* ec = nullptr;        // coarse correction
  double* w = nullptr;         // fine prolongated correction / temps
  double* t = nullptr;
  double* red = nullptr;       // [32 * 304 + 32] reduction scratch (coarse mean projection)
  // mixed precision (pc.precision == FV_PREC_FP32)
  int prec32 = 0;
  float* ghost32 = nullptr;    // FP32 ghost layer
  float *r32 = nullptr, *x32 = nullptr;                  // inner solve right-hand side / solution
  float *xc32 = nullptr, *ec32 = nullptr, *w32 = nullptr, *t32 = nullptr;  // FP32 two-level work
  cudaGraphExec_t inner_graph = nullptr;  // captured inner solve (r32 -> x32)
  int inner_warm = 0;
  // FGMRES workspace for this system (outer) sized lazily
  fv::Krylov* kry = nullptr;
  fv::BatchWork* batch = nullptr;  // fv_gmres_solve_batch workspace
  mutable int last_inner = 0;
  int level = 0;               // 0 fine, 1 coarse (kernel timing category offset)
  // learned coarse correction (fv_net.h), borrowed network
  fv_net* net = nullptr;
  int learned_its = 0, learned_flags = 0;
  int learned_on = 0;          // 0 while a failed learned solve is finished by the plain one
  double* xbak = nullptr;      // [n] x0 of the top-level solve (fallback after NaN)
  float *tc32 = nullptr, *dc32 = nullptr;  // [coarse n] FP32 residual / correction of the coarse iterations
  std::vector<void*> allocs;
};

namespace fv {

void set_error(const std::string& msg);
fv_status cuda_fail(cudaError_t e, const char* what);

// profile.cu: event brackets around one launch (slot -1 when timing is off)
int prof_begin(int category, cudaStream_t st);
bool prof_enabled();
void prof_end(int slot, cudaStream_t st);
struct ProfScope {
  int slot;
  cudaStream_t st;
  ProfScope(int category, cudaStream_t s) : slot(prof_begin(category, s)), st(s) {}
  ~ProfScope() { prof_end(slot, st); }
};

#define FV_CUDA(call)                                        \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return fv::cuda_fail(e_, #call);  \
  } while (0)

// grid.cpp
fv_status build_edge_table(fv_grid* g);
fv_status build_grid(const fv_grid_desc* desc, fv_grid** out);
void free_grid(fv_grid* g);

// apply.cu (tiled operator apply), ops.cu
fv_status apply_op(const fv_system* s, const double* x, double* y, cudaStream_t st);
fv_status apply_op32(const fv_system* s, const float* x, float* y, cudaStream_t st);
fv_status apply_op_noalloc(const fv_system* s, const double* x, double* y, cudaStream_t st);
fv_status ghost_fill(const Geo& G, const double* x, double* gh, int d, cudaStream_t st);
fv_status assemble_subdomains(fv_system* s);
// glue kernels of the time step
fv_status nonlinear_terms(const fv_grid* g, const fv_phys& ph, const double* fields, double* f, double* gh7,
                          cudaStream_t st);
fv_status face_divergence_uB(const fv_grid* g, const double* x7, double* bP, double* gh7, cudaStream_t st);
fv_status cell_gradient(const fv_grid* g, const double* x, int wall, double scale, double* out3, double* gh,
                        cudaStream_t st);

// precond.cu
fv_status build_subdomains(fv_system* s, const fv_grid* g);
fv_status ilu_factor(fv_system* s);
fv_status prepare_sweeps(fv_system* s, int prec);
fv_status sweeps_smem_attr(const fv_system* s);
fv_status precond_apply(const fv_system* s, const double* r, double* z, cudaStream_t st);
fv_status precond_apply32(const fv_system* s, const float* r, float* z, cudaStream_t st);
fv_status ras_apply(const fv_system* s, const double* r, double* z, cudaStream_t st);
fv_status restrict_mean(const fv_grid* g, int d, const double* x, double* xc, cudaStream_t st);
fv_status prolong_inject(const fv_grid* g, int d, const double* xc, double* x, cudaStream_t st);
fv_status restrict_coarse(const fv_system* s, const double* x, double* xc, cudaStream_t st);
void set_learned_active(fv_system* s, int on);
fv_status learned_guess(const fv_system* s, const double* b, double* x, cudaStream_t st);

// nn.cu: learned coarse correction (one sample, coarse vectors in the system layout)
fv_status net_forward64(fv_net* n, const double* r, double* e, cudaStream_t st);
fv_status net_forward32(fv_net* n, const float* r, float* e, cudaStream_t st);
bool net_matches(const fv_net* n, const fv_grid* coarse);

// krylov.cu
fv_status gmres(const fv_system* s, const double* b, double* x, const fv_gmres_opts* o, fv_solve_stats* stats,
                cudaStream_t st, bool inner);
void free_krylov(Krylov* k);
void free_batch(BatchWork* b);
fv_status axpby(long long n, double a, const double* x, double b, const double* y, double* out, cudaStream_t st);
fv_status axpby32(long long n, double a, const float* x, double b, const float* y, float* out, cudaStream_t st);
fv_status to_fp32(long long n, const double* x, float* out, cudaStream_t st);
fv_status to_fp64(long long n, const float* x, double* out, cudaStream_t st);
fv_status gmres32(const fv_system* s, const float* b, float* x, const fv_gmres_opts* o, fv_solve_stats* stats,
                  cudaStream_t st);
fv_status gmres_fixed32(const fv_system* s, const float* b, float* x, int m, cudaStream_t st);
fv_status weighted_mean_remove32(const fv_grid* g, float* x, cudaStream_t st, double* part, double* sums);
fv_status weighted_mean_remove(const fv_grid* g, double* x, cudaStream_t st, double* part, double* sums);

}  // namespace fv
