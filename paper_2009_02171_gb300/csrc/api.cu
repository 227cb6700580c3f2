// C ABI entry points of libfv (declared in include/fv.h).
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fv_net.h"
#include "fv_internal.h"

namespace fv {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

fv_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? FV_ENOMEM : FV_ECUDA;
}

static void free_system(fv_system* s) {
  if (!s) return;
  if (s->inner_graph) cudaGraphExecDestroy(s->inner_graph);
  if (s->coarse) free_system(s->coarse);
  free_krylov(s->kry);
  free_batch(s->batch);
  for (void* p : s->allocs) cudaFree(p);
  delete s;
}

static fv_status make_system(const fv_grid* g, int kind, const fv_phys* ph, const fv_pc_desc* pc, fv_system** out) {
  if (pc->inner_gs_passes < 0 || pc->inner_gs_passes > 2)
    return set_error("fv_assemble_system: inner_gs_passes must be 0, 1 or 2"), FV_EINVAL;
  if (pc->levels < 1 || pc->levels > 6) return set_error("fv_assemble_system: levels must be 1..6"), FV_EINVAL;
  if (pc->cp1 < 0 || pc->cp2 < 0 || pc->cp3 < 0)
    return set_error("fv_assemble_system: coarse box splits must be >= 0"), FV_EINVAL;
  if (pc->precision < FV_PREC_FP64 || pc->precision > FV_PREC_BF16)
    return set_error("fv_assemble_system: precision must be FV_PREC_FP64, FV_PREC_FP32 or FV_PREC_BF16"), FV_EINVAL;
  fv_system* s = new fv_system();
  s->grid = g, s->kind = kind, s->d = kind == FV_VTBE ? 7 : 2;
  s->n = s->d * g->h.N;
  s->phys = *ph, s->pc = *pc;
  s->prec32 = pc->precision != FV_PREC_FP64;
  fv_status rc = FV_OK;
  const size_t ng = (size_t)s->d * 6 * 4 * g->h.Nr * (g->h.Ns + 2);
  if (cudaMalloc(&s->ghost, ng * sizeof(double)) != cudaSuccess) {
    delete s;
    return set_error("fv_assemble_system: ghost layer allocation failed"), FV_ENOMEM;
  }
  s->allocs.push_back(s->ghost);
  if (s->prec32) {
    if (pc->inner_maxit < 1 || pc->inner_maxit > 31 || (pc->levels >= 2 && (pc->coarse_maxit < 1 || pc->coarse_maxit > 31))) {
      free_system(s);
      return set_error("fv_assemble_system: mixed precision needs inner_maxit and coarse_maxit in [1, 31]"),
             FV_EINVAL;
    }
    if (cudaMalloc(&s->ghost32, ng * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&s->r32, s->n * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&s->x32, s->n * sizeof(float)) != cudaSuccess) {
      free_system(s);
      return set_error("fv_assemble_system: FP32 work allocation failed"), FV_ENOMEM;
    }
    s->allocs.insert(s->allocs.end(), {s->ghost32, s->r32, s->x32});
  }
  if ((rc = build_subdomains(s, g)) || (rc = assemble_subdomains(s)) || (rc = ilu_factor(s)) ||
      (rc = prepare_sweeps(s, pc->precision == FV_PREC_BF16 ? 2 : s->prec32)) || (rc = sweeps_smem_attr(s))) {
    free_system(s);
    return rc;
  }
  if (pc->levels >= 2) {
    if (g->h.Ns % 2 || g->h.Nr % 2 || g->h.Ns < 8 || g->h.Nr < 4) {
      free_system(s);
      return set_error("fv_assemble_system: two levels need even Ns >= 8 and even Nr >= 4"), FV_EINVAL;
    }
    fv_grid* gm = const_cast<fv_grid*>(g);
    if (!gm->coarse) {
      fv_grid_desc cd{g->h.Ns / 2, g->h.Nr / 2, g->h.ri, g->h.ro};
      if ((rc = build_grid(&cd, &gm->coarse))) {
        free_system(s);
        return rc;
      }
    }
    // multilevel hybrid RAS (Sec. 3.3): the coarse system's own preconditioner is the same construction
    // with one level fewer, down to one-level RAS on the coarsest mesh
    fv_pc_desc cpc = *pc;
    cpc.levels = pc->levels - 1;
    cpc.overlap = pc->overlap_coarse;
    cpc.p1 = std::min(pc->cp1 > 0 ? pc->cp1 : pc->p1, g->h.Ns / 2);
    cpc.p2 = std::min(pc->cp2 > 0 ? pc->cp2 : pc->p2, g->h.Ns / 2);
    cpc.p3 = std::min(pc->cp3 > 0 ? pc->cp3 : pc->p3, g->h.Nr / 2);
    std::vector<int> cboxes;
    if (pc->nboxes > 0) {  // the coarse level uses the halved boxes (bounds must be even)
      for (int q = 0; q < 7 * pc->nboxes; ++q) {
        if (q % 7 && pc->boxes[q] % 2) {
          free_system(s);
          return set_error("fv_assemble_system: two levels need even box bounds"), FV_EINVAL;
        }
        cboxes.push_back(q % 7 ? pc->boxes[q] / 2 : pc->boxes[q]);
      }
      cpc.boxes = cboxes.data();
    }
    if ((rc = make_system(gm->coarse, kind, ph, &cpc, &s->coarse))) {
      free_system(s);
      return rc;
    }
    s->coarse->level = 1;
    const size_t n = (size_t)s->n, nc = (size_t)s->coarse->n;
    if (cudaMalloc(&s->xc, nc * sizeof(double)) != cudaSuccess || cudaMalloc(&s->ec, nc * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&s->w, n * sizeof(double)) != cudaSuccess || cudaMalloc(&s->t, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&s->red, (32 * 304 + 32) * sizeof(double)) != cudaSuccess) {
      free_system(s);
      return set_error("fv_assemble_system: two-level work allocation failed"), FV_ENOMEM;
    }
    s->allocs.insert(s->allocs.end(), {s->xc, s->ec, s->w, s->t, s->red});
    if (s->prec32) {
      if (cudaMalloc(&s->xc32, nc * sizeof(float)) != cudaSuccess ||
          cudaMalloc(&s->ec32, nc * sizeof(float)) != cudaSuccess ||
          cudaMalloc(&s->w32, n * sizeof(float)) != cudaSuccess || cudaMalloc(&s->t32, n * sizeof(float)) != cudaSuccess) {
        free_system(s);
        return set_error("fv_assemble_system: FP32 two-level work allocation failed"), FV_ENOMEM;
      }
      s->allocs.insert(s->allocs.end(), {s->xc32, s->ec32, s->w32, s->t32});
    }
  }
  FV_CUDA(cudaDeviceSynchronize());
  *out = s;
  return FV_OK;
}

}  // namespace fv

using namespace fv;

extern "C" {

const char* fv_last_error(void) { return g_err.c_str(); }

fv_status fv_build_grid(const fv_grid_desc* desc, fv_grid** out) { return build_grid(desc, out); }

fv_status fv_free_grid(fv_grid* g) {
  free_grid(g);
  return FV_OK;
}

fv_status fv_grid_cells(const fv_grid* g, long long* n) {
  if (!g || !n) return set_error("fv_grid_cells: null argument"), FV_EINVAL;
  *n = g->h.N;
  return FV_OK;
}

fv_status fv_assemble_system(const fv_grid* g, int kind, const fv_phys* phys, const fv_pc_desc* pc, fv_system** out) {
  if (!g || !phys || !pc || !out || (kind != FV_VTBE && kind != FV_PPBE))
    return set_error("fv_assemble_system: bad argument"), FV_EINVAL;
  if (!(phys->dt > 0) || !(phys->E > 0) || !(phys->Pr > 0) || !(phys->Pm > 0))
    return set_error("fv_assemble_system: E, Pr, Pm, dt must be positive"), FV_EINVAL;
  return make_system(g, kind, phys, pc, out);
}

fv_status fv_free_system(fv_system* s) {
  free_system(s);
  return FV_OK;
}

fv_status fv_system_size(const fv_system* s, long long* n) {
  if (!s || !n) return set_error("fv_system_size: null argument"), FV_EINVAL;
  *n = s->n;
  return FV_OK;
}

fv_status fv_apply_op(const fv_system* s, const double* x, double* y, void* stream) {
  if (!s || !x || !y || x == y) return set_error("fv_apply_op: bad argument"), FV_EINVAL;
  return apply_op(s, x, y, (cudaStream_t)stream);
}

fv_status fv_apply_op_noalloc(const fv_system* s, const double* x, double* y, void* stream) {
  if (!s || !x || !y || x == y) return set_error("fv_apply_op_noalloc: bad argument"), FV_EINVAL;
  return apply_op_noalloc(s, x, y, (cudaStream_t)stream);
}

fv_status fv_precond_apply(const fv_system* s, const double* r, double* z, void* stream) {
  if (!s || !r || !z || r == z) return set_error("fv_precond_apply: bad argument"), FV_EINVAL;
  s->last_inner = 0;
  return precond_apply(s, r, z, (cudaStream_t)stream);
}

fv_status fv_gmres_solve(const fv_system* s, const double* b, double* x, const fv_gmres_opts* opts,
                         fv_solve_stats* stats, void* stream) {
  if (!s || !b || !x || !opts || b == x) return set_error("fv_gmres_solve: bad argument"), FV_EINVAL;
  return gmres(s, b, x, opts, stats, (cudaStream_t)stream, false);
}

fv_status fv_coarse_system(const fv_system* s, const fv_system** coarse) {
  if (!s || !coarse) return set_error("fv_coarse_system: null argument"), FV_EINVAL;
  if (!s->coarse) return set_error("fv_coarse_system: the system has one level"), FV_EINVAL;
  *coarse = s->coarse;
  return FV_OK;
}

fv_status fv_restrict_coarse(const fv_system* s, const double* x, double* xc, void* stream) {
  if (!s || !x || !xc) return set_error("fv_restrict_coarse: null argument"), FV_EINVAL;
  if (!s->coarse) return set_error("fv_restrict_coarse: the system has one level"), FV_EINVAL;
  return restrict_coarse(s, x, xc, (cudaStream_t)stream);
}

fv_status fv_prolong_coarse(const fv_system* s, const double* xc, double* x, void* stream) {
  if (!s || !xc || !x || xc == x) return set_error("fv_prolong_coarse: bad argument"), FV_EINVAL;
  if (!s->coarse) return set_error("fv_prolong_coarse: the system has one level"), FV_EINVAL;
  return prolong_inject(s->grid, s->d, xc, x, (cudaStream_t)stream);
}

fv_status fv_pc_set_learned(fv_system* s, fv_net* net, int coarse_its, int flags) {
  if (!s) return set_error("fv_pc_set_learned: null system"), FV_EINVAL;
  if (!net) {
    set_learned_active(s, 0);
    s->net = nullptr;
    return FV_OK;
  }
  if (s->kind != FV_PPBE || !s->coarse) return set_error("fv_pc_set_learned: needs a two-level PPBE system"), FV_EINVAL;
  if (!net_matches(net, s->coarse->grid))
    return set_error("fv_pc_set_learned: the network's grid differs from the coarse grid"), FV_EINVAL;
  if (coarse_its < 0 || coarse_its > 31 || (flags & ~FV_LEARN_GUESS))
    return set_error("fv_pc_set_learned: coarse_its must be in [0, 31], flags in {0, FV_LEARN_GUESS}"), FV_EINVAL;
  if (!s->xbak) {
    if (cudaMalloc(&s->xbak, s->n * sizeof(double)) != cudaSuccess)
      return set_error("fv_pc_set_learned: allocation failed"), FV_ENOMEM;
    s->allocs.push_back(s->xbak);
  }
  if (s->prec32 && !s->tc32) {
    const size_t nc = (size_t)s->coarse->n;
    if (cudaMalloc(&s->tc32, nc * sizeof(float)) != cudaSuccess) return set_error("fv_pc_set_learned: allocation failed"), FV_ENOMEM;
    s->allocs.push_back(s->tc32);
    if (cudaMalloc(&s->dc32, nc * sizeof(float)) != cudaSuccess) return set_error("fv_pc_set_learned: allocation failed"), FV_ENOMEM;
    s->allocs.push_back(s->dc32);
  }
  set_learned_active(s, 0);
  s->net = net, s->learned_its = coarse_its, s->learned_flags = flags;
  set_learned_active(s, 1);
  return FV_OK;
}

}  // extern "C"
