// float64 instantiation: Gaussian, polynomial, sparse-product, low-rank and dense generators.
#include "pipeline.cuh"
#include "run.h"

namespace hbaca {

cudaError_t run_f64(Plan& p, RunCtx& rc, std::string& err) {
  const hbaca_gen& g = p.gens[0];
  cudaError_t e = cudaErrorInvalidValue;
  switch (g.kind) {
    case HBACA_GEN_DENSE: {
      GenDense gd{reinterpret_cast<const double*>(g.a), g.lda};
      e = run_baca(p, gd, rc, err);
      break;
    }
    case HBACA_GEN_GAUSSIAN: {  // one block or many: per-block points and widths
      GenGaussianBatch gg{reinterpret_cast<const GaussBlockParams*>(rc.ws + p.desc_region.off + p.gparams_off)};
      e = run_baca(p, gg, rc, err);
      break;
    }
    case HBACA_GEN_SPARSE_PRODUCT: {
      GenSparseProduct gs{g.p_rowptr, g.p_colidx, g.p_val, g.q_colptr, g.q_rowidx, g.q_val, g.p2, g.q2, g.n, g.r2};
      e = run_baca(p, gs, rc, err);
      break;
    }
    case HBACA_GEN_LOWRANK: {
      GenLowRank gl{reinterpret_cast<const double*>(g.lu), reinterpret_cast<const double*>(g.lv), g.m, g.n, g.lr};
      e = run_baca(p, gl, rc, err);
      break;
    }
    case HBACA_GEN_POLYNOMIAL: {
      GenPolynomial gp{g.x, g.y, g.dim, g.h};
      e = run_baca(p, gp, rc, err);
      break;
    }
    default:
      err = "generator kind not available for float64";
      return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  if (rc.baca_only) return cudaSuccess;
  return run_stages<double>(p, rc, err);
}

}  // namespace hbaca
