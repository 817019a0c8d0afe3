// complex128 instantiation: Helmholtz, EFIE2D (Hankel), low-rank and dense generators.
#include "pipeline.cuh"
#include "run.h"

namespace hbaca {

cudaError_t run_c128(Plan& p, RunCtx& rc, std::string& err) {
  const hbaca_gen& g = p.gens[0];
  cudaError_t e = cudaErrorInvalidValue;
  switch (g.kind) {
    case HBACA_GEN_DENSE: {
      GenDenseC gd{reinterpret_cast<const cplx*>(g.a), g.lda};
      e = run_baca(p, gd, rc, err);
      break;
    }
    case HBACA_GEN_HELMHOLTZ: {
      GenHelmholtz gh{g.x, g.y, g.dim, g.k / 3.14159265358979323846};
      e = run_baca(p, gh, rc, err);
      break;
    }
    case HBACA_GEN_LOWRANK: {
      GenLowRankC gl{reinterpret_cast<const cplx*>(g.lu), reinterpret_cast<const cplx*>(g.lv), g.m, g.n, g.lr};
      e = run_baca(p, gl, rc, err);
      break;
    }
    case HBACA_GEN_HANKEL2D: {
      GenHankel2D gk{g.x, g.y, g.dim, g.k};
      e = run_baca(p, gk, rc, err);
      break;
    }
    default:
      err = "generator kind not available for complex128";
      return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  if (rc.baca_only) return cudaSuccess;
  return run_stages<cplx>(p, rc, err);
}

}  // namespace hbaca
