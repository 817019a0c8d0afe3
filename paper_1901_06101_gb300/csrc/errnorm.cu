// Accuracy of a compression on the device: the squared Frobenius norms
// ||A(I,:) - U(I,:) diag(S) V||_F^2 and ||A(I,:)||_F^2 over a set of rows I
// (all rows, or a sample), the measure of the paper's accuracy study
// (Sec. 5.2: relative Frobenius error of the approximation).
//
// A is regenerated tile by tile from the entry generator; the product
// U diag(S) V of a 64 x 64 tile is accumulated in registers from 16-wide
// panels of U diag(S) and V staged in shared memory, then subtracted from the
// generated entries.  Persistent CTAs walk the tiles; every CTA leaves two
// partial sums and the host adds them in CTA order (a fixed order, so the
// result does not depend on scheduling).  This evaluator is separate from
// the compression kernels: it reads only the result factors and the
// generator.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "hbaca.h"
#include "hbaca_debug.h"
#include "run.h"

namespace hbaca {
namespace {

constexpr int kTile = 64;
constexpr int kPanel = 16;
constexpr int kErrThreads = 256;
constexpr int kErrCtasPerSm = 4;

template <typename Gen>
__global__ void __launch_bounds__(kErrThreads) errnorm_kernel(const Gen gen, const typename Gen::scalar* U, int64_t ldu,
                                                              const double* S, const typename Gen::scalar* V,
                                                              int64_t ldv, int r, const int64_t* rows, int64_t nrows,
                                                              int64_t n, double* part) {
  using T = typename Gen::scalar;
  __shared__ T Us[kTile][kPanel + 1];  // U(I, p) S(p), one panel
  __shared__ T Vs[kPanel][kTile];      // V(p, J), one panel
  __shared__ double red[2][kErrThreads / 32];
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int64_t tr = (nrows + kTile - 1) / kTile, tc = (n + kTile - 1) / kTile;
  double e2 = 0.0, a2 = 0.0;
  for (int64_t tile = blockIdx.x; tile < tr * tc; tile += gridDim.x) {
    const int64_t i0 = (tile / tc) * kTile, j0 = (tile % tc) * kTile;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = Traits<T>::zero();
    for (int p0 = 0; p0 < r; p0 += kPanel) {
      for (int e = tid; e < kTile * kPanel; e += kErrThreads) {
        const int ii = e % kTile, pp = e / kTile;
        const int64_t i = i0 + ii;
        T u = Traits<T>::zero();
        if (i < nrows && p0 + pp < r) {
          const int64_t row = rows ? rows[i] : i;
          u = scale(U[(int64_t)(p0 + pp) * ldu + row], S[p0 + pp]);
        }
        Us[ii][pp] = u;
      }
      for (int e = tid; e < kTile * kPanel; e += kErrThreads) {
        const int jj = e % kTile, pp = e / kTile;
        const int64_t j = j0 + jj;
        Vs[pp][jj] = (j < n && p0 + pp < r) ? V[(int64_t)(p0 + pp) * ldv + j] : Traits<T>::zero();
      }
      __syncthreads();
#pragma unroll 4
      for (int pp = 0; pp < kPanel; ++pp) {
        T u[4], v[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) u[a] = Us[ty + 16 * a][pp];
#pragma unroll
        for (int b = 0; b < 4; ++b) v[b] = Vs[pp][tx + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = mac(acc[a][b], u[a], v[b]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t i = i0 + ty + 16 * a;
      if (i >= nrows) continue;
      const int64_t row = rows ? rows[i] : i;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int64_t j = j0 + tx + 16 * b;
        if (j >= n) continue;
        const T av = gen(row, j);
        e2 += abs2(sub(av, acc[a][b]));
        a2 += abs2(av);
      }
    }
  }
  e2 = warp_sum(e2);
  a2 = warp_sum(a2);
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = e2;
    red[1][tid >> 5] = a2;
  }
  __syncthreads();
  if (tid == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < kErrThreads / 32; ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    part[2 * blockIdx.x] = s0;
    part[2 * blockIdx.x + 1] = s1;
  }
}

int err_grid(int sms) { return (sms > 0 ? sms : 152) * kErrCtasPerSm; }

// Calls f(generator functor) for the generator `g` describes (single block).
template <typename F>
cudaError_t visit_gen(const hbaca_gen& g, F&& f, std::string& err) {
  if (g.dtype == HBACA_F64) {
    switch (g.kind) {
      case HBACA_GEN_DENSE:
        return f(GenDense{reinterpret_cast<const double*>(g.a), g.lda});
      case HBACA_GEN_GAUSSIAN: {
        GenGaussian gg;
        gg.x = g.x;
        gg.y = g.y;
        gg.dim = g.dim;
        gg.c = -1.0 / (2.0 * g.h * g.h);
        return f(gg);
      }
      case HBACA_GEN_SPARSE_PRODUCT:
        return f(GenSparseProduct{g.p_rowptr, g.p_colidx, g.p_val, g.q_colptr, g.q_rowidx, g.q_val, g.p2, g.q2, g.n,
                                  g.r2});
      case HBACA_GEN_LOWRANK:
        return f(GenLowRank{reinterpret_cast<const double*>(g.lu), reinterpret_cast<const double*>(g.lv), g.m, g.n,
                            g.lr});
      case HBACA_GEN_POLYNOMIAL:
        return f(GenPolynomial{g.x, g.y, g.dim, g.h});
      default:
        break;
    }
  } else {
    switch (g.kind) {
      case HBACA_GEN_DENSE:
        return f(GenDenseC{reinterpret_cast<const cplx*>(g.a), g.lda});
      case HBACA_GEN_HELMHOLTZ:
        return f(GenHelmholtz{g.x, g.y, g.dim, g.k / 3.14159265358979323846});
      case HBACA_GEN_LOWRANK:
        return f(GenLowRankC{reinterpret_cast<const cplx*>(g.lu), reinterpret_cast<const cplx*>(g.lv), g.m, g.n,
                             g.lr});
      case HBACA_GEN_HANKEL2D:
        return f(GenHankel2D{g.x, g.y, g.dim, g.k});
      default:
        break;
    }
  }
  err = "generator kind not available for this dtype";
  return cudaErrorInvalidValue;
}

cudaError_t dispatch_err(const hbaca_gen& g, const hbaca_result& res, const int64_t* rows, int64_t nrows, double* part,
                         int grid, cudaStream_t st, std::string& err) {
  return visit_gen(
      g,
      [&](auto gen) -> cudaError_t {
        using T = typename decltype(gen)::scalar;
        errnorm_kernel<decltype(gen)><<<grid, kErrThreads, 0, st>>>(gen, reinterpret_cast<const T*>(res.U), res.ldu,
                                                                    res.S, reinterpret_cast<const T*>(res.V), res.ldv,
                                                                    (int)res.rank, rows, nrows, g.n, part);
        return cudaGetLastError();
      },
      err);
}

// An index outside the matrix gives NaN (the entry is not evaluated).
template <typename Gen>
__global__ void entries_kernel(const Gen gen, int64_t m, int64_t n, const int64_t* rows, const int64_t* cols,
                               int64_t count, typename Gen::scalar* out) {
  using T = typename Gen::scalar;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = rows[t], j = cols[t];
    out[t] = (i >= 0 && i < m && j >= 0 && j < n) ? gen(i, j) : scale(from_re<T>(1.0), __longlong_as_double(0x7ff8000000000000ll));
  }
}

}  // namespace
}  // namespace hbaca

extern "C" {

size_t hbaca_error_workspace_size(int64_t nrows) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 152;
  }
  const size_t part = ((size_t)hbaca::err_grid(sms) * 2 * sizeof(double) + 255) / 256 * 256;
  return part + (size_t)(nrows > 0 ? nrows : 0) * sizeof(int64_t);
}

hbaca_status hbaca_error_norms(hbaca_ctx* ctx, const hbaca_gen* gen, const hbaca_result* res, const int64_t* rows,
                               int64_t nrows, double* out, void* workspace, size_t ws_bytes, void* stream) {
  if (!ctx || !gen || !res || !out || !workspace) return hbaca::record_error(HBACA_INVALID_ARG, "NULL argument");
  if (res->rank < 0 || res->rank > 1024 || (res->rank > 0 && (!res->U || !res->S || !res->V)) ||
      res->ldu < gen->m || res->ldv < gen->n)
    return hbaca::record_error(HBACA_INVALID_ARG, "result needs a host rank in [0, 1024], U, S, V, ldu >= m, ldv >= n");
  if (gen->m < 1 || gen->n < 1 || (gen->dtype != HBACA_F64 && gen->dtype != HBACA_C128))
    return hbaca::record_error(HBACA_INVALID_ARG, "generator needs m, n >= 1 and a known dtype");
  if (nrows < 0 || (!rows && nrows != 0))
    return hbaca::record_error(HBACA_INVALID_ARG, "rows NULL needs nrows = 0 (all rows)");
  for (int64_t i = 0; rows && i < nrows; ++i)
    if (rows[i] < 0 || rows[i] >= gen->m) return hbaca::record_error(HBACA_INVALID_ARG, "a row index is outside [0, m)");
  if (reinterpret_cast<uintptr_t>(workspace) & 255u)
    return hbaca::record_error(HBACA_WORKSPACE, "workspace must be 256-byte aligned");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != hbaca::ctx_device(ctx)) {
    cudaGetLastError();
    return hbaca::record_error(HBACA_INVALID_ARG, "the current device is not the context's");
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = hbaca::err_grid(sms);
  const size_t part_bytes = ((size_t)grid * 2 * sizeof(double) + 255) / 256 * 256;
  if (ws_bytes < part_bytes + (size_t)(rows ? nrows : 0) * sizeof(int64_t))
    return hbaca::record_error(HBACA_WORKSPACE, "workspace smaller than hbaca_error_workspace_size(nrows)");
  const int64_t nr = rows ? nrows : gen->m;
  out[0] = 0.0;
  out[1] = 0.0;
  if (nr == 0) return HBACA_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double* part = reinterpret_cast<double*>(workspace);
  int64_t* drows = nullptr;
  cudaError_t e = cudaSuccess;
  if (rows) {
    drows = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(workspace) + part_bytes);
    e = cudaMemcpyAsync(drows, rows, (size_t)nrows * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return hbaca::record_error(HBACA_CUDA, std::string("row upload: ") + cudaGetErrorString(e));
  }
  std::string err;
  e = hbaca::dispatch_err(*gen, *res, drows, nr, part, grid, st, err);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return hbaca::record_error(err.empty() ? HBACA_CUDA : HBACA_INVALID_ARG,
                               err.empty() ? std::string("error kernel: ") + cudaGetErrorString(e) : err);
  }
  std::vector<double> h((size_t)grid * 2);
  e = cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return hbaca::record_error(HBACA_CUDA, std::string("error norms: ") + cudaGetErrorString(e));
  double s0 = 0.0, s1 = 0.0;
  for (int b = 0; b < grid; ++b) {
    s0 += h[2 * b];
    s1 += h[2 * b + 1];
  }
  out[0] = s0;
  out[1] = s1;
  hbaca::record_error(HBACA_OK, "");
  return HBACA_OK;
}

hbaca_status hbaca_debug_entries(const hbaca_gen* gen, const int64_t* rows, const int64_t* cols, int64_t count,
                                 void* out, void* stream) {
  if (!gen || (count > 0 && (!rows || !cols || !out)) || count < 0)
    return hbaca::record_error(HBACA_INVALID_ARG, "NULL argument or count < 0");
  if (count == 0) return HBACA_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::string err;
  const int grid = (int)std::min<int64_t>((count + 255) / 256, 4096);
  cudaError_t e = hbaca::visit_gen(
      *gen,
      [&](auto g) -> cudaError_t {
        using T = typename decltype(g)::scalar;
        hbaca::entries_kernel<decltype(g)><<<grid, 256, 0, st>>>(g, gen->m, gen->n, rows, cols, count,
                                                                 reinterpret_cast<T*>(out));
        return cudaGetLastError();
      },
      err);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return hbaca::record_error(err.empty() ? HBACA_CUDA : HBACA_INVALID_ARG,
                               err.empty() ? std::string("entries kernel: ") + cudaGetErrorString(e) : err);
  }
  hbaca::record_error(HBACA_OK, "");
  return HBACA_OK;
}

}  // extern "C"
