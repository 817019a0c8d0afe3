// Kernels of y = U diag(S) V X and of its reverse pass with frozen pivots
// (real double precision, Gaussian entry generator).
//
// The reverse pass differentiates the H-BACA map A -> U diag(S) V of Alg. 3
// with every discrete choice frozen: the BACA pivots I_k, J_k, the LRID
// column choice and ranks d_k (Alg. 2, Eqs. LRID1-2), and the truncation rank
// of the leaf re-compression and of every merge (Sec. 3.2, Eqs. columncomb,
// columnsvdmerge).  Each truncated SVD M -> T_s(M) is differentiated at the
// product level; its adjoint needs every singular triplet of the core (the
// kept ones and the discarded ones, through the singular-value gap
// 1 / (sigma_i^2 - sigma_j^2), i kept, j discarded).
#pragma once

#include <stdint.h>

namespace hbaca {

constexpr int kGemmTile = 64;
constexpr int kGemmK = 16;
constexpr int kGemmThreads = 256;

// C (M x N) = or += alpha op(A) op(B), op(A) M x K, op(B) K x N, element
// addresses given by strides and optional index maps:
//   op(A)(i, l) = A[amap(i) a_ri + akmap(l) a_ki] * (akscale ? akscale[l] : 1)
//   op(B)(l, j) = B[bkmap(l) b_ki + bmap(j) b_cj]
//   C(i, j)     at C[cmap_r(i) c_ri + cmap_c(j) c_cj]
// beta0 = 1 stores (ksplit must be 1 and no two tasks may write one element);
// beta0 = 0 adds atomically, so tasks may overlap and K may be split.
struct GemmTask {
  int32_t M, N, K, ksplit;
  int32_t tm, tn, beta0, pad;
  int64_t first;  // first CTA of the task in its launch
  double alpha;
  const double* A;
  int64_t a_ri, a_ki;
  const double* B;
  int64_t b_ki, b_cj;
  double* C;
  int64_t c_ri, c_cj;
  const int32_t* amap;
  const int32_t* akmap;
  const double* akscale;
  const int32_t* bkmap;
  const int32_t* bmap;
  const int32_t* cmap_r;
  const int32_t* cmap_c;
};

// dst(i, j) = src(i, j), or 0 when src is null (a fill).
struct CopyTask {
  int64_t rows, cols;
  const double* src;
  int64_t s_ri, s_cj;
  double* dst;
  int64_t d_ri, d_cj;
};

// Singular-value-gap coefficients of one node (i < s kept, s <= j < nout
// discarded, nd = nout - s):
//   E1(i, j-s) = sig_j (sig_j GB(i, j-s) + sig_i GC(j-s, i)) / (sig_i^2 - sig_j^2)
//   E2(j-s, i) = sig_j (sig_j GC(j-s, i) + sig_i GB(i, j-s)) / (sig_i^2 - sig_j^2)
// GB, E1: s x nd column-major (ld s); GC, E2: nd x s column-major (ld nd).
struct GapTask {
  int32_t s, nd;
  const double* sigma;
  const double* GB;
  const double* GC;
  double* E1;
  double* E2;
};

// Gaussian entry generator of one block (points, dimension, c = -1 / (2 h^2),
// h) and where its gradients go.
struct GaussAdj {
  const double* x;
  const double* y;
  int dim;
  double c;
  double h;
  double* dx;  // m x dim (may be null)
  double* dy;  // n x dim (may be null)
  double* dh;  // 1 (may be null)
};

// Gaussian entries of rows I(0..rows-1) of a leaf added to R (rows x n, row-major).
struct GenRowsTask {
  int32_t rows, n;
  const int32_t* I;  // leaf-local row indices
  double* R;
  int64_t row0, col0;  // leaf offsets in the matrix
  GaussAdj G;          // the leaf's block
};

// One reverse BACA iteration of one leaf: from R_k (dI x n, row-major), the
// block J_k, the LRID positions jbar (first dk kept) and Zbar = Vbar_k R_k^T
// (dk x dI, column-major), form W = R_k(:, J_k(jbar)) = Q T, its
// pseudo-inverse Z = W^+ = T^-1 Q^T (dk x dI, column-major, written), the adjoint
//   Wbar = (I - Q Q^T) Zbar^T (W^T W)^-1 - Z^T Zbar Z^T,
// added to Acols at rows I_k of columns r0 .. r0+dk-1, and slotcol[r0 + t] =
// J_k(jbar(t)).
struct LeafStepTask {
  int32_t dI, dk, n, m;
  int32_t r0, pad;
  const double* R;
  const int32_t* I;
  const int32_t* J;
  const int32_t* jbar;
  const double* Zbar;
  double* Z;
  double* Acols;  // m x rcap, column-major (ld m)
  int32_t* slotcol;
};

// Generator adjoint of one leaf: the adjoint entries of the kept columns
// (Acols, m x nslot, column index slotcol[t]) and of the residual rows
// (Arows, nrow x n, row index rowidx[t]) contracted with dA/dx_i, dA/dy_j,
// dA/dh of A(i, j) = exp(c ||x_i - y_j||^2), c = -1 / (2 h^2).
struct GenAdjTask {
  int32_t m, n, nslot, nrow;
  int64_t row0, col0;
  const double* Acols;
  const int32_t* slotcol;
  const double* Arows;
  const int32_t* rowidx;
  GaussAdj G;  // the leaf's block: entry generator and gradient outputs
};


// ------------------------------------------------------------------ GEMM
__global__ void __launch_bounds__(kGemmThreads) gemm_kernel(const GemmTask* tasks, int ntasks) {
  __shared__ double As[kGemmK][kGemmTile + 1];
  __shared__ double Bs[kGemmK][kGemmTile + 1];
  int lo = 0, hi = ntasks - 1;
  const int64_t cta = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].first <= cta) lo = mid;
    else hi = mid - 1;
  }
  const GemmTask T = tasks[lo];
  const int64_t local = cta - T.first;
  const int tiles = T.tm * T.tn;
  const int ks = (int)(local / tiles);
  const int tile = (int)(local % tiles);
  const int i0 = (tile % T.tm) * kGemmTile, j0 = (tile / T.tm) * kGemmTile;
  const int kchunk = (((T.K + T.ksplit - 1) / T.ksplit) + kGemmK - 1) / kGemmK * kGemmK;
  const int kb = ks * kchunk, ke = min(T.K, kb + kchunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  const bool a_rows_fast = T.a_ri == 1 && !T.amap;
  const bool b_cols_fast = T.b_cj == 1 && !T.bmap;
  for (int k0 = kb; k0 < ke; k0 += kGemmK) {
#pragma unroll
    for (int q = 0; q < (kGemmTile * kGemmK) / kGemmThreads; ++q) {
      const int e = tid + q * kGemmThreads;
      int r, kk;
      if (a_rows_fast) { r = e % kGemmTile; kk = e / kGemmTile; }
      else { kk = e % kGemmK; r = e / kGemmK; }
      const int i = i0 + r, l = k0 + kk;
      double v = 0.0;
      if (i < T.M && l < ke) {
        const int64_t ii = T.amap ? T.amap[i] : i;
        const int64_t ll = T.akmap ? T.akmap[l] : l;
        v = T.A[ii * T.a_ri + ll * T.a_ki];
        if (T.akscale) v *= T.akscale[l];
      }
      As[kk][r] = v;
    }
#pragma unroll
    for (int q = 0; q < (kGemmTile * kGemmK) / kGemmThreads; ++q) {
      const int e = tid + q * kGemmThreads;
      int c, kk;
      if (b_cols_fast) { c = e % kGemmTile; kk = e / kGemmTile; }
      else { kk = e % kGemmK; c = e / kGemmK; }
      const int j = j0 + c, l = k0 + kk;
      double v = 0.0;
      if (j < T.N && l < ke) {
        const int64_t jj = T.bmap ? T.bmap[j] : j;
        const int64_t ll = T.bkmap ? T.bkmap[l] : l;
        v = T.B[ll * T.b_ki + jj * T.b_cj];
      }
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGemmK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[kk][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Bs[kk][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty + 16 * u;
    if (i >= T.M) continue;
    const int64_t ii = T.cmap_r ? T.cmap_r[i] : i;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = j0 + tx + 16 * v;
      if (j >= T.N) continue;
      const int64_t jj = T.cmap_c ? T.cmap_c[j] : j;
      double* p = T.C + ii * T.c_ri + jj * T.c_cj;
      if (T.beta0) *p = T.alpha * acc[u][v];
      else atomicAdd(p, T.alpha * acc[u][v]);
    }
  }
}

// ------------------------------------------------------------------ copies / fills
__global__ void copy_kernel(const CopyTask* tasks) {
  const CopyTask T = tasks[blockIdx.y];
  const int64_t tot = T.rows * T.cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % T.rows, j = e / T.rows;
    T.dst[i * T.d_ri + j * T.d_cj] = T.src ? T.src[i * T.s_ri + j * T.s_cj] : 0.0;
  }
}

// ------------------------------------------------------------------ singular-value gap
__global__ void gap_kernel(const GapTask* tasks) {
  const GapTask T = tasks[blockIdx.y];
  const int64_t tot = (int64_t)T.s * T.nd;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % T.s), jd = (int)(e / T.s);
    const double si = T.sigma[i], sj = T.sigma[T.s + jd];
    const double gb = T.GB[i + (int64_t)jd * T.s], gc = T.GC[jd + (int64_t)i * T.nd];
    const double den = (si - sj) * (si + sj);
    double e1 = 0.0, e2 = 0.0;
    if (den > 0.0) {
      e1 = sj * (sj * gb + si * gc) / den;
      e2 = sj * (sj * gc + si * gb) / den;
    }
    T.E1[i + (int64_t)jd * T.s] = e1;
    T.E2[jd + (int64_t)i * T.nd] = e2;
  }
}

// ------------------------------------------------------------------ Gaussian entries
__device__ __forceinline__ double gauss_entry(const GaussAdj& G, int64_t i, int64_t j) {
  double d2 = 0.0;
  for (int t = 0; t < G.dim; ++t) {
    const double df = G.x[i * G.dim + t] - G.y[j * G.dim + t];
    d2 = fma(df, df, d2);
  }
  return exp(G.c * d2);
}

__global__ void genrows_kernel(const GenRowsTask* tasks) {
  const GenRowsTask T = tasks[blockIdx.y];
  const GaussAdj G = T.G;
  const int64_t tot = (int64_t)T.rows * T.n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / T.n), j = (int)(e % T.n);
    T.R[e] += gauss_entry(G, T.row0 + T.I[r], T.col0 + j);
  }
}

// ------------------------------------------------------------------ one reverse LRID step
// One warp per task; dI, dk <= 32.  Householder QR of W (dI x dk) in shared
// memory, Z = T^-1 Q^T, G = (W^T W)^-1 = T^-1 T^-T, then Wbar.  Matrices are
// 32 x 33 doubles, column-major (buf[col * 33 + row]), in dynamic shared
// memory (kLeafStepSmem bytes).
constexpr int kMaxD = 32;
constexpr int kLd = kMaxD + 1;
constexpr size_t kLeafStepSmem = 7 * (size_t)kMaxD * kLd * sizeof(double) + kMaxD * sizeof(double);

__device__ __forceinline__ double warp_sum_all(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(32) leafstep_kernel(const LeafStepTask* tasks) {
  extern __shared__ __align__(16) double lsm[];
  const LeafStepTask T = tasks[blockIdx.x];
  const int lane = threadIdx.x;
  const int dI = T.dI, dk = T.dk;
  double* W0 = lsm;                   // W (dI x dk); later ZZ = Zbar Z^T (dk x dk)
  double* Hq = W0 + kMaxD * kLd;      // Householder work, then Q (dI x dk); later F2 (dI x dk)
  double* Tm = Hq + kMaxD * kLd;      // R, then T^-1; later Q^T Zbar^T (dk x dk)
  double* Zs = Tm + kMaxD * kLd;      // Z (dk x dI)
  double* Zb = Zs + kMaxD * kLd;      // Zbar (dk x dI)
  double* F1 = Zb + kMaxD * kLd;      // scratch, then G (dk x dk)
  double* F3 = F1 + kMaxD * kLd;      // scratch
  double* tau = F3 + kMaxD * kLd;
  if (dk <= 0 || dI <= 0) return;
  for (int t = 0; t < dk; ++t) {
    const int col = T.J[T.jbar[t]];
    if (lane < dI) {
      const double v = T.R[(int64_t)lane * T.n + col];
      W0[t * kLd + lane] = v;
      Hq[t * kLd + lane] = v;
    }
    if (lane == 0) T.slotcol[T.r0 + t] = col;
  }
  for (int i = 0; i < dI; ++i)
    if (lane < dk) Zb[i * kLd + lane] = T.Zbar[lane + (int64_t)i * dk];
  __syncwarp();
  // Householder QR (column j: v = [1; x / (alpha - beta)], tau = (beta - alpha) / beta)
  for (int j = 0; j < dk; ++j) {
    double x2 = 0.0;
    for (int i = j + 1 + lane; i < dI; i += 32) x2 = fma(Hq[j * kLd + i], Hq[j * kLd + i], x2);
    x2 = warp_sum_all(x2);
    const double alpha = Hq[j * kLd + j];
    double beta, tj, scale;
    if (x2 == 0.0) { beta = alpha; tj = 0.0; scale = 0.0; }
    else {
      beta = -copysign(sqrt(alpha * alpha + x2), alpha);
      tj = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    __syncwarp();
    for (int i = j + 1 + lane; i < dI; i += 32) Hq[j * kLd + i] *= scale;
    __syncwarp();
    if (lane == 0) { Hq[j * kLd + j] = beta; tau[j] = tj; }
    __syncwarp();
    for (int c = j + 1; c < dk; ++c) {
      double w = 0.0;
      for (int i = j + 1 + lane; i < dI; i += 32) w = fma(Hq[j * kLd + i], Hq[c * kLd + i], w);
      w = warp_sum_all(w) + Hq[c * kLd + j];
      const double f = tj * w;
      __syncwarp();
      if (lane == 0) Hq[c * kLd + j] -= f;
      for (int i = j + 1 + lane; i < dI; i += 32) Hq[c * kLd + i] -= f * Hq[j * kLd + i];
      __syncwarp();
    }
  }
  for (int c = 0; c < dk; ++c)
    if (lane < dk) Tm[c * kLd + lane] = lane <= c ? Hq[c * kLd + lane] : 0.0;
  __syncwarp();
  // explicit thin Q (dI x dk) in F3: Q e_c, reflectors applied last to first; lane = row
  for (int c = 0; c < dk; ++c) {
    double q = (lane == c) ? 1.0 : 0.0;
    for (int j = dk - 1; j >= 0; --j) {
      const double vj = lane == j ? 1.0 : (lane > j && lane < dI ? Hq[j * kLd + lane] : 0.0);
      const double w = warp_sum_all(vj * q);
      q -= tau[j] * w * vj;
    }
    F3[c * kLd + lane] = q;
  }
  __syncwarp();
  for (int c = 0; c < dk; ++c) Hq[c * kLd + lane] = F3[c * kLd + lane];  // Hq = Q
  __syncwarp();
  // T^-1 (upper), lane = column c, into F1
  if (lane < dk) {
    const int c = lane;
    for (int r = dk - 1; r >= 0; --r) {
      double v = (r == c) ? 1.0 : 0.0;
      for (int t = r + 1; t <= c; ++t) v -= Tm[t * kLd + r] * F1[c * kLd + t];
      F1[c * kLd + r] = (r <= c) ? v / Tm[r * kLd + r] : 0.0;
    }
  }
  __syncwarp();
  for (int c = 0; c < dk; ++c)
    if (lane < dk) Tm[c * kLd + lane] = F1[c * kLd + lane];  // Tm = T^-1
  __syncwarp();
  // Z = T^-1 Q^T (dk x dI): Z(t, i) = sum_u Tinv(t, u) Q(i, u); lane = i
  if (lane < dI)
    for (int t = 0; t < dk; ++t) {
      double v = 0.0;
      for (int u = t; u < dk; ++u) v = fma(Tm[u * kLd + t], Hq[u * kLd + lane], v);
      Zs[lane * kLd + t] = v;
    }
  __syncwarp();
  for (int i = 0; i < dI; ++i)
    if (lane < dk) T.Z[lane + (int64_t)i * dk] = Zs[i * kLd + lane];
  // G(a, b) = sum_u Tinv(a, u) Tinv(b, u), lane = b, into F1
  if (lane < dk)
    for (int a = 0; a < dk; ++a) {
      double v = 0.0;
      for (int u = max(a, lane); u < dk; ++u) v = fma(Tm[u * kLd + a], Tm[u * kLd + lane], v);
      F1[lane * kLd + a] = v;
    }
  __syncwarp();
  // F2 = (I - W W^+) Zbar^T = (I - Q Q^T) Zbar^T (dI x dk), into Hq.  The
  // projector is formed from the orthonormal Q (not as I - W Z, whose
  // rounding error ~ cond(W) eps would be amplified by (W^T W)^-1); for a
  // square W it is exactly zero.
  if (dI > dk) {
    // QZ(a, b) = sum_i Q(i, a) Zbar(b, i), lane = b, into Tm
    if (lane < dk)
      for (int a = 0; a < dk; ++a) {
        double v = 0.0;
        for (int i = 0; i < dI; ++i) v = fma(Hq[a * kLd + i], Zb[i * kLd + lane], v);
        F3[lane * kLd + a] = v;
      }
    __syncwarp();
    for (int c = 0; c < dk; ++c)
      if (lane < dk) Tm[c * kLd + lane] = F3[c * kLd + lane];
    __syncwarp();
    // F2(i, b) = Zbar(b, i) - sum_a Q(i, a) QZ(a, b), lane = i
    if (lane < dI)
      for (int b = 0; b < dk; ++b) {
        double v = Zb[lane * kLd + b];
        for (int a = 0; a < dk; ++a) v -= Hq[a * kLd + lane] * Tm[b * kLd + a];
        F3[b * kLd + lane] = v;
      }
  } else {
    for (int b = 0; b < dk; ++b) F3[b * kLd + lane] = 0.0;
  }
  __syncwarp();
  for (int c = 0; c < dk; ++c) Hq[c * kLd + lane] = F3[c * kLd + lane];
  __syncwarp();
  // ZZ(a, b) = sum_i Zbar(a, i) Z(b, i), lane = b, into W0
  if (lane < dk)
    for (int a = 0; a < dk; ++a) {
      double v = 0.0;
      for (int i = 0; i < dI; ++i) v = fma(Zb[i * kLd + a], Zs[i * kLd + lane], v);
      F3[lane * kLd + a] = v;
    }
  __syncwarp();
  for (int c = 0; c < dk; ++c)
    if (lane < dk) W0[c * kLd + lane] = F3[c * kLd + lane];
  __syncwarp();
  // Wbar(i, b) = sum_a F2(i, a) G(a, b) - sum_a Z(a, i) ZZ(a, b); lane = i
  if (lane < dI)
    for (int b = 0; b < dk; ++b) {
      double v = 0.0;
      for (int a = 0; a < dk; ++a) v = fma(Hq[a * kLd + lane], F1[b * kLd + a], v);
      for (int a = 0; a < dk; ++a) v -= Zs[lane * kLd + a] * W0[b * kLd + a];
      T.Acols[T.I[lane] + (int64_t)(T.r0 + b) * T.m] += v;
    }
}

// ------------------------------------------------------------------ generator adjoint
// dA/dx_i = 2c A (x_i - y_j), dA/dy_j = -2c A (x_i - y_j), dA/dh = A d2 / h^3.
constexpr int kAdjThreads = 256;
constexpr int kMaxDim = 4;
constexpr int kAdjSlots = 64;  // columns (or rows) staged per pass

__device__ __forceinline__ double block_sum_adj(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

// grid (chunks of rows, task): thread = leaf row i; loops over the kept columns
__global__ void __launch_bounds__(kAdjThreads) genadj_cols_kernel(const GenAdjTask* tasks) {
  const GenAdjTask T = tasks[blockIdx.y];
  const GaussAdj G = T.G;
  __shared__ double ys[kAdjSlots][kMaxDim];
  __shared__ double dys[kAdjSlots][kMaxDim];
  __shared__ double red[32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = i < T.m;
  double xi[kMaxDim] = {0, 0, 0, 0}, dxi[kMaxDim] = {0, 0, 0, 0}, dh = 0.0;
  if (act)
    for (int t = 0; t < G.dim; ++t) xi[t] = G.x[(T.row0 + i) * G.dim + t];
  for (int s0 = 0; s0 < T.nslot; s0 += kAdjSlots) {
    const int ns = min(kAdjSlots, T.nslot - s0);
    __syncthreads();
    for (int e = threadIdx.x; e < ns * kMaxDim; e += blockDim.x) {
      const int sl = e / kMaxDim, t = e % kMaxDim;
      ys[sl][t] = t < G.dim ? G.y[(T.col0 + T.slotcol[s0 + sl]) * G.dim + t] : 0.0;
      dys[sl][t] = 0.0;
    }
    __syncthreads();
    for (int sl = 0; sl < ns; ++sl) {
      double g = act ? T.Acols[i + (int64_t)(s0 + sl) * T.m] : 0.0;
      double df[kMaxDim], d2 = 0.0;
#pragma unroll
      for (int t = 0; t < kMaxDim; ++t) {
        df[t] = t < G.dim ? xi[t] - ys[sl][t] : 0.0;
        d2 = fma(df[t], df[t], d2);
      }
      const double a = act ? exp(G.c * d2) : 0.0;
      const double ga = g * a;
      dh = fma(ga, d2, dh);
      const double f = 2.0 * G.c * ga;
#pragma unroll
      for (int t = 0; t < kMaxDim; ++t) {
        if (t >= G.dim) break;
        dxi[t] = fma(f, df[t], dxi[t]);
        double v = -f * df[t];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&dys[sl][t], v);
      }
    }
    __syncthreads();
    if (G.dy)
      for (int e = threadIdx.x; e < ns * G.dim; e += blockDim.x) {
        const int sl = e / G.dim, t = e % G.dim;
        const double v = dys[sl][t];
        if (v != 0.0) atomicAdd(&G.dy[(T.col0 + T.slotcol[s0 + sl]) * G.dim + t], v);
      }
  }
  if (act && G.dx)
    for (int t = 0; t < G.dim; ++t)
      if (dxi[t] != 0.0) atomicAdd(&G.dx[(T.row0 + i) * G.dim + t], dxi[t]);
  const double tot = block_sum_adj(dh, red);
  if (threadIdx.x == 0 && G.dh && tot != 0.0) atomicAdd(G.dh, tot / (G.h * G.h * G.h));
}

// grid (chunks of columns, task): thread = leaf column j; loops over the residual rows
__global__ void __launch_bounds__(kAdjThreads) genadj_rows_kernel(const GenAdjTask* tasks) {
  const GenAdjTask T = tasks[blockIdx.y];
  const GaussAdj G = T.G;
  __shared__ double xs[kAdjSlots][kMaxDim];
  __shared__ double dxs[kAdjSlots][kMaxDim];
  __shared__ double red[32];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = j < T.n;
  double yj[kMaxDim] = {0, 0, 0, 0}, dyj[kMaxDim] = {0, 0, 0, 0}, dh = 0.0;
  if (act)
    for (int t = 0; t < G.dim; ++t) yj[t] = G.y[(T.col0 + j) * G.dim + t];
  for (int s0 = 0; s0 < T.nrow; s0 += kAdjSlots) {
    const int ns = min(kAdjSlots, T.nrow - s0);
    __syncthreads();
    for (int e = threadIdx.x; e < ns * kMaxDim; e += blockDim.x) {
      const int sl = e / kMaxDim, t = e % kMaxDim;
      xs[sl][t] = t < G.dim ? G.x[(T.row0 + T.rowidx[s0 + sl]) * G.dim + t] : 0.0;
      dxs[sl][t] = 0.0;
    }
    __syncthreads();
    for (int sl = 0; sl < ns; ++sl) {
      double g = act ? T.Arows[(int64_t)(s0 + sl) * T.n + j] : 0.0;
      double df[kMaxDim], d2 = 0.0;
#pragma unroll
      for (int t = 0; t < kMaxDim; ++t) {
        df[t] = t < G.dim ? xs[sl][t] - yj[t] : 0.0;
        d2 = fma(df[t], df[t], d2);
      }
      const double a = act ? exp(G.c * d2) : 0.0;
      const double ga = g * a;
      dh = fma(ga, d2, dh);
      const double f = 2.0 * G.c * ga;
#pragma unroll
      for (int t = 0; t < kMaxDim; ++t) {
        if (t >= G.dim) break;
        dyj[t] = fma(-f, df[t], dyj[t]);
        double v = f * df[t];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&dxs[sl][t], v);
      }
    }
    __syncthreads();
    if (G.dx)
      for (int e = threadIdx.x; e < ns * G.dim; e += blockDim.x) {
        const int sl = e / G.dim, t = e % G.dim;
        const double v = dxs[sl][t];
        if (v != 0.0) atomicAdd(&G.dx[(T.row0 + T.rowidx[s0 + sl]) * G.dim + t], v);
      }
  }
  if (act && G.dy)
    for (int t = 0; t < G.dim; ++t)
      if (dyj[t] != 0.0) atomicAdd(&G.dy[(T.col0 + j) * G.dim + t], dyj[t]);
  const double tot = block_sum_adj(dh, red);
  if (threadIdx.x == 0 && G.dh && tot != 0.0) atomicAdd(G.dh, tot / (G.h * G.h * G.h));
}

}  // namespace hbaca
