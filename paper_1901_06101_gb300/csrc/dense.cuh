// Re-compression and hierarchical merge (Sec. 3.2 last paragraph; Alg. 3,
// Eqs. columncomb, columnsvdmerge) as batched kernels.
//
// Every task is "truncated SVD of a product whose factors are known":
//   LEAF   U V            : QR(U) = Q_A R_A, QR(V^H) = Q_B R_B, core M = R_A R_B^H
//   HORIZ  [U1 S1, U2 S2] diag(V1, V2)   : QR of the stacked U side, core M = R_A
//   VERT   diag(U1, U2) [S1 V1; S2 V2]   : QR of the stacked V^H side, core M = R_A
// SVD(M) = X S Y^H by one-sided Jacobi; s = eps-rank (Sec. 2); the Q side is
// Q_A [X_s; 0] and the other side is Q_B [Y_s; 0] (LEAF) or the block-diagonal
// factor times Y_s (HORIZ: V = Y_s^H diag(V1, V2); VERT: U = diag(U1, U2) Y_s).
// For the merges this is SVD(U_bar, eps) computed as QR followed by the SVD of
// the triangular factor, which equals the paper's SVD of the stacked factor.
//
// Tasks read their ranks from device memory, so a whole level is launched
// without a host round trip.  QR, Jacobi and Q-application kernels run one
// thread-block cluster per task; partial sums are combined across the cluster
// through distributed shared memory in a fixed order, so every CTA holds
// bit-identical reflector coefficients.
#pragma once

#include <cooperative_groups.h>
#include <climits>
#include <type_traits>

#include "common.cuh"
#include "types.h"

namespace cg = cooperative_groups;

namespace hbaca {

constexpr int kDenseThreads = 256;
// one CTA per task with a serial column loop (pivoted QR of the core): the
// widest block hides more of the latency of the per-column reductions
constexpr int kWideThreads = 1024;





template <typename T>
struct DenseParams {
  const SvdTask* tasks;
  TaskDims* dims;
  int ntasks;
  // BACA arenas and leaf table (LEAF tasks)
  T* Uar;
  T* Var;
  const int32_t* leaf_rank;  // stride leaf_rank_stride ints (LeafOut.rank)
  int leaf_rank_stride;
  // input / output block stores
  const BlockRef* in_blocks;
  const int32_t* in_rank;
  T* inU;
  const double* inS;
  T* inV;
  const BlockRef* out_blocks;
  int32_t* out_rank;
  T* outU;
  double* outS;
  T* outV;
  int64_t out_cap;     // rank capacity of output blocks
  // scratch
  T* qr;               // QR arena (operand B of LEAF tasks, stacked operands of merges)
  T* tau;
  T* core;             // M and Y matrices
  int32_t* ord;        // per-task column order after Jacobi
  int* status;
  double eps;
};

template <typename T>
__device__ __forceinline__ T* qr_a_ptr(const DenseParams<T>& P, const SvdTask& t) {
  return (t.a_in_baca ? P.Uar : P.qr) + t.a_off;
}

// Output addresses of a block: the caller's buffers for a block's final
// result, otherwise the output store arena plus the block's offsets.
template <typename T>
__device__ __forceinline__ T* out_u(const DenseParams<T>& P, const BlockRef& b) {
  return b.U ? reinterpret_cast<T*>(b.U) : P.outU + b.u_off;
}
template <typename T>
__device__ __forceinline__ T* out_v(const DenseParams<T>& P, const BlockRef& b) {
  return b.V ? reinterpret_cast<T*>(b.V) : P.outV + b.v_off;
}
template <typename T>
__device__ __forceinline__ double* out_s(const DenseParams<T>& P, const BlockRef& b) {
  return b.S ? b.S : P.outS + b.s_off;
}

// ------------------------------------------------------------------ pack
// Build the QR operands and the task dimensions.
template <typename T>
__global__ void pack_kernel(const DenseParams<T> P) {
  const int ti = blockIdx.y;
  if (ti >= P.ntasks) return;
  const SvdTask t = P.tasks[ti];
  int k = 0;
  if (t.kind == TASK_LEAF) {
    k = P.leaf_rank[(size_t)t.in1 * P.leaf_rank_stride];
    if (k < 0 || k > t.kcap) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_status(P.status, DS_RANK_CAPACITY);
      k = 0;
    }
    // B = V^H (rows_b x k): B(j, p) = conj(V(p, j)); the leaf V (k x n, ld n)
    // and B (n x k, ld n) share the index p * n + j
    const T* V = P.Var + t.src_v_off;
    T* B = P.qr + t.b_off;
    const int64_t tot = (int64_t)t.rows_b * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
      const int64_t j = e % t.rows_b, p = e / t.rows_b;
      B[p * t.rows_b + j] = conj_(V[p * t.rows_b + j]);
    }
    if (!t.a_in_baca) {  // QR operand A = a copy of the leaf's U (m x k, ld m)
      const T* U = P.Uar + t.src_u_off;
      T* A = P.qr + t.a_off;
      const int64_t tu = (int64_t)t.rows_a * k;
      for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tu; e += (int64_t)gridDim.x * blockDim.x)
        A[e] = U[e];
    }
  } else {
    const BlockRef b1 = P.in_blocks[t.in1], b2 = P.in_blocks[t.in2];
    const int r1 = P.in_rank[b1.rank_slot], r2 = P.in_rank[b2.rank_slot];
    k = r1 + r2;
    if (k > t.kcap) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_status(P.status, DS_RANK_CAPACITY);
      k = 0;
    }
    T* A = P.qr + t.a_off;
    const int rows = t.rows_a;
    const int64_t tot = (int64_t)rows * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
      const int64_t i = e % rows, p = e / rows;
      const BlockRef& b = p < r1 ? b1 : b2;
      const int64_t pp = p < r1 ? p : p - r1;
      const double sg = P.inS[b.s_off + pp];
      T v;
      if (t.kind == TASK_HORIZ) v = P.inU[b.u_off + pp * b.ldu + i];    // [U1 S1, U2 S2]
      else v = conj_(P.inV[b.v_off + pp * b.ldv + i]);                  // [V1^H S1, V2^H S2]
      A[p * t.lda + i] = scale(v, sg);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    TaskDims dm;
    dm.k = k;
    dm.kra = min(t.rows_a, k);
    dm.krb = t.kind == TASK_LEAF ? min(t.rows_b, k) : 0;
    dm.s = 0;
    dm.sweeps = 0;
    dm.nout = 0;
    dm.rotations = 0;
    dm.pad = 0;
    P.dims[ti] = dm;
  }
}

// ------------------------------------------------------------------ cluster groups
// A matrix with few companions in its stage is spread over G clusters (a
// cooperative launch keeps every CTA of the grid resident).  After each
// cluster has combined its CTAs' partial sums through DSMEM, its leader CTA
// publishes them in a global slot (double-buffered by step parity), counts
// itself in on the matrix's arrival counter and waits until all G clusters
// have arrived at that step; every CTA then sums the G slots in cluster
// order, so all CTAs of all clusters hold bit-identical totals.  The wait is
// bounded by kXWaitNs of wall time: on expiry the status word records
// DS_TIMEOUT and the clusters leave the column loop together.
constexpr unsigned long long kXWaitNs = 4000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One thread, after a __syncthreads that follows the CTA's slot writes.
__device__ __forceinline__ int xgroup_arrive_wait(unsigned* cnt, unsigned target, int* status) {
  __threadfence();
  atomicAdd(cnt, 1u);
  const unsigned long long t0 = global_ns();
  for (;;) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
    if (v >= target) return 1;
    if (global_ns() - t0 > kXWaitNs) {
      set_status(status, DS_TIMEOUT);
      return 0;
    }
    __nanosleep(100);
  }
}

// Launch shape (cluster size csize, njobs matrices, G clusters per matrix)
// and the inter-cluster exchange (slot stride xplen elements).
template <typename T>
struct XGroup {
  int G;
  int csize;
  int njobs;
  int xplen;
  T* xpart;       // [cluster of the grid][2][xplen]
  unsigned* xcnt; // [matrix of the launch]
};

// ------------------------------------------------------------------ QR
// Householder QR (LAPACK geqr2 convention) of a rows x k column-major matrix,
// in place: R in the upper triangle (diagonal = beta), reflector tails below,
// tau[j].  G clusters per matrix (one unless the stage has few matrices);
// CTA q of cluster g owns the contiguous slice g c + q of the rows.
// Per column: one pass forms the partial squared tail norm, the partial
// inner products of the tail with every trailing column and the head row;
// one cluster barrier; every CTA combines the partials in rank order (then
// across the G clusters through global memory).

template <typename T>
__global__ void __launch_bounds__(kDenseThreads) qr_kernel(const DenseParams<T> P, const QrJob* jobs, const XGroup<T> X) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int xok;
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank(), c = (int)cl.num_blocks();
  const int G = X.G;
  const int cid = blockIdx.x / c;
  const int job = cid / G, g = cid - job * G;
  if (c != X.csize || job >= X.njobs) {  // not the planned launch shape: touch nothing
    if (threadIdx.x == 0) set_status(P.status, DS_LAUNCH);
    return;
  }
  const QrJob jb = jobs[job];
  const SvdTask t = P.tasks[jb.task];
  const TaskDims dm = P.dims[jb.task];
  const int k = dm.k;
  const int rows = jb.which ? t.rows_b : t.rows_a;
  T* A = jb.which ? P.qr + t.b_off : qr_a_ptr(P, t);
  const int64_t lda = jb.which ? (int64_t)t.rows_b : t.lda;
  T* tau = P.tau + t.tau_off + (jb.which ? t.kcap : 0);
  const int kk = min(rows, k);
  if (kk <= 0) return;
  const int np = G * c, pi = g * c + q;
  const int chunk = (rows + np - 1) / np;
  const int ra = min(rows, pi * chunk), rb = min(rows, ra + chunk);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // partial buffer (double-buffered): [0] sig2 (re), [1] alpha, [2 + l] dot_l, [2 + kcap + l] head row value
  const int plen = 2 + 2 * t.kcap;
  T* part = reinterpret_cast<T*>(smem_raw);
  T* tot = part + 2 * plen;
  T* coef = tot + plen;  // [0] conj(tau), [1] sc, [2] beta (re), [3] tau
  for (int j = 0; j < kk; ++j) {
    T* pb = part + (j & 1) * plen;
    const int i0 = max(ra, j + 1);
    const int ncol = k - j;  // column j and trailing ones
    // two columns per warp: their inner products with column j share its
    // loads and are summed over the warp together
    for (int l0 = 2 * warp; l0 < ncol; l0 += 2 * nw) {
      const T* colj = A + (int64_t)j * lda;
      const T* c0 = A + (int64_t)(j + l0) * lda;
      const bool two = l0 + 1 < ncol;  // warp-uniform
      T a0 = Traits<T>::zero(), a1 = Traits<T>::zero();
      if (two) {
        for (int i = i0 + lane; i < rb; i += 32) {
          const T xj = colj[i];
          a0 = cmac(a0, xj, c0[i]);
          a1 = cmac(a1, xj, c0[lda + i]);
        }
      } else {
        for (int i = i0 + lane; i < rb; i += 32) a0 = cmac(a0, colj[i], c0[i]);
      }
      int col, comp;
      bool first;
      const double sum = warp_sum2<T>(a0, a1, lane, col, comp, first);
      const int l = l0 + col;
      if (first && l < ncol) {
        T* dst = l == 0 ? pb : pb + 2 + (l - 1);
        reinterpret_cast<double*>(dst)[comp] = sum;
      }
      if (lane < 2 && l0 + lane < ncol) {
        const int lh = l0 + lane;
        const bool own = (j >= ra && j < rb);
        if (lh == 0) pb[1] = own ? A[(int64_t)j * lda + j] : Traits<T>::zero();
        else pb[2 + t.kcap + (lh - 1)] = own ? A[(int64_t)(j + lh) * lda + j] : Traits<T>::zero();
      }
    }
    __syncthreads();
    cl.sync();
    for (int e = tid; e < 2 * ncol; e += blockDim.x) {
      const int idx = e < ncol ? (e == 0 ? 0 : 2 + (e - 1)) : (e == ncol ? 1 : 2 + t.kcap + (e - ncol - 1));
      T s = Traits<T>::zero();
      for (int r = 0; r < c; ++r) {
        const T* rp = cl.map_shared_rank(part + (j & 1) * plen, r);
        s = add(s, rp[idx]);
      }
      tot[idx] = s;
    }
    __syncthreads();
    if (G > 1) {
      auto slot_idx = [&](int e) {
        return e < ncol ? (e == 0 ? 0 : 2 + (e - 1)) : (e == ncol ? 1 : 2 + t.kcap + (e - ncol - 1));
      };
      if (q == 0) {
        T* xs = X.xpart + ((size_t)cid * 2 + (j & 1)) * X.xplen;
        for (int e = tid; e < 2 * ncol; e += blockDim.x) xs[slot_idx(e)] = tot[slot_idx(e)];
        __syncthreads();
        if (tid == 0) xok = xgroup_arrive_wait(X.xcnt + job, (unsigned)(j + 1) * G, P.status);
      }
      cl.sync();
      if (*cl.map_shared_rank(&xok, 0) == 0) break;
      for (int e = tid; e < 2 * ncol; e += blockDim.x) {
        const int idx = slot_idx(e);
        T s = Traits<T>::zero();
        for (int gg = 0; gg < G; ++gg) s = add(s, ldcg(X.xpart + ((size_t)(job * G + gg) * 2 + (j & 1)) * X.xplen + idx));
        tot[idx] = s;
      }
      __syncthreads();
    }
    if (tid == 0) {
      double beta;
      T tu, sc;
      householder(tot[1], re_(tot[0]), beta, tu, sc);
      coef[0] = conj_(tu);
      coef[1] = sc;
      coef[2] = from_re<T>(beta);
      coef[3] = tu;
      if (pi == 0) tau[j] = tu;
    }
    __syncthreads();
    const T ctau = coef[0], sc = coef[1];
    const T csc = conj_(sc);
    // w_l = a_jl + conj(sc) dot_l ; f_l = conj(tau) w_l (into the dot slots)
    for (int l = 1 + tid; l < ncol; l += blockDim.x) {
      const T w = mac(tot[2 + t.kcap + (l - 1)], csc, tot[2 + (l - 1)]);
      tot[2 + (l - 1)] = mul(ctau, w);
    }
    __syncthreads();
    // A(i, l) -= (x_i sc) f_l: one thread per row, four trailing columns per
    // step so that their loads are in flight together; the tail of column j
    // becomes the reflector x sc
    {
      const T* fv = tot + 1;  // f_l at fv[l]
      T* colj = A + (int64_t)j * lda;
      for (int i = i0 + tid; i < rb; i += blockDim.x) {
        const T xi = mul(colj[i], sc);
        int l = 1;
        for (; l + 3 < ncol; l += 4) {
          T* c0 = A + (int64_t)(j + l) * lda + i;
          const T v0 = c0[0], v1 = c0[lda], v2 = c0[2 * lda], v3 = c0[3 * lda];
          c0[0] = msub(v0, xi, fv[l]);
          c0[lda] = msub(v1, xi, fv[l + 1]);
          c0[2 * lda] = msub(v2, xi, fv[l + 2]);
          c0[3 * lda] = msub(v3, xi, fv[l + 3]);
        }
        for (; l < ncol; ++l) {
          T* c0 = A + (int64_t)(j + l) * lda + i;
          *c0 = msub(*c0, xi, fv[l]);
        }
        colj[i] = xi;
      }
      if (j >= ra && j < rb) {  // head row: A(j, l) -= f_l
        for (int l = 1 + tid; l < ncol; l += blockDim.x) {
          T* h = A + (int64_t)(j + l) * lda + j;
          *h = sub(*h, fv[l]);
        }
        if (tid == 0) colj[j] = coef[2];
      }
    }
    __syncthreads();
  }
  cl.sync();
}

// ------------------------------------------------------------------ core
// M = R_A R_B^H (LEAF, kra x krb) or M = R_A (merges, kra x k), column-major ld kcap.
template <typename T>
__global__ void core_kernel(const DenseParams<T> P) {
  const int ti = blockIdx.y;
  const SvdTask t = P.tasks[ti];
  const TaskDims dm = P.dims[ti];
  T* M = P.core + t.m_off;
  const T* A = qr_a_ptr(P, t);
  const int kra = dm.kra;
  if (t.kind == TASK_LEAF) {
    const T* B = P.qr + t.b_off;
    const int krb = dm.krb, k = dm.k;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kra * krb; e += gridDim.x * blockDim.x) {
      const int i = e % kra, j = e / kra;
      T s = Traits<T>::zero();
      for (int p = max(i, j); p < k; ++p) s = mac(s, A[(int64_t)p * t.lda + i], conj_(B[(int64_t)p * t.rows_b + j]));
      M[(int64_t)j * t.kcap + i] = s;
    }
  } else {
    const int k = dm.k;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kra * k; e += gridDim.x * blockDim.x) {
      const int i = e % kra, j = e / kra;
      M[(int64_t)j * t.kcap + i] = (i <= j) ? A[(int64_t)j * t.lda + i] : Traits<T>::zero();
    }
  }
}

// Block-wide max (identical in every CTA of a cluster).
__device__ __forceinline__ double block_max_dense(double v, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s = fmax(s, scratch[w]);
  __syncthreads();
  return s;
}

// Block-wide sum with a fixed order (identical in every CTA of a cluster).
__device__ __forceinline__ double block_sum_dense(double v, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += scratch[w];
  __syncthreads();
  return s;
}

// ------------------------------------------------------------------ QRCP of the core
// Preconditioning of the one-sided Jacobi SVD (Drmac & Veselic, "New fast and
// accurate Jacobi SVD algorithm", SIAM J. Matrix Anal. Appl. 2008): column-
// pivoted Householder QR of the core, M P = Q2 R2 (pivot = largest trailing
// column norm, recomputed explicitly), then the Jacobi sweeps run on the
// graded matrix X = R2^H (nc x p), which converges in a few sweeps.
// M (mr x nc) is overwritten by R2 (column perm[t] holds R2(0..t, t)) and the
// reflector tails; perm (nc ints) lists the pivot order followed by the
// unchosen columns; X = R2^H is written to the x_off region.  One cluster per
// task, column j owned by CTA j mod c: per step every CTA forms the norms of
// its columns and a local argmax, the cluster argmax is taken in rank order
// through DSMEM (ties to the smaller index, identical in every CTA), the
// owner of the pivot column builds the reflector, every CTA copies it to
// shared memory after a cluster barrier and updates its own columns.
struct QcArg {
  long long b;
  int i, pad;
};

template <typename T>
__global__ void __launch_bounds__(kWideThreads) qrcp_core_kernel(const DenseParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank(), c = (int)cl.num_blocks();
  const int ti = blockIdx.x / c;
  if (ti >= P.ntasks) return;  // uniform per cluster
  const SvdTask t = P.tasks[ti];
  const TaskDims dm = P.dims[ti];
  const int mr = dm.kra;
  const int nc = t.kind == TASK_LEAF ? dm.krb : dm.k;
  const int ld = t.kcap;
  if (mr <= 0 || nc <= 0) return;  // uniform per cluster
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  T* M = P.core + t.m_off;
  T* X = P.core + t.x_off;
  T* tau = P.tau + t.tau_off + 2 * t.kcap;
  int32_t* perm = P.ord + t.ord_off + t.kcap;
  // shared memory: [rv: kcap T][coef: 2 T][slots: 2 QcArg][nrm: kcap double]
  //                [wb: 32 ll][wi: 32 int][sh: 4 int][sperm: kcap int][chosen: kcap bytes]
  T* rv = reinterpret_cast<T*>(smem_raw);                        // reflector u (rows st..mr-1)
  T* coef = rv + t.kcap;                                         // [0] conj(tau), [1] beta (re)
  QcArg* aslot = reinterpret_cast<QcArg*>(coef + 2);             // argmax slots (step parity)
  double* nrm = reinterpret_cast<double*>(aslot + 2);            // this CTA's column norms
  long long* wb = reinterpret_cast<long long*>(nrm + t.kcap);    // 32
  int* wi = reinterpret_cast<int*>(wb + 32);                     // 32
  int* sh = wi + 32;                                             // [0] pivot
  int* sperm = sh + 4;                                           // pivot order (every CTA)
  uint8_t* chosen = reinterpret_cast<uint8_t*>(sperm + t.kcap);  // nc
  for (int j = tid; j < nc; j += blockDim.x) chosen[j] = 0;
  __syncthreads();
  const int p = min(mr, nc);
  const int own = (nc - q + c - 1) / c;  // columns q, q + c, ...
  for (int st = 0; st < p; ++st) {
    // norms of this CTA's unchosen columns, local argmax
    // two columns per warp, summed over the warp together
    for (int l = 2 * warp; l < own; l += 2 * nw) {
      const int j0 = q + l * c, j1 = j0 + c;
      const bool u0 = !chosen[j0], u1 = l + 1 < own && !chosen[j1];  // warp-uniform
      if (!u0 && !u1) continue;
      double a0 = 0.0, a1 = 0.0;
      for (int i = st + lane; i < mr; i += 32) {
        if (u0) a0 += abs2(M[(int64_t)j0 * ld + i]);
        if (u1) a1 += abs2(M[(int64_t)j1 * ld + i]);
      }
      warp_sum2_all(a0, a1, lane);
      if (lane == 0) {
        if (u0) nrm[j0] = a0;
        if (u1) nrm[j1] = a1;
      }
    }
    __syncthreads();
    long long bb = -1;
    int bi = INT_MAX;
    for (int l = tid; l < own; l += blockDim.x) {
      const int j = q + l * c;
      if (!chosen[j]) argmax_merge(bb, bi, nbits(nrm[j]), j);
    }
    warp_argmax(bb, bi);
    if (lane == 0) { wb[warp] = bb; wi[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      bb = lane < nw ? wb[lane] : -1;
      bi = lane < nw ? wi[lane] : INT_MAX;
      warp_argmax(bb, bi);
      if (lane == 0) { aslot[st & 1].b = bb; aslot[st & 1].i = bi; }
    }
    cl.sync();
    if (tid == 0) {  // cluster argmax in rank order
      long long gb = -1;
      int gi = INT_MAX;
      for (int r = 0; r < c; ++r) {
        const QcArg* rs = cl.map_shared_rank(aslot + (st & 1), r);
        argmax_merge(gb, gi, rs->b, rs->i);
      }
      sh[0] = gi;
      chosen[gi] = 1;
      sperm[st] = gi;
    }
    __syncthreads();
    const int pc = sh[0];
    T* col = M + (int64_t)pc * ld;
    const int owner = pc % c;
    if (q == owner && warp == 0) {
      const T alpha = col[st];  // read by every lane before lane 0 overwrites it
      double sig2 = 0.0;
      for (int i = st + 1 + lane; i < mr; i += 32) sig2 += abs2(col[i]);
      sig2 = warp_sum(sig2);
      double beta;
      T tu, sc;
      householder(alpha, sig2, beta, tu, sc);  // every lane: the same value
      for (int i = st + 1 + lane; i < mr; i += 32) col[i] = mul(col[i], sc);
      if (lane == 0) {
        coef[0] = conj_(tu);
        coef[1] = from_re<T>(beta);
        tau[st] = tu;
        col[st] = from_re<T>(beta);
      }
    }
    cl.sync();
    // the reflector u = [1; col(st+1:)] and conj(tau) from the owner
    for (int i = st + 1 + tid; i < mr; i += blockDim.x) rv[i] = ldcg(col + i);
    const T ctau = *cl.map_shared_rank(coef, owner);
    __syncthreads();
    for (int l = 2 * warp; l < own; l += 2 * nw) {  // two columns per warp
      const int j0 = q + l * c, j1 = j0 + c;
      const bool u0 = !chosen[j0], u1 = l + 1 < own && !chosen[j1];  // warp-uniform
      if (!u0 && !u1) continue;
      T* y0 = M + (int64_t)j0 * ld;
      T* y1 = M + (int64_t)j1 * ld;
      T w0 = Traits<T>::zero(), w1 = Traits<T>::zero();
      for (int i = st + 1 + lane; i < mr; i += 32) {
        const T r = rv[i];
        if (u0) w0 = cmac(w0, r, y0[i]);
        if (u1) w1 = cmac(w1, r, y1[i]);
      }
      warp_sum2_all(w0, w1, lane);
      if (u0) {
        const T f = mul(ctau, add(w0, y0[st]));
        __syncwarp();
        if (lane == 0) y0[st] = sub(y0[st], f);
        for (int i = st + 1 + lane; i < mr; i += 32) y0[i] = msub(y0[i], rv[i], f);
      }
      if (u1) {
        const T f = mul(ctau, add(w1, y1[st]));
        __syncwarp();
        if (lane == 0) y1[st] = sub(y1[st], f);
        for (int i = st + 1 + lane; i < mr; i += 32) y1[i] = msub(y1[i], rv[i], f);
      }
    }
    // the owner may overwrite coef only after every CTA has read it
    cl.sync();
  }
  if (tid == 0) {  // unchosen columns (nc > mr) follow in index order
    int qq = p;
    for (int j = 0; j < nc; ++j)
      if (!chosen[j]) sperm[qq++] = j;
  }
  __syncthreads();
  if (q == 0)
    for (int j = tid; j < nc; j += blockDim.x) perm[j] = sperm[j];
  // X = R2^H: X(j, i) = conj(R2(i, j)) = conj(M(i, perm[j])) for i <= j, i < p;
  // CTA q writes the rows j = q, q + c, ... (columns of other CTAs read through L2)
  for (int e = tid; e < own * p; e += blockDim.x) {
    const int j = q + (e % own) * c, i = e / own;
    X[(int64_t)i * ld + j] = i <= j ? conj_(ldcg(M + (int64_t)sperm[j] * ld + i)) : Traits<T>::zero();
  }
  cl.sync();
}

// ------------------------------------------------------------------ Jacobi SVD
// One-sided Jacobi (Hestenes) on M (mr x nc): M Y = X S.  Round-robin pairs;
// per pair the warp forms alpha = |a|^2, beta = |b|^2, gamma = a^H b and
// rotates [a, e^{-i phi} b] by the real angle that zeroes their inner product,
// accumulating the same rotation in Y.  The pairs of one round are spread over
// all warps of all CTAs in the cluster; a cluster barrier separates rounds.
// At the end singular values are column norms, sorted descending; s = eps-rank.
// Rotation of one Jacobi pair from alpha = |a|^2, beta = |b|^2, gamma = a^H b.
// Returns false when the pair counts as orthogonal: |gamma| below tol times
// |a| |b|, or both columns negligible, or a column in the denormal range.
//
// The chain runs on one thread per pair while the CTA's other warps wait (and
// an FP64 instruction costs the same pipe time whatever the number of active
// lanes), so its FP64 part is kept short.  Only two quantities must be
// accurate to a few ulp: the phase e^{-i phi} = conj(gamma) / |gamma| and the
// cosine-sine pair (cs^2 + sn^2 = 1), which make the rotation unitary; the
// angle itself only decides how much of gamma the rotation removes, and a
// relative error of 1e-7 there leaves a residual inner product of 1e-7 gamma
// that later sweeps remove (the convergence test is on the inner products
// the sweeps form, not on the angle).  So gamma is scaled by the power of two
// below its larger component (exact), q = |gamma / 2^e|^2 lies in [1, 4),
// and phase = conj(gamma / 2^e) rsqrt(q) in FP64; the tangent
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (beta - alpha) /
// (2 |gamma|), is formed in FP32 (in FP64 as 1 / (2 zeta) when |zeta| > 2^30)
// and widened exactly to FP64, where cs = rsqrt(1 + t^2) and sn = cs t.
__device__ __forceinline__ double pow2_below(double v) {  // 2^floor(log2 v), v > 0 normal
  return __longlong_as_double(__double_as_longlong(v) & 0x7ff0000000000000ll);
}
__device__ __forceinline__ double pow2_inverse(double p2) {  // 1 / p2 for a power of two in the normal range
  return __longlong_as_double(0x7fe0000000000000ll - __double_as_longlong(p2));
}

template <typename T>
__device__ __forceinline__ bool jacobi_rotation(double al, double be, T ga, double tol, double negl, double fro2,
                                                double& cs, double& sn, T& ph, double& tout, double& gabs) {
  if (al < 1e-290 || be < 1e-290 || fmax(al, be) < negl) return false;
  const double mx = fmax(fabs(re_(ga)), fabs(im_(ga)));
  if (!(mx >= 1e-300)) return false;                            // zero (or denormal) gamma
  const double rm = pow2_inverse(pow2_below(mx));               // exact: mx rm in [1, 2)
  const double gr = re_(ga) * rm, gi = im_(ga) * rm;
  const double q = fma(gr, gr, gi * gi);                        // |gamma rm|^2 in [1, 4)
  if (q < (tol * tol) * (al * rm) * (be * rm)) return false;    // |gamma| <= tol |a| |b|
  const double rq = rsqrt(q);
  // zeta = (beta - alpha) / (2 |gamma|), |gamma| = sqrt(q) / rm; for
  // |zeta| > 2^30 the tangent is 1 / (2 zeta) to double precision (and the
  // FP32 form would lose it), formed in FP64
  const double zeta = (be - al) * rm * 0.5 * rq;
  double tt;
  if (fabs(zeta) > 1073741824.0) {
    tt = __drcp_rn(2.0 * zeta);
  } else {
    const float zf = (float)zeta;
    tt = (double)copysignf(1.0f / (fabsf(zf) + sqrtf(fmaf(zf, zf, 1.0f))), zf);
  }
  cs = rsqrt(fma(tt, tt, 1.0));
  sn = cs * tt;
  tout = tt;
  gabs = q * rq * pow2_below(mx);  // |gamma| = sqrt(q) / rm
  if constexpr (Traits<T>::is_complex) ph = mk(gr * rq, -gi * rq);  // e^{-i phi}, gamma = |gamma| e^{i phi}
  else ph = gr >= 0.0 ? 1.0 : -1.0;
  return true;
}

constexpr int kJacRegs = 8;  // columns of up to 256 rows are held in registers
// columns of up to 32 * JacKeep<T>::n rows stay in registers from (1) to (3)
// (real data; complex columns are re-read, which keeps the kernel within the
// registers of three resident CTAs per SM)
template <typename T> struct JacKeep { static constexpr int n = 5; };
template <> struct JacKeep<cplx> { static constexpr int n = 0; };

// Loads of the Jacobi sweeps: columns in another CTA's shared memory are read
// with plain (distributed shared memory) loads, columns in global memory
// through L2.
template <typename T, bool kDsm>
__device__ __forceinline__ T jld(const T* p) {
  if constexpr (kDsm) return *p;
  else return ldcg(p);
}

// One element of a Jacobi rotation with the phase folded in:
// a' = cs a - sp b, b' = sn a + cp b with sp = sn ph, cp = cs ph (ph = e^{-i phi}).
__device__ __forceinline__ void rot_elem(double& a, double& b, double cs, double sn, double sp, double cp) {
  const double a0 = a, b0 = b;
  a = fma(-sp, b0, cs * a0);
  b = fma(cp, b0, sn * a0);
}
__device__ __forceinline__ void rot_elem(cplx& a, cplx& b, double cs, double sn, cplx sp, cplx cp) {
  const cplx a0 = a, b0 = b;
  a.re = fma(sp.im, b0.im, fma(-sp.re, b0.re, cs * a0.re));
  a.im = fma(-sp.im, b0.re, fma(-sp.re, b0.im, cs * a0.im));
  b.re = fma(-cp.im, b0.im, fma(cp.re, b0.re, sn * a0.re));
  b.im = fma(cp.im, b0.re, fma(cp.re, b0.im, sn * a0.im));
}

template <typename T, bool kDsm>
__device__ __forceinline__ void rotate_pair_t(T* a, T* b, int len, double cs, double sn, T sp, T cp, int lane) {
  for (int i = lane; i < len; i += 32) {
    T ai = jld<T, kDsm>(a + i), bi = jld<T, kDsm>(b + i);
    rot_elem(ai, bi, cs, sn, sp, cp);
    a[i] = ai;
    b[i] = bi;
  }
}

// Inner products of a pair posted by its warp, turned into the pair's
// rotation by one thread of the CTA.
template <typename T>
struct JPair {
  double al, be;
  T ga;
  double cs, sn;
  T sp, cp;
  int ok, a, b;  // a, b: the pair's columns
  float c2;      // |gamma|^2 / (alpha beta) of a rotation that counts against convergence
};
constexpr int kJSlotMax = 96;  // bytes reserved per pair slot (>= sizeof(JPair<cplx>))

// The sweeps of one task.  kDsm: column j of X and of the accumulated rotation
// W live in the shared memory of CTA j mod c of the cluster, slot j / c
// ([X(0..mr-1), W(0..nc-1)], stride ldc); otherwise X and W are in global
// memory (column j at M + j ld, Y + j ld).  A round's pairs are dealt to the
// warps of the cluster; each CTA (1) forms the inner products of all its
// pairs, (2) turns them into rotations, one thread per pair, (3) rotates its
// pairs' columns; one cluster barrier ends the round.
// A core too large for one cluster's shared memory may be swept by G
// clusters at once (columns in global memory, a cooperative launch): the
// pairs of a round are dealt over all G c CTAs, and a round ends with the
// cluster barrier plus an arrival count on the task's counter (bounded wait,
// HBACA_TIMEOUT on expiry); the per-sweep decisions are summed over the
// clusters through global slots.  Every rotation is formed and applied with
// the same arithmetic as with one cluster, so the result does not depend on G.
struct JGroup {
  int G;              // clusters per core (1: no grouping)
  unsigned* cnt;      // arrival counter per core of the launch (zeroed before it)
  double* slots;      // [cluster of the launch][2][4] per-sweep values
};

template <typename T, bool kDsm>
__device__ void jacobi_sweeps(cg::cluster_group& cl, int q, int c, int mr, int nc, int K, T* M, T* Y, int64_t ld,
                              T* dsm, int64_t ldc, double tol, double negl, double fro2, double& cmax, double eps,
                              int max_sweeps, int* flag, double* cmx, JPair<T>* slots, int& sweep, int& nrot,
                              bool acc_w, T* const* ctab, int* c2bits, bool& converged, double* gnrm,
                              int ql, int csz, const JGroup& jg, int tl, int g, int* xok, int* status) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // column addresses from the table (no division by the cluster size per access)
  auto colX = [&](int j) -> T* { return ctab[j]; };
  auto colW = [&](int j) -> T* {
    if constexpr (kDsm) return ctab[j] + mr + 1;
    else return Y + (int64_t)j * ld;
  };
  // The squared column norms (in the column's shared-memory slot after X, or
  // in gnrm[j] on the global-memory path) are formed exactly at the start of
  // every sweep and carried through the sweep's rotations by |a'|^2 = |a|^2 -
  // t |gamma|, |b'|^2 = |b|^2 + t |gamma| (t the tangent), so a pair's inner
  // product is gamma alone; an update that loses more than three digits to
  // cancellation (the new value below 1e-3 of the old) is marked -1 and the
  // norm is formed again with the pair's inner product.  Both paths do the
  // same arithmetic.
  auto nrm = [&](int j) -> double* {
    if constexpr (kDsm) return reinterpret_cast<double*>(ctab[j] + mr);
    else return gnrm + j;
  };
  auto nrm_ld = [&](int j) -> double {
    if constexpr (kDsm) return *nrm(j);
    else return ldcg(gnrm + j);
  };
  // the end of a round: every CTA of the cluster, and with G > 1 every
  // cluster of the core (columns written by one cluster are read by others
  // in the next round: each writer fences, the leader counts the cluster in)
  unsigned nbar = 0;
  auto group_barrier = [&]() -> bool {
    if (jg.G > 1) __threadfence();
    cl.sync();
    if (jg.G == 1) return true;
    ++nbar;
    if (ql == 0 && threadIdx.x == 0) *xok = xgroup_arrive_wait(jg.cnt + tl, nbar * (unsigned)jg.G, status);
    cl.sync();
    return *cl.map_shared_rank(xok, 0) != 0;
  };
  bool ok = true;
  const int per = (nc + c - 1) / c;
  const int npairs = K / 2;
  const int stride = c * nw;                             // pairs dealt per pass over the cluster's warps
  const int per_warp = (npairs + stride - 1) / stride;   // passes (pairs per warp) per round
  const bool regs = mr <= 32 * kJacRegs;
  constexpr int kJacKeep = JacKeep<T>::n > 0 ? JacKeep<T>::n : 1;
  const bool keep = JacKeep<T>::n > 0 && mr <= 32 * JacKeep<T>::n;
  auto pair_of = [&](int rd, int pi, int& a, int& b) {
    // circle method: pair 0 = (rd, K-1), pair i = ((rd+i) mod (K-1), (rd-i+K-1) mod (K-1))
    if (pi == 0) { a = rd; b = K - 1; }
    else { a = (rd + pi) % (K - 1); b = (rd - pi + K - 1) % (K - 1); }
    if (a > b) { int tmp = a; a = b; b = tmp; }
  };
  unsigned fb = 0;
  for (; sweep < max_sweeps && K > 1; ++sweep) {
    const double tau2 = 0.01 * eps * eps * cmax;
    double wmax = 0.0;
    if (tid == 0) { flag[fb & 1] = 0; *cmx = 0.0; c2bits[fb & 1] = 0; }
    for (int l = warp; l < per; l += nw) {  // this CTA's columns, exactly
      const int j = l * c + q;
      if (j >= nc) continue;
      const T* cj = colX(j);
      double v = 0.0;
      for (int i = lane; i < mr; i += 32) v = acc_abs2(v, jld<T, kDsm>(cj + i));
      v = warp_sum(v);
      if (lane == 0) *nrm(j) = v;
      wmax = fmax(wmax, v);
    }
    __syncthreads();
    if (!group_barrier()) break;
    __syncthreads();
    for (int rd = 0; rd < K - 1; ++rd) {
      // (1) inner products of this warp's pairs; the first pass keeps its
      // two columns in registers for (3)
      T ka[kJacKeep], kb[kJacKeep];
      for (int j = 0; j < per_warp; ++j) {
        // pairs are dealt to the CTAs first (pair j * stride + warp * c + q),
        // so a round with fewer pairs than warps spreads over all CTAs and
        // over the four schedulers of each SM (warps 0-3 first)
        const int pi = j * stride + warp * c + q;
        int a = 0, b = 0;
        bool act = pi < npairs;
        if (act) {
          pair_of(rd, pi, a, b);
          act = b < nc;  // else a padding column
        }
        double al = 0.0, be = 0.0;
        T ga = Traits<T>::zero();
        if (act) {
          const T* ca = colX(a);
          const T* cb = colX(b);
          // the pair's inner products over the rows; with_norms: also |a|^2, |b|^2
          auto dots = [&](auto with_norms) {
            constexpr bool kN = decltype(with_norms)::value;
            if (regs) {
#pragma unroll
              for (int u = 0; u < kJacRegs; ++u) {
                const int i = lane + 32 * u;
                if (32 * u < mr) {  // warp-uniform: no FP64 work on padding
                  const T xa = i < mr ? jld<T, kDsm>(ca + i) : Traits<T>::zero();
                  const T xb = i < mr ? jld<T, kDsm>(cb + i) : Traits<T>::zero();
                  if constexpr (kN) {
                    al = acc_abs2(al, xa);
                    be = acc_abs2(be, xb);
                  }
                  ga = cmac(ga, xa, xb);
                  if (u < kJacKeep && j == 0) {
                    ka[u < kJacKeep ? u : 0] = xa;
                    kb[u < kJacKeep ? u : 0] = xb;
                  }
                }
              }
            } else {
              for (int i = lane; i < mr; i += 32) {
                const T xa = jld<T, kDsm>(ca + i), xb = jld<T, kDsm>(cb + i);
                if constexpr (kN) {
                  al = acc_abs2(al, xa);
                  be = acc_abs2(be, xb);
                }
                ga = cmac(ga, xa, xb);
              }
            }
          };
          const double na = nrm_ld(a), nb = nrm_ld(b);
          if (na < 0.0 || nb < 0.0) {  // warp-uniform
            dots(std::true_type{});
            // the four sums by recursive halving (6 FP64 adds instead of 20),
            // then every lane takes them from the lanes that hold them
            double v4[4] = {al, be, re_(ga), im_(ga)};
            const double sum = warp_reduce_scatter<4>(v4, lane);
            al = __shfl_sync(0xffffffffu, sum, 0);
            be = __shfl_sync(0xffffffffu, sum, 8);
            if constexpr (Traits<T>::is_complex) ga = mk(__shfl_sync(0xffffffffu, sum, 16), __shfl_sync(0xffffffffu, sum, 24));
            else ga = __shfl_sync(0xffffffffu, sum, 16);
          } else {
            dots(std::false_type{});
            if constexpr (Traits<T>::is_complex) {
              double v2[2] = {ga.re, ga.im};
              const double sum = warp_reduce_scatter<2>(v2, lane);
              ga = mk(__shfl_sync(0xffffffffu, sum, 0), __shfl_sync(0xffffffffu, sum, 16));
            } else {
              ga = warp_sum(ga);
            }
            al = na;
            be = nb;
          }
        }
        if (lane == 0) {
          JPair<T>& sl = slots[j * nw + warp];
          sl.al = al;
          sl.be = be;
          sl.ga = ga;
          sl.ok = act ? 1 : 0;
          sl.a = a;
          sl.b = b;
        }
      }
      __syncthreads();
      // (2) rotations, one thread per pair
      for (int sidx = tid; sidx < per_warp * nw; sidx += blockDim.x) {
        JPair<T>& sl = slots[sidx];
        if (!sl.ok) continue;
        double cs, sn, tt, gabs;
        T ph;
        if (jacobi_rotation(sl.al, sl.be, sl.ga, tol, negl, fro2, cs, sn, ph, tt, gabs)) {
          sl.cs = cs;
          sl.sn = sn;
          sl.sp = scale(ph, sn);
          sl.cp = scale(ph, cs);
          if (fmax(sl.al, sl.be) >= tau2) {  // counts; the largest cosine^2 of the sweep's counted rotations
            sl.ok = 2;
            const float c2 = (float)(abs2(sl.ga) / (sl.al * sl.be));
            atomicMax(&c2bits[fb & 1], __float_as_int(c2));
          }
          {  // the pair's norms after the rotation
            const double na = fma(-tt, gabs, sl.al), nb = fma(tt, gabs, sl.be);
            sl.al = na >= 1e-3 * sl.al ? na : -1.0;
            sl.be = nb >= 1e-3 * sl.be ? nb : -1.0;
          }
        } else {
          sl.ok = 0;
        }
      }
      __syncthreads();
      // (3) rotate this warp's pairs
      for (int j = 0; j < per_warp; ++j) {
        const JPair<T>& sl = slots[j * nw + warp];
        if (!sl.ok) continue;  // warp-uniform
        const int a = sl.a, b = sl.b;
        const double cs = sl.cs, sn = sl.sn;
        const T spv = sl.sp, cpv = sl.cp;
        if (lane == 0) {
          if (sl.ok == 2) flag[fb & 1] = 1;
          *nrm(a) = sl.al;
          *nrm(b) = sl.be;
        }
        ++nrot;
        T* ca = colX(a);
        T* cb = colX(b);
        if (keep && j == 0) {
#pragma unroll
          for (int u = 0; u < kJacKeep; ++u) {
            const int i = lane + 32 * u;
            if (32 * u < mr && i < mr) {
              rot_elem(ka[u], kb[u], cs, sn, spv, cpv);
              ca[i] = ka[u];
              cb[i] = kb[u];
            }
          }
        } else {
          rotate_pair_t<T, kDsm>(ca, cb, mr, cs, sn, spv, cpv, lane);
        }
        if (acc_w) rotate_pair_t<T, kDsm>(colW(a), colW(b), nc, cs, sn, spv, cpv, lane);
      }
      if (!(ok = group_barrier())) break;
    }
    if (!ok) break;
    // the largest column norm^2 of this sweep, over the cluster (for the next tau)
    if (lane == 0) atomicMax(reinterpret_cast<unsigned long long*>(cmx), (unsigned long long)__double_as_longlong(wmax));
    __syncthreads();
    cl.sync();
    // any relevant rotation anywhere in the cluster this sweep?  And the
    // largest cosine among them: the sweeps converge quadratically, so after a
    // sweep whose cosines are all below 0.1 sqrt(tol) the next one would find
    // none above tol (its only work would be the inner products): stop here
    int any = 0, c2b = 0;
    double cm = 0.0;
    for (int r = 0; r < csz; ++r) {
      any |= *cl.map_shared_rank(&flag[fb & 1], r);
      cm = fmax(cm, *cl.map_shared_rank(cmx, r));
      c2b = max(c2b, *cl.map_shared_rank(&c2bits[fb & 1], r));
    }
    if (jg.G > 1) {  // over the clusters of the core, in cluster order
      double* mine = jg.slots + ((size_t)(tl * jg.G + g) * 2 + (fb & 1)) * 4;
      if (ql == 0 && threadIdx.x == 0) {
        mine[0] = (double)any;
        mine[1] = cm;
        mine[2] = (double)__int_as_float(c2b);
      }
      if (!group_barrier()) break;
      any = 0;
      c2b = 0;
      cm = 0.0;
      for (int gg = 0; gg < jg.G; ++gg) {
        const double* sl2 = jg.slots + ((size_t)(tl * jg.G + gg) * 2 + (fb & 1)) * 4;
        any |= ldcg(sl2) != 0.0;
        cm = fmax(cm, ldcg(sl2 + 1));
        c2b = max(c2b, __float_as_int((float)ldcg(sl2 + 2)));
      }
    }
    if (cm > 0.0) cmax = cm;
    ++fb;
    cl.sync();
    if (!any) { converged = true; break; }
    if ((double)__int_as_float(c2b) < 0.01 * tol) { converged = true; break; }  // sweep = executed - 1, as above
  }
}

template <typename T>
__global__ void __launch_bounds__(kDenseThreads, 3) jacobi_kernel(const DenseParams<T> P, int max_sweeps,
                                                                   int hdr_bytes, int slot_off, int64_t dsm_bytes,
                                                                   const int32_t* task_list, const JGroup jg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int xok;
  cg::cluster_group cl = cg::this_cluster();
  // ql / csz: rank in the cluster and cluster size; q / c: rank and number
  // of CTAs over the jg.G clusters that sweep one core (the same with G = 1)
  const int ql = (int)cl.block_rank(), csz = (int)cl.num_blocks();
  const int cid = (int)(blockIdx.x / csz);
  const int tl = cid / jg.G, g = cid - tl * jg.G;
  const int q = g * csz + ql, c = jg.G * csz;
  const int ti = task_list ? task_list[tl] : tl;
  const SvdTask t = P.tasks[ti];
  const TaskDims dm = P.dims[ti];
  // the sweeps orthogonalise the columns of X = R2^H (nc_M x p), accumulating W
  const int ncm = t.kind == TASK_LEAF ? dm.krb : dm.k;
  const int mr = ncm;
  const int nc = min(dm.kra, ncm);
  T* M = P.core + t.x_off;
  T* Y = P.core + t.y_off;
  const int ld = t.kcap;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  int* flag = reinterpret_cast<int*>(smem_raw);  // [0..1] rotation-applied flags (double-buffered)
  double* sv = reinterpret_cast<double*>(smem_raw + 16);  // nc singular values (CTA 0, sorting)
  if (mr <= 0 || nc <= 0) {
    if (q == 0 && tid == 0) {
      P.dims[ti].s = 0;
      P.dims[ti].nout = 0;
      P.out_rank[P.out_blocks[t.out].rank_slot] = 0;
      if (P.out_blocks[t.out].full_slot >= 0) P.out_rank[P.out_blocks[t.out].full_slot] = 0;
    }
    return;
  }
  // the task's columns fit the cluster's shared memory: sweep there (column j
  // in CTA j mod c), else in global memory
  // the rotations are accumulated (W) only for a taped output, which keeps
  // every triplet; otherwise the kept right vectors of X are recovered from
  // X^H z_i = sigma_i w_i after the sweeps (wsolve_kernel), and a column's
  // shared-memory slot holds X alone
  const bool acc_w = P.out_blocks[t.out].full_slot >= 0;
  const int per = (nc + c - 1) / c;
  const int64_t ldc = (int64_t)mr + 1 + (acc_w ? nc : 0);  // X, the squared norm, W
  T* dsm = reinterpret_cast<T*>(smem_raw + hdr_bytes);
  const bool use_dsm = jg.G == 1 && (int64_t)per * ldc * (int64_t)sizeof(T) <= dsm_bytes;
  if (use_dsm) {  // own columns: X from global memory, W = I
    for (int l = warp; l < per; l += nw) {
      const int j = l * c + q;
      if (j >= nc) continue;
      T* dst = dsm + (int64_t)l * ldc;
      for (int i = lane; i < mr; i += 32) dst[i] = M[(int64_t)j * ld + i];
      if (acc_w)
        for (int i = lane; i < nc; i += 32) dst[mr + 1 + i] = from_re<T>(i == j ? 1.0 : 0.0);
    }
  } else if (acc_w) {  // Y = I
    const int j0 = q * per, j1 = min(nc, j0 + per);
    for (int j = j0; j < j1; ++j)
      for (int i = tid; i < nc; i += blockDim.x) Y[(int64_t)j * ld + i] = from_re<T>(i == j ? 1.0 : 0.0);
  }
  const int K = nc + (nc & 1);
  const double tol = 4.0e-16 * (double)max(mr, 8);
  // ||M||_F^2 (rotation invariant) and the largest column norm^2, the same in
  // every CTA (fixed summation order)
  double fro2 = 0.0, cmax = 0.0;
  {
    double part = 0.0, pm = 0.0;
    for (int j = warp; j < nc; j += nw) {
      double cj = 0.0;
      for (int i = lane; i < mr; i += 32) cj += abs2(M[(int64_t)j * ld + i]);
      cj = warp_sum(cj);
      part += (lane == 0) ? cj : 0.0;
      pm = fmax(pm, cj);
    }
    fro2 = block_sum_dense(part, sv);
    cmax = block_max_dense(pm, sv);
  }
  // a pair of columns both below 1e-3 eps ||M||_F (<= 0.011 eps sigma_1 for
  // nc <= 128) cannot affect a singular value or vector above the eps-rank
  // threshold: such pairs are not rotated
  const double negl = 1e-6 * P.eps * P.eps * fro2;
  // a rotation counts against convergence only if it touches a column that can
  // still be kept (norm >= 0.1 eps max column norm); columns below that never
  // grow (a rotation always shrinks the smaller column of its pair), so they
  // cannot cross the eps-rank threshold.  All pairs are still rotated.
  double* cmx = reinterpret_cast<double*>(smem_raw + 8);  // largest column norm^2 seen this sweep
  int sweep = 0;
  int nrot = 0;  // rotations applied by this warp
  if (tid == 0) { flag[0] = 0; flag[1] = 0; }
  cl.sync();
  JPair<T>* slots = reinterpret_cast<JPair<T>*>(smem_raw + slot_off);
  // two ints of the header's slack just below the pair slots (slot_off is at
  // least 56 bytes past the order table)
  int* c2bits = reinterpret_cast<int*>(smem_raw + slot_off - 8);
  bool converged = false;
  // the squared column norms of the global-memory path, in the compact-X
  // area of the task (written only after the sweeps, by finish_kernel)
  double* gnrm = reinterpret_cast<double*>(P.core + t.xs_off);
  // column addresses of X for the sweeps, in the singular-value area (free
  // until the epilogue): column j in CTA j mod c (DSMEM) or in global memory
  T** ctab = reinterpret_cast<T**>(sv);
  for (int j = tid; j < nc; j += blockDim.x)
    ctab[j] = use_dsm ? cl.map_shared_rank(dsm, j % csz) + (int64_t)(j / csz) * ldc : M + (int64_t)j * ld;
  __syncthreads();
  if (use_dsm)
    jacobi_sweeps<T, true>(cl, q, c, mr, nc, K, M, Y, ld, dsm, ldc, tol, negl, fro2, cmax, P.eps, max_sweeps, flag, cmx,
                           slots, sweep, nrot, acc_w, ctab, c2bits, converged, gnrm, ql, csz, jg, tl, g, &xok, P.status);
  else
    jacobi_sweeps<T, false>(cl, q, c, mr, nc, K, M, Y, ld, dsm, ldc, tol, negl, fro2, cmax, P.eps, max_sweeps, flag,
                            cmx, slots, sweep, nrot, acc_w, ctab, c2bits, converged, gnrm, ql, csz, jg, tl, g, &xok, P.status);
  // the sweep cap was reached while relevant rotations were still being
  // applied: the singular values and the eps-rank come from an unconverged
  // SVD, which the call reports (the loop leaves through its convergence
  // test before the cap otherwise)
  if (K > 1 && !converged && q == 0 && tid == 0) set_status(P.status, DS_NOT_CONVERGED);
  __syncthreads();
  if (use_dsm) {  // the sweeps' result back to global memory for the epilogue and finish_kernel
    for (int l = warp; l < per; l += nw) {
      const int j = l * c + q;
      if (j >= nc) continue;
      const T* src = dsm + (int64_t)l * ldc;
      for (int i = lane; i < mr; i += 32) M[(int64_t)j * ld + i] = src[i];
      if (acc_w)
        for (int i = lane; i < nc; i += 32) Y[(int64_t)j * ld + i] = src[mr + 1 + i];
    }
  }
  cl.sync();
  if (lane == 0 && nrot) atomicAdd(&P.dims[ti].rotations, nrot);
  // the first cluster of the core finishes it (the others' columns are in
  // global memory, fenced before their last arrival)
  if (g != 0) return;
  // singular values and their order (CTA 0); then every CTA normalises a
  // share of the kept columns of M in place (X = M / sigma) and writes S
  int* ord = reinterpret_cast<int*>(sv + nc);
  int* sshare = ord + nc;
  if (q == 0) {
    for (int j = warp; j < nc; j += nw) {
      double s = 0.0;
      for (int i = lane; i < mr; i += 32) s += abs2(ldcg(M + (int64_t)j * ld + i));
      s = warp_sum(s);
      if (lane == 0) sv[j] = sqrt(s);
    }
    __syncthreads();
    for (int j = tid; j < nc; j += blockDim.x) {  // rank by (value desc, index asc)
      int rk = 0;
      const double vj = sv[j];
      for (int i = 0; i < nc; ++i) rk += (sv[i] > vj) || (sv[i] == vj && i < j);
      ord[rk] = j;
    }
    __syncthreads();
    for (int j = tid; j < nc; j += blockDim.x) P.ord[t.ord_off + j] = ord[j];
    if (tid == 0) {
      const double s1 = sv[ord[0]];
      int s = 0;
      if (s1 > 0.0 && isfinite(s1)) {
        const int pmax = min(nc, mr);
        if (t.trunc > 0) {
          // Frobenius rule: the fewest values whose discarded tail
          // sqrt(sum_{j >= s} sigma_j^2) is at most eps / sqrt(2L + 1) of
          // sqrt(sum_j sigma_j^2); the tail grows from the smallest value.
          // The values are scaled by the power of two below sigma_1 (exact,
          // so every comparison is the unscaled one; the squares cannot
          // overflow)
          const double budget = P.eps / sqrt((double)t.trunc);
          const double r2 = pow2_inverse(pow2_below(s1));
          double total = 0.0;
          for (int j = 0; j < pmax; ++j) {
            const double v = sv[ord[j]] * r2;
            total = fma(v, v, total);
          }
          const double lim = budget * sqrt(total);
          double tail = 0.0;
          s = pmax;
          while (s > 0) {
            const double v = sv[ord[s - 1]] * r2;
            const double nt = fma(v, v, tail);
            if (!(sqrt(nt) <= lim)) break;
            tail = nt;
            --s;
          }
        } else {
          while (s < pmax && sv[ord[s]] >= P.eps * s1) ++s;
        }
      }
      if (!isfinite(s1)) set_status(P.status, DS_NUMERICAL);
      const BlockRef ob = P.out_blocks[t.out];
      if (s > ob.cap) { set_status(P.status, DS_RANK_CAPACITY); s = ob.cap; }
      // a taped output keeps every triplet of the core (the kept ones first)
      const int nout = ob.full_slot >= 0 ? min(min(nc, mr), ob.store_cap) : s;
      sshare[0] = nout;
      P.dims[ti].s = s;
      P.dims[ti].nout = nout;
      P.dims[ti].sweeps = sweep;
      P.out_rank[ob.rank_slot] = s;
      if (ob.full_slot >= 0) P.out_rank[ob.full_slot] = nout;
    }
  }
  cl.sync();
  {
    const double* sv0 = cl.map_shared_rank(sv, 0);
    const int* ord0 = cl.map_shared_rank(ord, 0);
    const int s = *cl.map_shared_rank(sshare, 0);
    const BlockRef ob = P.out_blocks[t.out];
    for (int tc = ql * nw + warp; tc < s; tc += csz * nw) {
      const int j = ord0[tc];
      const double sg = sv0[j];
      const double inv = sg > 0.0 ? 1.0 / sg : 0.0;  // a zero singular value (taped outputs only)
      for (int i = lane; i < mr; i += 32) M[(int64_t)j * ld + i] = scale(ldcg(M + (int64_t)j * ld + i), inv);
      if (lane == 0) out_s(P, ob)[tc] = sg;
    }
  }
  cl.sync();
}

// ------------------------------------------------------------------ right vectors of X
// For an output that keeps only its eps-rank triplets the sweeps do not
// accumulate W; its kept columns come from the SVD relation X^H z_i = sigma_i
// w_i with X = R2^H, i.e. w_i = R2 z_i / sigma_i (R2 upper trapezoidal, the
// pivoted QR of the core left in place: pivoted column c at physical column
// perm[c]), written to W's column ord[tc] as the
// accumulated rotation would have been.  The error of w_i is about
// eps_mach sigma_1 / sigma_i (at most eps_mach / eps for kept triplets); one
// modified Gram-Schmidt pass over the s columns restores orthonormality.
// One CTA per task.
constexpr int kMaxWsolveCols = 1024;  // kept triplets of one output (rank caps are <= 1024)

template <typename T>
__global__ void __launch_bounds__(kDenseThreads) wsolve_kernel(const DenseParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank(), c = (int)cl.num_blocks();
  const int ti = blockIdx.x / c;
  const SvdTask t = P.tasks[ti];
  const BlockRef ob = P.out_blocks[t.out];
  if (ob.full_slot >= 0) return;  // taped: W was accumulated (uniform over the cluster)
  const TaskDims dm = P.dims[ti];
  const int s = min(dm.nout, kMaxWsolveCols);
  const int ncm = t.kind == TASK_LEAF ? dm.krb : dm.k;
  const int p = min(dm.kra, ncm);
  if (s <= 0 || p <= 0) return;
  const int ld = t.kcap;
  const T* R2 = P.core + t.m_off;   // R2(r, c) at R2[perm[c] ld + r], r <= c (columns not moved)
  const int32_t* perm = P.ord + t.ord_off + t.kcap;
  const T* Z = P.core + t.x_off;    // z_j (normalised for the kept j) at Z[j ld + i], i < ncm
  T* W = P.core + t.y_off;
  const int32_t* ord = P.ord + t.ord_off;
  const double* sg = out_s(P, ob);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // w_tc(r) = sum_{c >= r} R2(r, c) z_ord(c) / sigma_tc; a warp per tc (dealt
  // over the cluster), a lane per r
  for (int tc = q * nw + warp; tc < s; tc += c * nw) {
    const int j = ord[tc];
    const double inv = sg[tc] > 0.0 ? 1.0 / sg[tc] : 0.0;
    const T* z = Z + (int64_t)j * ld;
    T* w = W + (int64_t)j * ld;
    for (int r = lane; r < p; r += 32) {
      T acc = Traits<T>::zero();
      for (int cc = r; cc < ncm; ++cc) acc = mac(acc, R2[(int64_t)perm[cc] * ld + r], ldcg(z + cc));
      w[r] = scale(acc, inv);
    }
  }
  // one classical Gram-Schmidt pass in the sorted order (the columns are
  // orthonormal up to ~eps_mach / eps, so one pass suffices); CTA q of the
  // cluster owns a slice of the rows, and the inner products and norms are
  // summed over the cluster in rank order (the same totals in every CTA)
  T* part = reinterpret_cast<T*>(smem_raw);   // [2][s] partial inner products (step parity)
  T* dd = part + 2 * s;                        // [s] totals
  double* pn = reinterpret_cast<double*>(dd + s);  // [2] partial norms^2 (step parity)
  double* red = pn + 2;                        // [32]
  const int chunk = (p + c - 1) / c;
  const int ra = min(p, q * chunk), rb = min(p, ra + chunk);
  __syncthreads();
  cl.sync();  // every W column complete (other CTAs' rows are read through L2)
  for (int tc = 0; tc < s; ++tc) {
    T* wt = W + (int64_t)ord[tc] * ld;
    T* pb = part + (tc & 1) * s;
    for (int u = 2 * warp; u < tc; u += 2 * nw) {  // partial d_u = w_u^H w_tc, two per warp
      const bool two = u + 1 < tc;  // warp-uniform
      const T* wu0 = W + (int64_t)ord[u] * ld;
      const T* wu1 = W + (int64_t)ord[two ? u + 1 : u] * ld;
      T p0 = Traits<T>::zero(), p1 = Traits<T>::zero();
      for (int r = ra + lane; r < rb; r += 32) {
        const T x = ldcg(wt + r);
        p0 = cmac(p0, ldcg(wu0 + r), x);
        if (two) p1 = cmac(p1, ldcg(wu1 + r), x);
      }
      warp_sum2_all(p0, p1, lane);
      if (lane == 0) {
        pb[u] = p0;
        if (two) pb[u + 1] = p1;
      }
    }
    __syncthreads();
    if (tc > 0) {
      cl.sync();
      for (int u = tid; u < tc; u += blockDim.x) {
        T sum = Traits<T>::zero();
        for (int r = 0; r < c; ++r) sum = add(sum, cl.map_shared_rank(part + (tc & 1) * s, r)[u]);
        dd[u] = sum;
      }
      __syncthreads();
    }
    double nloc = 0.0;
    for (int r = ra + tid; r < rb; r += blockDim.x) {  // w_tc -= sum_u w_u d_u (own rows)
      T v = ldcg(wt + r);
      for (int u = 0; u < tc; ++u) v = msub(v, ldcg(W + (int64_t)ord[u] * ld + r), dd[u]);
      wt[r] = v;
      nloc += abs2(v);
    }
    nloc = warp_sum(nloc);
    if (lane == 0) red[warp] = nloc;
    __syncthreads();
    if (tid == 0) {
      double a = 0.0;
      for (int q2 = 0; q2 < nw; ++q2) a += red[q2];
      pn[tc & 1] = a;
    }
    cl.sync();
    double nrm = 0.0;
    for (int r = 0; r < c; ++r) nrm += *cl.map_shared_rank(pn + (tc & 1), r);
    const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
    for (int r = ra + tid; r < rb; r += blockDim.x) wt[r] = scale(wt[r], inv);
    __syncthreads();
  }
  cl.sync();  // the normalised W complete before any CTA leaves (DSMEM reads done)
}

// ------------------------------------------------------------------ finish
// Singular vectors of the core M from the preconditioned Jacobi: with
// X = R2^H, X W = Z S and M P = Q2 R2, M = (Q2 W) S (P Z)^H.  Writes, for the
// s kept columns in descending order, Xs = Q2 [W(:, ord); 0] (mr x s) and
// Ys(perm[j], :) = Z(j, ord) (nc x s).  One warp per output column.
template <typename T>
__global__ void finish_kernel(const DenseParams<T> P) {
  const int ti = blockIdx.y;
  const SvdTask t = P.tasks[ti];
  const TaskDims dm = P.dims[ti];
  const int s = dm.nout;  // columns written (the kept s, or all when taped)
  const int mr = dm.kra;
  const int nc = t.kind == TASK_LEAF ? dm.krb : dm.k;
  const int p = min(mr, nc);
  const int ld = t.kcap;
  const T* M = P.core + t.m_off;
  const T* W = P.core + t.y_off;
  const T* Z = P.core + t.x_off;
  T* Xs = P.core + t.xs_off;
  T* Ys = P.core + t.ys_off;
  const T* tau = P.tau + t.tau_off + 2 * t.kcap;
  const int32_t* ord = P.ord + t.ord_off;
  const int32_t* perm = P.ord + t.ord_off + t.kcap;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwt = (gridDim.x * blockDim.x) >> 5;
  for (int tc = gw; tc < s; tc += nwt) {
    const int jo = ord[tc];
    T* v = Xs + (int64_t)tc * ld;
    for (int i = lane; i < mr; i += 32) v[i] = i < p ? W[(int64_t)jo * ld + i] : Traits<T>::zero();
    __syncwarp();
    for (int st = p - 1; st >= 0; --st) {
      const T* u = M + (int64_t)perm[st] * ld;
      T w = Traits<T>::zero();
      for (int i = st + 1 + lane; i < mr; i += 32) w = cmac(w, u[i], v[i]);
      w = warp_sum(w);
      w = add(w, v[st]);
      const T f = mul(tau[st], w);
      __syncwarp();
      if (lane == 0) v[st] = sub(v[st], f);
      for (int i = st + 1 + lane; i < mr; i += 32) v[i] = msub(v[i], u[i], f);
      __syncwarp();
    }
    for (int j = lane; j < nc; j += 32) Ys[(int64_t)tc * ld + perm[j]] = Z[(int64_t)jo * ld + j];
  }
}

// ------------------------------------------------------------------ Q application
// D = Q [Z; 0] with Q = H_0 H_1 ... H_{kk-1} from qr_kernel (Z = X_s for the A
// side, Y_s for the B side), written to an output block: U side stored
// column-major, V side stored as V = D^H (row-major).  Reflectors are applied
// from the last to the first; each needs w = u^H D (cluster-wide partial sums
// combined through DSMEM) and a rank-1 update of this CTA's rows.

template <typename T>
__global__ void __launch_bounds__(kDenseThreads) qapply_kernel(const DenseParams<T> P, const QJob* jobs, const XGroup<T> X) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int xok;
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank(), c = (int)cl.num_blocks();
  const int G = X.G;
  const int cid = blockIdx.x / c;
  const int job = cid / G, g = cid - job * G;
  if (c != X.csize || job >= X.njobs) {  // not the planned launch shape: touch nothing
    if (threadIdx.x == 0) set_status(P.status, DS_LAUNCH);
    return;
  }
  const QJob jb = jobs[job];
  const SvdTask t = P.tasks[jb.task];
  const TaskDims dm = P.dims[jb.task];
  const int s = dm.nout;  // columns written (the kept s, or all when taped)
  const int rows = jb.which ? t.rows_b : t.rows_a;
  const int kk = jb.which ? dm.krb : dm.kra;
  const T* A = jb.which ? P.qr + t.b_off : qr_a_ptr(P, t);
  const int64_t lda = jb.which ? (int64_t)t.rows_b : t.lda;
  const T* tau = P.tau + t.tau_off + (jb.which ? t.kcap : 0);
  const T* Z = P.core + (jb.which ? t.ys_off : t.xs_off);  // compact, column tc
  const BlockRef ob = P.out_blocks[t.out];
  T* D = jb.to_v ? out_v(P, ob) : out_u(P, ob);
  const int64_t ldd = jb.to_v ? ob.ldv : ob.ldu;
  if (s <= 0) return;
  const int np = G * c;
  const int chunk = (rows + np - 1) / np;
  const int ra = min(rows, (g * c + q) * chunk), rb = min(rows, ra + chunk);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // reflectors are applied two at a time (H_{j-1} H_j): with a = u_j^H D,
  // b = u_{j-1}^H D and gamma = u_{j-1}^H u_j,
  //   H_{j-1} H_j D = D - u_j w - u_{j-1} w',  w = tau_j a,  w' = tau_{j-1} (b - gamma w),
  // so one pass over D forms both inner products and one pass updates it
  const int plen = 2 * s + 1;                 // a (s), b (s), gamma
  T* part = reinterpret_cast<T*>(smem_raw);  // 2 x plen partials (step parity)
  T* tot = part + 2 * plen;                   // plen combined, then w (s), w' (s)
  for (int tc = 0; tc < s; ++tc)
    for (int i = ra + tid; i < rb; i += blockDim.x)
      D[(int64_t)tc * ldd + i] = i < kk ? Z[(int64_t)tc * t.kcap + i] : Traits<T>::zero();
  __syncthreads();
  const T one = from_re<T>(1.0), zero = Traits<T>::zero();
  int step = 0;
  for (int j = kk - 1; j >= 0; j -= 2, ++step) {
    const bool pair = j >= 1;  // block-uniform
    const int jm = j - 1;
    T* pb = part + (step & 1) * plen;
    const T tj = tau[j];
    const T tjm = pair ? tau[jm] : zero;
    const int i0 = max(ra, pair ? jm : j);
    const T* uj = A + (int64_t)j * lda;
    const T* ujm = A + (int64_t)(pair ? jm : j) * lda;
    for (int tc = warp; tc < s; tc += nw) {
      const T* d = D + (int64_t)tc * ldd;
      T a0 = zero, a1 = zero;
      for (int i = i0 + lane; i < rb; i += 32) {
        const T x = d[i];
        const T vj = i < j ? zero : (i == j ? one : uj[i]);
        a0 = cmac(a0, vj, x);
        if (pair) a1 = cmac(a1, i == jm ? one : ujm[i], x);
      }
      int col, comp;
      bool first;
      const double sum = warp_sum2<T>(a0, a1, lane, col, comp, first);
      if (first) reinterpret_cast<double*>(pb + col * s + tc)[comp] = sum;
    }
    if (warp == nw - 1) {  // gamma over this CTA's rows (u_j vanishes above row j)
      T g = zero;
      if (pair)
        for (int i = max(ra, j) + lane; i < rb; i += 32) g = cmac(g, ujm[i], i == j ? one : uj[i]);
      g = warp_sum(g);
      if (lane == 0) pb[2 * s] = g;
    }
    __syncthreads();
    cl.sync();
    for (int e = tid; e < plen; e += blockDim.x) {
      T sum = zero;
      for (int r = 0; r < c; ++r) sum = add(sum, cl.map_shared_rank(part + (step & 1) * plen, r)[e]);
      tot[e] = sum;
    }
    __syncthreads();
    if (G > 1) {
      if (q == 0) {
        T* xs = X.xpart + ((size_t)cid * 2 + (step & 1)) * X.xplen;
        for (int e = tid; e < plen; e += blockDim.x) xs[e] = tot[e];
        __syncthreads();
        if (tid == 0) xok = xgroup_arrive_wait(X.xcnt + job, (unsigned)(step + 1) * G, P.status);
      }
      cl.sync();
      if (*cl.map_shared_rank(&xok, 0) == 0) break;
      for (int e = tid; e < plen; e += blockDim.x) {
        T sum = zero;
        for (int gg = 0; gg < G; ++gg) sum = add(sum, ldcg(X.xpart + ((size_t)(job * G + gg) * 2 + (step & 1)) * X.xplen + e));
        tot[e] = sum;
      }
      __syncthreads();
    }
    const T gam = tot[2 * s];
    for (int tc = tid; tc < s; tc += blockDim.x) {
      const T w = mul(tj, tot[tc]);
      tot[tc] = w;
      tot[s + tc] = pair ? mul(tjm, msub(tot[s + tc], gam, w)) : zero;
    }
    __syncthreads();
    // D(i, tc) -= u_j(i) w_tc + u_{j-1}(i) w'_tc: one thread per row, four columns per step
    const T* wa = tot;
    const T* wb = tot + s;
    for (int i = i0 + tid; i < rb; i += blockDim.x) {
      const T vj = i < j ? zero : (i == j ? one : uj[i]);
      const T vm = !pair ? zero : (i == jm ? one : ujm[i]);
      int tc = 0;
      for (; tc + 3 < s; tc += 4) {
        T* d0 = D + (int64_t)tc * ldd + i;
        T v0 = d0[0], v1 = d0[ldd], v2 = d0[2 * ldd], v3 = d0[3 * ldd];
        v0 = msub(msub(v0, vj, wa[tc]), vm, wb[tc]);
        v1 = msub(msub(v1, vj, wa[tc + 1]), vm, wb[tc + 1]);
        v2 = msub(msub(v2, vj, wa[tc + 2]), vm, wb[tc + 2]);
        v3 = msub(msub(v3, vj, wa[tc + 3]), vm, wb[tc + 3]);
        d0[0] = v0;
        d0[ldd] = v1;
        d0[2 * ldd] = v2;
        d0[3 * ldd] = v3;
      }
      for (; tc < s; ++tc) {
        T* d0 = D + (int64_t)tc * ldd + i;
        *d0 = msub(msub(*d0, vj, wa[tc]), vm, wb[tc]);
      }
    }
    __syncthreads();
  }
  if (jb.to_v)
    for (int tc = 0; tc < s; ++tc)
      for (int i = ra + tid; i < rb; i += blockDim.x) D[(int64_t)tc * ldd + i] = conj_(D[(int64_t)tc * ldd + i]);
  cl.sync();
}

// ------------------------------------------------------------------ block-diagonal side
// HORIZ: V_out = Y_s^H diag(V1, V2); VERT: U_out = diag(U1, U2) Y_s.
template <typename T>
__global__ void blockprod_kernel(const DenseParams<T> P) {
  const int ti = blockIdx.y;
  const SvdTask t = P.tasks[ti];
  if (t.kind == TASK_LEAF) return;
  const TaskDims dm = P.dims[ti];
  const int s = dm.nout;  // columns written (the kept s, or all when taped)
  const BlockRef b1 = P.in_blocks[t.in1], b2 = P.in_blocks[t.in2];
  const int r1 = P.in_rank[b1.rank_slot], r2 = P.in_rank[b2.rank_slot];
  const BlockRef ob = P.out_blocks[t.out];
  const T* Y = P.core + t.ys_off;  // compact, column tc
  if (t.kind == TASK_HORIZ) {
    const int n1 = b1.n, ntot = b1.n + b2.n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)ntot * s; e += (int64_t)gridDim.x * blockDim.x) {
      const int j = (int)(e % ntot), tc = (int)(e / ntot);
      T acc = Traits<T>::zero();
      if (j < n1) {
        const T* ys = Y + (int64_t)tc * t.kcap;
        for (int p = 0; p < r1; ++p) acc = cmac(acc, ys[p], P.inV[b1.v_off + (int64_t)p * b1.ldv + j]);
      } else {
        const T* ys = Y + (int64_t)tc * t.kcap + r1;
        for (int p = 0; p < r2; ++p) acc = cmac(acc, ys[p], P.inV[b2.v_off + (int64_t)p * b2.ldv + (j - n1)]);
      }
      out_v(P, ob)[(int64_t)tc * ob.ldv + j] = acc;
    }
  } else {
    const int m1 = b1.m, mtot = b1.m + b2.m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)mtot * s; e += (int64_t)gridDim.x * blockDim.x) {
      const int i = (int)(e % mtot), tc = (int)(e / mtot);
      T acc = Traits<T>::zero();
      if (i < m1) {
        const T* ys = Y + (int64_t)tc * t.kcap;
        for (int p = 0; p < r1; ++p) acc = mac(acc, P.inU[b1.u_off + (int64_t)p * b1.ldu + i], ys[p]);
      } else {
        const T* ys = Y + (int64_t)tc * t.kcap + r1;
        for (int p = 0; p < r2; ++p) acc = mac(acc, P.inU[b2.u_off + (int64_t)p * b2.ldu + (i - m1)], ys[p]);
      }
      out_u(P, ob)[(int64_t)tc * ob.ldu + i] = acc;
    }
  }
}

// ------------------------------------------------------------------ taped root
// With a tape the root node of block b is kept (all triplets) in the store;
// its first s triplets (s = its eps-rank) go to the caller's result.
template <typename T>
__global__ void copyroot_kernel(const BlockRef* refs, int32_t* ranks, const T* fullU, const double* fullS,
                                const T* fullV, int root_first, int user_first) {
  const int b = blockIdx.y;
  const BlockRef src = refs[root_first + b], dst = refs[user_first + b];
  const int s = ranks[src.rank_slot];
  T* U = reinterpret_cast<T*>(dst.U);
  T* V = reinterpret_cast<T*>(dst.V);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t e = t0; e < (int64_t)src.m * s; e += stride) {
    const int64_t i = e % src.m, p = e / src.m;
    U[p * dst.ldu + i] = fullU[src.u_off + p * src.ldu + i];
  }
  for (int64_t e = t0; e < (int64_t)src.n * s; e += stride) {
    const int64_t j = e % src.n, p = e / src.n;
    V[p * dst.ldv + j] = fullV[src.v_off + p * src.ldv + j];
  }
  for (int64_t e = t0; e < s; e += stride) dst.S[e] = fullS[src.s_off + e];
  if (t0 == 0) ranks[dst.rank_slot] = s;
}

}  // namespace hbaca
