// Leaf-level BACA (Alg. 2) as one persistent kernel.
//
// A thread-block cluster of `c` CTAs owns one leaf at a time (leaves are
// pulled from a device work counter).  CTA q of the cluster owns a contiguous
// slice of the leaf's rows and a contiguous slice of its columns.  Every
// iteration k runs, with cluster barriers between the steps:
//   C_k = A(:, J_k) - U V(:, J_k)        entries generated in registers (line 3)
//   I_k = greedy QRCP pivots of C_k^t    DSMEM argmax per pivot   (line 4, Eq. QRIk)
//   R_k = A(I_k, :) - U(I_k, :) V                                 (line 5)
//   J_{k+1} = greedy QRCP pivots of R_k                           (line 6, Eq. QRJk)
//   W_k = C_k(I_k, :), LRID: QR(W_k, eps), U_k, V_k = T^-1 Q^H R_k (lines 7-9, Eqs. LRID1-2)
//   nu = ||U_k V_k||_F, mu update (Gram form)                     (lines 10-11, Eqs. numu, normup)
//   append, stop if nu < eps mu                                   (lines 12-14)
// Pivot-dependent small work (QRCP of W_k, T^-1 Q^H) is done redundantly and
// bit-identically by every CTA of the cluster, so no broadcast is needed.
#pragma once

#include <cooperative_groups.h>
#include <climits>

#include "common.cuh"
#include "types.h"

namespace cg = cooperative_groups;

namespace hbaca {

constexpr int kBacaThreads = 256;
constexpr int kMaxD = 32;




template <typename Gen>
struct BacaParams {
  using T = typename Gen::scalar;
  Gen gen;
  const LeafDesc* leaves;
  const int32_t* order;  // processing order of the leaves (largest first)
  LeafOut* out;
  int nleaves;
  int* queue;
  int* status;
  T* Uar;
  T* Var;
  T* Cscr;  // per cluster: m_max x d (column-major, ld m)
  T* Rscr;  // per cluster: d x n_max (row-major, ld n)
  T* Gscr;  // per cluster: 2 * c * rcap_max * d partial Gram entries
  int64_t cscr_stride, rscr_stride, gscr_stride;
  int32_t* tape_int;
  double* tape_dbl;
  double eps;
  int d;
  uint64_t seed;
  int mr_max, nc_max, rcap_max;
  double srrqr_f2;  // > 0: pivot sets refined by strong RRQR with threshold f^2
};

struct ArgSlot {
  long long bits;
  int idx;
  int pad;
};

template <typename T>
struct BacaSmem {
  T* work;       // max(mr_max * d, d * nc_max)
  T* slotvec;    // 2 * d: this CTA's candidate pivot vector, double-buffered
  T* hv;         // d: winning pivot vector / Householder vector u
  T* Wm;         // d * d: W_k, column-major (ld d), reduced in place
  T* Em;         // d * d: T11^-1 Q^H (rows 0..dk-1), column-major (ld d)
  T* tauv;       // d
  double* betav; // d
  ArgSlot* slot; // 2
  long long* wb; // 32
  int* wi;       // 32
  double* red;   // 96: reductions [0..63]; norms^2 of the chosen pivots [64..95]
  int* sI;       // d
  int* sJ;       // d
  int* sJn;      // d
  int* sjbar;    // d
  int* sint;     // 16 scratch ints
  uint8_t* kept_row;  // mr_max
  uint8_t* kept_col;  // nc_max
  uint8_t* cand;      // max(mr_max, nc_max)
};

template <typename T>
__host__ __device__ inline size_t baca_smem_bytes(int mr_max, int nc_max, int d) {
  size_t w = (size_t)mr_max * d;
  size_t w2 = (size_t)d * nc_max;
  if (w2 > w) w = w2;
  size_t b = 0;
  b += w * sizeof(T);
  b += (size_t)(2 * d + d + 2 * d * d + d) * sizeof(T);
  b += (size_t)d * sizeof(double);
  b += 2 * sizeof(ArgSlot) + 32 * sizeof(long long) + 32 * sizeof(int) + 96 * sizeof(double);
  b += (size_t)(4 * d + 16) * sizeof(int);
  int mx = mr_max > nc_max ? mr_max : nc_max;
  b += (size_t)mr_max + nc_max + mx + 64;
  return b;
}

template <typename T>
__device__ inline BacaSmem<T> carve(unsigned char* base, int mr_max, int nc_max, int d) {
  BacaSmem<T> s;
  size_t w = (size_t)mr_max * d;
  size_t w2 = (size_t)d * nc_max;
  if (w2 > w) w = w2;
  T* tp = reinterpret_cast<T*>(base);
  s.work = tp; tp += w;
  s.slotvec = tp; tp += 2 * d;
  s.hv = tp; tp += d;
  s.Wm = tp; tp += d * d;
  s.Em = tp; tp += d * d;
  s.tauv = tp; tp += d;
  double* dp = reinterpret_cast<double*>(tp);
  s.betav = dp; dp += d;
  s.slot = reinterpret_cast<ArgSlot*>(dp);
  long long* lp = reinterpret_cast<long long*>(s.slot + 2);
  s.wb = lp; lp += 32;
  dp = reinterpret_cast<double*>(lp);
  s.red = dp; dp += 96;
  int* ip = reinterpret_cast<int*>(dp);
  s.wi = ip; ip += 32;
  s.sI = ip; ip += d;
  s.sJ = ip; ip += d;
  s.sJn = ip; ip += d;
  s.sjbar = ip; ip += d;
  s.sint = ip; ip += 16;
  uint8_t* bp = reinterpret_cast<uint8_t*>(ip);
  s.kept_row = bp; bp += mr_max;
  s.kept_col = bp; bp += nc_max;
  s.cand = bp;
  return s;
}

// SplitMix64 (Steele, Lea & Flood 2014): state += golden gamma; variant-13 mix.
__device__ __forceinline__ uint64_t splitmix_next(uint64_t& s) {
  s += 0x9E3779B97F4A7C15ull;
  uint64_t z = s;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Random initial block J_1 (Alg. 2 line 1): partial Fisher-Yates shuffle of
// [0, n) driven by the block's counter-based stream; d swaps tracked in a
// small list (single thread).
__device__ inline int initial_columns(uint64_t seed, int64_t stream_id, int n, int d, int* J, int* scratch_pos, int* scratch_val) {
  int dd = d < n ? d : n;
  uint64_t s = seed ^ ((uint64_t)stream_id * 0xD1342543DE82EF95ull);
  int nsw = 0;  // explicit (position -> value) overrides of the identity permutation
  auto get = [&](int pos) {
    for (int a = nsw - 1; a >= 0; --a)
      if (scratch_pos[a] == pos) return scratch_val[a];
    return pos;
  };
  auto set = [&](int pos, int val) {
    for (int a = 0; a < nsw; ++a)
      if (scratch_pos[a] == pos) { scratch_val[a] = val; return; }
    scratch_pos[nsw] = pos;
    scratch_val[nsw] = val;
    ++nsw;
  };
  for (int t = 0; t < dd; ++t) {
    uint64_t z = splitmix_next(s);
    int j = t + (int)(((z >> 32) * (uint64_t)(n - t)) >> 32);
    int vt = get(t), vj = get(j);
    set(t, vj);
    set(j, vt);
    J[t] = vj;
  }
  return dd;
}

// Greedy QRCP over vectors spread across the cluster (Eqs. QRIk / QRJk read as
// their definition: at each step the candidate with the largest residual norm
// after the previous Householder reflections, recomputed explicitly, wins;
// ties go to the smaller index).  work[cc * ldw + v] is component cc of local
// vector v.  Chosen global indices go to piv[] (identical in every CTA).
template <typename T>
__device__ int qrcp_cluster(cg::cluster_group& cl, const BacaSmem<T>& S, int ldw, int nloc, int p,
                            int kmax, int gbase, int d, int* piv, unsigned& ctr) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int q = (int)cl.block_rank(), c = (int)cl.num_blocks();
  T* work = S.work;
  uint8_t* cand = S.cand;
  for (int t = 0; t < kmax; ++t) {
    const int buf = ctr & 1u;
    ++ctr;
    // 1. local argmax of the trailing squared norm
    long long bb = -1;
    int bi = INT_MAX;
    for (int v = tid; v < nloc; v += blockDim.x) {
      if (!cand[v]) continue;
      double s = 0.0;
      for (int cc = t; cc < p; ++cc) s += abs2(work[(size_t)cc * ldw + v]);
      argmax_merge(bb, bi, nbits(s), v);
    }
    warp_argmax(bb, bi);
    if (lane == 0) { S.wb[warp] = bb; S.wi[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      bb = lane < nw ? S.wb[lane] : -1;
      bi = lane < nw ? S.wi[lane] : INT_MAX;
      warp_argmax(bb, bi);
      if (lane == 0) {
        S.slot[buf].bits = bb;
        S.slot[buf].idx = (bi == INT_MAX) ? -1 : gbase + bi;
        S.sint[0] = bi;
      }
    }
    __syncthreads();
    {
      int li = S.sint[0];
      if (li != INT_MAX)
        for (int cc = t + tid; cc < p; cc += blockDim.x) S.slotvec[buf * d + (cc - t)] = work[(size_t)cc * ldw + li];
    }
    cl.sync();
    // 2. cluster-wide argmax over the c slots (warp 0), broadcast through smem
    if (warp == 0) {
      long long gb = -1;
      int gi = INT_MAX, own = -1;
      if (lane < c) {
        const ArgSlot* rs = cl.map_shared_rank(&S.slot[buf], lane);
        if (rs->idx >= 0) { gb = rs->bits; gi = rs->idx; own = lane; }
      }
      long long b2 = gb;
      int i2 = gi;
      warp_argmax(b2, i2);
      unsigned ownmask = __ballot_sync(0xffffffffu, own >= 0 && gi == i2 && i2 != INT_MAX);
      if (lane == 0) {
        S.sint[1] = i2;
        S.sint[2] = ownmask ? (__ffs(ownmask) - 1) : -1;
        if (t < 32) S.red[64 + t] = __longlong_as_double(b2);  // the pivot's residual norm^2
      }
    }
    __syncthreads();
    const int gi = S.sint[1], owner = S.sint[2];
    if (gi == INT_MAX) return t;
    if (tid == 0) piv[t] = gi;
    const int L = p - t;
    {
      const T* rv = cl.map_shared_rank(S.slotvec + buf * d, owner);
      for (int cc = tid; cc < L; cc += blockDim.x) S.hv[cc] = rv[cc];
    }
    if (owner == q && tid == 0) cand[gi - gbase] = 0;
    __syncthreads();
    // 3. Householder reflector of the pivot vector
    if (tid == 0) {
      double sig2 = 0.0;
      for (int cc = 1; cc < L; ++cc) sig2 += abs2(S.hv[cc]);
      double beta;
      T tau, sc;
      householder(S.hv[0], sig2, beta, tau, sc);
      for (int cc = 1; cc < L; ++cc) S.hv[cc] = mul(S.hv[cc], sc);
      S.hv[0] = from_re<T>(1.0);
      S.tauv[0] = conj_(tau);
    }
    __syncthreads();
    // 4. apply H^H to the remaining local candidates (components t..p-1)
    const T ctau = S.tauv[0];
    if (L > 1) {
      for (int v = tid; v < nloc; v += blockDim.x) {
        if (!cand[v]) continue;
        T w = Traits<T>::zero();
        for (int cc = 0; cc < L; ++cc) w = cmac(w, S.hv[cc], work[(size_t)(t + cc) * ldw + v]);
        T f = mul(ctau, w);
        for (int cc = 0; cc < L; ++cc) {
          size_t o = (size_t)(t + cc) * ldw + v;
          work[o] = msub(work[o], S.hv[cc], f);
        }
      }
    }
    __syncthreads();
  }
  return kmax;
}

// LRID (Alg. 2 function LRID; Eqs. LRID1-2) on W (dI x dJ, column-major ld d,
// in smem), done by warp 0: Householder QRCP with the QR(W, eps) rank rule
// |T_tt| >= eps |T_11|; fills sjbar[0..dk) and Em = T11^-1 (Q^H)(0:dk, :)
// (dk x dI, column-major ld d).  Returns dk.
template <typename T>
__device__ int lrid_small(const BacaSmem<T>& S, int dI, int dJ, int d, double eps) {
  const int lane = threadIdx.x & 31;
  T* W = S.Wm;
  bool chosen = false;  // lane = column of W
  int dk = 0;
  double t00 = 0.0;
  const int kmax = dI < dJ ? dI : dJ;
  for (int t = 0; t < kmax; ++t) {
    long long bb = -1;
    int bi = INT_MAX;
    if (lane < dJ && !chosen) {
      double s = 0.0;
      for (int r = t; r < dI; ++r) s += abs2(W[lane * d + r]);
      bb = nbits(s);
      bi = lane;
    }
    warp_argmax(bb, bi);
    if (bi == INT_MAX) break;
    double nrm = sqrt(__longlong_as_double(bb));
    if (t == 0) {
      if (nrm == 0.0) break;
      t00 = nrm;
    } else if (nrm < eps * t00) {
      break;
    }
    if (lane == bi) chosen = true;
    // reflector from column bi, rows t..dI-1 (lane 0 computes, then broadcast via smem)
    if (lane == 0) {
      T* x = W + bi * d;
      double sig2 = 0.0;
      for (int r = t + 1; r < dI; ++r) sig2 += abs2(x[r]);
      double beta;
      T tau, sc;
      householder(x[t], sig2, beta, tau, sc);
      for (int r = t + 1; r < dI; ++r) x[r] = mul(x[r], sc);  // u tail stored below the diagonal
      x[t] = from_re<T>(beta);
      S.betav[t] = beta;
      S.tauv[t] = tau;
      S.sjbar[t] = bi;
    }
    __syncwarp();
    // apply H^H to the other unchosen columns
    if (lane < dJ && !chosen) {
      const T* u = W + bi * d;
      T* y = W + lane * d;
      T w = y[t];  // u_t = 1
      for (int r = t + 1; r < dI; ++r) w = cmac(w, u[r], y[r]);
      T f = mul(conj_(S.tauv[t]), w);
      y[t] = sub(y[t], f);
      for (int r = t + 1; r < dI; ++r) y[r] = msub(y[r], u[r], f);
    }
    __syncwarp();
    dk = t + 1;
  }
  // Em(:, col) = first dk rows of H_{dk-1}^H ... H_0^H e_col, then T11^{-1}
  if (dk > 0 && lane < dI) {
    T* e = S.Em + lane * d;
    for (int r = 0; r < dI; ++r) e[r] = from_re<T>(r == lane ? 1.0 : 0.0);
    for (int t = 0; t < dk; ++t) {
      const T* u = W + S.sjbar[t] * d;
      T w = e[t];
      for (int r = t + 1; r < dI; ++r) w = cmac(w, u[r], e[r]);
      T f = mul(conj_(S.tauv[t]), w);
      e[t] = sub(e[t], f);
      for (int r = t + 1; r < dI; ++r) e[r] = msub(e[r], u[r], f);
    }
    // back substitution with T11(s, t) = W(s, jbar[t]) (s < t), T11(t, t) = beta_t
    for (int t = dk - 1; t >= 0; --t) {
      T v = e[t];
      for (int s2 = t + 1; s2 < dk; ++s2) v = msub(v, W[S.sjbar[s2] * d + t], e[s2]);
      e[t] = scale(v, 1.0 / S.betav[t]);
    }
  }
  __syncwarp();
  return dk;
}

// Strong rank-revealing QR (Gu & Eisenstat, SIAM J. Sci. Comput. 17, 1996) as
// a refinement of the k pivots qrcp_cluster chose among this cluster's
// vectors -- one of the subset-selection methods Sec. 3.2 names beside QRCP.
// With the chosen vectors as columns, M(:, piv) = Q R11, R12 = Q^H M(:, j)
// and gamma_j = the norm of the rest of the reflected vector j, the criterion
// rho_ij = |(R11^{-1} R12)_ij|^2 + (omega_i gamma_j)^2 (omega_i = norm of row
// i of R11^{-1}) is the squared factor by which swapping chosen i for
// candidate j multiplies |det R11|; while the largest rho exceeds f^2 that
// pair is swapped (ties: smaller j, then smaller i; the candidate takes the
// chosen one's position).  The vectors are re-read from their global copy
// (vec(g, cc): component cc of vector g); every CTA factors the chosen set
// itself (bit-identical), forms rho for its own candidates, and the cluster
// argmax is taken in rank order through DSMEM, so every CTA takes the same
// swaps.  At most 4k + 4 swaps (each multiplies a volume by more than f > 1).
// Returns the number of swaps; piv and the candidate flags are updated.
template <typename T, typename VecF>
__device__ int srrqr_cluster(cg::cluster_group& cl, const BacaSmem<T>& S, int ldw, int nloc, int p, int k,
                             int gbase, int d, int* piv, VecF vec, double f2, unsigned& ctr) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int q = (int)cl.block_rank(), c = (int)cl.num_blocks();
  T* work = S.work;
  uint8_t* cand = S.cand;
  const int max_swaps = 4 * k + 4;
  int swaps = 0;
  while (swaps < max_swaps) {
    // 1. the chosen vectors as the columns of Em (p x k), Householder QR by warp 0
    for (int e = tid; e < p * k; e += blockDim.x) {
      const int cc = e % p, t = e / p;
      S.Em[t * d + cc] = vec(piv[t], cc);
    }
    __syncthreads();
    if (warp == 0) {
      for (int t = 0; t < k; ++t) {
        if (lane == 0) {
          T* x = S.Em + t * d;
          double sig2 = 0.0;
          for (int r = t + 1; r < p; ++r) sig2 += abs2(x[r]);
          double beta;
          T tau, sc;
          householder(x[t], sig2, beta, tau, sc);
          for (int r = t + 1; r < p; ++r) x[r] = mul(x[r], sc);
          x[t] = from_re<T>(beta);
          S.betav[t] = beta;
          S.tauv[t] = tau;
        }
        __syncwarp();
        if (lane > t && lane < k) {  // apply H_t^H to the later chosen columns
          const T* u = S.Em + t * d;
          T* y = S.Em + lane * d;
          T w = y[t];
          for (int r = t + 1; r < p; ++r) w = cmac(w, u[r], y[r]);
          const T fct = mul(conj_(S.tauv[t]), w);
          y[t] = sub(y[t], fct);
          for (int r = t + 1; r < p; ++r) y[r] = msub(y[r], u[r], fct);
        }
        __syncwarp();
      }
      // 2. Ri = R11^{-1} (column-major ld d in Wm), lane = column; R11(s, t) = Em[t d + s]
      if (lane < k) {
        T* col = S.Wm + lane * d;
        for (int t = k - 1; t >= 0; --t) {
          T v = from_re<T>(t == lane ? 1.0 : 0.0);
          for (int s2 = t + 1; s2 < k; ++s2) v = msub(v, S.Em[s2 * d + t], col[s2]);
          col[t] = S.betav[t] != 0.0 ? scale(v, 1.0 / S.betav[t]) : Traits<T>::zero();
        }
      }
      __syncwarp();
      // 3. omega_i = norm of row i of Ri
      if (lane < k) {
        double o = 0.0;
        for (int t = lane; t < k; ++t) o += abs2(S.Wm[t * d + lane]);
        S.red[lane] = o;  // omega_i^2
      }
    }
    __syncthreads();
    bool singular = false;
    for (int t = 0; t < k; ++t) singular |= (S.betav[t] == 0.0);
    if (singular) break;
    // 4. this CTA's candidates: reflect, rho over the chosen positions
    long long bb = -1;
    int bkey = INT_MAX;
    for (int v = tid; v < nloc; v += blockDim.x) {
      if (!cand[v]) continue;
      for (int cc = 0; cc < p; ++cc) work[(size_t)cc * ldw + v] = vec(gbase + v, cc);
      for (int t = 0; t < k; ++t) {
        const T* u = S.Em + t * d;
        T w = work[(size_t)t * ldw + v];
        for (int cc = t + 1; cc < p; ++cc) w = cmac(w, u[cc], work[(size_t)cc * ldw + v]);
        const T fct = mul(conj_(S.tauv[t]), w);
        work[(size_t)t * ldw + v] = sub(work[(size_t)t * ldw + v], fct);
        for (int cc = t + 1; cc < p; ++cc) work[(size_t)cc * ldw + v] = msub(work[(size_t)cc * ldw + v], u[cc], fct);
      }
      double gam2 = 0.0;
      for (int cc = k; cc < p; ++cc) gam2 += abs2(work[(size_t)cc * ldw + v]);
      for (int i = 0; i < k; ++i) {
        T b = Traits<T>::zero();
        for (int t = i; t < k; ++t) b = mac(b, S.Wm[t * d + i], work[(size_t)t * ldw + v]);
        const double rho = abs2(b) + S.red[i] * gam2;
        argmax_merge(bb, bkey, nbits(rho), (gbase + v) * 32 + i);
      }
    }
    warp_argmax(bb, bkey);
    if (lane == 0) { S.wb[warp] = bb; S.wi[warp] = bkey; }
    __syncthreads();
    const int buf = ctr & 1u;
    ++ctr;
    if (warp == 0) {
      bb = lane < nw ? S.wb[lane] : -1;
      bkey = lane < nw ? S.wi[lane] : INT_MAX;
      warp_argmax(bb, bkey);
      if (lane == 0) {
        S.slot[buf].bits = bb;
        S.slot[buf].idx = bkey;
      }
    }
    cl.sync();
    if (warp == 0) {  // cluster argmax in rank order (every CTA the same)
      long long gb = lane < c ? cl.map_shared_rank(&S.slot[buf], lane)->bits : -1;
      int gk = lane < c ? cl.map_shared_rank(&S.slot[buf], lane)->idx : INT_MAX;
      warp_argmax(gb, gk);
      if (lane == 0) {
        S.sint[5] = gk;
        S.sint[6] = (gb >= 0 && gk != INT_MAX && __longlong_as_double(gb) > f2) ? 1 : 0;
      }
    }
    __syncthreads();
    const int key = S.sint[5];
    const int doswap = S.sint[6];
    // the owner CTAs may overwrite their slots only after every CTA has read them
    cl.sync();
    if (!doswap) break;
    const int i = key % 32, jn = key / 32, old = piv[i];
    __syncthreads();
    if (tid == 0) {
      piv[i] = jn;
      if (jn >= gbase && jn < gbase + nloc) cand[jn - gbase] = 0;
      if (old >= gbase && old < gbase + nloc) cand[old - gbase] = 1;
    }
    __syncthreads();
    ++swaps;
  }
  (void)q;
  return swaps;
}

// Whether a greedy pivot set is refined: its smallest pivot residual norm at
// least 1e-8 of the larger of the first one and the current mu (below that the
// block is numerically rank-deficient or at the rounding level, where volume
// gains compare rounding noise).  The norms^2 are those qrcp_cluster recorded.
__device__ __forceinline__ bool srrqr_refine(const double* pn2, int k, double mu) {
  if (k <= 0) return false;
  double mn = pn2[0];
  for (int t = 1; t < k; ++t) mn = fmin(mn, pn2[t]);
  const double ref = fmax(sqrt(fmax(pn2[0], 0.0)), mu);
  return sqrt(fmax(mn, 0.0)) >= 1e-8 * ref;
}

template <typename T>
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// panel columns (C_k) or rows (R_k) one thread forms together
constexpr int kPanel = 4;

template <typename Gen>
__global__ void __launch_bounds__(kBacaThreads) baca_leaf_kernel(const BacaParams<Gen> P) {
  using T = typename Gen::scalar;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank(), c = (int)cl.num_blocks();
  const int tid = threadIdx.x;
  const int cid = blockIdx.x / c;
  const int d = P.d;
  BacaSmem<T> S = carve<T>(smem_raw, P.mr_max, P.nc_max, d);
  T* Cg = P.Cscr + (size_t)cid * P.cscr_stride;
  T* Rg = P.Rscr + (size_t)cid * P.rscr_stride;
  T* Gg = P.Gscr + (size_t)cid * P.gscr_stride;
  unsigned ctr = 0;

  for (;;) {
    if (q == 0 && tid == 0) {
      const int slot = atomicAdd(P.queue, 1);
      S.sint[8] = slot < P.nleaves ? P.order[slot] : P.nleaves;
    }
    cl.sync();
    int leaf;
    {
      const int* rl = cl.map_shared_rank(&S.sint[8], 0);
      leaf = *rl;
    }
    if (leaf >= P.nleaves) break;
    const LeafDesc Lf = P.leaves[leaf];
    const auto gen = P.gen.bind(Lf.block);
    const int m = Lf.m, n = Lf.n;
    const int mchunk = (m + c - 1) / c, nchunk = (n + c - 1) / c;
    const int ra = min(m, q * mchunk), mr = min(m, ra + mchunk) - ra;
    const int ca = min(n, q * nchunk), nc = min(n, ca + nchunk) - ca;
    T* U = P.Uar + Lf.u_off;  // m x rcap, ld m
    T* V = P.Var + Lf.v_off;  // rcap x n, ld n
    int32_t* tpi = P.tape_int + Lf.tape_off;
    double* tpd = P.tape_dbl + Lf.taped_off;
    const int rec = 4 + 3 * d;
    for (int i = tid; i < mr; i += blockDim.x) S.kept_row[i] = 0;
    for (int j = tid; j < nc; j += blockDim.x) S.kept_col[j] = 0;
    if (tid == 0)  // swap list needs up to 2d (position, value) pairs: W / E scratch holds them
      S.sint[3] = initial_columns(P.seed, Lf.stream_id, n, d, S.sJ, reinterpret_cast<int*>(S.Wm), reinterpret_cast<int*>(S.Em));
    __syncthreads();
    int dJ = S.sint[3];
    int r = 0, it = 0, stop = STOP_ITERS;
    double mu2 = 0.0;
    const int itmax = min(m, n);
    for (; it < itmax; ++it) {
      if (dJ == 0) { stop = STOP_NO_COLS; break; }
      // ---- C_k = A(:, J_k) - U V(:, J_k)   (line 3)
      // a thread takes one row and kPanel columns of the panel, so each entry
      // of U is loaded once per kPanel columns (the sums run over p in the
      // same order as for one column)
      {
        const int ngrp = (dJ + kPanel - 1) / kPanel;
        for (int e = tid; e < mr * ngrp; e += blockDim.x) {
          const int il = e % mr, j0 = (e / mr) * kPanel, i = ra + il;
          const int nj = min(kPanel, dJ - j0);
          T acc[kPanel];
          const T* vp[kPanel];
#pragma unroll
          for (int u = 0; u < kPanel; ++u) {
            acc[u] = Traits<T>::zero();
            vp[u] = V + S.sJ[j0 + (u < nj ? u : 0)];
          }
          const T* up = U + i;
          for (int p = 0; p < r; ++p) {
            const T uv = up[(size_t)p * m];
#pragma unroll
            for (int u = 0; u < kPanel; ++u)
              if (u < nj) acc[u] = mac(acc[u], uv, ldcg(vp[u] + (size_t)p * n));
          }
#pragma unroll
          for (int u = 0; u < kPanel; ++u) {
            if (u >= nj) continue;
            const int j = j0 + u, jc = S.sJ[j];
            const T val = sub(gen(Lf.row0 + i, Lf.col0 + jc), acc[u]);
            S.work[(size_t)j * mr + il] = val;
            Cg[(size_t)j * m + i] = val;
          }
        }
      }
      for (int i = tid; i < mr; i += blockDim.x) S.cand[i] = !S.kept_row[i];
      __syncthreads();
      // ---- I_k: greedy QRCP of C_k^t over unkept rows   (line 4)
      const int dI = qrcp_cluster<T>(cl, S, mr, mr, dJ, min(d, dJ), ra, d, S.sI, ctr);
      __syncthreads();
      if (dI == 0) { stop = STOP_NO_ROWS; break; }
      if (P.srrqr_f2 > 0.0 && srrqr_refine(S.red + 64, dI, sqrt(fmax(mu2, 0.0)))) {
        // strong-RRQR refinement of I_k over the rows (vector of row g: C(g, :))
        srrqr_cluster<T>(cl, S, mr, mr, dJ, dI, ra, d, S.sI,
                         [&](int g, int cc) { return ldcg(Cg + (size_t)cc * m + g); }, P.srrqr_f2, ctr);
        __syncthreads();
      }
      // ---- R_k = A(I_k, :) - U(I_k, :) V   (line 5)
      // a thread takes one column and kPanel rows of the panel (each entry of
      // V loaded once per kPanel rows; the same order of the sums)
      {
        const int ngrp = (dI + kPanel - 1) / kPanel;
        for (int e = tid; e < nc * ngrp; e += blockDim.x) {
          const int jl = e % nc, s0 = (e / nc) * kPanel, j = ca + jl;
          const int ns = min(kPanel, dI - s0);
          T acc[kPanel];
          const T* up[kPanel];
#pragma unroll
          for (int u = 0; u < kPanel; ++u) {
            acc[u] = Traits<T>::zero();
            up[u] = U + S.sI[s0 + (u < ns ? u : 0)];
          }
          const T* vp = V + j;
          for (int p = 0; p < r; ++p) {
            const T vv = vp[(size_t)p * n];
#pragma unroll
            for (int u = 0; u < kPanel; ++u)
              if (u < ns) acc[u] = mac(acc[u], ldcg(up[u] + (size_t)p * m), vv);
          }
#pragma unroll
          for (int u = 0; u < kPanel; ++u) {
            if (u >= ns) continue;
            const int s = s0 + u, i = S.sI[s];
            const T val = sub(gen(Lf.row0 + i, Lf.col0 + j), acc[u]);
            S.work[(size_t)s * nc + jl] = val;
            Rg[(size_t)s * n + j] = val;
          }
        }
      }
      for (int jl = tid; jl < nc; jl += blockDim.x) {
        bool ex = S.kept_col[jl];
        for (int t = 0; t < dJ; ++t) ex |= (S.sJ[t] == ca + jl);
        S.cand[jl] = !ex;
      }
      __syncthreads();
      // ---- J_{k+1}: greedy QRCP of R_k over unkept columns outside J_k   (line 6)
      const int dJn = qrcp_cluster<T>(cl, S, nc, nc, dI, min(d, dI), ca, d, S.sJn, ctr);
      __syncthreads();
      if (P.srrqr_f2 > 0.0 && srrqr_refine(S.red + 64, dJn, sqrt(fmax(mu2, 0.0)))) {
        // the same for J_{k+1} over the columns (vector of column g: R(:, g))
        srrqr_cluster<T>(cl, S, nc, nc, dI, dJn, ca, d, S.sJn,
                         [&](int g, int s2) { return ldcg(Rg + (size_t)s2 * n + g); }, P.srrqr_f2, ctr);
      }
      cl.sync();  // C_k and R_k (global scratch) complete in every CTA
      // ---- W_k and LRID   (lines 7-8)
      for (int e = tid; e < dI * dJ; e += blockDim.x) {
        const int s = e % dI, t = e / dI;
        S.Wm[t * d + s] = ldcg(Cg + (size_t)t * m + S.sI[s]);
      }
      __syncthreads();
      if (tid < 32) {
        int dk0 = lrid_small<T>(S, dI, dJ, d, P.eps);
        if (tid == 0) S.sint[4] = dk0;
      }
      __syncthreads();
      const int dk = S.sint[4];
      if (r + dk > Lf.rcap) {
        stop = STOP_CAPACITY;
        if (q == 0 && tid == 0) set_status(P.status, DS_RANK_CAPACITY);
        break;
      }
      // U_k = C_k(:, Jbar), V_k = T^-1 Q^H R_k, appended at column / row r   (line 12)
      for (int e = tid; e < mr * dk; e += blockDim.x) {
        const int il = e % mr, s = e / mr, i = ra + il;
        U[(size_t)(r + s) * m + i] = Cg[(size_t)S.sjbar[s] * m + i];
      }
      for (int e = tid; e < nc * dk; e += blockDim.x) {
        const int jl = e % nc, s = e / nc, j = ca + jl;
        T acc = Traits<T>::zero();
        for (int t = 0; t < dI; ++t) acc = mac(acc, S.Em[t * d + s], Rg[(size_t)t * n + j]);
        V[(size_t)(r + s) * n + j] = acc;
      }
      cl.sync();
      // ---- nu = LRnorm(U_k, V_k), mu = LRnormUp(...)   (lines 10-11): partial Grams
      const int Pn = r + dk;
      T* GU = Gg + (size_t)q * P.rcap_max * d;
      T* GV = Gg + (size_t)(c + q) * P.rcap_max * d;
      for (int e = tid; e < Pn * dk; e += blockDim.x) {
        const int s = e % dk, p = e / dk;
        T a = Traits<T>::zero();
        const T* up = U + (size_t)p * m + ra;
        const T* uk = U + (size_t)(r + s) * m + ra;
        for (int il = 0; il < mr; ++il) a = cmac(a, up[il], uk[il]);
        GU[(size_t)p * d + s] = a;
        T b = Traits<T>::zero();
        const T* vpp = V + (size_t)p * n + ca;
        const T* vk = V + (size_t)(r + s) * n + ca;
        for (int jl = 0; jl < nc; ++jl) b = cmac(b, vk[jl], vpp[jl]);
        GV[(size_t)p * d + s] = b;
      }
      cl.sync();
      double nu2p = 0.0, crp = 0.0;
      for (int e = tid; e < Pn * dk; e += blockDim.x) {
        const int s = e % dk, p = e / dk;
        T gu = Traits<T>::zero(), gv = Traits<T>::zero();
        for (int qq = 0; qq < c; ++qq) {
          gu = add(gu, ldcg(Gg + ((size_t)qq * P.rcap_max + p) * d + s));
          gv = add(gv, ldcg(Gg + ((size_t)(c + qq) * P.rcap_max + p) * d + s));
        }
        double v = re_(gu) * re_(gv) + im_(gu) * im_(gv);  // Re(gu conj(gv))
        if (p >= r) nu2p += v; else crp += v;
      }
      const double nu2 = block_sum<T>(nu2p, S.red);
      const double cr = block_sum<T>(crp, S.red + 32);
      const double nu = dk ? sqrt(fmax(nu2, 0.0)) : 0.0;
      if (dk) mu2 = mu2 + nu2 + 2.0 * cr;
      const double mu = sqrt(fmax(mu2, 0.0));
      // ---- tape, kept sets, append   (lines 9, 12)
      if (q == 0 && it < Lf.tape_iters) {
        int32_t* rp = tpi + (size_t)it * rec;
        for (int t = tid; t < rec; t += blockDim.x) {
          int v = -1;
          if (t == 0) v = dI;
          else if (t == 1) v = dJ;
          else if (t == 2) v = dk;
          else if (t >= 4 && t < 4 + d) v = (t - 4) < dI ? S.sI[t - 4] : -1;
          else if (t >= 4 + d && t < 4 + 2 * d) v = (t - 4 - d) < dJ ? S.sJ[t - 4 - d] : -1;
          else if (t >= 4 + 2 * d) v = (t - 4 - 2 * d) < dk ? S.sjbar[t - 4 - 2 * d] : -1;
          rp[t] = v;
        }
        if (tid == 0) { tpd[2 * it] = nu; tpd[2 * it + 1] = mu; }
      }
      __syncthreads();
      for (int s = tid; s < dk; s += blockDim.x) {
        const int i = S.sI[s];
        if (i >= ra && i < ra + mr) S.kept_row[i - ra] = 1;
        const int j = S.sJ[S.sjbar[s]];
        if (j >= ca && j < ca + nc) S.kept_col[j - ca] = 1;
      }
      r += dk;
      __syncthreads();
      if (!isfinite(nu) || !isfinite(mu)) {
        stop = STOP_NUMERICAL;
        if (q == 0 && tid == 0) set_status(P.status, DS_NUMERICAL);
        ++it;
        break;
      }
      if (nu < P.eps * mu) { stop = STOP_CONVERGED; ++it; break; }
      for (int t = tid; t < dJn; t += blockDim.x) S.sJ[t] = S.sJn[t];
      dJ = dJn;
      __syncthreads();
    }
    if (q == 0 && tid == 0) {
      LeafOut o;
      o.rank = r;
      o.iters = it;
      o.stop = stop;
      o.status = 0;
      o.mu = sqrt(fmax(mu2, 0.0));
      P.out[leaf] = o;
    }
    cl.sync();
  }
  cl.sync();
}

}  // namespace hbaca
