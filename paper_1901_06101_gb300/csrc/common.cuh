// Shared device-side building blocks of libhbaca: scalar arithmetic for
// float64 and interleaved complex128, the O(1) entry generators that the
// residual kernels evaluate in registers, and warp / block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hbaca.h"
#include "types.h"

namespace hbaca {

// ------------------------------------------------------------------ scalars
struct __align__(16) cplx {
  double re, im;
};

__host__ __device__ __forceinline__ cplx mk(double r, double i) { cplx z; z.re = r; z.im = i; return z; }

template <typename T> struct Traits;
template <> struct Traits<double> {
  static constexpr bool is_complex = false;
  __device__ __forceinline__ static double zero() { return 0.0; }
};
template <> struct Traits<cplx> {
  static constexpr bool is_complex = true;
  __device__ __forceinline__ static cplx zero() { return mk(0.0, 0.0); }
};

__device__ __forceinline__ double conj_(double a) { return a; }
__device__ __forceinline__ cplx conj_(cplx a) { return mk(a.re, -a.im); }
__device__ __forceinline__ double re_(double a) { return a; }
__device__ __forceinline__ double re_(cplx a) { return a.re; }
__device__ __forceinline__ double im_(double) { return 0.0; }
__device__ __forceinline__ double im_(cplx a) { return a.im; }
__device__ __forceinline__ double abs2(double a) { return a * a; }
__device__ __forceinline__ double abs2(cplx a) { return fma(a.re, a.re, a.im * a.im); }
// acc + |a|^2 as fused multiply-adds
__device__ __forceinline__ double acc_abs2(double acc, double a) { return fma(a, a, acc); }
__device__ __forceinline__ double acc_abs2(double acc, cplx a) { return fma(a.re, a.re, fma(a.im, a.im, acc)); }
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ cplx add(cplx a, cplx b) { return mk(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ double sub(double a, double b) { return a - b; }
__device__ __forceinline__ cplx sub(cplx a, cplx b) { return mk(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ double mul(double a, double b) { return a * b; }
__device__ __forceinline__ cplx mul(cplx a, cplx b) {
  return mk(fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re));
}
__device__ __forceinline__ double scale(double a, double s) { return a * s; }
__device__ __forceinline__ cplx scale(cplx a, double s) { return mk(a.re * s, a.im * s); }
// acc + a * b
__device__ __forceinline__ double mac(double acc, double a, double b) { return fma(a, b, acc); }
__device__ __forceinline__ cplx mac(cplx acc, cplx a, cplx b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a) * b
__device__ __forceinline__ double cmac(double acc, double a, double b) { return fma(a, b, acc); }
__device__ __forceinline__ cplx cmac(cplx acc, cplx a, cplx b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
// acc - a * b
__device__ __forceinline__ double msub(double acc, double a, double b) { return fma(-a, b, acc); }
__device__ __forceinline__ cplx msub(cplx acc, cplx a, cplx b) {
  acc.re = fma(-a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(-a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
// a / b
__device__ __forceinline__ double div_(double a, double b) { return a / b; }
__device__ __forceinline__ cplx div_(cplx a, cplx b) {
  double d = 1.0 / abs2(b);
  return mk((a.re * b.re + a.im * b.im) * d, (a.im * b.re - a.re * b.im) * d);
}
template <typename T> __device__ __forceinline__ T from_re(double r);
template <> __device__ __forceinline__ double from_re<double>(double r) { return r; }
template <> __device__ __forceinline__ cplx from_re<cplx>(double r) { return mk(r, 0.0); }

// Loads of data written by other CTAs of the cluster earlier in the same
// kernel go through L2 (ld.global.cg), never a possibly stale L1 line.
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ cplx ldcg(const cplx* p) {
  double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return mk(v.x, v.y);
}

// |z| without squaring (no underflow for tiny z) and the exact unit phase
// conj(z) / |z| (sign for real z).
__device__ __forceinline__ double absval(double a) { return fabs(a); }
__device__ __forceinline__ double absval(cplx a) { return hypot(a.re, a.im); }
__device__ __forceinline__ double conj_phase(double a, double) { return a >= 0.0 ? 1.0 : -1.0; }
__device__ __forceinline__ cplx conj_phase(cplx a, double mag) { return mk(a.re / mag, -a.im / mag); }

// Non-negative doubles order like their bit patterns: argmax reductions on
// norms compare 64-bit integers and keep the FP64 pipe for arithmetic.
__device__ __forceinline__ long long nbits(double nonneg) { return __double_as_longlong(nonneg); }

// Householder reflector (LAPACK larfg convention) for a vector x of length
// len with head alpha = x[0] and tail squared norm sig2: beta, tau and the
// scale 1/(alpha - beta) of the tail.  H = I - tau u u^H, u = [1; x(1:)*sc],
// H^H x = beta e_1.  tau = 0 (H = I) when the tail is zero and alpha is real.
template <typename T>
__device__ __forceinline__ void householder(T alpha, double sig2, double& beta, T& tau, T& sc) {
  double ar = re_(alpha), ai = im_(alpha);
  if (sig2 == 0.0 && ai == 0.0) {
    beta = ar;
    tau = Traits<T>::zero();
    sc = Traits<T>::zero();
    return;
  }
  double nrm = sqrt(ar * ar + ai * ai + sig2);
  beta = (ar >= 0.0) ? -nrm : nrm;
  T b = from_re<T>(beta);
  tau = div_(sub(b, alpha), b);
  sc = div_(from_re<T>(1.0), sub(alpha, b));
}

// ------------------------------------------------------------------ generators
// Each generator maps global (row, column) indices to one entry.  They are
// passed by value into the kernels and inlined into the residual updates.
struct GenDense {
  __device__ __forceinline__ GenDense bind(int) const { return *this; }
  using scalar = double;
  const double* a;
  int64_t lda;
  __device__ __forceinline__ double operator()(int64_t i, int64_t j) const { return a[j * lda + i]; }
};
struct GenDenseC {
  __device__ __forceinline__ GenDenseC bind(int) const { return *this; }
  using scalar = cplx;
  const cplx* a;
  int64_t lda;
  __device__ __forceinline__ cplx operator()(int64_t i, int64_t j) const { return a[j * lda + i]; }
};

struct GenGaussian {
  __device__ __forceinline__ GenGaussian bind(int) const { return *this; }
  using scalar = double;
  const double* x;
  const double* y;
  int dim;
  double c;  // -1 / (2 h^2)
  __device__ __forceinline__ double operator()(int64_t i, int64_t j) const {
    const double* xi = x + i * dim;
    const double* yj = y + j * dim;
    double s = 0.0;
    if (dim == 3) {
      double t0 = xi[0] - yj[0], t1 = xi[1] - yj[1], t2 = xi[2] - yj[2];
      s = fma(t0, t0, fma(t1, t1, t2 * t2));
    } else {
      for (int t = 0; t < dim; ++t) {
        double u = xi[t] - yj[t];
        s = fma(u, u, s);
      }
    }
    return exp(s * c);
  }
};

struct GenHelmholtz {
  __device__ __forceinline__ GenHelmholtz bind(int) const { return *this; }
  using scalar = cplx;
  const double* x;
  const double* y;
  int dim;
  double kpi;  // k / pi: sincospi(kpi * r) = (sin, cos)(k r)
  __device__ __forceinline__ cplx operator()(int64_t i, int64_t j) const {
    const double* xi = x + i * dim;
    const double* yj = y + j * dim;
    double s = 0.0;
    for (int t = 0; t < dim; ++t) {
      double u = xi[t] - yj[t];
      s = fma(u, u, s);
    }
    double rinv = rsqrt(s);
    double r = s * rinv;
    double sn, cs;
    sincospi(kpi * r, &sn, &cs);
    return mk(cs * rinv, sn * rinv);
  }
};

struct GenLowRank {
  __device__ __forceinline__ GenLowRank bind(int) const { return *this; }
  using scalar = double;
  const double* lu;  // m x lr, column-major, ld = m
  const double* lv;  // lr x n, row-major, ld = n
  int64_t m, n, lr;
  __device__ __forceinline__ double operator()(int64_t i, int64_t j) const {
    double s = 0.0;
    for (int64_t t = 0; t < lr; ++t) s = fma(lu[t * m + i], lv[t * n + j], s);
    return s;
  }
};
struct GenLowRankC {
  __device__ __forceinline__ GenLowRankC bind(int) const { return *this; }
  using scalar = cplx;
  const cplx* lu;
  const cplx* lv;
  int64_t m, n, lr;
  __device__ __forceinline__ cplx operator()(int64_t i, int64_t j) const {
    cplx s = mk(0.0, 0.0);
    for (int64_t t = 0; t < lr; ++t) s = mac(s, lu[t * m + i], lv[t * n + j]);
    return s;
  }
};

// A(i,j) = sum_k P(i,k) Q(k,j) + sum_t P2(i,t) Q2(t,j): a sorted-list
// intersection of row i of P (CSR) with column j of Q (CSC), then the dense term.
struct GenSparseProduct {
  __device__ __forceinline__ GenSparseProduct bind(int) const { return *this; }
  using scalar = double;
  const int32_t* prp;
  const int32_t* pci;
  const double* pv;
  const int32_t* qcp;
  const int32_t* qri;
  const double* qv;
  const double* p2;
  const double* q2;
  int64_t n;
  int r2;
  __device__ __forceinline__ double operator()(int64_t i, int64_t j) const {
    int a = prp[i], ae = prp[i + 1];
    int b = qcp[j], be = qcp[j + 1];
    double s = 0.0;
    while (a < ae && b < be) {
      int ka = pci[a], kb = qri[b];
      if (ka == kb) {
        s = fma(pv[a], qv[b], s);
        ++a;
        ++b;
      } else if (ka < kb) {
        ++a;
      } else {
        ++b;
      }
    }
    double t = 0.0;
    for (int u = 0; u < r2; ++u) t = fma(p2[i * r2 + u], q2[u * n + j], t);
    return s + t;
  }
};

// Polynomial kernel (x_i^t y_j + h)^2 (Sec. 5, kernel 5).
struct GenPolynomial {
  __device__ __forceinline__ GenPolynomial bind(int) const { return *this; }
  using scalar = double;
  const double* x;
  const double* y;
  int dim;
  double h;
  __device__ __forceinline__ double operator()(int64_t i, int64_t j) const {
    const double* xi = x + i * dim;
    const double* yj = y + j * dim;
    double s = h;
    for (int t = 0; t < dim; ++t) s = fma(xi[t], yj[t], s);
    return s * s;
  }
};

// Hankel function of the second kind of order 0, H0^(2)(z) = J0(z) - i Y0(z),
// for real z > 0 (the EFIE2D kernel of Sec. 5, kernel 2).
//  z <  20: J_n(z) by Miller's backward recurrence J_{n-1} = (2n/z) J_n -
//           J_{n+1} from a large even start N (J_{N+1} = 0), normalised by
//           J_0 + 2 sum_k J_2k = 1; Y0 from Neumann's series
//           Y0 = (2/pi)(ln(z/2) + gamma) J0 - (4/pi) sum_k (-1)^k J_2k / k
//           (Abramowitz & Stegun 9.1.88, 9.12).
//  z >= 20: Hankel's asymptotic expansion H0^(2)(z) = sqrt(2/(pi z))
//           (P - i Q) exp(-i (z - pi/4)) with P = sum_k (-1)^k c_2k / (8z)^2k,
//           Q = sum_k (-1)^(k+1) c_(2k+1) / (8z)^(2k+1),
//           c_m = prod_{j<=m} (2j-1)^2 / m! (A&S 9.2.5, 9.2.9, 9.2.10), summed
//           until the terms fall below 1e-17 (their smallest size is about
//           exp(-2z) < 1e-17 for z >= 20).
__device__ inline cplx hankel2_0(double z) {
  const double kPi = 3.141592653589793238462643383;
  if (z < 20.0) {
    const int N = 2 * (int)((z + 24.0 + 4.0 * cbrt(z)) * 0.5) + 2;
    const double iz = 1.0 / z;
    double jp = 0.0, jn = 1e-30;  // J_{n+1}, J_n (unnormalised), from n = N down
    double even = 0.0, neu = 0.0;  // sum_k J_2k and sum_k (-1)^k J_2k / k (k >= 1)
    for (int n = N; n >= 1; --n) {
      if ((n & 1) == 0) {
        even += jn;
        const int k = n >> 1;
        neu += ((k & 1) ? -jn : jn) / (double)k;
      }
      const double jm = 2.0 * n * iz * jn - jp;  // J_{n-1}
      jp = jn;
      jn = jm;
      if (fabs(jn) > 1e250) {  // rescale all running values
        jp *= 1e-250;
        jn *= 1e-250;
        even *= 1e-250;
        neu *= 1e-250;
      }
    }
    const double norm = 1.0 / (jn + 2.0 * even);
    const double j0 = jn * norm;
    const double kGamma = 0.57721566490153286060651209;
    const double y0 = (2.0 / kPi) * (log(0.5 * z) + kGamma) * j0 - (4.0 / kPi) * neu * norm;
    return mk(j0, -y0);
  }
  const double w = 1.0 / (8.0 * z);
  double P = 1.0, Q = 0.0, t = 1.0;
  for (int m = 1; m < 80; ++m) {
    t *= (double)((2 * m - 1) * (2 * m - 1)) * w / (double)m;
    const int k = m >> 1;
    if (m & 1) Q += (k & 1) ? t : -t;  // m = 2k + 1: sign (-1)^(k+1)
    else P += (k & 1) ? -t : t;        // m = 2k: sign (-1)^k
    if (t < 1e-17) break;
  }
  double sn, cs;
  sincos(z, &sn, &cs);
  const double amp = sqrt(2.0 / (kPi * z)) * 0.70710678118654752440;  // and 1/sqrt(2) of exp(i pi/4)
  // exp(-i (z - pi/4)) = ((cos z + sin z) + i (cos z - sin z)) / sqrt(2)
  const double er = cs + sn, ei = cs - sn;
  return mk(amp * (P * er + Q * ei), amp * (P * ei - Q * er));
}

// EFIE2D kernel H0^(2)(k ||x_i - y_j||) (Sec. 5, kernel 2).
struct GenHankel2D {
  __device__ __forceinline__ GenHankel2D bind(int) const { return *this; }
  using scalar = cplx;
  const double* x;
  const double* y;
  int dim;
  double k;
  __device__ __forceinline__ cplx operator()(int64_t i, int64_t j) const {
    const double* xi = x + i * dim;
    const double* yj = y + j * dim;
    double s = 0.0;
    for (int t = 0; t < dim; ++t) {
      double u = xi[t] - yj[t];
      s = fma(u, u, s);
    }
    return hankel2_0(k * sqrt(s));
  }
};

// Batched Gaussian blocks: each block b has its own points and width; a leaf
// binds the generator of its block once (batched form of Alg. 2 / Alg. 3).
struct GenGaussianBatch {
  using scalar = double;
  const GaussBlockParams* blocks;
  __device__ __forceinline__ GenGaussian bind(int b) const {
    const GaussBlockParams q = blocks[b];
    GenGaussian g;
    g.x = q.x;
    g.y = q.y;
    g.dim = q.dim;
    g.c = q.c;
    return g;
  }
};

// ------------------------------------------------------------------ reductions
template <typename T> __device__ __forceinline__ T shfl_xor(T v, int m);
template <> __device__ __forceinline__ double shfl_xor<double>(double v, int m) {
  return __shfl_xor_sync(0xffffffffu, v, m);
}
template <> __device__ __forceinline__ cplx shfl_xor<cplx>(cplx v, int m) {
  return mk(__shfl_xor_sync(0xffffffffu, v.re, m), __shfl_xor_sync(0xffffffffu, v.im, m));
}
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = add(v, shfl_xor(v, o));
  return v;
}

// Warp sums of N doubles per lane (N a power of two <= 32) by recursive
// halving: at the shuffle distance 16 >> t a lane keeps half of its values
// and adds its partner's copies of them, so every FP64 add is a full-warp
// one (N - 1 + 5 - log2 N adds for N sums instead of 5 N).  Returns, in lane
// L, the sum of value reduce_scatter_index<N>(L).
template <int N>
__device__ __forceinline__ double warp_reduce_scatter(double (&v)[N], int lane) {
  static_assert(N >= 1 && N <= 32 && (N & (N - 1)) == 0, "N must be a power of two <= 32");
#pragma unroll
  for (int t = 0; (N >> t) > 1; ++t) {
    const int o = 16 >> t, half = N >> (t + 1);
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const double send = up ? v[k] : v[k + half];
      const double keep = up ? v[k + half] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  constexpr int lg = N >= 32 ? 5 : N >= 16 ? 4 : N >= 8 ? 3 : N >= 4 ? 2 : N >= 2 ? 1 : 0;
#pragma unroll
  for (int o = 16 >> lg; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
  return v[0];
}
template <int N>
__device__ __forceinline__ int reduce_scatter_index(int lane) {
  int idx = 0;
#pragma unroll
  for (int t = 0; (N >> t) > 1; ++t) idx += ((lane >> (4 - t)) & 1) * (N >> (t + 1));
  return idx;
}

// Warp sums of two values of type T per lane: lane L ends with component
// comp of value col (T = double: one component), and it is the first lane
// holding that sum when (L & mask) == 0.
template <typename T>
__device__ __forceinline__ double warp_sum2(T a0, T a1, int lane, int& col, int& comp, bool& first);
template <>
__device__ __forceinline__ double warp_sum2<double>(double a0, double a1, int lane, int& col, int& comp, bool& first) {
  double v[2] = {a0, a1};
  const double s = warp_reduce_scatter<2>(v, lane);
  col = reduce_scatter_index<2>(lane);
  comp = 0;
  first = (lane & 15) == 0;
  return s;
}
template <>
__device__ __forceinline__ double warp_sum2<cplx>(cplx a0, cplx a1, int lane, int& col, int& comp, bool& first) {
  double v[4] = {a0.re, a0.im, a1.re, a1.im};
  const double s = warp_reduce_scatter<4>(v, lane);
  const int idx = reduce_scatter_index<4>(lane);
  col = idx >> 1;
  comp = idx & 1;
  first = (lane & 7) == 0;
  return s;
}

// Both warp sums of two values per lane, in every lane.
__device__ __forceinline__ void warp_sum2_all(double& a0, double& a1, int lane) {
  double v[2] = {a0, a1};
  const double s = warp_reduce_scatter<2>(v, lane);
  a0 = __shfl_sync(0xffffffffu, s, 0);
  a1 = __shfl_sync(0xffffffffu, s, 16);
}
__device__ __forceinline__ void warp_sum2_all(cplx& a0, cplx& a1, int lane) {
  double v[4] = {a0.re, a0.im, a1.re, a1.im};
  const double s = warp_reduce_scatter<4>(v, lane);
  a0 = mk(__shfl_sync(0xffffffffu, s, 0), __shfl_sync(0xffffffffu, s, 8));
  a1 = mk(__shfl_sync(0xffffffffu, s, 16), __shfl_sync(0xffffffffu, s, 24));
}

// (bits, index) argmax: larger bits win, ties go to the smaller index.
__device__ __forceinline__ void argmax_merge(long long& b, int& i, long long ob, int oi) {
  if (ob > b || (ob == b && oi < i)) {
    b = ob;
    i = oi;
  }
}
__device__ __forceinline__ void warp_argmax(long long& b, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    long long ob = __shfl_xor_sync(0xffffffffu, b, o);
    int oi = __shfl_xor_sync(0xffffffffu, i, o);
    argmax_merge(b, i, ob, oi);
  }
}

// Device status word values (first error wins).
enum DevStatus : int {
  DS_OK = 0,
  DS_RANK_CAPACITY = 2,
  DS_TIMEOUT = 4,
  DS_NUMERICAL = 6,
  DS_LAUNCH = 8,  // a kernel found a launch shape other than the planned one
  DS_NOT_CONVERGED = 10,  // a Jacobi SVD reached its sweep cap still rotating
};
__device__ __forceinline__ void set_status(int* st, int code) { atomicCAS(st, 0, code); }

}  // namespace hbaca
