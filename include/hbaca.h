/*
 * hbaca.h -- C ABI of the GB300 (sm_103a) H-BACA library, libhbaca.so.
 *
 * The method is H-BACA (Liu, Sid-Lakhdar, Rebrova, Ghysels, Li, "A Parallel
 * Hierarchical Blocked Adaptive Cross Approximation Algorithm", arXiv
 * 1901.06101): every leaf block of an L-level partition (n_b = 4^L leaves)
 * is compressed by blocked adaptive cross approximation (Alg. 2) from an
 * O(1) entry function, re-compressed by QR + truncated SVD (Sec. 3.2, last
 * paragraph), and the leaves are merged pairwise up two binary index trees
 * (Alg. 3, Eqs. columncomb, columnsvdmerge).  The result is an approximate
 * truncated SVD A ~ U diag(S) V with ||A - U S V||_F <~ eps ||A||_F (the
 * problem statement of Alg. 1-3; the bound is heuristic, Eq. aca_stop).
 *
 * Conventions
 *  - All matrix and point pointers are DEVICE pointers unless stated.  The
 *    caller allocates every device buffer (factors, workspace); the library
 *    never calls cudaMalloc / cudaFree.
 *  - U is column-major (element (i, p) at U[p * ldu + i]); V is row-major
 *    (element (p, j) at V[p * ldv + j]).  Complex data is interleaved
 *    (real, imaginary) pairs of double, 16-byte aligned.
 *  - Every entry point is synchronous with respect to the host unless
 *    HBACA_FLAG_ASYNC is set: it enqueues work on `stream` (a cudaStream_t;
 *    NULL = the legacy default stream), synchronises that stream once at the
 *    end and returns the rank on the host.
 *  - No exception crosses the ABI.  Errors are reported as hbaca_status;
 *    hbaca_last_error() gives a message for the calling thread.
 *  - Device-side failures (rank capacity exceeded, NaN/Inf in a norm or a
 *    pivot) are written to a status word in the workspace and mapped to
 *    the return code when the call synchronises.
 */
#ifndef HBACA_H
#define HBACA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hbaca_status {
  HBACA_OK = 0,
  HBACA_INVALID_ARG = 1,    /* a NULL pointer, a size out of range, an unknown kind */
  HBACA_RANK_CAPACITY = 2,  /* a leaf or merged rank exceeded its capacity */
  HBACA_CUDA = 3,           /* a CUDA runtime call failed (message has the detail) */
  HBACA_TIMEOUT = 4,        /* a bounded device-side wait expired (the inter-cluster wait of
                               the QR / Q application, 4 s; see HBACA_FLAG_SINGLE_CLUSTER) */
  HBACA_NO_TAPE = 5,        /* backward called on a result without a recorded tape */
  HBACA_NUMERICAL = 6,      /* NaN or Inf in a norm, a pivot or a singular value */
  HBACA_WORKSPACE = 7,      /* workspace too small or misaligned (256-byte alignment) */
  HBACA_NOT_CONVERGED = 8   /* the one-sided Jacobi SVD of a re-compression or merge core
                               (Sec. 2, SVD(A, eps)) reached its sweep cap (40) while still
                               rotating: singular values and eps-ranks are unreliable */
} hbaca_status;

/* Entry generators: A(i, j) computable in O(1) (abstract; Sec. 5 kernels). */
typedef enum hbaca_gen_kind {
  HBACA_GEN_DENSE = 0,          /* explicit matrix a (column-major, lda >= m)             */
  HBACA_GEN_GAUSSIAN = 1,       /* exp(-||x_i - y_j||^2 / (2 h^2))       (Sec. 5, kernel 1) */
  HBACA_GEN_HELMHOLTZ = 2,      /* exp(i k r) / r, r = ||x_i - y_j||     (complex128)       */
  HBACA_GEN_SPARSE_PRODUCT = 3, /* sum_k P(i,k) Q(k,j) + sum_t P2(i,t) Q2(t,j)              */
  HBACA_GEN_LOWRANK = 4,        /* sum_t LU(i,t) LV(t,j)        (Sec. 5, kernel 6)          */
  HBACA_GEN_POLYNOMIAL = 5,     /* (x_i^t y_j + h)^2            (Sec. 5, kernel 5; float64) */
  HBACA_GEN_HANKEL2D = 6        /* H0^(2)(k ||x_i - y_j||), the EFIE2D kernel (Sec. 5,
                                   kernel 2; complex128); x_i != y_j (H0^(2) is singular
                                   at 0) */
} hbaca_gen_kind;

typedef enum hbaca_dtype { HBACA_F64 = 0, HBACA_C128 = 1 } hbaca_dtype;

/* Description of one matrix A (m x n).  Only the fields of `kind` are read. */
typedef struct hbaca_gen {
  int32_t kind;        /* hbaca_gen_kind */
  int32_t dtype;       /* hbaca_dtype; HELMHOLTZ requires C128, GAUSSIAN and
                          SPARSE_PRODUCT require F64 */
  int64_t m, n;        /* rows, columns (1 <= m, n < 2^31) */
  /* GAUSSIAN, HELMHOLTZ, POLYNOMIAL, HANKEL2D: points, row-major, `dim` doubles each */
  const double* x;     /* m x dim */
  const double* y;     /* n x dim */
  int32_t dim;         /* 1 .. 64 */
  int32_t pad0;
  double h;            /* Gaussian width (finite, > 0); POLYNOMIAL: the shift h (finite) */
  double k;            /* Helmholtz / HANKEL2D wavenumber (finite; HANKEL2D: > 0) */
  /* DENSE */
  const void* a;       /* m x n column-major, scalar = dtype */
  int64_t lda;
  /* LOWRANK: LU (m x lr, column-major, ld = m), LV (lr x n, row-major, ld = n) */
  const void* lu;
  const void* lv;
  int64_t lr;
  /* SPARSE_PRODUCT: P (m x K) in CSR, Q (K x n) in CSC, indices sorted
     ascending within a row of P / a column of Q; P2 (m x r2) and Q2 (r2 x n)
     dense row-major. */
  int64_t K;
  const int32_t* p_rowptr;  /* m + 1 */
  const int32_t* p_colidx;
  const double* p_val;
  const int32_t* q_colptr;  /* n + 1 */
  const int32_t* q_rowidx;
  const double* q_val;
  const double* p2;
  const double* q2;
  int32_t r2;               /* 0 .. 16 */
  int32_t pad1;
} hbaca_gen;

/* Flags */
#define HBACA_FLAG_ASYNC 1u    /* do not synchronise; the rank goes to result.d_rank only */
#define HBACA_FLAG_PROFILE 2u  /* record CUDA events around each phase on `stream`
                                  (read with hbaca_phase_times after the call) */
#define HBACA_FLAG_TAPE 4u     /* keep, in the workspace, every intermediate block of the
                                  merge tree with ALL singular triplets of its core (not
                                  only the eps-rank kept ones), for hbaca_apply_backward.
                                  The kept results agree with an untaped call to rounding
                                  (a taped call accumulates the Jacobi rotations, an
                                  untaped one recovers the kept right vectors); the
                                  workspace is larger (no store is reused across levels) */
#define HBACA_FLAG_GRAPH 8u    /* capture the call into a CUDA graph and replay it: the first
                                  call with a given plan, caller buffers, workspace and
                                  options runs normally (sizing its launches by the actual
                                  ranks) and then captures itself; later identical calls on
                                  the same context only launch the graph (one graph is kept
                                  per context).  The workspace must not be used by other
                                  calls between replays.  New data in the same buffers is
                                  allowed: results are exact, only the launch shapes were
                                  chosen for the first call's ranks. */
#define HBACA_FLAG_SINGLE_CLUSTER 16u  /* one thread-block cluster per matrix in the QR and Q
                                  application of every merge stage.  By default a stage
                                  with few matrices spreads each over several clusters
                                  that exchange partial sums through global memory and
                                  wait for one another (a cooperative launch keeps them
                                  resident; waits are bounded, HBACA_TIMEOUT on expiry).
                                  This flag is for tools that serialise or re-launch
                                  kernels (profilers), which cannot keep them resident. */
#define HBACA_FLAG_FROB 32u    /* truncate every leaf re-compression and merge by the
                                  Frobenius rule instead of the eps-rank of Sec. 2: keep
                                  the fewest singular triplets whose discarded tail
                                  sqrt(sum_{j>t} sigma_j^2) is at most eps / sqrt(2L + 1)
                                  of the block's Frobenius norm (L: the block's merge
                                  levels; a block passes through 2L + 1 truncations, so
                                  their budgets add up to eps in quadrature, the relative
                                  Frobenius error of Sec. 5.2).  BACA's own stopping test
                                  (nu < eps mu) is unchanged. */

/* Options of one compression (Alg. 3 inputs n_b, d, eps). */
typedef struct hbaca_opts {
  double eps;             /* relative tolerance, 0 < eps < 1 */
  int32_t d;              /* BACA block size, 1 .. 32 (d = 1 is ACA, Sec. 3.2) */
  int32_t levels;         /* L >= 0: n_b = 4^L leaves, 2^L <= min(m, n); L < 0: per
                             block, the smallest L whose leaves have at most -L rows
                             and columns (limited by 2^L <= min(m, n)) */
  uint64_t seed;          /* seed of the random initial column blocks J_1 */
  int64_t rank_cap;       /* column capacity of U / rows of V (output and every
                             merged block), <= 1024; 0 = min(m, n, 1024) */
  int64_t leaf_rank_cap;  /* capacity of a leaf's BACA factors before
                             re-compression, <= 1024; 0 = min(m_leaf, n_leaf, 1024) */
  uint32_t flags;         /* HBACA_FLAG_* (any other bit: HBACA_INVALID_ARG) */
  int32_t cluster;        /* CTAs per leaf (1, 2, 4, 8, 16); 0 = choose automatically */
  double srrqr_f;         /* 0: the greedy QRCP pivots of Alg. 2.  f > 1: each greedy
                             pivot set I_k / J_{k+1} whose smallest pivot residual is
                             at least 1e-8 of max(first pivot residual, mu) is then
                             refined by strong rank-revealing QR (Gu & Eisenstat 1996,
                             one of the subset selections Sec. 3.2 names): a chosen
                             vector is swapped for a candidate while that multiplies
                             the chosen set's volume by more than f (at most 4k + 4
                             swaps per set) */
} hbaca_opts;

/* Output factors (caller-owned device memory) and the rank. */
typedef struct hbaca_result {
  void* U;            /* m x rank_cap, column-major, ld = ldu >= m */
  int64_t ldu;
  double* S;          /* rank_cap singular values, descending */
  void* V;            /* rank_cap x n, row-major, ld = ldv >= n */
  int64_t ldv;
  int32_t* d_rank;    /* optional device int receiving the rank (may be NULL) */
  int64_t rank;       /* OUT (host): the rank r; rows/columns beyond r are unspecified */
  int32_t leaf_rank_max;   /* OUT: largest leaf BACA rank before re-compression */
  int32_t leaf_iters_max;  /* OUT: largest number of BACA iterations of a leaf */
} hbaca_result;

typedef struct hbaca_ctx hbaca_ctx;

/* Create / destroy a context bound to the current CUDA device. */
hbaca_status hbaca_create(hbaca_ctx** ctx);
hbaca_status hbaca_destroy(hbaca_ctx* ctx);

/* Bytes of device workspace hbaca_compress needs for (gen, opts); 0 when the
   arguments are invalid (hbaca_last_error() says why). */
size_t hbaca_workspace_size(const hbaca_gen* gen, const hbaca_opts* opts);

/* H-BACA(A, n_b = 4^L, d, eps) (Alg. 3): leaf BACA (Alg. 2) with on-device
   entry generation, leaf SVD re-compression (Sec. 3.2), hierarchical merge
   (Eqs. columncomb, columnsvdmerge).  `workspace` must hold
   hbaca_workspace_size(gen, opts) bytes, 256-byte aligned; it is overwritten
   and, after the call, holds the per-leaf pivot tape read by
   hbaca_read_leaf_trace.  Returns HBACA_RANK_CAPACITY when a rank exceeds
   rank_cap / leaf_rank_cap. */
hbaca_status hbaca_compress(hbaca_ctx* ctx, const hbaca_gen* gen, const hbaca_opts* opts,
                            hbaca_result* out, void* workspace, void* stream);

/* Batched H-BACA: `nblocks` independent matrices (HOST array `gens`, all the
   same kind and dtype; kind GAUSSIAN when nblocks > 1), each compressed as by
   hbaca_compress with its own tree depth (opts.levels, see above) and written
   to its own result outs[b] (HOST array).  All leaves of all blocks share one
   persistent BACA launch, largest leaves first; every merge level of all
   blocks is one batch of launches.  The workspace must hold
   hbaca_workspace_size_batched(nblocks, gens, opts) bytes, 256-byte aligned.
   This is the batched form of Alg. 2 / Alg. 3 over many admissible blocks. */
size_t hbaca_workspace_size_batched(int32_t nblocks, const hbaca_gen* gens, const hbaca_opts* opts);
hbaca_status hbaca_compress_batched(hbaca_ctx* ctx, int32_t nblocks, const hbaca_gen* gens, const hbaca_opts* opts,
                                    hbaca_result* outs, void* workspace, void* stream);

/* hbaca_compress with a workspace built into the library instead of one from
   the caller; the paper has no counterpart (it is an interface convenience).
   Meant for callers that cannot allocate device memory themselves: a C
   program with no device allocator of its own, a caller whose device memory
   all belongs to another runtime's pool, or a latency-bound caller that must
   not allocate per call.  The area is HBACA_NOALLOC_WORKSPACE_BYTES per
   device; a problem whose hbaca_workspace_size exceeds it is rejected with
   HBACA_WORKSPACE before anything is enqueued.  Every call looks up the
   area's address on the current device (cudaGetSymbolAddress, no stale
   address after a device reset); the first call on a device loads the
   module there, so make it before any stream capture.  The current device
   must be the context's (HBACA_INVALID_ARG otherwise).  HBACA_FLAG_GRAPH
   and HBACA_FLAG_TAPE are rejected with HBACA_INVALID_ARG: a graph replay
   would read descriptor tables that a later call on the shared area has
   replaced, and a tape in the area cannot be handed to
   hbaca_apply_backward, which needs its workspace pointer.  With
   HBACA_FLAG_ASYNC the rank is delivered through result.d_rank only.  No
   device memory is allocated or freed.  All calls on one device share the
   area, so calls that overlap in time (other threads, or other streams
   with work still pending) race on it: serialise them.  Results, ranks
   and status are as for hbaca_compress; the leaf records in the area are
   overwritten by the next call. */
#define HBACA_NOALLOC_WORKSPACE_BYTES (64u << 20)
hbaca_status hbaca_compress_noalloc(hbaca_ctx* ctx, const hbaca_gen* gen, const hbaca_opts* opts,
                                    hbaca_result* out, void* stream);

/* ---- Apply and reverse pass (real F64; the reverse pass: GAUSSIAN generator) ----

   y = U diag(S) V X for a compressed result (A ~ U diag(S) V, the output of
   Alg. 3).  X: n x nrhs, column-major (ldx >= n); Y: m x nrhs, column-major
   (ldy >= m), overwritten.  `workspace` (device, 256-byte aligned) holds
   hbaca_apply_workspace_size(rank, nrhs) bytes.  Synchronises `stream`. */
size_t hbaca_apply_workspace_size(int64_t rank, int64_t nrhs);
hbaca_status hbaca_apply(hbaca_ctx* ctx, const hbaca_gen* gen, const hbaca_result* res, const void* X, int64_t nrhs,
                         int64_t ldx, void* Y, int64_t ldy, void* workspace, void* stream);

/* Reverse pass of Y = (U diag(S) V) X with every discrete choice of the
   forward frozen: the BACA pivots and LRID ranks of each leaf (Alg. 2), and
   the truncation rank of the leaf re-compression and of every merge
   (Sec. 3.2; Alg. 3).  Given dY = dL/dY it returns
     d_x = dL/dx (m x dim, row-major like x), d_y = dL/dy (n x dim),
     d_h = dL/dh (one double), dX = dL/dX = (U diag(S) V)^T dY (n x nrhs,
     column-major, ldx >= n; NULL to skip),
   for the GAUSSIAN generator A(i, j) = exp(-||x_i - y_j||^2 / (2 h^2)),
   real F64.  Each truncated SVD is differentiated with the singular-value-gap
   coefficients 1 / (sigma_i^2 - sigma_j^2) (i kept, j discarded), which is
   why the forward must run with HBACA_FLAG_TAPE (every merge node keeps all
   its singular triplets); the BACA residual rows are regenerated from the
   factors, not stored.  gen, opts and workspace are those of the forward
   call, res its result; all output arrays are device memory and are
   overwritten (any of d_h, d_x, d_y may be NULL).  `bwd_workspace` (device,
   256-byte aligned) holds hbaca_backward_workspace_size(...) bytes, a size
   that depends on the ranks of the forward: the size query reads them from
   `workspace` (and synchronises `stream`).  No counterpart in the paper,
   which has no reverse pass; the adjoint is of the map the paper defines. */
size_t hbaca_backward_workspace_size(const hbaca_gen* gen, const hbaca_opts* opts, const void* workspace, int64_t nrhs,
                                     void* stream);
hbaca_status hbaca_apply_backward(hbaca_ctx* ctx, const hbaca_gen* gen, const hbaca_opts* opts, const hbaca_result* res,
                                  const void* workspace, const void* X, int64_t nrhs, int64_t ldx, const void* dY,
                                  int64_t lddy, double* d_h, double* d_x, double* d_y, void* dX, int64_t lddx,
                                  void* bwd_workspace, size_t bwd_bytes, void* stream);

/* Reverse pass over the blocks of one taped hbaca_compress_batched call
   (GAUSSIAN, F64): per block b the same as hbaca_apply_backward with X[b]
   (n_b x nrhs, ld n_b), dY[b] (m_b x nrhs, ld m_b), dX[b] (n_b x nrhs, ld n_b;
   dX or dX[b] may be NULL), d_x[b] (m_b x dim), d_y[b] (n_b x dim) and d_h[b]
   (d_h: a device array of nblocks doubles; any of d_h, d_x, d_y may be NULL).
   X, dY, dX, d_x, d_y are HOST arrays of device pointers; gens, results are the
   forward's host arrays.  The size query reads the forward's ranks. */
size_t hbaca_backward_workspace_size_batched(int32_t nblocks, const hbaca_gen* gens, const hbaca_opts* opts,
                                             const void* workspace, int64_t nrhs, void* stream);
hbaca_status hbaca_apply_backward_batched(hbaca_ctx* ctx, int32_t nblocks, const hbaca_gen* gens,
                                          const hbaca_opts* opts, const hbaca_result* results, const void* workspace,
                                          const void* const* X, int64_t nrhs, const void* const* dY, double* d_h,
                                          double* const* d_x, double* const* d_y, void* const* dX,
                                          void* bwd_workspace, size_t bwd_bytes, void* stream);

/* Autotuner of the batched (or single, nblocks = 1) call: times the
   persistent leaf BACA launch (Alg. 2 over all leaves) with clusters of 1, 2,
   4, 8 and 16 CTAs per leaf (every size whose plan fits `workspace_bytes`)
   and returns the fastest in *best_cluster and its device time in *best_ms.
   The cluster size does not change any result (every CTA of a cluster takes
   the same pivot decisions); set opts.cluster to the returned value.  Uses
   `workspace` as scratch and synchronises `stream`.  No counterpart in the
   paper. */
hbaca_status hbaca_autotune_batched(hbaca_ctx* ctx, int32_t nblocks, const hbaca_gen* gens, const hbaca_opts* opts,
                                    void* workspace, size_t workspace_bytes, void* stream, int32_t* best_cluster,
                                    double* best_ms);

/* Accuracy of a compression, measured on the device (the relative Frobenius
   error of the paper's accuracy study, Sec. 5.2): out[0] = ||A(I,:) -
   U(I,:) diag(S) V||_F^2 and out[1] = ||A(I,:)||_F^2 (HOST array of two
   doubles) over the rows I = rows[0 .. nrows-1] (a HOST array of row indices
   in [0, m), each counted as often as it appears), or over all rows when rows
   is NULL and nrows = 0.  The relative error is sqrt(out[0] / out[1]).  The
   entries of A are regenerated from `gen` tile by tile; the factors are read
   from `res` (U, S, V, ldu, ldv and the HOST rank res->rank, as a synchronous
   hbaca_compress left them).  `workspace` (device, 256-byte aligned) holds
   hbaca_error_workspace_size(nrows) bytes.  Synchronises `stream`.  Returns
   HBACA_INVALID_ARG for a row index outside [0, m), a missing rank or an
   unsupported generator. */
size_t hbaca_error_workspace_size(int64_t nrows);
hbaca_status hbaca_error_norms(hbaca_ctx* ctx, const hbaca_gen* gen, const hbaca_result* res, const int64_t* rows,
                               int64_t nrows, double* out, void* workspace, size_t workspace_bytes, void* stream);

/* ---- Geometry (host only; no device memory, no stream) ----

   KD-tree ordering of n points (HOST, row-major n x dim): perm (HOST, n
   entries) receives an ordering in which every node of the H-BACA index tree
   (Alg. 3: a node of s indices has a first child of ceil(s/2)) down to nodes
   of at most `leaf` points is one side of a split of its parent's points
   along the widest side of their bounding box.  Compressing A(perm_x,
   perm_y) is the setting of the paper's experiments (Sec. 5: rows and
   columns permuted by a KD-tree partitioning), in which every leaf is a
   spatial cell. */
hbaca_status hbaca_kdtree_order(const double* points, int64_t n, int32_t dim, int64_t leaf, int64_t* perm);

/* Blocks of a hierarchical-matrix partition of the kernel matrix between
   ordered point sets x (m x dim) and y (n x dim) (HOST, row-major, each
   ordered by hbaca_kdtree_order with the same leaf size): the block cluster
   tree of the two halving trees, a block (tau, sigma) being admissible when
   min(diam tau, diam sigma) <= eta dist(tau, sigma) (bounding boxes); an
   inadmissible block is split (its larger side first) until both sides have
   at most `leaf` points.  blocks (HOST, 5 x max_blocks int64) receives per
   block (row start, rows, column start, columns, admissible 0/1), in tree
   order; returns the number of blocks (-1 on invalid arguments; blocks may
   be NULL to query the count).  The blocks tile the matrix.  Every
   admissible block is a low-rank block for H-BACA (Sec. 1: H-BACA as the
   compression tool of hierarchical matrices); hbaca_compress_batched
   compresses them all in one call. */
int64_t hbaca_hmatrix_blocks(const double* x, int64_t m, const double* y, int64_t n, int32_t dim, int64_t leaf,
                             double eta, int64_t* blocks, int64_t max_blocks);

/* Per-leaf record of one BACA run (Alg. 2), copied to HOST arrays provided
   by the caller.  Leaf (a, b) of the 2^L x 2^L partition has index
   a * 2^L + b.  Arrays I, J, jbar hold `max_iters * d` entries (row-major by
   iteration, unused slots -1); dI, dJ, dk, nu, mu hold `max_iters` entries.
   I: row pivots of QR(C_k^t, d) in pivot order (before the shrink of line 9);
   J: column block J_k (before LRID); jbar: positions into J of the columns
   LRID keeps (Eq. IkJkUp); dI = |I_k|, dJ = |J_k|, dk = d_k; nu, mu: the
   norms of lines 10-11.  Indices are local to the leaf. */
typedef struct hbaca_leaf_trace {
  int32_t iters;      /* OUT: iterations run */
  int32_t rank_baca;  /* OUT: BACA rank before re-compression */
  int32_t rank;       /* OUT: rank after re-compression */
  int32_t stop;       /* OUT: 0 converged, 1 iteration bound, 2 no columns left,
                         3 no rows left, 4 rank capacity, 5 NaN/Inf */
  int32_t max_iters;  /* IN: capacity of the arrays below, in iterations */
  int32_t d;          /* IN: row stride of I, J, jbar (must equal opts.d) */
  int32_t* I;
  int32_t* J;
  int32_t* jbar;
  int32_t* dI;
  int32_t* dJ;
  int32_t* dk;
  double* nu;
  double* mu;
} hbaca_leaf_trace;

hbaca_status hbaca_read_leaf_trace(const hbaca_gen* gen, const hbaca_opts* opts,
                                   const void* workspace, int64_t leaf,
                                   hbaca_leaf_trace* trace, void* stream);

/* The same record for leaf `leaf` of block `block` of a batched call. */
hbaca_status hbaca_read_leaf_trace_batched(int32_t nblocks, const hbaca_gen* gens, const hbaca_opts* opts,
                                           const void* workspace, int32_t block, int64_t leaf,
                                           hbaca_leaf_trace* trace, void* stream);

/* Device time of the phases of the last hbaca_compress on `ctx` that ran with
   HBACA_FLAG_PROFILE, from CUDA events recorded on the call's stream:
   ms[0] leaf BACA kernel (Alg. 2), ms[1] leaf re-compression (Sec. 3.2),
   ms[2] hierarchical merges (Alg. 3), ms[3] whole call.  *launches receives
   the number of kernels the call launched.  Synchronises on the events. */
hbaca_status hbaca_phase_times(hbaca_ctx* ctx, double ms[4], int32_t* launches);

/* Device time per kernel class of the last hbaca_compress(_batched) on `ctx`
   that ran with HBACA_FLAG_PROFILE (CUDA events around every launch, on the
   call's stream).  Classes, in order: leaf BACA (Alg. 2), QR-operand
   packing, Householder QR, core product, pivoted QR of the core, Jacobi SVD
   of the core, singular vectors of the core, reflector application,
   block-diagonal product, root copy (taped calls).  ms[c] is the time during
   which at least one launch of class c ran (launches of a class that run
   concurrently on two streams count once), launches[c] the number of
   launches.  Synchronises on the events. */
#define HBACA_KERNEL_CLASSES 10
hbaca_status hbaca_kernel_times(hbaca_ctx* ctx, double ms[HBACA_KERNEL_CLASSES], int32_t launches[HBACA_KERNEL_CLASSES]);

/* Message of the last failed call on this thread ("" if none). */
const char* hbaca_last_error(void);

/* Library version string. */
const char* hbaca_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HBACA_H */
