// Plain descriptor structs shared by the host planner and the kernels.
#pragma once

#include <stdint.h>

namespace hbaca {

// Per-block parameters of a batched Gaussian compression.
struct GaussBlockParams {
  const double* x;
  const double* y;
  int dim;
  int pad;
  double c;  // -1 / (2 h^2)
};

struct LeafDesc {
  int64_t row0, col0;     // offsets of the leaf in its block's matrix
  int32_t m, n;           // leaf size
  int32_t rcap;           // BACA rank capacity of this leaf
  int32_t tape_iters;     // iteration capacity of the tape
  int64_t stream_id;      // counter-based stream of J_1
  int64_t u_off, v_off;   // element offsets of U (m x rcap, ld m) and V (rcap x n, ld n)
  int64_t tape_off;       // int offset into tape_int (records of 4 + 3d ints)
  int64_t taped_off;      // double offset into tape_dbl (records of 2 doubles)
  int32_t block;          // block of a batched call (0 for a single matrix)
  int32_t pad;
};

struct LeafOut {
  int32_t rank, iters, stop, status;
  double mu;
};

enum StopReason : int {
  STOP_CONVERGED = 0,
  STOP_ITERS = 1,
  STOP_NO_COLS = 2,
  STOP_NO_ROWS = 3,
  STOP_CAPACITY = 4,
  STOP_NUMERICAL = 5,
};

enum TaskKind : int { TASK_LEAF = 0, TASK_HORIZ = 1, TASK_VERT = 2 };

// A stored low-rank block U diag(S) V (U column-major ld m, V row-major ld n).
struct BlockRef {
  int64_t u_off, s_off, v_off;  // element offsets (U, V: scalars; S: doubles) in the store arenas
  int64_t ldu, ldv;             // U column-major (ld >= m), V row-major (ld >= n)
  int32_t m, n;
  int32_t rank_slot;            // index into the rank array
  int32_t cap;                  // rank capacity (columns of U, rows of V)
  int32_t store_cap;            // columns of U / rows of V the storage holds (>= cap)
  int32_t full_slot;            // rank-array index receiving the number of stored singular
                                // triplets (all of them, not only the kept ones), or -1
  void* U;                      // caller buffers of a block's final factors: when set they
  double* S;                    // replace the arena + offset addresses
  void* V;
};

struct SvdTask {
  int32_t kind;
  int32_t kcap;        // capacity of k (columns of the QR operand)
  // inputs (LEAF: leaf index into the BACA arenas; merges: blocks of the input store)
  int32_t in1, in2;
  // QR operand A: rows_a x k, column-major, ld = lda (LEAF: the BACA U arena in place)
  int64_t a_off;       // offset in the arena selected by a_in_baca
  int32_t rows_a, a_in_baca;
  int64_t lda;
  // QR operand B (LEAF only): rows_b x k, column-major (V^H), in the QR arena
  int64_t b_off;
  int32_t rows_b;
  int32_t trunc;       // truncation rule: 0 the eps-rank (Sec. 2); n > 0 the Frobenius
                       // rule with budget eps / sqrt(n), n = 2L + 1 (HBACA_FLAG_FROB)
  int64_t src_v_off;   // LEAF: offset of the leaf's V (k x rows_b, row-major) in the BACA V arena
  int64_t tau_off;     // 3 * kcap scalars: reflectors of QR(A), QR(B), QRCP of the core
  int64_t m_off;       // core M (kcap x kcap, column-major ld kcap); QRCP in place
  int64_t y_off;       // W: Jacobi rotations accumulated (kcap x kcap)
  int64_t x_off;       // X = R2^H, the matrix the Jacobi sweeps orthogonalise (kcap x kcap)
  int64_t xs_off;      // left singular vectors of M, sorted, compact (kcap x kcap)
  int64_t ys_off;      // right singular vectors of M, sorted, compact (kcap x kcap)
  int64_t ord_off;     // 2 * kcap ints: Jacobi column order, then the QRCP permutation
  int32_t out;         // block index in the output store
  int32_t m1;          // HORIZ / VERT: rows (VERT) or columns (HORIZ) of the first child
  int64_t src_u_off;   // LEAF with a_in_baca = 0: offset of the leaf's U in the BACA U arena
                       // (the QR then works on a copy and the BACA factors survive the call)
};

// Device-side per-task sizes written by the kernels.
struct TaskDims {
  int32_t k;       // columns of the QR operand(s) (LEAF: BACA rank; merges: r1 + r2)
  int32_t kra;     // rows of R_A = min(rows_a, k)
  int32_t krb;     // rows of R_B (LEAF) = min(rows_b, k)
  int32_t s;       // truncated rank
  int32_t sweeps;  // Jacobi sweeps run
  int32_t nout;    // singular triplets written to the output (s, or all of them when taped)
  int32_t rotations;  // Jacobi rotations applied (all sweeps, all CTAs of the task)
  int32_t pad;
};

// Cluster slots of the inter-cluster partial-sum exchange of one QR or
// Q-application launch (matrices x clusters per matrix).
constexpr int kXSlots = 64;

struct QrJob {
  int32_t task;
  int32_t which;  // 0: operand A, 1: operand B
};

struct QJob {
  int32_t task;
  int32_t which;   // 0: operand A with X_s, 1: operand B with Y_s
  int32_t to_v;    // 1: the result is stored as V = D^H in the output block
  int32_t pad;
};

}  // namespace hbaca
