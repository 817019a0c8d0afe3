/*
 * hbaca_debug.h -- inspection entry points of libhbaca.so for tests and
 * debugging (not needed to use the library).
 */
#ifndef HBACA_DEBUG_H
#define HBACA_DEBUG_H

#include "hbaca.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Copy one intermediate low-rank block U diag(S) V of an H-BACA call out of
   its workspace into HOST buffers, after hbaca_compress returned.
   store 0: blocks after the vertical merge of level `level` (level 0 = the
   re-compressed leaves; levels 0 .. L-1); store 1: blocks after the
   horizontal merge of level `level` (1 .. L).  Block (a, b) of a store level
   with nb column nodes has index a * nb + b (Alg. 3 node order).
   U (m x rank, column-major, ld m), S (rank), V (rank x n, row-major, ld n)
   must hold m * cap, cap and cap * n elements where cap = opts.rank_cap (as
   resolved by the library; *cap_out receives it).  *m_out, *n_out, *rank_out
   receive the block's size and rank. */
hbaca_status hbaca_debug_read_block(const hbaca_gen* gen, const hbaca_opts* opts, const void* workspace,
                                    int32_t store, int32_t level, int64_t block, void* U, double* S, void* V,
                                    int64_t* m_out, int64_t* n_out, int64_t* rank_out, int64_t* cap_out,
                                    void* stream);

/* The BACA factors of leaf `leaf` (Alg. 2 output before re-compression) of
   a call made with HBACA_FLAG_TAPE (only then do they survive the call),
   copied into HOST buffers: U (m_leaf x rank, column-major, ld m_leaf) and
   V (rank x n_leaf, row-major, ld n_leaf), which must hold m_leaf * cap and
   cap * n_leaf scalars for the leaf's rank capacity cap (opts.leaf_rank_cap
   as resolved; at most min(m_leaf, n_leaf, 1024)).  *m_out, *n_out,
   *rank_out receive the leaf's size and BACA rank. */
hbaca_status hbaca_debug_read_leaf_factors(const hbaca_gen* gen, const hbaca_opts* opts, const void* workspace,
                                           int64_t leaf, void* U, void* V, int64_t* m_out, int64_t* n_out,
                                           int64_t* rank_out, void* stream);

/* Every launch of the last call made with HBACA_FLAG_PROFILE on `ctx`: its
   kernel class (the order of hbaca_kernel_times), its stage (the index of the
   re-compression or merge stage in plan order; -1 for the leaf BACA launch),
   its start and its duration in ms (CUDA events on the launching stream,
   start relative to the call's first event).  Fills at most `max` entries of
   each (NULL arrays are skipped) and returns the number of launches, or -1. */
int32_t hbaca_debug_launch_times(hbaca_ctx* ctx, int32_t* cls, int32_t* stage, double* start_ms, double* ms,
                                 int32_t max);

/* Write a JSON description of the workspace layout of (gen, opts) (region
   byte offsets, stage task tables) into buf (NUL-terminated, truncated to
   len).  Returns the length the full text needs. */
size_t hbaca_debug_plan_json(const hbaca_gen* gen, const hbaca_opts* opts, char* buf, size_t len);

/* Layout of the reverse pass for a taped forward (gen, opts, workspace) with
   nrhs right-hand sides, as JSON in buf (NUL-terminated, truncated to len):
   per leaf the byte offsets, in the backward workspace, of the BACA factor
   adjoints, the column and row adjoint arrays and their index maps; per merge
   node its kept and stored triplet counts and buffer offsets.  Reads the
   sizes from `workspace` (synchronises `stream`).  Returns the length the
   full text needs, or -1. */
int64_t hbaca_debug_backward_json(const hbaca_gen* gen, const hbaca_opts* opts, const void* workspace, int64_t nrhs,
                                  char* buf, int64_t len, void* stream);

/* Entries A(rows[t], cols[t]), t < count, of the matrix described by `gen`,
   evaluated on the device by the same entry generators the compression uses
   (rows, cols: DEVICE int64 arrays; out: DEVICE array of count scalars of
   gen->dtype; a pair outside [0, m) x [0, n) gives NaN).
   Enqueued on `stream`, not synchronised.  For tests of the generators. */
hbaca_status hbaca_debug_entries(const hbaca_gen* gen, const int64_t* rows, const int64_t* cols, int64_t count,
                                 void* out, void* stream);

/* Cluster size (CTAs per core, 1 .. 16) that every later synchronous call in
   this process gives the one-sided Jacobi SVD of every core (raised where a
   core's columns do not fit the shared memory of that many CTAs); 0 restores
   the per-stage choice.  Returns the previous setting.  Results do not depend
   on it (every rotation is formed and applied with the same arithmetic
   whatever CTA runs it); it exists to time the launch shapes. */
int32_t hbaca_debug_set_jacobi_cluster(int32_t cluster);

/* Cluster size (CTAs per matrix, 1 .. 16) of the Householder QR and the Q
   application of every merge and re-compression stage in every later
   synchronous call in this process, one cluster per matrix; 0 restores the
   per-stage choice (which may spread a matrix over several clusters).
   Returns the previous setting.  The partial sums are combined in CTA order,
   so results depend on it at the rounding level; it exists to time the
   launch shapes. */
int32_t hbaca_debug_set_qr_cluster(int32_t cluster);

/* Upper bound (1 .. 32) on the number of 8-CTA clusters that the QR and the Q
   application of a stage with few matrices spread one matrix over, in every
   later synchronous call in this process (fewer than 3: one 16-CTA cluster
   per matrix); 0 restores the automatic choice.  Returns the previous
   setting.  Partial sums are combined in cluster order, so results depend on
   it at the rounding level; it exists to time the launch shapes. */
int32_t hbaca_debug_set_qr_groups(int32_t groups);

/* Clusters of 16 CTAs per core (1 .. 32) for the one-sided Jacobi SVD of the
   cores whose columns do not fit one cluster's shared memory, in every later
   synchronous call in this process: 1 keeps one cluster per core, 0 restores
   the automatic choice (several clusters sweep one such core through global
   memory, with bounded waits; HBACA_TIMEOUT on expiry).  Returns the previous
   setting.  Results do not depend on it (every rotation is formed and applied
   with the same arithmetic whichever CTA runs it). */
int32_t hbaca_debug_set_jacobi_groups(int32_t groups);

/* Sweep cap of the one-sided Jacobi SVD (Sec. 2, SVD(A, eps)) used by every
   later call in this process: sweeps > 0 sets it, 0 restores the default
   (40).  Returns the cap in force before the call.  For tests that make a
   core stop short of convergence (the call then returns
   HBACA_NOT_CONVERGED). */
int32_t hbaca_debug_set_jacobi_sweeps(int32_t sweeps);

#ifdef __cplusplus
}
#endif

#endif /* HBACA_DEBUG_H */
