// Host-side planning of an H-BACA call over one or many blocks: the two
// index trees of every block (Alg. 3 line 1; first child of a node of size s
// has ceil(s/2) indices), the leaf table and its processing order, the merge
// tasks of every level, and the byte layout of the caller's workspace.
// Everything here is plain host C++.
#pragma once

#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "hbaca.h"

namespace hbaca {

struct LeafDesc;
struct SvdTask;
struct BlockRef;
struct QrJob;
struct QJob;

using Span = std::pair<int64_t, int64_t>;  // (start, size)

// Nodes of an L-level binary tree on [0, n): levels[l] lists the nodes of
// level l (0 = leaves, L = root) left to right.
std::vector<std::vector<Span>> tree_levels(int64_t n, int L);

struct Region {
  size_t off = 0, bytes = 0;
};

// One batch of tasks launched together (a stage of Alg. 3, or a chunk of one).
struct Stage {
  int kind;                      // TaskKind
  std::vector<SvdTask>* tasks_h; // host copy (owned by Plan)
  int ntasks = 0;
  size_t tasks_off = 0, dims_off = 0, qrjobs_off = 0, qjobs_off = 0;
  int nqr = 0, nq = 0;
  int kcap = 0;
  int rows_max = 0;
  int in_store = -1, out_store = -1;  // block-store arenas: 0 = full, 1 = half
  size_t jlist_off = 0;                // element offset of this stage's Jacobi task lists in jlist
};

struct Plan {
  // inputs
  std::vector<hbaca_gen> gens;  // one per block
  hbaca_opts opts;
  bool cplx = false;
  size_t esz = 8;
  int d = 1;
  int nblocks = 0;
  int Lmax = 0;
  std::vector<int> Lb;            // levels of each block
  std::vector<int64_t> cap_b;     // rank capacity of each block's output
  int64_t rank_cap_max = 0;
  std::vector<int> leaf_first;    // first leaf of each block
  // leaves
  int nleaves = 0;
  int mmax = 0, nmax = 0, rcap_max = 0;
  int baca_cluster = 1;
  int mr_max = 0, nc_max = 0;
  size_t baca_smem = 0;
  int baca_clusters = 0;  // persistent clusters launched (set at launch time)
  // host descriptor tables, uploaded to ws + desc_region.off
  std::vector<char> desc;
  Region desc_region;
  size_t leafdesc_off = 0, order_off = 0, gparams_off = 0, refs_off = 0;
  int nrefs = 0;
  int nslots = 0;                 // length of the rank array (refs, then full-triplet counts)
  int user_ref_first = 0;         // global ref index of block 0's result
  bool tape = false;              // HBACA_FLAG_TAPE: every node keeps all its singular triplets
  bool frob = false;              // HBACA_FLAG_FROB: Frobenius truncation rule
  int root_tape_first = -1;       // tape: global ref index of block 0's root node
  // device-written tables
  size_t leafout_off = 0, ranks_off = 0;
  // workspace regions
  Region status, queue, uar, var, cscr, rscr, gscr, tape_int, tape_dbl;
  Region full_u, full_s, full_v, half_u, half_s, half_v;
  Region qr, tau, core, ord;
  Region jlist;                   // task index lists of the Jacobi launches (one slot per stage)
  Region xpart, xcnt;             // inter-cluster partial sums (kXSlots x 2 x xplen) and arrival counters
  int xplen = 0;
  int64_t cscr_stride = 0, rscr_stride = 0, gscr_stride = 0;
  int max_clusters_scratch = 0;
  // global ref index of node (a, c) of block b: full store at level l, half store at level l
  std::vector<std::vector<std::vector<int>>> full_idx, half_idx;  // [b][l][a * ncols + c]
  // stages
  std::vector<std::vector<SvdTask>> task_storage;
  std::vector<Stage> stages;
  size_t total = 0;
};

// Validate the arguments and lay out the workspace for `nblocks` matrices
// (one generator each, same kind and dtype).  `sms` is the device's SM count
// (0 when unknown).  Returns false with a message.
bool make_plan(const hbaca_gen* gens, int nblocks, const hbaca_opts& o, int sms, Plan& p, std::string& err);

// Point block b's result entry at the caller's buffers.
void bind_user_result(Plan& p, int b, const hbaca_result& r);

// Levels of a block for opts.levels (>= 0: that L; < 0: leaves of at most
// -levels rows and columns), or -1 when invalid.
int block_levels(int64_t m, int64_t n, int levels);

}  // namespace hbaca
