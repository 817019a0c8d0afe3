// Host-side planning of one H-BACA call: the two L-level index trees
// (Alg. 3 line 1; first child of a node of size s has ceil(s/2) indices),
// the leaf table, the per-level merge tasks and the byte layout of the
// caller's workspace.  Everything here is plain host C++.
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

// One merge (or leaf re-compression) stage: a batch of tasks launched together.
struct Stage {
  int kind;                      // TaskKind
  std::vector<SvdTask>* tasks_h; // host copy (owned by Plan)
  int ntasks = 0;
  size_t tasks_off = 0, dims_off = 0, qrjobs_off = 0, qjobs_off = 0;
  int nqr = 0, nq = 0;
  int kcap = 0;
  int rows_max = 0;
  int in_store = -1, out_store = -1;  // store ids: 0 = full, 1 = half, 2 = user
  int in_level = 0, out_level = 0;    // level index into the BlockRef tables
};

struct StoreLevel {
  size_t refs_off = 0;   // BlockRef array (device)
  size_t rank_off = 0;   // int32 ranks (device)
  int nblocks = 0;
};

struct Plan {
  // inputs
  hbaca_gen gen;
  hbaca_opts opts;
  bool cplx = false;
  size_t esz = 8;
  int L = 0, d = 1;
  int64_t m = 0, n = 0;
  int64_t rank_cap = 0, leaf_cap_opt = 0;
  std::vector<std::vector<Span>> rows, cols;
  // leaves
  int nleaves = 0;
  int mmax = 0, nmax = 0, rcap_max = 0;
  int baca_cluster = 1;
  int mr_max = 0, nc_max = 0;
  size_t baca_smem = 0;
  int baca_clusters = 0;  // persistent clusters launched (set at launch time)
  // host descriptor tables
  std::vector<char> desc;  // staged descriptor bytes, uploaded to ws + desc_region.off
  Region desc_region;
  size_t leafdesc_off = 0, leafout_off = 0;
  // workspace regions
  Region status, queue, uar, var, cscr, rscr, gscr, tape_int, tape_dbl;
  Region full_u, full_s, full_v, half_u, half_s, half_v;
  Region qr, tau, core, ord;
  int64_t cscr_stride = 0, rscr_stride = 0, gscr_stride = 0;
  int max_clusters_scratch = 0;
  // stores: [level] for full (0..L) and half (1..L)
  std::vector<StoreLevel> full_lv, half_lv;
  StoreLevel user_lv;
  size_t user_ref_off = 0;
  // stages
  std::vector<std::vector<SvdTask>> task_storage;
  std::vector<Stage> stages;
  size_t total = 0;
};

// Validate the arguments and lay out the workspace.  `sms` is the SM count of
// the device (0 when only the size is wanted).  Returns false with a message.
bool make_plan(const hbaca_gen& g, const hbaca_opts& o, int sms, Plan& p, std::string& err);

// Fill the descriptor tables that depend on the caller's result buffers.
void bind_user_result(Plan& p, const hbaca_result& r);

}  // namespace hbaca
