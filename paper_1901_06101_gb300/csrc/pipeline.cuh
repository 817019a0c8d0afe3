// Launch sequence of one H-BACA call for scalar type T: the persistent leaf
// BACA kernel, the leaf re-compression stage, then for every level l = 1..L
// the horizontal stage (step l - 1/2) and the vertical stage (step l) of
// Alg. 3.  All launches go to one stream; task sizes live on the device.
#pragma once

#include <string>
#include <vector>

#include "baca.cuh"
#include "dense.cuh"
#include "plan.h"
#include "run.h"

namespace hbaca {

#define HB_TRY(call)                                                              \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      err = std::string(#call) + ": " + cudaGetErrorString(e_);                   \
      return e_;                                                                  \
    }                                                                             \
  } while (0)

constexpr size_t kJacobiSmemLimit = 220 * 1024;  // dynamic shared memory of one Jacobi CTA

// Bracket one launch with profiling events when the call is profiled.
#define HB_TIMED(cls, ...)                                   \
  do {                                                       \
    if (rc.kt) HB_TRY(rc.kt->begin((cls), rc.st));           \
    __VA_ARGS__;                                             \
    if (rc.kt) HB_TRY(rc.kt->end(rc.st));                    \
  } while (0)

template <typename K>
cudaError_t cluster_config(K kern, int grid, int cluster, size_t smem, cudaStream_t st, bool coop,
                           cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int threads = kDenseThreads) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (cluster > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cfg = cudaLaunchConfig_t{};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = coop ? 2 : 1;
  return cudaSuccess;
}

// coop: all CTAs of the grid resident at once (kernels whose clusters wait
// on one another)
template <typename K, typename... Args>
cudaError_t launch_cluster_x(K kern, int grid, int cluster, size_t smem, cudaStream_t st, bool coop, Args... args) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[2];
  cudaError_t e = cluster_config(kern, grid, cluster, smem, st, coop, cfg, attr);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename K, typename... Args>
cudaError_t launch_cluster(K kern, int grid, int cluster, size_t smem, cudaStream_t st, Args... args) {
  return launch_cluster_x(kern, grid, cluster, smem, st, false, args...);
}

// Clusters of `cluster` CTAs with `smem` bytes that can be resident at once.
template <typename K>
int resident_clusters(K kern, int cluster, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[2];
  if (cluster_config(kern, cluster, cluster, smem, st, false, cfg, attr) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

inline int pick_cluster(int jobs, int rows, int sms, int min_rows_per_cta) {
  int c = 1;
  while (c < 16 && (int64_t)jobs * c < 2 * sms && rows / (2 * c) >= min_rows_per_cta) c *= 2;
  return c;
}

// CTAs per matrix of the QR and the Q application: the smallest of 1, 2, 4,
// 8, 12, 16 that gives each CTA at most 420 rows, stepped down while the
// stage would exceed 256 CTAs with more than 4 per matrix (at least 64 rows
// per CTA).  From a sweep of forced sizes on the 20000^2 workload (QR + Q
// application ms per stage, sizes 4 / 8 / 12 / 16): 1250-row matrices of the
// leaf stage (512 of them) 140 / 153 / 218 / 233; 64 merges of 2500 rows 50
// / 56 / 56 / 62; 32 of 2500 rows 33 / 27 / 31 / 31; 16 of 5000 rows 59 / 49
// / 35 / 38; 8 of 5000 rows 55 / 29 / 20 / 26.  A stage that would still
// leave half of the SMs idle is bound by the latency of its column steps and
// takes as many CTAs per matrix as keep 60 rows each (the 2000^2 Gaussian
// workload, QR + Q application ms per stage with 2 / 8 / 16 CTAs: 32 matrices
// of 500 rows 1.45 / 1.13 / 1.23; 8 of 1000 rows 2.21 / 1.17 / 1.06; one of
// 2000 rows 4.27 / 1.50 / 1.22).  Stages of at most four matrices spread
// each over several clusters instead (pick_groups).
inline int pick_qr_cluster(int jobs, int rows, int sms, int min_rows_per_cta) {
  static const int kSizes[] = {1, 2, 4, 8, 12, 16};
  int k = 0;
  while (k < 5 && rows > 420 * kSizes[k]) ++k;
  while (k > 0 && kSizes[k] > 4 && (int64_t)jobs * kSizes[k] > 256) --k;
  if ((int64_t)jobs * kSizes[k] * 2 < sms)
    while (k < 5 && rows / kSizes[k + 1] >= 60) ++k;
  while (k > 0 && rows / kSizes[k] < min_rows_per_cta) --k;
  return kSizes[k];
}

// Clusters per matrix when a stage has too few matrices to fill the machine
// with one 12- or 16-CTA cluster each: 8-CTA clusters, as many per matrix as two
// CTAs per SM, the resident clusters and the exchange slots allow, with at
// least min_rows_per_cta rows per CTA; 1 when that is not more than 16 CTAs.
// (The column steps of such a stage are bound by each CTA's own FP64 work:
// on the 50000-row root of the sparse-product workload QR + Q application
// took 3394 / 1932 / 1405 / 974 / 625 ms with 4 / 8 / 12 / 19 / 37 clusters.
// Each step also waits for every cluster of its matrix, which costs more
// than the rows it saves below about 128 rows per CTA: the 10000- and
// 20000-row top stages of the 20000^2 workload, 132 columns, took 14.9 and
// 15.7 ms with 18 and 37 clusters, 14.35 and 14.95 with 9 and 18.)
inline int pick_groups(int jobs, int rows, int sms, int resident, int min_rows_per_cta) {
  int G = 1;
  while (jobs * (G + 1) <= kXSlots && jobs * (G + 1) * 8 <= 2 * sms && jobs * (G + 1) <= resident &&
         rows / ((G + 1) * 8) >= min_rows_per_cta)
    ++G;
  return G * 8 > 16 ? G : 1;
}

template <typename Gen>
cudaError_t run_baca(Plan& p, const Gen& gen, RunCtx& rc, std::string& err) {
  const NvtxRange range("hbaca leaf BACA (Alg. 2)");
  using T = typename Gen::scalar;
  char* ws = rc.ws;
  BacaParams<Gen> P;
  P.gen = gen;
  P.leaves = reinterpret_cast<const LeafDesc*>(ws + p.desc_region.off + p.leafdesc_off);
  P.order = reinterpret_cast<const int32_t*>(ws + p.desc_region.off + p.order_off);
  P.out = reinterpret_cast<LeafOut*>(ws + p.leafout_off);
  P.nleaves = p.nleaves;
  P.queue = reinterpret_cast<int*>(ws + p.queue.off);
  P.status = reinterpret_cast<int*>(ws + p.status.off);
  P.Uar = reinterpret_cast<T*>(ws + p.uar.off);
  P.Var = reinterpret_cast<T*>(ws + p.var.off);
  P.Cscr = reinterpret_cast<T*>(ws + p.cscr.off);
  P.Rscr = reinterpret_cast<T*>(ws + p.rscr.off);
  P.Gscr = reinterpret_cast<T*>(ws + p.gscr.off);
  P.cscr_stride = p.cscr_stride;
  P.rscr_stride = p.rscr_stride;
  P.gscr_stride = p.gscr_stride;
  P.tape_int = reinterpret_cast<int32_t*>(ws + p.tape_int.off);
  P.tape_dbl = reinterpret_cast<double*>(ws + p.tape_dbl.off);
  P.eps = p.opts.eps;
  P.d = p.d;
  P.seed = p.opts.seed;
  P.mr_max = p.mr_max;
  P.nc_max = p.nc_max;
  P.rcap_max = p.rcap_max;
  P.srrqr_f2 = p.opts.srrqr_f > 0.0 ? p.opts.srrqr_f * p.opts.srrqr_f : 0.0;
  auto kern = baca_leaf_kernel<Gen>;
  const int c = p.baca_cluster;
  HB_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.baca_smem));
  if (c > 8) HB_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c, 1, 1);
  cfg.blockDim = dim3(kBacaThreads, 1, 1);
  cfg.dynamicSmemBytes = p.baca_smem;
  cfg.stream = rc.st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = c;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int ncl = 0;
  HB_TRY(cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg));
  if (ncl < 1) {
    err = "BACA kernel cannot be made resident (cluster " + std::to_string(c) + ", smem " + std::to_string(p.baca_smem) + ")";
    return cudaErrorInvalidConfiguration;
  }
  int nclusters = std::min(std::min(p.nleaves, ncl), p.max_clusters_scratch);
  p.baca_clusters = nclusters;
  cfg.gridDim = dim3(nclusters * c, 1, 1);
  HB_TIMED(KC_BACA, HB_TRY(cudaLaunchKernelEx(&cfg, kern, P)));
  ++rc.launches;
  return cudaSuccess;
}

template <typename T>
cudaError_t run_stage(Plan& p, int si, const Stage& sg, RunCtx& rc, std::string& err) {
  char* ws = rc.ws;
  if (rc.kt) rc.kt->stage = si;
  char* desc = ws + p.desc_region.off;
  DenseParams<T> D;
  D.tasks = reinterpret_cast<const SvdTask*>(desc + sg.tasks_off);
  D.dims = reinterpret_cast<TaskDims*>(ws + sg.dims_off);
  D.ntasks = sg.ntasks;
  D.Uar = reinterpret_cast<T*>(ws + p.uar.off);
  D.Var = reinterpret_cast<T*>(ws + p.var.off);
  D.leaf_rank = reinterpret_cast<const int32_t*>(ws + p.leafout_off);
  D.leaf_rank_stride = (int)(sizeof(LeafOut) / sizeof(int32_t));
  // every block reference and its rank live in one table / one array; the
  // stage's input and output store arenas are the full (0) or half (1) store
  auto arena = [&](int id, T*& U, double*& S, T*& V) {
    if (id == 0) {
      U = reinterpret_cast<T*>(ws + p.full_u.off);
      S = reinterpret_cast<double*>(ws + p.full_s.off);
      V = reinterpret_cast<T*>(ws + p.full_v.off);
    } else if (id == 1) {
      U = reinterpret_cast<T*>(ws + p.half_u.off);
      S = reinterpret_cast<double*>(ws + p.half_s.off);
      V = reinterpret_cast<T*>(ws + p.half_v.off);
    } else {
      U = nullptr;
      S = nullptr;
      V = nullptr;
    }
  };
  const BlockRef* refs = reinterpret_cast<const BlockRef*>(desc + p.refs_off);
  int32_t* ranks = reinterpret_cast<int32_t*>(ws + p.ranks_off);
  D.in_blocks = refs;
  D.in_rank = ranks;
  D.out_blocks = refs;
  D.out_rank = ranks;
  {
    double* in_s = nullptr;
    arena(sg.in_store, D.inU, in_s, D.inV);
    D.inS = in_s;
    arena(sg.out_store, D.outU, D.outS, D.outV);
  }
  D.out_cap = p.rank_cap_max;
  D.qr = reinterpret_cast<T*>(ws + p.qr.off);
  D.tau = reinterpret_cast<T*>(ws + p.tau.off);
  D.core = reinterpret_cast<T*>(ws + p.core.off);
  D.ord = reinterpret_cast<int32_t*>(ws + p.ord.off);
  D.status = reinterpret_cast<int*>(ws + p.status.off);
  D.eps = p.opts.eps;
  const int nt = sg.ntasks;
  const QrJob* qj = reinterpret_cast<const QrJob*>(desc + sg.qrjobs_off);
  const QJob* aj = reinterpret_cast<const QJob*>(desc + sg.qjobs_off);

  HB_TIMED(KC_PACK, pack_kernel<T><<<dim3(64, nt), 256, 0, rc.st>>>(D); HB_TRY(cudaGetLastError()));
  int cq = pick_qr_cluster(sg.nqr, sg.rows_max, rc.sms, 32);
  if (qr_forced_cluster() > 0) cq = qr_forced_cluster();
  const size_t qr_smem = (size_t)(3 * (2 + 2 * sg.kcap) + 4) * sizeof(T);
  const size_t qa_cols = p.tape ? std::max<size_t>((size_t)p.rank_cap_max, (size_t)sg.kcap) : (size_t)p.rank_cap_max;
  const size_t qa_smem = (6 * qa_cols + 3) * sizeof(T) + 64;
  XGroup<T> X{1, cq, sg.nqr, p.xplen, reinterpret_cast<T*>(ws + p.xpart.off),
              reinterpret_cast<unsigned*>(ws + p.xcnt.off)};
  // a stage of large matrices (12 or 16 CTAs each) too few to fill the SMs
  // spreads each over several clusters (the 8 matrices of 5000 rows of the
  // 20000^2 workload: QR + Q application 21.8 -> 15.9 ms with 4 clusters each)
  if (rc.xgroups && qr_forced_cluster() == 0 && cq >= 12 && sg.nqr == sg.nq && sg.nqr * 16 < rc.sms) {
    const int res = std::min(resident_clusters(qr_kernel<T>, 8, qr_smem, rc.st),
                             resident_clusters(qapply_kernel<T>, 8, qa_smem, rc.st));
    int G = pick_groups(sg.nqr, sg.rows_max, rc.sms, res, 128);
    if (qr_forced_groups() > 0 && G > qr_forced_groups()) G = qr_forced_groups() * 8 > 16 ? qr_forced_groups() : 1;
    if (G > 1) {
      cq = 8;
      X.G = G;
      X.csize = cq;
    }
  }
  const bool coop = X.G > 1;
  if (coop) HB_TRY(cudaMemsetAsync(X.xcnt, 0, kXSlots * sizeof(unsigned), rc.st));
  HB_TIMED(KC_QR, HB_TRY(launch_cluster_x(qr_kernel<T>, sg.nqr * X.G * cq, cq, qr_smem, rc.st, coop, D, qj, X)));
  HB_TIMED(KC_CORE, core_kernel<T><<<dim3(16, nt), 256, 0, rc.st>>>(D); HB_TRY(cudaGetLastError()));
  // pivoted QR of the cores: up to 8 CTAs per core while the stage leaves SMs idle
  const size_t qc_smem = (size_t)sg.kcap * (sizeof(T) + 8 + 4 + 1) + 2 * sizeof(T) + 2 * sizeof(QcArg) + 32 * 12 +
                         16 + 64;
  int cqc = 1;
  while (cqc < 8 && nt * cqc * 2 <= rc.sms) cqc *= 2;
  {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    HB_TRY(cluster_config(qrcp_core_kernel<T>, nt * cqc, cqc, qc_smem, rc.st, false, cfg, attr, kWideThreads));
    HB_TIMED(KC_QRCP, HB_TRY(cudaLaunchKernelEx(&cfg, qrcp_core_kernel<T>, D)));
  }
  // a stage's Jacobi launches: the largest (by CTAs) on the call's stream, the
  // others concurrently on the auxiliary stream (fork after the task lists
  // are in place, join before the next kernel)
  const JGroup jg1{1, nullptr, nullptr};
  auto jacobi_group_launches = [&](const std::vector<JacobiLaunch>& all) -> cudaError_t {
    std::vector<JacobiLaunch> ls, grouped;
    for (const JacobiLaunch& jl : all) (jl.groups > 1 ? grouped : ls).push_back(jl);
    size_t main_i = 0;
    for (size_t i = 1; i < ls.size(); ++i)
      if ((int64_t)ls[i].count * ls[i].cluster > (int64_t)ls[main_i].count * ls[main_i].cluster) main_i = i;
    const bool fork = rc.aux && rc.fork_ev && rc.join_ev && ls.size() > 1;
    if (fork) {
      HB_TRY(cudaEventRecord(rc.fork_ev, rc.st));
      HB_TRY(cudaStreamWaitEvent(rc.aux, rc.fork_ev, 0));
    }
    rc.launches += (int)ls.size();
    for (size_t i = 0; i < ls.size(); ++i) {
      const JacobiLaunch& jl = ls[i];
      cudaStream_t s2 = (fork && i != main_i) ? rc.aux : rc.st;
      const int32_t* lst = reinterpret_cast<const int32_t*>(ws + p.jlist.off) + jl.list_off;
      if (rc.kt) HB_TRY(rc.kt->begin(KC_JACOBI, s2));
      HB_TRY(launch_cluster(jacobi_kernel<T>, jl.count * jl.cluster, jl.cluster, jl.hdr + jl.dsm, s2, D, jacobi_max_sweeps(), (int)jl.hdr,
                            (int)jl.base, (int64_t)jl.dsm, lst, jg1));
      if (rc.kt) HB_TRY(rc.kt->end(s2));
    }
    if (fork) {
      HB_TRY(cudaEventRecord(rc.join_ev, rc.aux));
      HB_TRY(cudaStreamWaitEvent(rc.st, rc.join_ev, 0));
    }
    // cores swept by several clusters: a cooperative launch on the call's
    // stream after the others (arrival counters zeroed first)
    for (const JacobiLaunch& jl : grouped) {
      const int32_t* lst = reinterpret_cast<const int32_t*>(ws + p.jlist.off) + jl.list_off;
      const JGroup jg{jl.groups, X.xcnt, reinterpret_cast<double*>(X.xpart)};
      ++rc.launches;
      HB_TRY(cudaMemsetAsync(X.xcnt, 0, kXSlots * sizeof(unsigned), rc.st));
      if (rc.kt) HB_TRY(rc.kt->begin(KC_JACOBI, rc.st));
      HB_TRY(launch_cluster_x(jacobi_kernel<T>, jl.count * jl.groups * jl.cluster, jl.cluster, jl.hdr, rc.st, true, D,
                              jacobi_max_sweeps(), (int)jl.hdr, (int)jl.base, (int64_t)0, lst, jg));
      if (rc.kt) HB_TRY(rc.kt->end(rc.st));
    }
    return cudaSuccess;
  };
  if (rc.replay) {
    // captured call: the launch shapes a synchronous call chose (task lists
    // already in the workspace); kernels still check every task's sizes
    std::vector<JacobiLaunch> ls;
    for (const JacobiLaunch& jl : *rc.replay)
      if (jl.stage == si) ls.push_back(jl);
    HB_TRY(jacobi_group_launches(ls));
  } else if (rc.sizes_known) {
    // the cores' sizes are known: group the tasks by the cluster size that
    // gives each warp about one pair per round, with exactly the shared memory
    // the group's largest core needs (columns in distributed shared memory
    // when they fit 16 CTAs; otherwise the sweeps run in global memory)
    std::vector<TaskDims> dh(nt);
    HB_TRY(cudaMemcpyAsync(dh.data(), ws + sg.dims_off, (size_t)nt * sizeof(TaskDims), cudaMemcpyDeviceToHost, rc.st));
    HB_TRY(cudaStreamSynchronize(rc.st));
    const size_t j_base = (16 + (size_t)sg.kcap * 12 + 64 + 15) & ~(size_t)15;
    // pair slots: (pairs of a round per CTA, rounded up to whole passes over its warps)
    auto j_hdr_of = [&](int cc) {
      const size_t pairs = ((size_t)sg.kcap + 1) / 2;
      const size_t per_cta = (pairs + (size_t)cc * 8 - 1) / ((size_t)cc * 8) * 8;
      return j_base + per_cta * kJSlotMax;
    };
    // cluster size: about three resident CTAs per SM in all (a stage with
    // many cores is bound by the FP64 rate and takes 4-CTA clusters; one with
    // few cores by the latency of its rounds and spreads each core over up to
    // 16 CTAs), at least four pairs of a round per CTA (one per scheduler of
    // its SM), raised where a core's columns do not fit that many CTAs'
    // shared memory.  Measured on the 20000^2 workload: 4 CTAs for the 256,
    // 128 and 64 cores of the leaf and first merge stages, 8 for 32 cores, 16
    // for 16 or fewer (cluster sizes do not change any result).
    std::vector<std::vector<int32_t>> groups(17);
    std::vector<size_t> need(17, 0);
    const std::vector<SvdTask>& th = *sg.tasks_h;
    auto share_of = [&](int i, int cc) {
      const int ncm = th[i].kind == TASK_LEAF ? dh[i].krb : dh[i].k;
      const int nc = std::min(dh[i].kra, ncm), mr = ncm;
      // a column's slot: X (mr rows), its squared norm, and W (nc rows) when
      // the call is taped
      return (size_t)((nc + cc - 1) / cc) * (size_t)(mr + 1 + (p.tape ? nc : 0)) * sizeof(T);
    };
    auto fit = [&](int i, int cc) {
      while (cc < 16 && share_of(i, cc) + j_hdr_of(cc) > kJacobiSmemLimit) ++cc;
      return cc;
    };
    auto add_task = [&](int i, int cc) {
      groups[cc].push_back(i);
      const size_t sh = share_of(i, cc) + j_hdr_of(cc) <= kJacobiSmemLimit ? share_of(i, cc) : 0;
      need[cc] = std::max(need[cc], sh);
    };
    int c_stage = 4;
    while (c_stage < 16 && (int64_t)nt * c_stage * 2 <= 3 * (int64_t)rc.sms) c_stage *= 2;
    // cores whose columns do not fit 16 CTAs' shared memory and have at least
    // 256 pairs a round: swept by several 16-CTA clusters at once
    std::vector<int32_t> huge;
    int huge_pairs = 0;
    for (int i = 0; i < nt; ++i) {
      const int ncm = th[i].kind == TASK_LEAF ? dh[i].krb : dh[i].k;
      const int pairs = (std::min(dh[i].kra, ncm) + 1) / 2;
      int c = c_stage;
      while (c > 1 && pairs < 4 * c) c /= 2;
      if (jacobi_forced_cluster() > 0) c = jacobi_forced_cluster();
      c = fit(i, c);
      if (rc.xgroups && jacobi_forced_groups() != 1 && c == 16 && pairs >= 256 &&
          share_of(i, 16) + j_hdr_of(16) > kJacobiSmemLimit) {
        huge.push_back(i);
        huge_pairs = std::max(huge_pairs, pairs);
      } else {
        add_task(i, c);
      }
    }
    int G = 1;
    if (!huge.empty()) {
      // every cluster of the cooperative launch resident, one arrival counter
      // per core, about one pair per warp and round
      const int nh = (int)huge.size();
      const int res = resident_clusters(jacobi_kernel<T>, 16, j_hdr_of(16), rc.st);
      const int cap = std::min(res / nh, kXSlots / nh);
      G = std::min(cap, (huge_pairs + 16 * 8 - 1) / (16 * 8));
      if (jacobi_forced_groups() > 1) G = std::min(cap, jacobi_forced_groups());
      if (G < 2) {
        for (int i : huge) add_task(i, 16);
        huge.clear();
      }
    }
    size_t off = sg.jlist_off;
    std::vector<JacobiLaunch> ls;
    for (int g = 1; g <= 16; ++g) {
      if (groups[g].empty()) continue;
      int32_t* lst = reinterpret_cast<int32_t*>(ws + p.jlist.off) + off;
      HB_TRY(cudaMemcpyAsync(lst, groups[g].data(), groups[g].size() * 4, cudaMemcpyHostToDevice, rc.st));
      ls.push_back(JacobiLaunch{si, g, (int)groups[g].size(), j_hdr_of(g), j_base, need[g], off});
      off += groups[g].size();
    }
    if (!huge.empty()) {
      int32_t* lst = reinterpret_cast<int32_t*>(ws + p.jlist.off) + off;
      HB_TRY(cudaMemcpyAsync(lst, huge.data(), huge.size() * 4, cudaMemcpyHostToDevice, rc.st));
      ls.push_back(JacobiLaunch{si, 16, (int)huge.size(), j_hdr_of(16), j_base, 0, off, G});
      off += huge.size();
    }
    HB_TRY(jacobi_group_launches(ls));
    if (rc.record) rc.record->insert(rc.record->end(), ls.begin(), ls.end());
  } else {
    const int cj = pick_cluster(nt, sg.kcap, rc.sms, 16);
    // header (flags, singular values, order, pair slots) then, up to the
    // shared-memory limit, room for a task's columns of X and W (used when
    // they fit)
    const size_t j_base = (16 + (size_t)sg.kcap * 12 + 64 + 15) & ~(size_t)15;
    const size_t j_hdr = j_base + (((size_t)sg.kcap + 1) / 2 + (size_t)cj * 8 - 1) / ((size_t)cj * 8) * 8 * kJSlotMax;
    const size_t j_cap = ((size_t)sg.kcap + cj - 1) / cj * (2 * (size_t)sg.kcap + 1) * sizeof(T);
    const size_t j_dsm = std::min(j_cap, (size_t)kJacobiSmemLimit - j_hdr);
    HB_TIMED(KC_JACOBI, HB_TRY(launch_cluster(jacobi_kernel<T>, nt * cj, cj, j_hdr + j_dsm, rc.st, D, jacobi_max_sweeps(), (int)j_hdr,
                                              (int)j_base, (int64_t)j_dsm, (const int32_t*)nullptr, jg1)));
    ++rc.launches;
  }
  if (!p.tape) {
    // a cluster per task (rows of the Gram-Schmidt pass split over it) while
    // the stage has fewer tasks than SMs
    int cw = 1;
    while (cw < 16 && (int64_t)nt * cw * 2 <= rc.sms) cw *= 2;
    const int wcols = p.tape ? sg.kcap : (int)std::min<int64_t>(sg.kcap, p.rank_cap_max);
    const size_t ws_smem = (size_t)3 * std::min(wcols, kMaxWsolveCols) * sizeof(T) + 34 * sizeof(double);
    HB_TIMED(KC_FINISH, HB_TRY(launch_cluster(wsolve_kernel<T>, nt * cw, cw, ws_smem, rc.st, D)));
    ++rc.launches;
  }
  {
    // one warp per output column of every task: enough CTAs for the widest
    // output, within about eight CTAs per SM over the stage
    const int cols = p.tape ? sg.kcap : (int)std::min<int64_t>(sg.kcap, p.rank_cap_max);
    const int gx = std::max(8, std::min((cols + 7) / 8, std::max(8, 8 * rc.sms / std::max(nt, 1))));
    HB_TIMED(KC_FINISH, finish_kernel<T><<<dim3(gx, nt), 256, 0, rc.st>>>(D); HB_TRY(cudaGetLastError()));
  }
  ++rc.launches;
  X.njobs = sg.nq;
  // the block-diagonal side of a merge needs only the core's right (or left)
  // vectors, not the Q application: it runs on the auxiliary stream beside it
  // (fork after finish, join at the end of the stage)
  const bool side = sg.kind != TASK_LEAF && rc.aux && rc.fork_ev && rc.join_ev;
  if (side) {
    HB_TRY(cudaEventRecord(rc.fork_ev, rc.st));
    HB_TRY(cudaStreamWaitEvent(rc.aux, rc.fork_ev, 0));
  }
  if (coop) HB_TRY(cudaMemsetAsync(X.xcnt, 0, kXSlots * sizeof(unsigned), rc.st));
  HB_TIMED(KC_QAPPLY, HB_TRY(launch_cluster_x(qapply_kernel<T>, sg.nq * X.G * cq, cq, qa_smem, rc.st, coop, D, aj, X)));
  rc.launches += 5;  // pack, QR, core, pivoted QR of the core, Q application
  if (sg.kind != TASK_LEAF) {
    // element-parallel; a stage with few (large) tasks spreads each over more CTAs
    const int gx = std::max(64, std::min(1024, 8 * rc.sms / std::max(nt, 1)));
    cudaStream_t s2 = side ? rc.aux : rc.st;
    if (rc.kt) HB_TRY(rc.kt->begin(KC_BLOCKPROD, s2));
    blockprod_kernel<T><<<dim3(gx, nt), 256, 0, s2>>>(D);
    HB_TRY(cudaGetLastError());
    if (rc.kt) HB_TRY(rc.kt->end(s2));
    ++rc.launches;
    if (side) {
      HB_TRY(cudaEventRecord(rc.join_ev, rc.aux));
      HB_TRY(cudaStreamWaitEvent(rc.st, rc.join_ev, 0));
    }
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t run_stages(Plan& p, RunCtx& rc, std::string& err) {
  if (rc.ev[1]) HB_TRY(cudaEventRecord(rc.ev[1], rc.st));  // leaf BACA done
  for (size_t i = 0; i < p.stages.size(); ++i) {
    const Stage& sg = p.stages[i];
    const NvtxRange range(std::string("hbaca stage ") + std::to_string(i) +
                          (sg.kind == TASK_LEAF ? " leaf re-compression" : sg.kind == TASK_HORIZ ? " horizontal merge"
                                                                                                 : " vertical merge") +
                          " (" + std::to_string(sg.ntasks) + " tasks)");
    if (rc.ev[2] && sg.kind != TASK_LEAF && (i == 0 || p.stages[i - 1].kind == TASK_LEAF))
      HB_TRY(cudaEventRecord(rc.ev[2], rc.st));  // leaf re-compression done
    cudaError_t e = run_stage<T>(p, (int)i, sg, rc, err);
    if (e != cudaSuccess) return e;
  }
  if (rc.ev[2] && (p.stages.empty() || p.stages.back().kind == TASK_LEAF)) HB_TRY(cudaEventRecord(rc.ev[2], rc.st));
  if (p.tape) {
    char* ws = rc.ws;
    HB_TIMED(KC_COPYROOT, copyroot_kernel<T><<<dim3(64, p.nblocks), 256, 0, rc.st>>>(
                              reinterpret_cast<const BlockRef*>(ws + p.desc_region.off + p.refs_off),
                              reinterpret_cast<int32_t*>(ws + p.ranks_off), reinterpret_cast<const T*>(ws + p.full_u.off),
                              reinterpret_cast<const double*>(ws + p.full_s.off),
                              reinterpret_cast<const T*>(ws + p.full_v.off), p.root_tape_first, p.user_ref_first);
             HB_TRY(cudaGetLastError()));
    ++rc.launches;
  }
  return cudaSuccess;
}

}  // namespace hbaca
