// Entry points of the two scalar-type translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>
#include <utility>
#include <vector>

#include "plan.h"

namespace hbaca {

// A named range on the host timeline (NVTX) around a call or a phase, for
// timeline and profiling tools (ncu --nvtx); it costs nothing measurable when
// no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  explicit NvtxRange(const std::string& name) { nvtxRangePushA(name.c_str()); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Kernel classes timed under HBACA_FLAG_PROFILE (hbaca_kernel_times).
enum KernelClass {
  KC_BACA = 0, KC_PACK, KC_QR, KC_CORE, KC_QRCP, KC_JACOBI, KC_FINISH, KC_QAPPLY, KC_BLOCKPROD, KC_COPYROOT,
  KC_COUNT
};

// Event pairs around every launch of a profiled call; events are created on
// first use and reused by later calls of the same context.
struct KernelTimer {
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, size_t>> marks;  // (class, index of the start event; the stop is next)
  std::vector<int> mark_stage;                // stage of each mark (-1: the leaf BACA launch)
  int stage = -1;                             // stage whose launches are being recorded
  size_t used = 0;
  void reset() { marks.clear(); mark_stage.clear(); stage = -1; used = 0; }
  cudaError_t record(cudaStream_t st) {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      pool.push_back(e);
    }
    return cudaEventRecord(pool[used++], st);
  }
  cudaError_t begin(int cls, cudaStream_t st) {
    marks.emplace_back(cls, used);
    mark_stage.push_back(stage);
    return record(st);
  }
  cudaError_t end(cudaStream_t st) { return record(st); }
  ~KernelTimer() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

// Launch shape of one Jacobi launch of a stage, as sized by a synchronous call
// (replayed when the call is captured into a CUDA graph).
struct JacobiLaunch {
  int stage, cluster, count;
  size_t hdr, base, dsm, list_off;
  int groups = 1;  // clusters per core (> 1: a cooperative launch, columns in global memory)
};

struct RunCtx {
  char* ws;
  cudaStream_t st;
  int sms;
  const hbaca_result* res;
  int launches = 0;  // kernels launched by the call
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // profile: after BACA, after leaf stage, end
  KernelTimer* kt = nullptr;                                   // profile: per-launch events
  bool sizes_known = false;  // the call may synchronise between stages to size launches by the actual ranks
  std::vector<JacobiLaunch>* record = nullptr;       // sized launches are appended here
  const std::vector<JacobiLaunch>* replay = nullptr;  // capture: launch these shapes, no host sync
  bool baca_only = false;                             // autotuning: the leaf BACA launch alone
  bool xgroups = true;  // QR / Q application may spread a matrix over several clusters
  // auxiliary stream and fork / join events: a stage's smaller Jacobi launch
  // groups run on `aux` concurrently with its largest one (null: one stream)
  cudaStream_t aux = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
};
cudaError_t run_f64(Plan& p, RunCtx& rc, std::string& err);
cudaError_t run_c128(Plan& p, RunCtx& rc, std::string& err);
// Set the calling thread's hbaca_last_error() message; returns s.
hbaca_status record_error(hbaca_status s, const std::string& msg);
// Device ordinal a context was created on.
int ctx_device(const hbaca_ctx* ctx);
// Sweep cap of the one-sided Jacobi SVD launches (hbaca_debug_set_jacobi_sweeps).
int jacobi_max_sweeps();
// Jacobi cluster size forced on every core of a synchronous call (0: chosen
// per stage; hbaca_debug_set_jacobi_cluster).
int jacobi_forced_cluster();
// CTAs per matrix of the QR and Q-application launches forced by
// hbaca_debug_set_qr_cluster (0: the per-stage choice).
int qr_forced_cluster();
// Clusters per core of the Jacobi SVD of cores too large for one cluster's
// shared memory, forced by hbaca_debug_set_jacobi_groups (0: the per-stage
// choice; 1: never more than one).
int jacobi_forced_groups();
// Largest number of 8-CTA clusters per matrix of the QR and Q application of
// stages with few matrices, forced by hbaca_debug_set_qr_groups (0: the
// per-stage choice).
int qr_forced_groups();
}  // namespace hbaca
