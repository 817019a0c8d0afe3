// C ABI of libhbaca (include/hbaca.h): argument checks, planning, launches,
// device status mapping.  No exception crosses this boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>
#include <vector>

#include "hbaca.h"
#include "hbaca_debug.h"
#include "plan.h"
#include "run.h"
#include "types.h"

struct hbaca_ctx {
  int device;
  int sms;
  cudaEvent_t ev[4];
  bool have_times;
  int launches;
  hbaca::KernelTimer kt;
  // HBACA_FLAG_GRAPH: the last captured call, its plan and what identifies it
  // (the raw call arguments)
  cudaGraphExec_t gexec;
  std::vector<char> gkey;
  hbaca::Plan gplan;
  cudaStream_t cap_stream;  // captures run on this stream (the legacy default stream cannot be captured)
  // concurrent Jacobi launch groups of one stage (created on first use)
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
};

namespace {

thread_local std::string tls_err;

// A taped call leaves this byte pattern in the status region (after the
// status word); hbaca_apply_backward refuses a workspace without it.
constexpr size_t kTapeMarkOffset = 16;
constexpr int kTapeMarkByte = 0x5A;

hbaca_status fail(hbaca_status s, const std::string& m) {
  tls_err = m;
  return s;
}

int current_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 152; }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) { cudaGetLastError(); return 152; }
  return sms > 0 ? sms : 152;
}

// The auxiliary stream and its fork / join events (created once per context).
cudaError_t ensure_aux(hbaca_ctx* ctx) {
  cudaError_t e = cudaSuccess;
  if (!ctx->aux_stream) e = cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && !ctx->fork_ev) e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming);
  if (e == cudaSuccess && !ctx->join_ev) e = cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming);
  return e;
}

void use_aux(hbaca_ctx* ctx, hbaca::RunCtx& rc) {
  rc.aux = ctx->aux_stream;
  rc.fork_ev = ctx->fork_ev;
  rc.join_ev = ctx->join_ev;
}

hbaca_status map_device_status(int ds) {
  switch (ds) {
    case 0: return HBACA_OK;
    case 2: return HBACA_RANK_CAPACITY;
    case 4: return HBACA_TIMEOUT;
    case 6: return HBACA_NUMERICAL;
    case 10: return HBACA_NOT_CONVERGED;
    default: return HBACA_CUDA;
  }
}

constexpr int kDefaultJacobiSweeps = 40;
std::atomic<int> g_jacobi_sweeps{kDefaultJacobiSweeps};
std::atomic<int> g_jacobi_cluster{0};
std::atomic<int> g_qr_cluster{0};
std::atomic<int> g_jacobi_groups{0};
std::atomic<int> g_qr_groups{0};

}  // namespace

namespace hbaca {
hbaca_status record_error(hbaca_status s, const std::string& msg) { return fail(s, msg); }
int ctx_device(const hbaca_ctx* ctx) { return ctx->device; }
int jacobi_max_sweeps() { return g_jacobi_sweeps.load(std::memory_order_relaxed); }
int jacobi_forced_cluster() { return g_jacobi_cluster.load(std::memory_order_relaxed); }
int qr_forced_cluster() { return g_qr_cluster.load(std::memory_order_relaxed); }
int jacobi_forced_groups() { return g_jacobi_groups.load(std::memory_order_relaxed); }
int qr_forced_groups() { return g_qr_groups.load(std::memory_order_relaxed); }
}  // namespace hbaca

extern "C" {

const char* hbaca_version(void) { return "hbaca-gb300 0.1 (sm_103a)"; }

const char* hbaca_last_error(void) { return tls_err.c_str(); }

hbaca_status hbaca_create(hbaca_ctx** ctx) {
  if (!ctx) return fail(HBACA_INVALID_ARG, "ctx is NULL");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(HBACA_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  int major = 0, minor = 0, sms = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (major * 10 + minor != 103)
    return fail(HBACA_CUDA, "libhbaca is built for sm_103a (GB300); device is sm_" + std::to_string(major * 10 + minor));
  hbaca_ctx* c = new (std::nothrow)
      hbaca_ctx{dev, sms, {nullptr, nullptr, nullptr, nullptr}, false, 0, {}, nullptr, {}, {}, nullptr, nullptr, nullptr,
                nullptr};
  if (!c) return fail(HBACA_INVALID_ARG, "out of host memory");
  for (int i = 0; i < 4; ++i) {
    e = cudaEventCreate(&c->ev[i]);
    if (e != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaEventDestroy(c->ev[j]);
      delete c;
      return fail(HBACA_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
    }
  }
  *ctx = c;
  tls_err.clear();
  return HBACA_OK;
}

hbaca_status hbaca_destroy(hbaca_ctx* ctx) {
  if (ctx) {
    for (int i = 0; i < 4; ++i)
      if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
  }
  delete ctx;
  return HBACA_OK;
}

size_t hbaca_workspace_size(const hbaca_gen* gen, const hbaca_opts* opts) {
  return hbaca_workspace_size_batched(1, gen, opts);
}

size_t hbaca_workspace_size_batched(int32_t nblocks, const hbaca_gen* gens, const hbaca_opts* opts) {
  if (!gens || !opts || nblocks < 1) { tls_err = "gens or opts is NULL, or nblocks < 1"; return 0; }
  hbaca::Plan p;
  std::string err;
  if (!hbaca::make_plan(gens, nblocks, *opts, current_sms(), p, err)) { tls_err = err; return 0; }
  return p.total;
}

static hbaca_status compress_blocks(hbaca_ctx* ctx, int32_t nblocks, const hbaca_gen* gens, const hbaca_opts* opts,
                                    hbaca_result* outs, void* workspace, void* stream) {
  if (!ctx || !gens || !opts || !outs || nblocks < 1) return fail(HBACA_INVALID_ARG, "NULL ctx, gens, opts or results");
  const hbaca::NvtxRange range(nblocks > 1 ? "hbaca_compress_batched" : "hbaca_compress");
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return fail(HBACA_WORKSPACE, "workspace must be a non-NULL, 256-byte aligned device pointer");
  for (int b = 0; b < nblocks; ++b) {
    if (!outs[b].U || !outs[b].S || !outs[b].V) return fail(HBACA_INVALID_ARG, "result U, S and V must be set");
    if (outs[b].ldu < gens[b].m || outs[b].ldv < gens[b].n)
      return fail(HBACA_INVALID_ARG, "result needs ldu >= m and ldv >= n");
  }
  {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
      cudaGetLastError();
      return fail(HBACA_CUDA, "cudaGetDevice failed");
    }
    if (cur != ctx->device)
      return fail(HBACA_INVALID_ARG, "the current device (" + std::to_string(cur) + ") is not the context's (" +
                                         std::to_string(ctx->device) + ")");
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = reinterpret_cast<char*>(workspace);
  const bool graph = (opts->flags & HBACA_FLAG_GRAPH) != 0;
  std::vector<char> key;
  if (graph) {  // a captured call is identified by its raw arguments
    auto add = [&](const void* ptr, size_t bytes) {
      const char* c = reinterpret_cast<const char*>(ptr);
      key.insert(key.end(), c, c + bytes);
    };
    add(&nblocks, sizeof(nblocks));
    add(gens, sizeof(hbaca_gen) * (size_t)nblocks);
    add(opts, sizeof(hbaca_opts));
    for (int b = 0; b < nblocks; ++b) {
      add(&outs[b].U, sizeof(void*));
      add(&outs[b].ldu, sizeof(int64_t));
      add(&outs[b].S, sizeof(void*));
      add(&outs[b].V, sizeof(void*));
      add(&outs[b].ldv, sizeof(int64_t));
    }
    add(&workspace, sizeof(workspace));
  }
  const bool replay = graph && ctx->gexec && key == ctx->gkey;
  hbaca::Plan fresh;
  std::string err;
  if (!replay) {
    if (!hbaca::make_plan(gens, nblocks, *opts, ctx->sms, fresh, err)) return fail(HBACA_INVALID_ARG, err);
    for (int b = 0; b < nblocks; ++b) hbaca::bind_user_result(fresh, b, outs[b]);
  }
  hbaca::Plan& p = replay ? ctx->gplan : fresh;
  cudaError_t e = cudaSuccess;
  ctx->have_times = false;
  if (replay) {
    e = cudaGraphLaunch(ctx->gexec, st);
    if (e != cudaSuccess) return fail(HBACA_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
    ctx->launches = 0;
  } else {
    hbaca::RunCtx rc{ws, st, ctx->sms, &outs[0], 0};
    rc.xgroups = (opts->flags & HBACA_FLAG_SINGLE_CLUSTER) == 0;
    rc.sizes_known = (opts->flags & HBACA_FLAG_ASYNC) == 0;
    e = ensure_aux(ctx);
    if (e != cudaSuccess) return fail(HBACA_CUDA, std::string("auxiliary stream: ") + cudaGetErrorString(e));
    use_aux(ctx, rc);
    std::vector<hbaca::JacobiLaunch> recipe;
    if (graph) rc.record = &recipe;
    const bool prof = (opts->flags & HBACA_FLAG_PROFILE) != 0 && !graph;
    if (prof) {
      for (int i = 0; i < 4; ++i) rc.ev[i] = ctx->ev[i];
      ctx->kt.reset();
      rc.kt = &ctx->kt;
      cudaError_t pe = cudaEventRecord(ctx->ev[0], st);
      if (pe != cudaSuccess) return fail(HBACA_CUDA, std::string("cudaEventRecord: ") + cudaGetErrorString(pe));
    }
    // status word and leaf work counter live in separate 256-byte regions
    auto reset = [&](cudaStream_t sx) {
      cudaError_t r = cudaMemsetAsync(ws + p.status.off, 0, p.status.bytes, sx);
      if (r == cudaSuccess) r = cudaMemsetAsync(ws + p.queue.off, 0, p.queue.bytes, sx);
      if (r == cudaSuccess) r = cudaMemsetAsync(ws + p.ranks_off, 0, (size_t)p.nslots * 4, sx);
      return r;
    };
    e = reset(st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ws + p.desc_region.off, p.desc.data(), p.desc.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(HBACA_CUDA, std::string("workspace set-up: ") + cudaGetErrorString(e));
    e = p.cplx ? hbaca::run_c128(p, rc, err) : hbaca::run_f64(p, rc, err);
    if (e != cudaSuccess) return fail(HBACA_CUDA, err.empty() ? cudaGetErrorString(e) : err);
    ctx->launches = rc.launches;
    if (p.tape) {  // mark the workspace as holding a complete tape of this call
      e = cudaMemsetAsync(ws + p.status.off + kTapeMarkOffset, kTapeMarkByte, 4, st);
      if (e != cudaSuccess) return fail(HBACA_CUDA, std::string("tape mark: ") + cudaGetErrorString(e));
    }
    if (prof) {
      e = cudaEventRecord(ctx->ev[3], st);
      if (e != cudaSuccess) return fail(HBACA_CUDA, std::string("cudaEventRecord: ") + cudaGetErrorString(e));
      ctx->have_times = true;
    }
    if (graph) {
      // capture the same call with the recorded launch shapes: resets, the
      // persistent leaf kernel, every stage; no host synchronisation inside
      if (!ctx->cap_stream) {
        e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(HBACA_CUDA, std::string("capture stream: ") + cudaGetErrorString(e));
      }
      cudaStream_t cs = ctx->cap_stream;
      hbaca::RunCtx rg{ws, cs, ctx->sms, &outs[0], 0};
      rg.xgroups = (opts->flags & HBACA_FLAG_SINGLE_CLUSTER) == 0;
      use_aux(ctx, rg);
      rg.replay = &recipe;
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        std::string gerr;
        cudaError_t ce = reset(cs);
        if (ce == cudaSuccess) ce = p.cplx ? hbaca::run_c128(p, rg, gerr) : hbaca::run_f64(p, rg, gerr);
        if (ce == cudaSuccess && p.tape) ce = cudaMemsetAsync(ws + p.status.off + kTapeMarkOffset, kTapeMarkByte, 4, cs);
        e = cudaStreamEndCapture(cs, &g);
        if (ce != cudaSuccess) e = ce;
      }
      cudaGraphExec_t ex = nullptr;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HBACA_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      }
      if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
      ctx->gexec = ex;
      ctx->gkey.swap(key);
      ctx->gplan = fresh;  // a copy: this call still reads its ranks through `p`
      // the stages' host task tables point into the plan's own storage
      for (size_t i = 0; i < ctx->gplan.stages.size(); ++i) ctx->gplan.stages[i].tasks_h = &ctx->gplan.task_storage[i];
    }
  }
  const int32_t* d_ranks = reinterpret_cast<const int32_t*>(ws + p.ranks_off) + p.user_ref_first;
  for (int b = 0; b < nblocks; ++b) {
    outs[b].rank = -1;
    if (outs[b].d_rank) {
      e = cudaMemcpyAsync(outs[b].d_rank, d_ranks + b, 4, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return fail(HBACA_CUDA, std::string("rank copy: ") + cudaGetErrorString(e));
    }
  }
  if (opts->flags & HBACA_FLAG_ASYNC) {
    tls_err.clear();
    return HBACA_OK;
  }
  int status = 0;
  std::vector<int32_t> ranks(nblocks);
  std::vector<hbaca::LeafOut> lo(p.nleaves);
  e = cudaMemcpyAsync(&status, ws + p.status.off, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ranks.data(), d_ranks, (size_t)nblocks * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(lo.data(), ws + p.leafout_off, lo.size() * sizeof(hbaca::LeafOut), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(HBACA_CUDA, std::string("kernel execution: ") + cudaGetErrorString(e));
  for (int b = 0; b < nblocks; ++b) {
    int rmax = 0, imax = 0;
    const int nl = 1 << (2 * p.Lb[b]);
    for (int i = 0; i < nl; ++i) {
      rmax = std::max(rmax, lo[p.leaf_first[b] + i].rank);
      imax = std::max(imax, lo[p.leaf_first[b] + i].iters);
    }
    outs[b].rank = ranks[b];
    outs[b].leaf_rank_max = rmax;
    outs[b].leaf_iters_max = imax;
  }
  hbaca_status hs = map_device_status(status);
  if (hs != HBACA_OK) {
    const char* what = hs == HBACA_RANK_CAPACITY ? "a rank exceeded rank_cap or leaf_rank_cap"
                       : hs == HBACA_NUMERICAL   ? "NaN or Inf in a norm or a singular value"
                       : hs == HBACA_TIMEOUT     ? "the clusters of a QR / Q application did not meet within 4 s "
                                                   "(not resident together; HBACA_FLAG_SINGLE_CLUSTER avoids the wait)"
                       : hs == HBACA_NOT_CONVERGED ? "a Jacobi SVD of a re-compression or merge core reached its "
                                                     "sweep cap while still rotating"
                       : status == 8             ? "a QR / Q-application kernel ran with another launch shape than "
                                                   "planned (nothing was touched)"
                                                 : "device-side failure";
    return fail(hs, what);
  }
  tls_err.clear();
  return HBACA_OK;
}

hbaca_status hbaca_autotune_batched(hbaca_ctx* ctx, int32_t nblocks, const hbaca_gen* gens, const hbaca_opts* opts,
                                    void* workspace, size_t workspace_bytes, void* stream, int32_t* best_cluster,
                                    double* best_ms) {
  if (!ctx || !gens || !opts || !workspace || !best_cluster || nblocks < 1) return fail(HBACA_INVALID_ARG, "NULL argument");
  if (reinterpret_cast<uintptr_t>(workspace) & 255u) return fail(HBACA_WORKSPACE, "workspace must be 256-byte aligned");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = reinterpret_cast<char*>(workspace);
  cudaEvent_t e0 = ctx->ev[0], e1 = ctx->ev[1];
  int best = 0;
  double bms = 0.0;
  std::string last;
  for (int c = 1; c <= 16; c *= 2) {
    hbaca_opts o = *opts;
    o.cluster = c;
    o.flags &= ~(HBACA_FLAG_GRAPH | HBACA_FLAG_PROFILE);
    hbaca::Plan p;
    std::string err;
    if (!hbaca::make_plan(gens, nblocks, o, ctx->sms, p, err) || p.total > workspace_bytes) {
      last = err.empty() ? "workspace too small for cluster " + std::to_string(c) : err;
      continue;
    }
    double ms = -1.0;
    for (int rep = 0; rep < 2; ++rep) {  // the second run is timed (the first warms up)
      hbaca::RunCtx rc{ws, st, ctx->sms, nullptr, 0};
      rc.xgroups = (opts->flags & HBACA_FLAG_SINGLE_CLUSTER) == 0;
      rc.baca_only = true;
      cudaError_t e = cudaMemsetAsync(ws + p.status.off, 0, p.status.bytes, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(ws + p.queue.off, 0, p.queue.bytes, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(ws + p.desc_region.off, p.desc.data(), p.desc.size(), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      if (e == cudaSuccess) e = p.cplx ? hbaca::run_c128(p, rc, err) : hbaca::run_f64(p, rc, err);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float t = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (e != cudaSuccess) {
        cudaGetLastError();
        last = err.empty() ? cudaGetErrorString(e) : err;
        ms = -1.0;
        break;
      }
      ms = t;
    }
    if (ms >= 0.0 && (best == 0 || ms < bms)) {
      best = c;
      bms = ms;
    }
  }
  if (best == 0) return fail(HBACA_INVALID_ARG, "no cluster size could run: " + last);
  *best_cluster = best;
  if (best_ms) *best_ms = bms;
  ctx->have_times = false;
  tls_err.clear();
  return HBACA_OK;
}

hbaca_status hbaca_compress(hbaca_ctx* ctx, const hbaca_gen* gen, const hbaca_opts* opts, hbaca_result* out,
                            void* workspace, void* stream) {
  return compress_blocks(ctx, 1, gen, opts, out, workspace, stream);
}

hbaca_status hbaca_compress_batched(hbaca_ctx* ctx, int32_t nblocks, const hbaca_gen* gens, const hbaca_opts* opts,
                                    hbaca_result* outs, void* workspace, void* stream) {
  return compress_blocks(ctx, nblocks, gens, opts, outs, workspace, stream);
}

static hbaca_status read_trace(int32_t nblocks, const hbaca_gen* gens, const hbaca_opts* opts, const void* workspace,
                               int32_t block, int64_t leaf, hbaca_leaf_trace* tr, void* stream) {
  if (!gens || !opts || !workspace || !tr || nblocks < 1) return fail(HBACA_INVALID_ARG, "NULL argument");
  hbaca::Plan p;
  std::string err;
  if (!hbaca::make_plan(gens, nblocks, *opts, current_sms(), p, err)) return fail(HBACA_INVALID_ARG, err);
  if (block < 0 || block >= nblocks) return fail(HBACA_INVALID_ARG, "block index out of range");
  const int nl = 1 << (2 * p.Lb[block]);
  if (leaf < 0 || leaf >= nl) return fail(HBACA_INVALID_ARG, "leaf index out of range");
  if (tr->d != p.d) return fail(HBACA_INVALID_ARG, "trace.d must equal opts.d");
  const int64_t gl = p.leaf_first[block] + leaf;
  hbaca::LeafDesc L;
  std::memcpy(&L, p.desc.data() + p.leafdesc_off + gl * sizeof(hbaca::LeafDesc), sizeof(L));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const char* ws = reinterpret_cast<const char*>(workspace);
  hbaca::LeafOut lo;
  int rank_after = 0;
  cudaError_t e = cudaMemcpyAsync(&lo, ws + p.leafout_off + gl * sizeof(hbaca::LeafOut), sizeof(lo),
                                  cudaMemcpyDeviceToHost, st);
  const int ref = p.Lb[block] == 0 ? p.user_ref_first + block : p.full_idx[block][0][leaf];
  if (e == cudaSuccess) e = cudaMemcpyAsync(&rank_after, ws + p.ranks_off + (size_t)ref * 4, 4, cudaMemcpyDeviceToHost, st);
  const int rec = 4 + 3 * p.d;
  const int nit = std::min(L.tape_iters, tr->max_iters);
  std::vector<int32_t> ti((size_t)std::max(nit, 1) * rec);
  std::vector<double> td((size_t)std::max(nit, 1) * 2);
  if (e == cudaSuccess && nit > 0)
    e = cudaMemcpyAsync(ti.data(), ws + p.tape_int.off + L.tape_off * 4, (size_t)nit * rec * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && nit > 0)
    e = cudaMemcpyAsync(td.data(), ws + p.tape_dbl.off + L.taped_off * 8, (size_t)nit * 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(HBACA_CUDA, std::string("trace copy: ") + cudaGetErrorString(e));
  tr->iters = lo.iters;
  tr->rank_baca = lo.rank;
  tr->rank = rank_after;
  tr->stop = lo.stop;
  const int d = p.d;
  for (int it = 0; it < nit && it < lo.iters; ++it) {
    const int32_t* r = ti.data() + (size_t)it * rec;
    if (tr->dI) tr->dI[it] = r[0];
    if (tr->dJ) tr->dJ[it] = r[1];
    if (tr->dk) tr->dk[it] = r[2];
    for (int s2 = 0; s2 < d; ++s2) {
      if (tr->I) tr->I[(size_t)it * d + s2] = r[4 + s2];
      if (tr->J) tr->J[(size_t)it * d + s2] = r[4 + d + s2];
      if (tr->jbar) tr->jbar[(size_t)it * d + s2] = r[4 + 2 * d + s2];
    }
    if (tr->nu) tr->nu[it] = td[2 * it];
    if (tr->mu) tr->mu[it] = td[2 * it + 1];
  }
  tls_err.clear();
  return HBACA_OK;
}

hbaca_status hbaca_read_leaf_trace(const hbaca_gen* gen, const hbaca_opts* opts, const void* workspace, int64_t leaf,
                                   hbaca_leaf_trace* trace, void* stream) {
  return read_trace(1, gen, opts, workspace, 0, leaf, trace, stream);
}

hbaca_status hbaca_read_leaf_trace_batched(int32_t nblocks, const hbaca_gen* gens, const hbaca_opts* opts,
                                           const void* workspace, int32_t block, int64_t leaf,
                                           hbaca_leaf_trace* trace, void* stream) {
  return read_trace(nblocks, gens, opts, workspace, block, leaf, trace, stream);
}

hbaca_status hbaca_debug_read_block(const hbaca_gen* gen, const hbaca_opts* opts, const void* workspace,
                                    int32_t store, int32_t level, int64_t block, void* U, double* S, void* V,
                                    int64_t* m_out, int64_t* n_out, int64_t* rank_out, int64_t* cap_out,
                                    void* stream) {
  if (!gen || !opts || !workspace) return fail(HBACA_INVALID_ARG, "NULL argument");
  hbaca::Plan p;
  std::string err;
  if (!hbaca::make_plan(gen, 1, *opts, current_sms(), p, err)) return fail(HBACA_INVALID_ARG, err);
  const std::vector<int>* idx = nullptr;
  const hbaca::Region *ru, *rs, *rv;
  if (store == 0 && level >= 0 && level < p.Lb[0]) {
    idx = &p.full_idx[0][level];
    ru = &p.full_u; rs = &p.full_s; rv = &p.full_v;
  } else if (store == 1 && level >= 1 && level <= p.Lb[0]) {
    idx = &p.half_idx[0][level];
    ru = &p.half_u; rs = &p.half_s; rv = &p.half_v;
  } else {
    return fail(HBACA_INVALID_ARG, "no such store level");
  }
  if (block < 0 || block >= (int64_t)idx->size()) return fail(HBACA_INVALID_ARG, "block index out of range");
  hbaca::BlockRef b;
  std::memcpy(&b, p.desc.data() + p.refs_off + (size_t)(*idx)[block] * sizeof(b), sizeof(b));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const char* ws = reinterpret_cast<const char*>(workspace);
  int32_t rank = 0;
  cudaError_t e = cudaMemcpyAsync(&rank, ws + p.ranks_off + (size_t)b.rank_slot * 4, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && rank > 0) {
    if (U) e = cudaMemcpyAsync(U, ws + ru->off + b.u_off * p.esz, (size_t)b.m * rank * p.esz, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && S) e = cudaMemcpyAsync(S, ws + rs->off + b.s_off * 8, (size_t)rank * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && V) e = cudaMemcpyAsync(V, ws + rv->off + b.v_off * p.esz, (size_t)rank * b.n * p.esz, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) return fail(HBACA_CUDA, std::string("block copy: ") + cudaGetErrorString(e));
  if (m_out) *m_out = b.m;
  if (n_out) *n_out = b.n;
  if (rank_out) *rank_out = rank;
  if (cap_out) *cap_out = b.cap;
  tls_err.clear();
  return HBACA_OK;
}

hbaca_status hbaca_debug_read_leaf_factors(const hbaca_gen* gen, const hbaca_opts* opts, const void* workspace,
                                           int64_t leaf, void* U, void* V, int64_t* m_out, int64_t* n_out,
                                           int64_t* rank_out, void* stream) {
  if (!gen || !opts || !workspace) return fail(HBACA_INVALID_ARG, "NULL argument");
  if (!(opts->flags & HBACA_FLAG_TAPE))
    return fail(HBACA_INVALID_ARG, "leaf factors survive the call only with HBACA_FLAG_TAPE");
  hbaca::Plan p;
  std::string err;
  if (!hbaca::make_plan(gen, 1, *opts, current_sms(), p, err)) return fail(HBACA_INVALID_ARG, err);
  if (leaf < 0 || leaf >= p.nleaves) return fail(HBACA_INVALID_ARG, "leaf index out of range");
  hbaca::LeafDesc L;
  std::memcpy(&L, p.desc.data() + p.leafdesc_off + leaf * sizeof(hbaca::LeafDesc), sizeof(L));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const char* ws = reinterpret_cast<const char*>(workspace);
  hbaca::LeafOut lo;
  cudaError_t e = cudaMemcpyAsync(&lo, ws + p.leafout_off + leaf * sizeof(hbaca::LeafOut), sizeof(lo),
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const int r = std::max(0, std::min(lo.rank, L.rcap));
  if (e == cudaSuccess && r > 0 && U)
    e = cudaMemcpyAsync(U, ws + p.uar.off + (size_t)L.u_off * p.esz, (size_t)L.m * r * p.esz, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && r > 0 && V)
    e = cudaMemcpyAsync(V, ws + p.var.off + (size_t)L.v_off * p.esz, (size_t)r * L.n * p.esz, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(HBACA_CUDA, std::string("leaf factor copy: ") + cudaGetErrorString(e));
  if (m_out) *m_out = L.m;
  if (n_out) *n_out = L.n;
  if (rank_out) *rank_out = r;
  tls_err.clear();
  return HBACA_OK;
}

hbaca_status hbaca_phase_times(hbaca_ctx* ctx, double ms[4], int32_t* launches) {
  if (!ctx || !ms) return fail(HBACA_INVALID_ARG, "NULL argument");
  if (launches) *launches = ctx->launches;
  if (!ctx->have_times) return fail(HBACA_INVALID_ARG, "the last call did not run with HBACA_FLAG_PROFILE");
  float t[3];
  cudaError_t e = cudaEventSynchronize(ctx->ev[3]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t[0], ctx->ev[0], ctx->ev[1]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t[1], ctx->ev[1], ctx->ev[2]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t[2], ctx->ev[2], ctx->ev[3]);
  if (e != cudaSuccess) return fail(HBACA_CUDA, std::string("event timing: ") + cudaGetErrorString(e));
  ms[0] = t[0];
  ms[1] = t[1];
  ms[2] = t[2];
  ms[3] = (double)t[0] + t[1] + t[2];
  tls_err.clear();
  return HBACA_OK;
}

hbaca_status hbaca_kernel_times(hbaca_ctx* ctx, double ms[HBACA_KERNEL_CLASSES], int32_t launches[HBACA_KERNEL_CLASSES]) {
  if (!ctx || !ms || !launches) return fail(HBACA_INVALID_ARG, "NULL argument");
  if (!ctx->have_times) return fail(HBACA_INVALID_ARG, "the last call did not run with HBACA_FLAG_PROFILE");
  for (int i = 0; i < HBACA_KERNEL_CLASSES; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  cudaError_t e = cudaEventSynchronize(ctx->ev[3]);
  // launch intervals on the call's clock (from the start event); launches of
  // one class that overlap (concurrent streams) count once: the class time is
  // the length of the union of its intervals
  std::vector<std::vector<std::pair<float, float>>> iv(HBACA_KERNEL_CLASSES);
  for (const auto& mk : ctx->kt.marks) {
    if (e != cudaSuccess) break;
    float t0 = 0.f, t1 = 0.f;
    e = cudaEventElapsedTime(&t0, ctx->ev[0], ctx->kt.pool[mk.second]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, ctx->ev[0], ctx->kt.pool[mk.second + 1]);
    if (e == cudaSuccess && mk.first >= 0 && mk.first < HBACA_KERNEL_CLASSES) {
      iv[mk.first].emplace_back(t0, t1);
      launches[mk.first] += 1;
    }
  }
  for (int c = 0; c < HBACA_KERNEL_CLASSES; ++c) {
    std::sort(iv[c].begin(), iv[c].end());
    double tot = 0.0, a = 0.0, b = -1.0;
    for (const auto& x : iv[c]) {
      if (x.first > b) {
        if (b > a) tot += b - a;
        a = x.first;
        b = x.second;
      } else if (x.second > b) {
        b = x.second;
      }
    }
    if (b > a) tot += b - a;
    ms[c] = tot;
  }
  if (e != cudaSuccess) return fail(HBACA_CUDA, std::string("event timing: ") + cudaGetErrorString(e));
  tls_err.clear();
  return HBACA_OK;
}

int32_t hbaca_debug_set_jacobi_cluster(int32_t cluster) {
  const int v = cluster >= 1 && cluster <= 16 ? cluster : 0;
  return g_jacobi_cluster.exchange(v);
}

int32_t hbaca_debug_set_jacobi_groups(int32_t groups) {
  const int v = groups >= 1 && groups <= hbaca::kXSlots ? groups : 0;
  return g_jacobi_groups.exchange(v);
}

int32_t hbaca_debug_set_qr_groups(int32_t groups) {
  const int v = groups >= 1 && groups <= hbaca::kXSlots ? groups : 0;
  return g_qr_groups.exchange(v);
}

int32_t hbaca_debug_set_qr_cluster(int32_t cluster) {
  const int v = cluster >= 1 && cluster <= 16 ? cluster : 0;
  return g_qr_cluster.exchange(v);
}

int32_t hbaca_debug_set_jacobi_sweeps(int32_t sweeps) {
  const int v = sweeps > 0 ? sweeps : kDefaultJacobiSweeps;
  return g_jacobi_sweeps.exchange(v);
}

int32_t hbaca_debug_launch_times(hbaca_ctx* ctx, int32_t* cls, int32_t* stage, double* start_ms, double* ms,
                                 int32_t max) {
  if (!ctx || !ctx->have_times) {
    tls_err = "the last call did not run with HBACA_FLAG_PROFILE";
    return -1;
  }
  if (cudaEventSynchronize(ctx->ev[3]) != cudaSuccess) {
    cudaGetLastError();
    tls_err = "event synchronisation failed";
    return -1;
  }
  const int n = (int)ctx->kt.marks.size();
  for (int i = 0; i < n && i < max; ++i) {
    const auto& mk = ctx->kt.marks[i];
    float t0 = 0.f, t1 = 0.f;
    if (cudaEventElapsedTime(&t0, ctx->ev[0], ctx->kt.pool[mk.second]) != cudaSuccess ||
        cudaEventElapsedTime(&t1, ctx->ev[0], ctx->kt.pool[mk.second + 1]) != cudaSuccess) {
      cudaGetLastError();
      tls_err = "event timing failed";
      return -1;
    }
    if (cls) cls[i] = mk.first;
    if (stage) stage[i] = ctx->kt.mark_stage[i];
    if (start_ms) start_ms[i] = t0;
    if (ms) ms[i] = (double)t1 - t0;
  }
  tls_err.clear();
  return n;
}

size_t hbaca_debug_plan_json(const hbaca_gen* gen, const hbaca_opts* opts, char* buf, size_t len) {
  if (!gen || !opts) return 0;
  hbaca::Plan p;
  std::string err;
  if (!hbaca::make_plan(gen, 1, *opts, current_sms(), p, err)) { tls_err = err; return 0; }
  std::string j = "{";
  auto reg = [&](const char* name, const hbaca::Region& r) {
    j += std::string("\"") + name + "\": [" + std::to_string(r.off) + ", " + std::to_string(r.bytes) + "], ";
  };
  reg("status", p.status); reg("queue", p.queue); reg("desc", p.desc_region);
  reg("uar", p.uar); reg("var", p.var); reg("qr", p.qr); reg("tau", p.tau); reg("core", p.core); reg("ord", p.ord);
  reg("full_u", p.full_u); reg("full_s", p.full_s); reg("full_v", p.full_v);
  reg("half_u", p.half_u); reg("half_s", p.half_s); reg("half_v", p.half_v);
  reg("cscr", p.cscr); reg("rscr", p.rscr); reg("gscr", p.gscr); reg("tape_int", p.tape_int);
  reg("tape_dbl", p.tape_dbl); reg("jlist", p.jlist); reg("xpart", p.xpart); reg("xcnt", p.xcnt);
  j += "\"leafout\": " + std::to_string(p.leafout_off) + ", \"leafdesc\": " + std::to_string(p.leafdesc_off) + ", ";
  j += "\"baca_cluster\": " + std::to_string(p.baca_cluster) + ", \"rank_cap\": " + std::to_string(p.rank_cap_max) + ", ";
  j += "\"stages\": [";
  for (size_t si = 0; si < p.stages.size(); ++si) {
    const hbaca::Stage& st = p.stages[si];
    j += "{\"kind\": " + std::to_string(st.kind) + ", \"ntasks\": " + std::to_string(st.ntasks) +
         ", \"kcap\": " + std::to_string(st.kcap) + ", \"dims\": " + std::to_string(st.dims_off) + ", \"tasks\": [";
    for (size_t ti = 0; ti < st.tasks_h->size(); ++ti) {
      const hbaca::SvdTask& t = (*st.tasks_h)[ti];
      j += "{\"a_off\": " + std::to_string(t.a_off) + ", \"rows_a\": " + std::to_string(t.rows_a) +
           ", \"lda\": " + std::to_string(t.lda) + ", \"a_in_baca\": " + std::to_string(t.a_in_baca) +
           ", \"b_off\": " + std::to_string(t.b_off) + ", \"rows_b\": " + std::to_string(t.rows_b) +
           ", \"tau_off\": " + std::to_string(t.tau_off) + ", \"m_off\": " + std::to_string(t.m_off) +
           ", \"y_off\": " + std::to_string(t.y_off) + ", \"ord_off\": " + std::to_string(t.ord_off) +
           ", \"kcap\": " + std::to_string(t.kcap) + ", \"in1\": " + std::to_string(t.in1) +
           ", \"in2\": " + std::to_string(t.in2) + ", \"out\": " + std::to_string(t.out) +
           ", \"trunc\": " + std::to_string(t.trunc) + "}";
      if (ti + 1 < st.tasks_h->size()) j += ", ";
    }
    j += "]}";
    if (si + 1 < p.stages.size()) j += ", ";
  }
  j += "], \"total\": " + std::to_string(p.total) + "}";
  if (buf && len) {
    size_t n = std::min(len - 1, j.size());
    std::memcpy(buf, j.data(), n);
    buf[n] = 0;
  }
  return j.size() + 1;
}

}  // extern "C"
