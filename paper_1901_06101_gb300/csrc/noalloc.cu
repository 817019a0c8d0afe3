// hbaca_compress_noalloc: hbaca_compress whose workspace is a fixed area of
// device memory owned by this library, for callers that cannot hand over a
// workspace of their own.  Those are callers with no device allocator at
// hand (a plain C program that links only libhbaca and the CUDA runtime),
// callers whose device memory is entirely owned by another runtime's pool,
// and latency-bound callers that must not pay for an allocation per call.
// Problems are limited to HBACA_NOALLOC_WORKSPACE_BYTES of workspace.
//
// The area is a file-scope __device__ array, so every device context that
// loads this module has its own copy.  Its address is looked up once per
// device, on the first call made with that device current; that first call
// should come before any stream capture.  The function itself never
// allocates or frees device memory.  All calls on one device share the
// area: calls that overlap in time (other host threads, or other streams
// whose work has not finished) race on it and must be serialised by the
// caller.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "hbaca.h"
#include "run.h"

static __device__ __align__(256) unsigned char hbaca_noalloc_scratch[HBACA_NOALLOC_WORKSPACE_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch[kMaxDevices] = {};

}  // namespace

extern "C" hbaca_status hbaca_compress_noalloc(hbaca_ctx* ctx, const hbaca_gen* gen, const hbaca_opts* opts,
                                               hbaca_result* out, void* stream) {
  if (!ctx || !gen || !opts || !out) return hbaca::record_error(HBACA_INVALID_ARG, "NULL ctx, gen, opts or result");
  const size_t need = hbaca_workspace_size(gen, opts);
  if (need == 0) return HBACA_INVALID_ARG;  // message set by hbaca_workspace_size
  if (need > (size_t)HBACA_NOALLOC_WORKSPACE_BYTES)
    return hbaca::record_error(HBACA_WORKSPACE,
                               "problem needs " + std::to_string(need) + " bytes of workspace; the built-in area holds " +
                                   std::to_string((size_t)HBACA_NOALLOC_WORKSPACE_BYTES) +
                                   " (use hbaca_compress with a caller workspace)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hbaca::record_error(HBACA_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return hbaca::record_error(HBACA_INVALID_ARG, "device ordinal out of range");
  void* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch[dev]) {
      e = cudaGetSymbolAddress(&g_scratch[dev], hbaca_noalloc_scratch);
      if (e != cudaSuccess) {
        g_scratch[dev] = nullptr;
        return hbaca::record_error(HBACA_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
    }
    ws = g_scratch[dev];
  }
  // hbaca_compress clears the parts of the workspace that must start at zero
  // (status word, leaf work counter, rank slots) on `stream` before its
  // kernels run; everything else is written before it is read.
  return hbaca_compress(ctx, gen, opts, out, ws, stream);
}
