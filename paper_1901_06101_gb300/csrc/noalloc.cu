// hbaca_compress_noalloc: hbaca_compress whose workspace is a fixed area of
// device memory owned by this library, for callers that cannot hand over a
// workspace of their own.  Those are callers with no device allocator at
// hand (a plain C program that links only libhbaca and the CUDA runtime),
// callers whose device memory is entirely owned by another runtime's pool,
// and latency-bound callers that must not pay for an allocation per call.
// Problems are limited to HBACA_NOALLOC_WORKSPACE_BYTES of workspace.
//
// The area is a file-scope __device__ array, so every device context that
// loads this module has its own copy.  Its address is looked up on every
// call, on the current device (the first call on a device loads the module
// there, so it should come before any stream capture; later lookups are
// cheap, and an address is never reused after a device reset).  The
// function itself never allocates or frees device memory.  All calls on one
// device share the area: calls that overlap in time (other host threads, or
// other streams whose work has not finished) race on it and must be
// serialised by the caller.  Graph capture and the reverse-pass tape are
// refused: a replayed graph would read descriptor tables that a later call
// has replaced in the shared area, and a tape there could not be passed to
// hbaca_apply_backward, which takes the workspace pointer.
#include <cuda_runtime.h>

#include <string>

#include "hbaca.h"
#include "run.h"

static __device__ __align__(256) unsigned char hbaca_noalloc_scratch[HBACA_NOALLOC_WORKSPACE_BYTES];

extern "C" hbaca_status hbaca_compress_noalloc(hbaca_ctx* ctx, const hbaca_gen* gen, const hbaca_opts* opts,
                                               hbaca_result* out, void* stream) {
  if (!ctx || !gen || !opts || !out) return hbaca::record_error(HBACA_INVALID_ARG, "NULL ctx, gen, opts or result");
  if (opts->flags & (HBACA_FLAG_GRAPH | HBACA_FLAG_TAPE))
    return hbaca::record_error(HBACA_INVALID_ARG,
                               "HBACA_FLAG_GRAPH and HBACA_FLAG_TAPE need a workspace of the caller's "
                               "(use hbaca_compress)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hbaca::record_error(HBACA_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != hbaca::ctx_device(ctx))
    return hbaca::record_error(HBACA_INVALID_ARG, "the current device is not the context's");
  // the current device is the context's, so this plan is the one
  // hbaca_compress builds (same SM count)
  const size_t need = hbaca_workspace_size(gen, opts);
  if (need == 0) return HBACA_INVALID_ARG;  // message set by hbaca_workspace_size
  if (need > (size_t)HBACA_NOALLOC_WORKSPACE_BYTES)
    return hbaca::record_error(HBACA_WORKSPACE,
                               "problem needs " + std::to_string(need) + " bytes of workspace; the built-in area holds " +
                                   std::to_string((size_t)HBACA_NOALLOC_WORKSPACE_BYTES) +
                                   " (use hbaca_compress with a caller workspace)");
  void* ws = nullptr;
  e = cudaGetSymbolAddress(&ws, hbaca_noalloc_scratch);
  if (e != cudaSuccess || !ws) {
    cudaGetLastError();
    return hbaca::record_error(HBACA_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  }
  // hbaca_compress clears the parts of the workspace that must start at zero
  // (status word, leaf work counter, rank slots) on `stream` before its
  // kernels run; everything else is written before it is read.
  return hbaca_compress(ctx, gen, opts, out, ws, stream);
}
