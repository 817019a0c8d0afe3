// Entry points of the two scalar-type translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "plan.h"

namespace hbaca {
struct RunCtx {
  char* ws;
  cudaStream_t st;
  int sms;
  const hbaca_result* res;
  int launches = 0;  // kernels launched by the call
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // profile: after BACA, after leaf stage, end
};
cudaError_t run_f64(Plan& p, RunCtx& rc, std::string& err);
cudaError_t run_c128(Plan& p, RunCtx& rc, std::string& err);
// Set the calling thread's hbaca_last_error() message; returns s.
hbaca_status record_error(hbaca_status s, const std::string& msg);
}  // namespace hbaca
