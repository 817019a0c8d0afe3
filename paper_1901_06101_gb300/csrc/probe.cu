// FP64 unit-rate probe (DFMA and FP64 mma.sync) for the benchmark's report.
// Every thread writes one result; loops are bounded by the iteration count.
#include <cuda_runtime.h>

#include "hbaca.h"
#include "hbaca_probe.h"

namespace {

__global__ void dfma_loop(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void dmma_loop(double* out, int iters, double a, double b) {
  double acc[4][2];
  for (int j = 0; j < 4; ++j) { acc[j][0] = threadIdx.x + j; acc[j][1] = threadIdx.x - j; }
  const double av = a + threadIdx.x * 1e-9, bv = b - threadIdx.x * 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(acc[j][0]), "+d"(acc[j][1]) : "d"(av), "d"(bv));
  }
  double s = 0;
  for (int j = 0; j < 4; ++j) s += acc[j][0] + acc[j][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" hbaca_status hbaca_debug_fp64_probe(double* dfma_tflops, double* dmma_tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HBACA_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256;
  double* buf = nullptr;
  // the probe is a measurement utility, not part of the compression path
  if (cudaMalloc(&buf, sizeof(double) * blocks * threads) != cudaSuccess) return HBACA_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  const int it = 4000, itm = 800;
  dfma_loop<<<blocks, threads>>>(buf, 100, 0.999, 1e-3);
  cudaEventRecord(e0);
  dfma_loop<<<blocks, threads>>>(buf, it, 0.999, 1e-3);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  if (dfma_tflops) *dfma_tflops = 2.0 * 8 * (double)it * blocks * threads / ms / 1e9;
  dmma_loop<<<blocks, threads>>>(buf, 10, 0.999, 1e-3);
  cudaEventRecord(e0);
  dmma_loop<<<blocks, threads>>>(buf, itm, 0.999, 1e-3);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  if (dmma_tflops) *dmma_tflops = 2.0 * 8 * 8 * 4 * 4 * (double)itm * blocks * (threads / 32) / ms / 1e9;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t err = cudaGetLastError();
  cudaFree(buf);
  return err == cudaSuccess ? HBACA_OK : HBACA_CUDA;
}
