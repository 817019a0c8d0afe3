/* FP64 unit-rate probe, built as its own library (libhbaca_probe.so) for the
   benchmark's report; it is not part of the compression library. */
#ifndef HBACA_PROBE_H
#define HBACA_PROBE_H

#include "hbaca.h"

#ifdef __cplusplus
extern "C" {
#endif

/* FP64 throughput on the current device: a DFMA loop and an FP64 MMA
   (mma.sync m8n8k4) loop over all SMs; results in TFLOP/s, written to the
   non-NULL pointers.  Allocates and frees a scratch buffer of its own.
   HBACA_CUDA on a CUDA error. */
hbaca_status hbaca_debug_fp64_probe(double* dfma_tflops, double* dmma_tflops);

#ifdef __cplusplus
}
#endif

#endif
