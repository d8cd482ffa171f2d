// Internal hooks of the run-time counters (see metrics.cu).
#pragma once

#include <cuda_runtime.h>

namespace rgf {
bool gemm_timing_enabled();
void gemm_timing_before(cudaStream_t st, cudaEvent_t* a);
void gemm_timing_after(cudaStream_t st, cudaEvent_t a, double flops);
}  // namespace rgf
