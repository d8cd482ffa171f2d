// Peak probes of the CUDA-core pipes that bound the FP64 path and the FP32
// seed inverse: a grid of independent fused multiply-add chains, timed with
// CUDA events.  Used only for measurement (the denominators of the FP64 and
// FP32 roofline fractions); no transport step calls them.
#include <cuda_runtime.h>

#include "../../include/rgf_kernels.h"
#include "common.cuh"

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread (hides the pipe latency)

template <typename R>
__global__ void k_fma_loop(int iters, R x, R y, R* out) {
    R a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (R)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
    }
    R s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    // x and y are chosen by the caller so that the chains stay finite; the
    // store only keeps the compiler from dropping the loop.
    if (s == (R)12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename R>
rgf_status run(int blocks_per_sm, int iters, double* tflops, double* ms_out) {
    int dev = 0, sms = 0;
    RGF_CUDA_TRY(cudaGetDevice(&dev));
    RGF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256;
    const int blocks = sms * blocks_per_sm;
    R* out = nullptr;
    RGF_CUDA_TRY(cudaMalloc(&out, sizeof(R) * (size_t)blocks * threads));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const R x = (R)0.999999, y = (R)1e-7;
    k_fma_loop<R><<<blocks, threads>>>(iters / 10 + 1, x, y, out);  // warm-up
    RGF_LAUNCH_CHECK();
    cudaEventRecord(a);
    k_fma_loop<R><<<blocks, threads>>>(iters, x, y, out);
    RGF_LAUNCH_CHECK();
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess) {
        rgf::set_error("rgf_peak_fma: %s", cudaGetErrorString(e));
        return RGF_E_CUDA;
    }
    const double flops = 2.0 * kChains * (double)iters * threads * blocks;
    if (tflops) *tflops = flops / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return RGF_OK;
}

}  // namespace

extern "C" {

rgf_status rgf_peak_fma(int kind, int blocks_per_sm, int iters, double* tflops, double* ms) {
    if (blocks_per_sm < 1 || blocks_per_sm > 32 || iters < 1 || iters > (1 << 24)) {
        rgf::set_error("rgf_peak_fma: invalid arguments");
        return RGF_E_INVALID;
    }
    if (kind == 0) return run<double>(blocks_per_sm, iters, tflops, ms);
    if (kind == 1) return run<float>(blocks_per_sm, iters, tflops, ms);
    rgf::set_error("rgf_peak_fma: kind %d is neither 0 (FP64) nor 1 (FP32)", kind);
    return RGF_E_INVALID;
}

}  // extern "C"
