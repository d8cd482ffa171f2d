/*
 * rgf_kernels.h - kernel-level entry points of the RGF library, for tests
 * and benchmarks of single building blocks (same conventions as rgf.h:
 * complex matrices are row-major (re, im) double pairs, batch-major; all
 * pointers are HOST memory; the calls are synchronous; a non-OK status
 * leaves a message for rgf_last_error()).  They allocate their own
 * temporary device memory for the duration of the call.
 */
#ifndef RGF_KERNELS_H
#define RGF_KERNELS_H

#include "rgf.h"

#ifdef __cplusplus
extern "C" {
#endif

/* C[i] = A[i] B[i], i < batch; A m x k, B k x n, C m x n, all FP64 (the
 * FP64 path's CUDA-core GEMM). */
rgf_status rgf_kernel_zgemm_f64(int batch, int m, int n, int k, const double* A, const double* B, double* C);

/* In-place inverse of batch b x b matrices by the FP64 path's blocked
 * Gauss-Jordan elimination with partial pivoting.  flags[i] (may be NULL)
 * gets RGF_FLAG_SINGULAR for an exactly zero pivot. */
rgf_status rgf_kernel_inverse_f64(int batch, int b, double* A, int* flags);

/* In-place FP32 inverse (the mixed path's seed): A holds complex64 values
 * as (re, im) float pairs.  Blocked Gauss-Jordan with partial pivoting: the
 * 32-column panels on the CUDA cores, each trailing update on the tensor
 * cores (three BF16 splits per operand, FP32 accumulation, FP32-accurate;
 * RGF_GJ_TC=0 in the environment selects CUDA-core updates).  Returns
 * RGF_E_CUDA if the tensor-core pipeline's bounded waits run out. */
rgf_status rgf_kernel_inverse_c64(int batch, int b, float* A, int* flags);

/* C[i] = A[i] B[i] by the mixed path's slice-product GEMM: A and B are
 * rounded to double-float, split into six BF16 slices each and multiplied
 * on the tensor cores; C is the double-float result widened to FP64.
 * core = 0: tcgen05 (TMA, TMEM accumulators); core = 1: the legacy
 * warp-level mma.sync path. */
rgf_status rgf_kernel_zgemm_mixed(int batch, int m, int n, int k, const double* A, const double* B, double* C,
                                  int core);

/* Failure-path probe of the tcgen05 GEMM's bounded waits: runs a small
 * slice-product GEMM whose producer skips the loads of the first K chunk,
 * with every mbarrier wait limited to wait_us microseconds, so the waits
 * run out.  Expected result: RGF_E_CUDA with *status_bits nonzero (bit 0x2:
 * the MMA issuer gave up on data, 0x1: the producer gave up on a free
 * stage), the CTAs having released their tensor memory; the context stays
 * usable for the next call.  No GPU fault is involved. */
rgf_status rgf_kernel_tc_timeout_probe(int wait_us, int* status_bits);

/* C[i] = A[i] B[i] by the high-precision slice-product GEMM of the mixed
 * path's lead decimation: FP64 operands split into seven BF16 slices (56
 * bits relative to each row / column maximum), 28 products on the tcgen05
 * tensor cores, FP64 result. */
rgf_status rgf_kernel_zgemm_hp(int batch, int m, int n, int k, const double* A, const double* B, double* C);

/* C[i] = A[i] B[i] by the slice-product GEMM with a chosen number of slices
 * per operand, on the tcgen05 core; the sweep and the decimation use the
 * shorter forms only for products whose error is not amplified (see the
 * nsl field of the GEMM arguments).  fp64_operands = 0: double-float
 * operands (as rgf_kernel_zgemm_mixed), nsl in {4, 5, 6}; fp64_operands =
 * 1: FP64 operands (as rgf_kernel_zgemm_hp), nsl in {5, 7}.  Host buffers,
 * blocking; RGF_E_INVALID for another nsl. */
rgf_status rgf_kernel_zgemm_slices(int batch, int m, int n, int k, const double* A, const double* B, double* C,
                                   int fp64_operands, int nsl);

/* Allocation-free FP64 batched inverse.  The paper has no counterpart: this
 * entry point exists for callers that cannot or must not allocate device
 * memory, e.g. code running while another framework owns the device memory
 * pool, or a latency-critical thread that cannot afford the implicit device
 * synchronisation of cudaMalloc/cudaFree.  It inverts, in place, batch
 * matrices b x b of complex128 values at the DEVICE pointer A (row-major
 * (re, im) pairs, batch-major), with the same blocked Gauss-Jordan kernels
 * as rgf_kernel_inverse_f64; flags (DEVICE pointer, may be NULL) receives
 * RGF_FLAG_SINGULAR per matrix (it is cleared first).  The work is enqueued
 * on cuda_stream (a cudaStream_t; NULL = legacy default stream) and the call
 * returns without waiting for it.
 *
 * Scratch: a fixed file-scope device array of rgf_inverse_f64_noalloc_limit()
 * bytes (16 MiB), present on every GPU that loads the library until the
 * process exits.  A call whose workspace would exceed it (about 60 matrices
 * of b = 256) is rejected with RGF_E_INVALID and a message; so is b outside
 * 1..512.  Invalid calls return before anything is enqueued (flags are left
 * as they were).  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current) and caches it per
 * device ordinal; make that first call before any stream capture.  The cache
 * is not refreshed after cudaDeviceReset, which unloads the module: do not
 * call this entry point on a device after resetting it in the same process.
 * A, flags and cuda_stream must belong to the current device.  All calls on
 * a device share the one array, which keeps the last call's contents, so
 * calls that overlap on the GPU (different streams, no ordering) race. */
rgf_status rgf_inverse_f64_noalloc(int batch, int b, double* A, int* flags, void* cuda_stream);

/* Size in bytes of that fixed scratch array. */
size_t rgf_inverse_f64_noalloc_limit(void);

/* Peak probe of a CUDA-core pipe, the denominator of the FP64 path's and the
 * FP32 seed inverse's roofline fractions (no counterpart in the paper, which
 * reports no GPU numbers).  kind 0 = FP64, 1 = FP32.  Launches
 * blocks_per_sm x (SM count) CTAs of 256 threads, each thread running 8
 * independent chains of iters fused multiply-adds (2 flops each), once as
 * warm-up and once timed with CUDA events on the legacy default stream;
 * blocks until done.  Writes the achieved TFLOP/s and the timed launch's
 * milliseconds (either may be NULL).  Allocates and frees a small output
 * buffer.  RGF_E_INVALID for kind outside {0, 1}, blocks_per_sm outside
 * 1..32 or iters outside 1..2^24. */
rgf_status rgf_peak_fma(int kind, int blocks_per_sm, int iters, double* tflops, double* ms);

/* Debug build (no counterpart in the paper).  librgf_debug.so is the same
 * library compiled with -DRGF_DEBUG: the indices that kernels take from data
 * (pivot rows of the Gauss-Jordan inverses, entries of the server's slot
 * table) are checked on the device, and a failed check sets a bit
 * (1: pivot row out of range, 2: slot-table entry out of range, 4: null
 * block or result pointer of an active slot) instead of faulting; the kernel
 * goes on with a safe index or skips the access.  rgf_debug_build() is 1 in
 * that library and 0 in the normal one; rgf_debug_flags() returns the bits
 * set since the last call and clears them (0 in the normal build). */
int rgf_debug_build(void);
unsigned rgf_debug_flags(void);

/* Counters for measurement (process-wide, thread-safe). */

/* Number of CUDA kernel launches issued by the library since load. */
unsigned long long rgf_launch_count(void);

/* CUDA-event timing of the mixed path's slice-product GEMM (tcgen05 core),
 * recorded on the stream each launch runs on.  A call returns the totals of
 * the launches recorded since the previous call (total_ms: summed launch
 * durations; launches; flops: BF16 tensor flops executed, 21 slice-pair
 * products of 2 M N K each), clears them, and turns recording on
 * (enable != 0) or off.  Outputs may be NULL.  Only launches without an
 * energy mask are recorded. */
rgf_status rgf_gemm_timing(int enable, double* total_ms, long long* launches, double* flops);

#ifdef __cplusplus
}
#endif

#endif /* RGF_KERNELS_H */
