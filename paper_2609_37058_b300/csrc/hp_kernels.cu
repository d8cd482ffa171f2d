// Seven-digit BF16 slicing of FP64 complex matrices for the high-precision
// slice-product GEMM (used by the mixed path's lead decimation).
//
// For a row (A operand) or column (B operand) whose largest |entry| is below
// 2^e, an entry x is written as sign(x) 2^e sum_{s=0..6} d_s 2^(-7-8s) with
// balanced digits |d_s| <= 128.  The digits are taken from the FP64 bit
// pattern with 64-bit integer arithmetic (no FP64 arithmetic): Y =
// round(|x| 2^(55-e)) < 2^55, then base-256 digits from the bottom with a
// carry whenever a digit exceeds 127.  Rounding error: 2^-56 of 2^e.
#include <atomic>

#include "mixed.h"
#include "slice_strip.cuh"

namespace rgf {

namespace {

__device__ __forceinline__ int exp_above_f64(double m) {
    if (!(m > 0.0)) return 0;
    int e;
    frexp(m, &e);
    return e;
}

__device__ __forceinline__ void digits7(double x, int e, float out[kSlicesHP]) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const bool neg = (bits >> 63) != 0;
    const int E = (int)((bits >> 52) & 0x7FF);
    unsigned long long Y = 0;
    if (E != 0 && E != 0x7FF) {
        const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = E - 1020 - e;  // <= 2 because |x| < 2^e
        if (sh >= 0) {
            Y = mant << sh;
        } else if (sh > -60) {
            Y = (mant + (1ull << (-sh - 1))) >> (-sh);
        }
    }
    int d[kSlicesHP];
#pragma unroll
    for (int s = kSlicesHP - 1; s >= 1; --s) {
        int v = (int)(Y & 0xFFull);
        Y >>= 8;
        if (v >= 128) {
            v -= 256;
            Y += 1;
        }
        d[s] = v;
    }
    d[0] = (int)Y;
#pragma unroll
    for (int s = 0; s < kSlicesHP; ++s) {
        const float v = ldexpf((float)(neg ? -d[s] : d[s]), e - 7 - 8 * s);
        out[s] = v;
    }
}

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

__global__ void __launch_bounds__(256) k_slice_rows_f64(int m, int k, const double2* __restrict__ A, long sA,
                                                        __nv_bfloat16* __restrict__ out, int Kp,
                                                        const int* __restrict__ active) {
    const int bi = blockIdx.y;
    if (active && !active[bi]) return;
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= m) return;
    const double2* row = A + (long)bi * sA + (long)r * k;
    double mx = 0.0;
    for (int j = lane; j < k; j += 32) {
        const double2 v = row[j];
        mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
    }
    mx = warp_max_d(mx);
    const int e = exp_above_f64(mx);
    for (int j = lane; j < k; j += 32) {
        const double2 v = row[j];
        float sr[kSlicesHP], si[kSlicesHP];
        digits7(v.x, e, sr);
        digits7(v.y, e, si);
#pragma unroll
        for (int s = 0; s < kSlicesHP; ++s) {
            __nv_bfloat162 p;
            p.x = __float2bfloat16_rn(sr[s]);
            p.y = __float2bfloat16_rn(si[s]);
            *reinterpret_cast<__nv_bfloat162*>(out + (((long)bi * kSlicesHP + s) * m + r) * Kp + 2 * j) = p;
        }
    }
}

// Two-pass column slicer for strips that do not fit in shared memory: one
// CTA per strip of 32 columns, column exponents first, then 32 x 32 tiles
// through shared memory (layout as the double-float column slicer).
__global__ void __launch_bounds__(256) k_slice_cols_f64(int k, int n, const double2* __restrict__ B, long sB,
                                                        __nv_bfloat16* __restrict__ out, int Kp,
                                                        const int* __restrict__ active) {
    const int bi = blockIdx.y;
    if (active && !active[bi]) return;
    __shared__ double2 tile[32][33];
    __shared__ double cmax[8][32];
    __shared__ int cexp[32];
    const int c0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const double2* Bb = B + (long)bi * sB;
    {
        const int c = c0 + tx;
        double mx = 0.0;
        if (c < n)
            for (int j = ty; j < k; j += 8) {
                const double2 v = Bb[(long)j * n + c];
                mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
            }
        cmax[ty][tx] = mx;
    }
    __syncthreads();
    if (ty == 0) {
        double mx = cmax[0][tx];
#pragma unroll
        for (int w = 1; w < 8; ++w) mx = fmax(mx, cmax[w][tx]);
        cexp[tx] = exp_above_f64(mx);
    }
    const long rows = 2L * n;
    for (int j0 = 0; j0 < k; j0 += 32) {
        __syncthreads();
        for (int jj = ty; jj < 32; jj += 8) {
            const int j = j0 + jj, c = c0 + tx;
            tile[jj][tx] = (j < k && c < n) ? Bb[(long)j * n + c] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        for (int cc = ty; cc < 32; cc += 8) {
            const int c = c0 + cc, j = j0 + tx;
            if (c >= n || j >= k) continue;
            const double2 v = tile[tx][cc];
            const int e = cexp[cc];
            float sr[kSlicesHP], si[kSlicesHP];
            digits7(v.x, e, sr);
            digits7(v.y, e, si);
#pragma unroll
            for (int s = 0; s < kSlicesHP; ++s) {
                __nv_bfloat16* base = out + (((long)bi * kSlicesHP + s) * rows) * Kp;
                __nv_bfloat162 p0, p1;
                p0.x = __float2bfloat16_rn(sr[s]);
                p0.y = __float2bfloat16_rn(-si[s]);
                p1.x = __float2bfloat16_rn(si[s]);
                p1.y = __float2bfloat16_rn(sr[s]);
                *reinterpret_cast<__nv_bfloat162*>(base + (2L * c) * Kp + 2 * j) = p0;
                *reinterpret_cast<__nv_bfloat162*>(base + (2L * c + 1) * Kp + 2 * j) = p1;
            }
        }
    }
}

}  // namespace

rgf_status slice_rows_f64(int batch, int m, int k, const double2* A, long sA, __nv_bfloat16* out, int Kp,
                          const int* active, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_slice_rows_f64<<<dim3(ceil_div(m, 8), batch), 256, 0, st>>>(m, k, A, sA, out, Kp, active);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

struct F64Strip {
    static constexpr int kMinBlocks = 3;
    using T = double2;
    using M = double;
    static constexpr int NS = kSlicesHP;
    __device__ static T zero() { return make_double2(0.0, 0.0); }
    __device__ static M amax(const T& v) { return fmax(fabs(v.x), fabs(v.y)); }
    __device__ static M vmax(M a, M b) { return fmax(a, b); }
    __device__ static M shfl_xor(M v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
    __device__ static int expo(M m) { return exp_above_f64(m); }
    __device__ static void split(const T& v, int e, float* sr, float* si) {
        digits7(v.x, e, sr);
        digits7(v.y, e, si);
    }
};

rgf_status slice_cols_f64(int batch, int k, int n, const double2* B, long sB, __nv_bfloat16* out, int Kp,
                          const int* active, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    if (strip_fits(k)) {
        static std::atomic<bool> attr{false};
        if (!attr.load()) {
            // Idempotent: threads that race here all set the same value.
            RGF_CUDA_TRY(cudaFuncSetAttribute(k_slice_cols_strip<F64Strip>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, kStripMaxSmem));
            attr.store(true);
        }
        k_slice_cols_strip<F64Strip><<<dim3(ceil_div(n, kStripCols), batch), kStripCols * 32, strip_smem_bytes(k),
                                       st>>>(k, n, B, sB, out, Kp, active, kSlicesHP);
        RGF_LAUNCH_CHECK();
        return RGF_OK;
    }
    k_slice_cols_f64<<<dim3(ceil_div(n, 32), batch), 256, 0, st>>>(k, n, B, sB, out, Kp, active);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

}  // namespace rgf
