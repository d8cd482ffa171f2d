// Column slicer with the strip resident in shared memory.  One CTA takes
// kStripCols columns of one batch entry: it reads the k x kStripCols strip
// from HBM once into shared memory (computing the column maxima on the way),
// then each warp turns one column into its slices.  The two-pass slicer read
// every strip twice and, with ~1200 strips of 128 KB resident at once, the
// second read missed L2.
//
// Output layout (the B operand of the slice-product GEMM, transposed and
// complex-expanded; rows of Kp BF16):
//   slice s, row 2c  : (Re, -Im) of B[j][c] at K positions (2j, 2j+1)
//   slice s, row 2c+1: (Im,  Re)
// Only c < n, j < k and the first `planes` slices are written (the K padding
// is zeroed once by the owner).
//
// Traits supply the element type (16 bytes: float4 double-float or double2),
// the magnitude used for the column exponent, the exponent rule and the
// per-element split into NS slices of the real and imaginary parts, and the
// CTAs per SM the register budget is sized for.
#pragma once

#include <cuda_bf16.h>

namespace rgf {

constexpr int kStripCols = 8;                 // columns per CTA = warps per CTA
constexpr int kStripPitch = kStripCols + 1;   // padded row: conflict-free column reads
constexpr int kStripMaxSmem = 200 * 1024;     // dynamic shared memory bound of the strip path

inline size_t strip_smem_bytes(int k) { return (size_t)k * kStripPitch * 16; }
inline bool strip_fits(int k) { return strip_smem_bytes(k) <= (size_t)kStripMaxSmem; }

template <class Tr>
__global__ void __launch_bounds__(kStripCols * 32, Tr::kMinBlocks) k_slice_cols_strip(int k, int n, const typename Tr::T* __restrict__ B,
                                                                      long sB, __nv_bfloat16* __restrict__ out, int Kp,
                                                                      const int* __restrict__ active, int planes) {
    using T = typename Tr::T;
    using M = typename Tr::M;
    constexpr int NS = Tr::NS;
    constexpr int kThreads = kStripCols * 32;
    constexpr int kRowsPerPass = kThreads / kStripCols;
    const int bi = blockIdx.y;
    if (active && !active[bi]) return;
    extern __shared__ __align__(16) unsigned char strip_raw[];
    T* tile = reinterpret_cast<T*>(strip_raw);
    __shared__ M wmax[kStripCols][kStripCols];  // [warp][column]
    __shared__ int cexp[kStripCols];
    const int c0 = blockIdx.x * kStripCols;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int col = tid % kStripCols;
    const int c = c0 + col;
    const T* Bb = B + (long)bi * sB;

    // Pass over HBM: strip into shared memory, per-thread column maxima.
    M mx = M(0);
#pragma unroll 4
    for (int j = tid / kStripCols; j < k; j += kRowsPerPass) {
        T v = Tr::zero();
        if (c < n) v = Bb[(long)j * n + c];
        tile[j * kStripPitch + col] = v;
        mx = Tr::vmax(mx, Tr::amax(v));
    }
    // Lanes l, l ^ 8, l ^ 16, l ^ 24 hold the same column.
#pragma unroll
    for (int off = kStripCols; off < 32; off <<= 1) mx = Tr::vmax(mx, Tr::shfl_xor(mx, off));
    if (lane < kStripCols) wmax[warp][lane] = mx;
    __syncthreads();
    if (tid < kStripCols) {
        M m = wmax[0][tid];
#pragma unroll
        for (int w = 1; w < kStripCols; ++w) m = Tr::vmax(m, wmax[w][tid]);
        cexp[tid] = Tr::expo(m);
    }
    __syncthreads();

    // Warp w slices column c0 + w; lanes run along j (coalesced writes).
    const int cw = c0 + warp;
    if (cw >= n) return;
    const int e = cexp[warp];
    const long rows = 2L * n;
    for (int j = lane; j < k; j += 32) {
        const T v = tile[j * kStripPitch + warp];
        float sr[NS], si[NS];
        Tr::split(v, e, sr, si);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (s >= planes) break;
            __nv_bfloat16* base = out + (((long)bi * NS + s) * rows) * Kp;
            __nv_bfloat162 p0, p1;
            p0.x = __float2bfloat16_rn(sr[s]);
            p0.y = __float2bfloat16_rn(-si[s]);
            p1.x = __float2bfloat16_rn(si[s]);
            p1.y = __float2bfloat16_rn(sr[s]);
            *reinterpret_cast<__nv_bfloat162*>(base + (2L * cw) * Kp + 2 * j) = p0;
            *reinterpret_cast<__nv_bfloat162*>(base + (2L * cw + 1) * Kp + 2 * j) = p1;
        }
    }
}

}  // namespace rgf
