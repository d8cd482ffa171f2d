// Mixed-precision kernels: BF16 slicing of double-float operands, the
// legacy-path reference core of the slice-product complex GEMM, and the
// double-float elementwise steps (block formation, decimation updates,
// broadenings, Newton-Schulz bookkeeping, the FP64 trace reduction).
#include <atomic>
#include <cstdlib>
#include "df.cuh"
#include "engine.h"
#include "mixed.h"
#include "slice_strip.cuh"

namespace rgf {

static inline int grid_for2(long n, int threads, int cap = 1024) {
    long g = (n + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// ------------------------------------------------------------------ slicing
// x = hi + lo, scaled by 2^(7 - e) where every |x| of the row is below 2^e:
// then |y| < 128 and the slices are q_s = rint of the running remainder
// times 256^s, |q_s| <= 128, value weight 2^(e - 7 - 8 s).
__device__ __forceinline__ void slice6(float hi, float lo, int e, float out[kSlices]) {
    float yh = ldexpf(hi, 7 - e);
    float yl = ldexpf(lo, 7 - e);
    float w = ldexpf(1.0f, e - 7);
#pragma unroll
    for (int s = 0; s < kSlices; ++s) {
        const float q = rintf(yh);
        out[s] = q * w;
        const float r = yh - q;
        const float2 t = two_sum(r * 256.0f, yl * 256.0f);
        yh = t.x;
        yl = t.y;
        w *= (1.0f / 256.0f);
    }
}

__device__ __forceinline__ int exp_above(float m) {
    // smallest e with m < 2^e (m > 0); 0 for m == 0
    if (!(m > 0.0f)) return 0;
    int e;
    frexpf(m, &e);
    return e;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

__global__ void __launch_bounds__(256) k_slice_rows(int m, int k, const float4* __restrict__ A, long sA,
                                                    __nv_bfloat16* __restrict__ out, int Kp,
                                                    const int* __restrict__ active, int planes) {
    const int bi = blockIdx.y;
    if (active && !active[bi]) return;
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= m) return;
    const float4* row = A + (long)bi * sA + (long)r * k;
    float mx = 0.0f;
    for (int j = lane; j < k; j += 32) {
        const float4 v = row[j];
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.z)));
    }
    mx = warp_max(mx);
    const int e = exp_above(mx);
    for (int j = lane; j < k; j += 32) {
        const float4 v = row[j];
        float sr[kSlices], si[kSlices];
        slice6(v.x, v.y, e, sr);
        slice6(v.z, v.w, e, si);
#pragma unroll
        for (int s = 0; s < kSlices; ++s) {
            if (s >= planes) break;
            __nv_bfloat162 p;
            p.x = __float2bfloat16_rn(sr[s]);
            p.y = __float2bfloat16_rn(si[s]);
            __nv_bfloat16* o = out + (((long)bi * kSlices + s) * m + r) * Kp + 2 * j;
            *reinterpret_cast<__nv_bfloat162*>(o) = p;
        }
    }
}

// (zr + i zi) S' - H' in df for one element (S', H' already conjugated
// when the caller needs the conjugate transpose).
__device__ __forceinline__ float4 zsh_df(float2 zr, float2 zi, float4 sv, float4 hv) {
    const float2 sr = re_of(sv), sim = im_of(sv);
    const float2 re = df_sub(df_sub(df_mul(zr, sr), df_mul(zi, sim)), re_of(hv));
    const float2 im = df_sub(df_add(df_mul(zr, sim), df_mul(zi, sr)), im_of(hv));
    return cdf(re, im);
}
__device__ __forceinline__ float4 conj_df(float4 v) { return make_float4(v.x, v.y, -v.z, -v.w); }

// Slices of the formed element v (row r, column j) in the A layout, and of
// the element at row i of column c in the B layout of the K-interleaved
// product (rows 2c: (Re, -Im), 2c + 1: (Im, Re)).
__device__ __forceinline__ void put_row_slices(__nv_bfloat16* out, int bi, int b, int r, int Kp, int j, float4 v,
                                               int e) {
    float sr[kSlices], si[kSlices];
    slice6(v.x, v.y, e, sr);
    slice6(v.z, v.w, e, si);
#pragma unroll
    for (int s = 0; s < kSlices; ++s) {
        __nv_bfloat162 p;
        p.x = __float2bfloat16_rn(sr[s]);
        p.y = __float2bfloat16_rn(si[s]);
        *reinterpret_cast<__nv_bfloat162*>(out + (((long)bi * kSlices + s) * b + r) * Kp + 2 * j) = p;
    }
}
__device__ __forceinline__ void put_col_slices(__nv_bfloat16* out, int bi, int b, int c, int Kp, int i, float4 v,
                                               int e) {
    float sr[kSlices], si[kSlices];
    slice6(v.x, v.y, e, sr);
    slice6(v.z, v.w, e, si);
    const long rows = 2L * b;
#pragma unroll
    for (int s = 0; s < kSlices; ++s) {
        __nv_bfloat16* base = out + (((long)bi * kSlices + s) * rows) * Kp;
        __nv_bfloat162 p0, p1;
        p0.x = __float2bfloat16_rn(sr[s]);
        p0.y = __float2bfloat16_rn(-si[s]);
        p1.x = __float2bfloat16_rn(si[s]);
        p1.y = __float2bfloat16_rn(sr[s]);
        *reinterpret_cast<__nv_bfloat162*>(base + (2L * c) * Kp + 2 * i) = p0;
        *reinterpret_cast<__nv_bfloat162*>(base + (2L * c + 1) * Kp + 2 * i) = p1;
    }
}

// One warp forms the b elements of a row (or column) with form(i), finds
// their largest |Re|, |Im| for the slice exponent and writes the slices with
// put(i, v, e).  The first 32 * kFormCache elements stay in registers between
// the two passes (all of them for b <= 256); the rest are formed again.
constexpr int kFormCache = 8;
template <typename Form, typename Put>
__device__ __forceinline__ void form_slice_warp(int b, int lane, Form form, Put put) {
    float4 cache[kFormCache];
    float mx = 0.0f;
#pragma unroll
    for (int t = 0; t < kFormCache; ++t) {
        const int i = lane + 32 * t;
        cache[t] = i < b ? form(i) : make_float4(0.f, 0.f, 0.f, 0.f);
        mx = fmaxf(mx, fmaxf(fabsf(cache[t].x), fabsf(cache[t].z)));
    }
    for (int i = lane + 32 * kFormCache; i < b; i += 32) {
        const float4 v = form(i);
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.z)));
    }
    mx = warp_max(mx);
    const int e = exp_above(mx);
#pragma unroll
    for (int t = 0; t < kFormCache; ++t) {
        const int i = lane + 32 * t;
        if (i < b) put(i, cache[t], e);
    }
    for (int i = lane + 32 * kFormCache; i < b; i += 32) put(i, form(i), e);
}

// A-operand slices of tau = z S - H (one warp per row, one batch entry per
// energy; S, H shared b x b df blocks): the formed matrix never goes to
// memory.  Same layout as k_slice_rows.
__global__ void __launch_bounds__(256) k_form_slice_rows(int b, const double* __restrict__ E, double eta,
                                                         const float4* __restrict__ S, const float4* __restrict__ H,
                                                         __nv_bfloat16* __restrict__ out, int Kp) {
    const int bi = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= b) return;
    const float2 zr = df_from_double(E[bi]), zi = df_from_double(eta);
    const float4* Sr = S + (long)r * b;
    const float4* Hr = H + (long)r * b;
    form_slice_warp(
        b, lane, [&](int j) { return zsh_df(zr, zi, Sr[j], Hr[j]); },
        [&](int j, float4 v, int e) { put_row_slices(out, bi, b, r, Kp, j, v, e); });
}

// B-operand slices of tau' = z S^dagger - H^dagger (one warp per column c of
// tau', i.e. per row c of S and H, read contiguously): same layout as
// k_slice_cols, with no transposition pass.
__global__ void __launch_bounds__(256) k_form_slice_cols_dag(int b, const double* __restrict__ E, double eta,
                                                             const float4* __restrict__ S,
                                                             const float4* __restrict__ H,
                                                             __nv_bfloat16* __restrict__ out, int Kp) {
    const int bi = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= b) return;
    const float2 zr = df_from_double(E[bi]), zi = df_from_double(eta);
    const float4* Sc = S + (long)c * b;
    const float4* Hc = H + (long)c * b;
    form_slice_warp(
        b, lane, [&](int i) { return zsh_df(zr, zi, conj_df(Sc[i]), conj_df(Hc[i])); },
        [&](int i, float4 v, int e) { put_col_slices(out, bi, b, c, Kp, i, v, e); });
}

// Table-driven forms of the two kernels above for the server's energy
// slots: entry s reads its own coupling blocks tab[s].Sl, tab[s].Hl and
// energy tab[s].E + i tab[s].eta, and is skipped unless mask[s].
__global__ void __launch_bounds__(256) k_form_slice_rows_tab(int b, const SlotTab* __restrict__ tab,
                                                             const int* __restrict__ mask,
                                                             __nv_bfloat16* __restrict__ out, int Kp) {
    const int bi = blockIdx.y;
    if (!mask[bi]) return;
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= b) return;
    const SlotTab t = tab[bi];
    const float2 zr = df_from_double(t.E), zi = df_from_double(t.eta);
    const float4* Sr = t.Sl + (long)r * b;
    const float4* Hr = t.Hl + (long)r * b;
    form_slice_warp(
        b, lane, [&](int j) { return zsh_df(zr, zi, Sr[j], Hr[j]); },
        [&](int j, float4 v, int e) { put_row_slices(out, bi, b, r, Kp, j, v, e); });
}

__global__ void __launch_bounds__(256) k_form_slice_cols_dag_tab(int b, const SlotTab* __restrict__ tab,
                                                                 const int* __restrict__ mask,
                                                                 __nv_bfloat16* __restrict__ out, int Kp) {
    const int bi = blockIdx.y;
    if (!mask[bi]) return;
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= b) return;
    const SlotTab t = tab[bi];
    const float2 zr = df_from_double(t.E), zi = df_from_double(t.eta);
    const float4* Sc = t.Sl + (long)c * b;
    const float4* Hc = t.Hl + (long)c * b;
    form_slice_warp(
        b, lane, [&](int i) { return zsh_df(zr, zi, conj_df(Sc[i]), conj_df(Hc[i])); },
        [&](int i, float4 v, int e) { put_col_slices(out, bi, b, c, Kp, i, v, e); });
}

rgf_status form_slice_rows_tab(int S, int b, const SlotTab* tab, const int* mask, __nv_bfloat16* out, int Kp,
                               cudaStream_t st) {
    if (S <= 0) return RGF_OK;
    k_form_slice_rows_tab<<<dim3(ceil_div(b, 8), S), 256, 0, st>>>(b, tab, mask, out, Kp);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

rgf_status form_slice_cols_dag_tab(int S, int b, const SlotTab* tab, const int* mask, __nv_bfloat16* out, int Kp,
                                   cudaStream_t st) {
    if (S <= 0) return RGF_OK;
    k_form_slice_cols_dag_tab<<<dim3(ceil_div(b, 8), S), 256, 0, st>>>(b, tab, mask, out, Kp);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

rgf_status form_slice_rows(int W, int b, const double* E, double eta, const float4* S, const float4* H,
                           __nv_bfloat16* out, int Kp, cudaStream_t st) {
    if (W <= 0) return RGF_OK;
    k_form_slice_rows<<<dim3(ceil_div(b, 8), W), 256, 0, st>>>(b, E, eta, S, H, out, Kp);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

rgf_status form_slice_cols_dag(int W, int b, const double* E, double eta, const float4* S, const float4* H,
                               __nv_bfloat16* out, int Kp, cudaStream_t st) {
    if (W <= 0) return RGF_OK;
    k_form_slice_cols_dag<<<dim3(ceil_div(b, 8), W), 256, 0, st>>>(b, E, eta, S, H, out, Kp);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

rgf_status slice_rows(int batch, int m, int k, const float4* A, long sA, __nv_bfloat16* out, int Kp,
                      const int* active, cudaStream_t st, int planes) {
    if (batch <= 0) return RGF_OK;
    dim3 grid(ceil_div(m, 8), batch);
    k_slice_rows<<<grid, 256, 0, st>>>(m, k, A, sA, out, Kp, active, planes);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

// Two-pass column slicer for operands whose strip does not fit in shared
// memory (k above ~1400): one CTA per strip of 32 columns of one batch
// entry, first the column maxima (exponents) over all k rows, then 32 (j) x
// 32 (c) tiles through shared memory so that both the df reads (along c) and
// the slice writes (along j) are coalesced.  The second pass re-reads the
// strip.
__global__ void __launch_bounds__(256) k_slice_cols(int k, int n, const float4* __restrict__ B, long sB,
                                                    __nv_bfloat16* __restrict__ out, int Kp,
                                                    const int* __restrict__ active, int planes) {
    const int bi = blockIdx.y;
    if (active && !active[bi]) return;
    __shared__ float4 tile[32][33];
    __shared__ float cmax[8][32];
    __shared__ int cexp[32];
    const int c0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const float4* Bb = B + (long)bi * sB;
    {
        const int c = c0 + tx;
        float mx = 0.0f;
        if (c < n)
            for (int j = ty; j < k; j += 8) {
                const float4 v = Bb[(long)j * n + c];
                mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.z)));
            }
        cmax[ty][tx] = mx;
    }
    __syncthreads();
    if (ty == 0) {
        float mx = cmax[0][tx];
#pragma unroll
        for (int w = 1; w < 8; ++w) mx = fmaxf(mx, cmax[w][tx]);
        cexp[tx] = exp_above(mx);
    }
    const long rows = 2L * n;
    for (int j0 = 0; j0 < k; j0 += 32) {
        __syncthreads();
        for (int jj = ty; jj < 32; jj += 8) {
            const int j = j0 + jj, c = c0 + tx;
            tile[jj][tx] = (j < k && c < n) ? Bb[(long)j * n + c] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        for (int cc = ty; cc < 32; cc += 8) {
            const int c = c0 + cc, j = j0 + tx;
            if (c >= n || j >= k) continue;
            const float4 v = tile[tx][cc];
            const int e = cexp[cc];
            float sr[kSlices], si[kSlices];
            slice6(v.x, v.y, e, sr);
            slice6(v.z, v.w, e, si);
#pragma unroll
            for (int s = 0; s < kSlices; ++s) {
                if (s >= planes) break;
                __nv_bfloat16* base = out + (((long)bi * kSlices + s) * rows) * Kp;
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

struct DfStrip {
    static constexpr int kMinBlocks = 4;
    using T = float4;
    using M = float;
    static constexpr int NS = kSlices;
    __device__ static T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static M amax(const T& v) { return fmaxf(fabsf(v.x), fabsf(v.z)); }
    __device__ static M vmax(M a, M b) { return fmaxf(a, b); }
    __device__ static M shfl_xor(M v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
    __device__ static int expo(M m) { return exp_above(m); }
    __device__ static void split(const T& v, int e, float* sr, float* si) {
        slice6(v.x, v.y, e, sr);
        slice6(v.z, v.w, e, si);
    }
};

rgf_status slice_cols(int batch, int k, int n, const float4* B, long sB, __nv_bfloat16* out, int Kp,
                      const int* active, cudaStream_t st, int planes) {
    if (batch <= 0) return RGF_OK;
    if (strip_fits(k)) {
        static std::atomic<bool> attr{false};
        if (!attr.load()) {
            // Idempotent: threads that race here all set the same value.
            RGF_CUDA_TRY(cudaFuncSetAttribute(k_slice_cols_strip<DfStrip>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, kStripMaxSmem));
            attr.store(true);
        }
        k_slice_cols_strip<DfStrip><<<dim3(ceil_div(n, kStripCols), batch), kStripCols * 32, strip_smem_bytes(k),
                                      st>>>(k, n, B, sB, out, Kp, active, planes);
        RGF_LAUNCH_CHECK();
        return RGF_OK;
    }
    k_slice_cols<<<dim3(ceil_div(n, 32), batch), 256, 0, st>>>(k, n, B, sB, out, Kp, active, planes);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

// ------------------------------------------------------------------ epilogue
// Combine the group sums of one real output into a df value: groups 0..3
// (each about 2^-8 of the previous) through exact TwoSums, the tail group
// into the low word.
__device__ __forceinline__ float2 combine_groups(const float* g) {
    const float2 s = two_sum(g[0], g[1]);
    const float2 t = two_sum(s.x, g[2]);
    const float2 u = two_sum(t.x, g[3]);
    float lo = s.y + t.y;
    lo += u.y;
    lo += g[4];
    return fast_two_sum(u.x, lo);
}

__device__ __forceinline__ float4 oz_finish(const OzGemm& g, int bi, int r, int c, float2 re, float2 im) {
    if (g.alpha < 0.0f) {
        re = df_neg(re);
        im = df_neg(im);
    }
    if (g.D) {
        const float4 d = g.D[(long)bi * g.sD + (long)r * g.n + c];
        re = df_add(re, re_of(d));
        im = df_add(im, im_of(d));
    }
    if (g.add_identity && r == c) re = df_add(re, make_float2(1.0f, 0.0f));
    return cdf(re, im);
}

// ------------------------------------------------------------------ mma.sync core
// 64 x 64 real output tile per CTA, 8 warps of 32 x 16, K chunk 32.
constexpr int MM_BM = 64, MM_BN = 64, MM_BK = 32, MM_PITCH = 40;

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(256) k_oz_mma(OzGemm g) {
    const int bi = blockIdx.z;
    if (g.active && !g.active[bi]) return;
    extern __shared__ __align__(16) unsigned char smem_mm[];
    __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem_mm);   // [6][64][40]
    __nv_bfloat16* Bs = As + kSlices * MM_BM * MM_PITCH;               // [6][64][40]
    const int m0 = blockIdx.y * MM_BM, n0 = blockIdx.x * MM_BN;        // n0 in real columns
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int wm = w >> 2, wn = w & 3;
    const int gq = lane >> 2, tq = lane & 3;
    const long rowsB = 2L * g.n;
    float acc[kGroups][2][2][4];
#pragma unroll
    for (int a = 0; a < kGroups; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int d = 0; d < 4; ++d) acc[a][b][c][d] = 0.0f;

    const __nv_bfloat16* Ab = g.As + (long)bi * kSlices * g.m * g.Kp;
    const __nv_bfloat16* Bb = g.Bs + (long)bi * kSlices * rowsB * g.Kp;
    for (int kc = 0; kc < g.Kp; kc += MM_BK) {
        // 6 slices x 64 rows x 32 elements = 1536 16-byte pieces per operand.
        for (int i = tid; i < kSlices * MM_BM * 4; i += blockDim.x) {
            const int s = i / (MM_BM * 4), rem = i % (MM_BM * 4), r = rem >> 2, q = rem & 3;
            uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
            if (m0 + r < g.m)
                va = *reinterpret_cast<const uint4*>(Ab + ((long)s * g.m + m0 + r) * g.Kp + kc + q * 8);
            if (n0 + r < rowsB)
                vb = *reinterpret_cast<const uint4*>(Bb + ((long)s * rowsB + n0 + r) * g.Kp + kc + q * 8);
            *reinterpret_cast<uint4*>(As + (s * MM_BM + r) * MM_PITCH + q * 8) = va;
            *reinterpret_cast<uint4*>(Bs + (s * MM_BN + r) * MM_PITCH + q * 8) = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < MM_BK; kk += 16) {
#pragma unroll
            for (int si = 0; si < kSlices; ++si) {
                uint32_t af[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const __nv_bfloat16* base = As + (si * MM_BM + wm * 32 + mt * 16 + gq) * MM_PITCH + kk + 2 * tq;
                    af[mt][0] = *reinterpret_cast<const uint32_t*>(base);
                    af[mt][1] = *reinterpret_cast<const uint32_t*>(base + 8 * MM_PITCH);
                    af[mt][2] = *reinterpret_cast<const uint32_t*>(base + 8);
                    af[mt][3] = *reinterpret_cast<const uint32_t*>(base + 8 * MM_PITCH + 8);
                }
#pragma unroll
                for (int sj = 0; sj < kSlices; ++sj) {
                    if (si + sj > kSlices - 1) continue;
                    const int grp = (si + sj) < (kGroups - 1) ? (si + sj) : (kGroups - 1);
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) {
                        const __nv_bfloat16* bb = Bs + (sj * MM_BN + wn * 16 + nt * 8 + gq) * MM_PITCH + kk + 2 * tq;
                        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(bb);
                        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(bb + 8);
#pragma unroll
                        for (int mt = 0; mt < 2; ++mt) mma_bf16(acc[grp][mt][nt], af[mt], b0, b1);
                    }
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int r = m0 + wm * 32 + mt * 16 + gq + half * 8;
            if (r >= g.m) continue;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int col = n0 + wn * 16 + nt * 8 + 2 * tq;  // even real column
                const int c = col >> 1;
                if (c >= g.n) continue;
                float gr[kGroups], gi[kGroups];
#pragma unroll
                for (int q = 0; q < kGroups; ++q) {
                    gr[q] = acc[q][mt][nt][2 * half];
                    gi[q] = acc[q][mt][nt][2 * half + 1];
                }
                g.C[(long)bi * g.sC + (long)r * g.n + c] = oz_finish(g, bi, r, c, combine_groups(gr), combine_groups(gi));
            }
        }
    }
}

rgf_status oz_gemm_mma(const OzGemm& g, cudaStream_t st) {
    if (g.batch <= 0) return RGF_OK;
    const size_t smem = 2ull * kSlices * MM_BM * MM_PITCH * sizeof(__nv_bfloat16);
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        RGF_CUDA_TRY(cudaFuncSetAttribute(k_oz_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr.store(true);
    }
    dim3 grid(ceil_div(2L * g.n, MM_BN), ceil_div(g.m, MM_BM), g.batch);
    k_oz_mma<<<grid, 256, smem, st>>>(g);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

rgf_status oz_gemm(const OzGemm& g, int core, cudaStream_t st) {
    return core == 1 ? oz_gemm_mma(g, st) : oz_gemm_tc(g, st);
}

// ------------------------------------------------------------------ elementwise
__global__ void k_to_dfc(long n, const double2* __restrict__ src, float4* __restrict__ dst) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double2 v = src[i];
        dst[i] = cdf(df_from_double(v.x), df_from_double(v.y));
    }
}

rgf_status to_dfc(long n, const double2* src, float4* dst, cudaStream_t st) {
    if (n <= 0) return RGF_OK;
    k_to_dfc<<<grid_for2(n, 256, 4096), 256, 0, st>>>(n, src, dst);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_form_dfc(int W, int b, const double* __restrict__ E, double eta, FormSrcDf src,
                           float4* __restrict__ out, const float4* __restrict__ sub, const int* __restrict__ active) {
    const int be = blockIdx.y;
    if (active && !active[be]) return;
    const int s = be / W, e = be % W;
    const float2 zr = df_from_double(E[e]);
    const float2 zi = df_from_double(eta);
    const float4* S = src.S[s];
    const float4* H = src.H[s];
    const int tr = src.trans[s];
    const long nn = (long)b * b;
    float4* o = out + (long)be * nn;
    const float4* sb = sub ? sub + (long)be * nn : nullptr;
    // One warp per row, lanes along the columns (no index division).
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int r = blockIdx.x * warps + (threadIdx.x >> 5); r < b; r += gridDim.x * warps) {
        for (int c = lane; c < b; c += 32) {
            const long idx = (long)r * b + c;
            const long si = tr ? (long)c * b + r : idx;
            float4 sv = S ? S[si] : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 hv = H[si];
            if (tr) {
                sv.z = -sv.z;
                sv.w = -sv.w;
                hv.z = -hv.z;
                hv.w = -hv.w;
            }
            // (zr + i zi)(Sr + i Si) - (Hr + i Hi)
            const float2 sr = re_of(sv), sim = im_of(sv);
            float2 re = df_sub(df_sub(df_mul(zr, sr), df_mul(zi, sim)), re_of(hv));
            float2 im = df_sub(df_add(df_mul(zr, sim), df_mul(zi, sr)), im_of(hv));
            if (sb) {
                const float4 d = sb[idx];
                re = df_sub(re, re_of(d));
                im = df_sub(im, im_of(d));
            }
            o[idx] = cdf(re, im);
        }
    }
}

rgf_status form_dfc(int W, int nsrc, int b, const double* E, double eta, const FormSrcDf& src, float4* out,
                    const float4* sub, const int* active, cudaStream_t st) {
    if (W <= 0) return RGF_OK;
    k_form_dfc<<<dim3(ceil_div(b, 8), W * nsrc), 256, 0, st>>>(W, b, E, eta, src, out, sub,
                                                                                  active);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_dfc_hi_to_c64(int b, const float4* X, float2* Y, const int* active) {
    if (active && !active[blockIdx.y]) return;
    const long nn = (long)b * b, off = (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const float4 v = X[off + i];
        Y[off + i] = make_float2(v.x + v.y, v.z + v.w);
    }
}

rgf_status dfc_hi_to_c64(int batch, int b, const float4* X, float2* Y, const int* active, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_dfc_hi_to_c64<<<dim3(grid_for2((long)b * b, 256, 64), batch), 256, 0, st>>>(b, X, Y, active);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_c64_to_dfc(int b, const float2* X, float4* Y, const int* active) {
    if (active && !active[blockIdx.y]) return;
    const long nn = (long)b * b, off = (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const float2 v = X[off + i];
        Y[off + i] = make_float4(v.x, 0.f, v.y, 0.f);
    }
}

rgf_status c64_to_dfc(int batch, int b, const float2* X, float4* Y, const int* active, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_c64_to_dfc<<<dim3(grid_for2((long)b * b, 256, 64), batch), 256, 0, st>>>(b, X, Y, active);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_copy_dfc(int b, float4* dst, const float4* src, const int* active) {
    if (active && !active[blockIdx.y]) return;
    const long nn = (long)b * b, off = (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x)
        dst[off + i] = src[off + i];
}

rgf_status copy_dfc(int batch, int b, float4* dst, const float4* src, const int* active, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_copy_dfc<<<dim3(grid_for2((long)b * b, 256, 64), batch), 256, 0, st>>>(b, dst, src, active);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_identity_dfc(int b, float4* A) {
    const long nn = (long)b * b;
    float4* Ab = A + (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x)
        Ab[i] = make_float4((i / b) == (i % b) ? 1.f : 0.f, 0.f, 0.f, 0.f);
}

rgf_status set_identity_dfc(int batch, int b, float4* A, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_identity_dfc<<<dim3(grid_for2((long)b * b, 256, 64), batch), 256, 0, st>>>(b, A);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_dec_update_dfc(int b, float4* eps_s, float4* eps, const float4* agb, const float4* bga,
                                 const int* active) {
    if (active && !active[blockIdx.y]) return;
    const long nn = (long)b * b, off = (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const float4 x = agb[off + i], y = bga[off + i];
        eps_s[off + i] = cdf_sub(eps_s[off + i], x);
        eps[off + i] = cdf_sub(cdf_sub(eps[off + i], x), y);
    }
}

rgf_status dec_update_dfc(int batch, int b, float4* eps_s, float4* eps, const float4* agb, const float4* bga,
                          const int* active, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_dec_update_dfc<<<dim3(grid_for2((long)b * b, 256, 64), batch), 256, 0, st>>>(b, eps_s, eps, agb, bga,
                                                                                     active);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__device__ double block_sum_d(double v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;
}

// Sum of squares in FP32 per thread (the values only decide a stopping
// test or a norm estimate), reduced in FP64.
__global__ void k_dec_check_dfc(int b, const float4* alpha, const float4* beta, const double* anorm, double tol,
                                int it, int* active, int* iters, int* remaining) {
    const int bi = blockIdx.x;
    if (!active[bi]) return;
    __shared__ double sh[32];
    const long nn = (long)b * b, off = (long)bi * nn;
    float sa = 0.f, sb = 0.f;
    for (long i = threadIdx.x; i < nn; i += blockDim.x) {
        const float4 a = alpha[off + i], c = beta[off + i];
        sa = fmaf(a.x, a.x, fmaf(a.z, a.z, sa));
        sb = fmaf(c.x, c.x, fmaf(c.z, c.z, sb));
    }
    const double ta = block_sum_d((double)sa, sh);
    const double tb = block_sum_d((double)sb, sh);
    if (threadIdx.x == 0) {
        iters[bi] = it;
        const double lim = tol * anorm[bi];
        if (sqrt(ta) <= lim && sqrt(tb) <= lim)
            active[bi] = 0;
        else
            atomicAdd(remaining, 1);
    }
}

rgf_status dec_check_dfc(int batch, int b, const float4* alpha, const float4* beta, const double* anorm, double tol,
                         int it, int* active, int* iters, int* remaining, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_dec_check_dfc<<<batch, 256, 0, st>>>(b, alpha, beta, anorm, tol, it, active, iters, remaining);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_fro_norm_dfc(int b, const float4* A, double* out) {
    __shared__ double sh[32];
    const long nn = (long)b * b, off = (long)blockIdx.x * nn;
    float s = 0.f;
    for (long i = threadIdx.x; i < nn; i += blockDim.x) {
        const float4 a = A[off + i];
        s = fmaf(a.x, a.x, fmaf(a.z, a.z, s));
    }
    const double t = block_sum_d((double)s, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = sqrt(t);
}

rgf_status fro_norm_dfc(int batch, int b, const float4* A, double* out, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_fro_norm_dfc<<<batch, 256, 0, st>>>(b, A, out);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_gamma_dfc(int b, const float4* sigma, float4* gamma) {
    const long nn = (long)b * b, off = (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / b), c = (int)(i % b);
        const float4 s = sigma[off + i];
        const float4 t = sigma[off + (long)c * b + r];
        // i (s - conj(t)) = -(s.im + t.im) + i (s.re - t.re)
        const float2 re = df_neg(df_add(im_of(s), im_of(t)));
        const float2 im = df_sub(re_of(s), re_of(t));
        gamma[off + i] = cdf(re, im);
    }
}

rgf_status gamma_dfc(int batch, int b, const float4* sigma, float4* gamma, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_gamma_dfc<<<dim3(grid_for2((long)b * b, 256, 64), batch), 256, 0, st>>>(b, sigma, gamma);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_axpy_dfc(int b, float alpha, const float4* X, float4* Y) {
    const long nn = (long)b * b, off = (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        float4 x = X[off + i];
        if (alpha < 0.f) x = make_float4(-x.x, -x.y, -x.z, -x.w);
        Y[off + i] = cdf_add(Y[off + i], x);
    }
}

rgf_status axpy_dfc(int batch, int b, float alpha, const float4* X, float4* Y, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_axpy_dfc<<<dim3(grid_for2((long)b * b, 256, 64), batch), 256, 0, st>>>(b, alpha, X, Y);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_ns_check(int W, int b, const float4* R, double* err, int* flags, int step, int max_steps,
                           const int* act, int* next_act, int* bad, int* bad_count, double2* theta,
                           int* more_count, double tol, const float* rsq, const double2* rtr) {
    const int bi = blockIdx.x;
    if (act && !act[bi]) {
        if (threadIdx.x == 0) {
            next_act[bi] = 0;
            if (step <= 1) bad[bi] = 0;
            if (step == 0) theta[bi] = make_double2(1.0, 0.0);
        }
        return;
    }
    __shared__ double sh[32];
    const long nn = (long)b * b, off = (long)bi * nn;
    double s = 0.0;
    double tr_re = 0.0, tr_im = 0.0;
    if (rsq) {
        // The residual GEMM's per-block sums, added in a fixed order.
        const int ns = rstat_slots(b);
        for (int i = threadIdx.x; i < ns; i += blockDim.x) s += (double)rsq[(long)bi * ns + i];
        if (step == 0 && rtr)
            for (int i = threadIdx.x; i < ns; i += blockDim.x) {
                const double2 v = rtr[(long)bi * ns + i];
                tr_re += v.x;
                tr_im += v.y;
            }
    } else {
        float sf = 0.f;
        for (long i = threadIdx.x; i < nn; i += blockDim.x) {
            const float4 a = R[off + i];
            sf = fmaf(a.x, a.x, fmaf(a.z, a.z, sf));
        }
        s = (double)sf;
        if (step == 0) {
            for (int i = threadIdx.x; i < b; i += blockDim.x) {
                const float4 a = R[off + (long)i * b + i];
                tr_re += df_to_double(re_of(a));
                tr_im += df_to_double(im_of(a));
            }
        }
    }
    const double t = sqrt(block_sum_d(s, sh));
    if (step == 0) {
        tr_re = block_sum_d(tr_re, sh);
        tr_im = block_sum_d(tr_im, sh);
    }
    if (threadIdx.x == 0) {
        const int e = bi % W;
        const bool num_ok = isfinite(t);
        if (step == 0) {
            // A seed that does not contract near a resonance has R = I - M X0
            // dominated by one rank-1 term u v^H whose eigenvalue is about
            // tr R; then (I - R)^-1 = I + R / (1 - tr R) (Sherman-Morrison) and
            // the first correction is scaled by theta = 1 / (1 - tr R).  Other
            // seeds keep theta = 1.
            double2 th = make_double2(1.0, 0.0);
            if (num_ok && t >= 0.5) {
                const double dr = 1.0 - tr_re, di = -tr_im, d2 = dr * dr + di * di;
                if (d2 > 1e-12) th = make_double2(dr / d2, -di / d2);
            }
            theta[bi] = th;
        }
        if (step == 1) {
            // Entries that still do not contract are reseeded in FP64.
            const bool is_bad = (!num_ok) || (t >= 0.5);
            bad[bi] = is_bad ? 1 : 0;
            if (is_bad) {
                atomicAdd(bad_count, 1);
                atomicOr(flags + e, RGF_FLAG_REFINE);
            }
        }
        const bool more = !(t <= tol);
        next_act[bi] = more ? 1 : 0;
        if (more && more_count) atomicAdd(more_count, 1);
        if (more && step == max_steps - 1) atomicOr(flags + e, RGF_FLAG_REFINE);
        // Error estimate of the finished inverse: after this step's correction
        // the residual is about t^2; an entry that never got there reports
        // its last residual.
        double est = -1.0;
        if (!more) est = t * t;
        else if (step == max_steps - 1) est = num_ok ? t : 1e300;
        if (est >= 0.0)
            atomicMax(reinterpret_cast<unsigned long long*>(err + e), (unsigned long long)__double_as_longlong(est));
    }
}

rgf_status ns_check(int batch, int W, int b, const float4* R, double* err, int* flags, int step, int max_steps,
                    const int* act, int* next_act, int* bad, int* bad_count, double2* theta, cudaStream_t st,
                    int* more_count, const float* rsq, const double2* rtr) {
    if (batch <= 0) return RGF_OK;
    k_ns_check<<<batch, 256, 0, st>>>(W, b, R, err, flags, step, max_steps, act, next_act, bad, bad_count, theta,
                                      more_count, kNsTol, rsq, rtr);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

// Same bookkeeping as k_ns_check for an FP64 residual.
__global__ void k_ns_check_f64(int W, int b, const double2* R, double* err, int* flags, int step, int max_steps,
                               const int* act, int* next_act, int* bad, int* bad_count, int* more_count) {
    const int bi = blockIdx.x;
    if (act && !act[bi]) {
        if (threadIdx.x == 0) {
            next_act[bi] = 0;
            if (step == 0) bad[bi] = 0;
        }
        return;
    }
    __shared__ double sh[32];
    const long nn = (long)b * b, off = (long)bi * nn;
    double s = 0.0;
    for (long i = threadIdx.x; i < nn; i += blockDim.x) {
        const double2 a = R[off + i];
        s += a.x * a.x + a.y * a.y;
    }
    const double t = sqrt(block_sum_d(s, sh));
    if (threadIdx.x == 0) {
        const int e = bi % W;
        const bool num_ok = isfinite(t);
        if (step == 0) {
            const bool is_bad = (!num_ok) || (t >= kHpBad);
            bad[bi] = is_bad ? 1 : 0;
            if (is_bad) {
                atomicAdd(bad_count, 1);
                atomicOr(flags + e, RGF_FLAG_REFINE);
            }
        }
        const bool more = !(t <= 3e-7);
        next_act[bi] = more ? 1 : 0;
        if (more && more_count) atomicAdd(more_count, 1);
        if (more && step == max_steps - 1) atomicOr(flags + e, RGF_FLAG_REFINE);
    }
}

rgf_status ns_check_f64(int batch, int W, int b, const double2* R, double* err, int* flags, int step, int max_steps,
                        const int* act, int* next_act, int* bad, int* bad_count, cudaStream_t st, int* more_count) {
    if (batch <= 0) return RGF_OK;
    k_ns_check_f64<<<batch, 256, 0, st>>>(W, b, R, err, flags, step, max_steps, act, next_act, bad, bad_count,
                                          more_count);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_c128_to_c64(int b, const double2* X, float2* Y, const int* mask) {
    if (mask && !mask[blockIdx.y]) return;
    const long nn = (long)b * b, off = (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const double2 v = X[off + i];
        Y[off + i] = make_float2((float)v.x, (float)v.y);
    }
}

rgf_status c128_to_c64(int batch, int b, const double2* X, float2* Y, const int* mask, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_c128_to_c64<<<dim3(grid_for2((long)b * b, 256, 64), batch), 256, 0, st>>>(b, X, Y, mask);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_c64_to_c128(int b, const float2* X, double2* Y, const int* mask) {
    if (mask && !mask[blockIdx.y]) return;
    const long nn = (long)b * b, off = (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const float2 v = X[off + i];
        Y[off + i] = make_double2(v.x, v.y);
    }
}

rgf_status c64_to_c128(int batch, int b, const float2* X, double2* Y, const int* mask, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_c64_to_c128<<<dim3(grid_for2((long)b * b, 256, 64), batch), 256, 0, st>>>(b, X, Y, mask);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_dfc_to_c128(int b, const float4* X, double2* Y, const int* mask) {
    if (mask && !mask[blockIdx.y]) return;
    const long nn = (long)b * b, off = (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const float4 v = X[off + i];
        Y[off + i] = make_double2(df_to_double(re_of(v)), df_to_double(im_of(v)));
    }
}

rgf_status dfc_to_c128(int batch, int b, const float4* X, double2* Y, const int* mask, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_dfc_to_c128<<<dim3(grid_for2((long)b * b, 256, 64), batch), 256, 0, st>>>(b, X, Y, mask);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_c128_to_dfc(int b, const double2* X, float4* Y, const int* mask) {
    if (mask && !mask[blockIdx.y]) return;
    const long nn = (long)b * b, off = (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const double2 v = X[off + i];
        Y[off + i] = cdf(df_from_double(v.x), df_from_double(v.y));
    }
}

rgf_status c128_to_dfc(int batch, int b, const double2* X, float4* Y, const int* mask, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_c128_to_dfc<<<dim3(grid_for2((long)b * b, 256, 64), batch), 256, 0, st>>>(b, X, Y, mask);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_scale_theta(int b, float4* R, const double2* theta, const int* act) {
    const int bi = blockIdx.y;
    if (act && !act[bi]) return;
    const double2 th = theta[bi];
    if (th.x == 1.0 && th.y == 0.0) return;
    const float4 tf = cdf(df_from_double(th.x), df_from_double(th.y));
    const long nn = (long)b * b, off = (long)bi * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x)
        R[off + i] = cdf_mul(R[off + i], tf);
}

rgf_status scale_theta(int batch, int b, float4* R, const double2* theta, const int* act, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_scale_theta<<<dim3(grid_for2((long)b * b, 256, 64), batch), 256, 0, st>>>(b, R, theta, act);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_mask_init(int batch, const int* act, int* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < batch) out[i] = act ? act[i] : 1;
}

rgf_status mask_init(int batch, const int* act, int* out, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_mask_init<<<ceil_div(batch, 256), 256, 0, st>>>(batch, act, out);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

// Second look at FP64 inverses whose seed was replaced by a nearby inverse:
// for mask entries, still_bad = (|R|_F >= kHpBad or not finite), counted into
// *count, and next_act = |R|_F > 3e-7 (or still bad); other entries keep
// next_act and get still_bad = 0.
__global__ void k_recheck_f64(int b, const double2* R, const int* mask, int* still_bad, int* count, int* next_act) {
    const int bi = blockIdx.x;
    if (!mask[bi]) {
        if (threadIdx.x == 0) still_bad[bi] = 0;
        return;
    }
    __shared__ double sh[32];
    const long nn = (long)b * b, off = (long)bi * nn;
    double s = 0.0;
    for (long i = threadIdx.x; i < nn; i += blockDim.x) {
        const double2 a = R[off + i];
        s += a.x * a.x + a.y * a.y;
    }
    const double t = sqrt(block_sum_d(s, sh));
    if (threadIdx.x == 0) {
        const bool sb = !(isfinite(t) && t < kHpBad);
        still_bad[bi] = sb ? 1 : 0;
        if (sb) atomicAdd(count, 1);
        next_act[bi] = (sb || t > 3e-7) ? 1 : 0;
    }
}

rgf_status recheck_f64(int batch, int b, const double2* R, const int* mask, int* still_bad, int* count,
                       int* next_act, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_recheck_f64<<<batch, 256, 0, st>>>(b, R, mask, still_bad, count, next_act);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_accumulate_count(long long* acc, const int* count) { *acc += *count; }

rgf_status accumulate_count(long long* acc, const int* count, cudaStream_t st) {
    k_accumulate_count<<<1, 1, 0, st>>>(acc, count);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_trace_dfc(int b, const float4* X, const float4* Y, double* T, double* Ti) {
    __shared__ double sh[32];
    const long nn = (long)b * b, off = (long)blockIdx.x * nn;
    double re = 0.0, im = 0.0;
    for (long i = threadIdx.x; i < nn; i += blockDim.x) {
        const float4 x4 = X[off + i], y4 = Y[off + i];
        const double xr = df_to_double(re_of(x4)), xi = df_to_double(im_of(x4));
        const double yr = df_to_double(re_of(y4)), yi = df_to_double(im_of(y4));
        re += xr * yr + xi * yi;
        im += xi * yr - xr * yi;
    }
    const double tr = block_sum_d(re, sh);
    const double ti = block_sum_d(im, sh);
    if (threadIdx.x == 0) {
        T[blockIdx.x] = tr;
        if (Ti) Ti[blockIdx.x] = ti;
    }
}

rgf_status trace_dfc(int batch, int b, const float4* X, const float4* Y, double* T, double* Ti, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_trace_dfc<<<batch, 256, 0, st>>>(b, X, Y, T, Ti);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

}  // namespace rgf
