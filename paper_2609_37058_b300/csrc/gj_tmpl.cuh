// Batched complex GEMM and blocked Gauss-Jordan inverse on the CUDA cores,
// templated on the complex element type (double2 for the FP64 path, float2
// for the FP32 seed inverse of the mixed path).
#pragma once

#include <atomic>
#include <mutex>
#include <type_traits>
#include <vector>

#include "kernels.h"

namespace rgf {

template <typename T2> struct CT;
template <> struct CT<double2> {
    using R = double;
    static __host__ __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};
template <> struct CT<float2> {
    using R = float;
    static __host__ __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
};

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// Raises a kernel's dynamic shared-memory limit once per function pointer.
// A kernel template instantiated from this header in several translation
// units is registered once per unit, and a launch uses its own unit's
// registration, so the limit is tracked per pointer, not per kernel.
inline rgf_status smem_limit_once(const void* fn, int bytes) {
    static std::mutex mu;
    static std::vector<const void*> done;
    std::lock_guard<std::mutex> lock(mu);
    for (const void* f : done)
        if (f == fn) return RGF_OK;
    RGF_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done.push_back(fn);
    return RGF_OK;
}

// x = o[0] + o[1] + o[2] within 2^-24 |x|: each BF16 value is the rounded
// remainder, and the remainders x - o[0] and x - o[0] - o[1] are exact in FP32.
__device__ __forceinline__ void split3_bf16(float x, __nv_bfloat16 (&o)[kGjSplits]) {
    o[0] = __float2bfloat16_rn(x);
    float r = x - __bfloat162float(o[0]);
    o[1] = __float2bfloat16_rn(r);
    r -= __bfloat162float(o[1]);
    o[2] = __float2bfloat16_rn(r);
}
__device__ __forceinline__ void store_bf2(__nv_bfloat16* p, __nv_bfloat16 x, __nv_bfloat16 y) {
    __nv_bfloat162 v;
    v.x = x;
    v.y = y;
    *reinterpret_cast<__nv_bfloat162*>(p) = v;
}

// 64 x 64 complex output tile per CTA, K step 16, 256 threads each owning a
// 4 x 4 set of outputs strided by 16 so shared-memory reads are broadcasts
// (A) or consecutive (B).
constexpr int ZG_BM = 64, ZG_BN = 64, ZG_BK = 16;

template <typename T2>
__global__ void __launch_bounds__(256) k_zgemm(GemmArgs<T2> g) {
    using C = CT<T2>;
    const int bi = blockIdx.z;
    if (g.active && !g.active[bi]) return;
    const int m0 = blockIdx.y * ZG_BM, n0 = blockIdx.x * ZG_BN;
    if (n0 >= g.skip0 && n0 + ZG_BN <= g.skip1) return;
    const T2* __restrict__ A = g.A + (long)bi * g.sA;
    const T2* __restrict__ B = g.B + (long)bi * g.sB;
    __shared__ T2 As[ZG_BK][ZG_BM];
    __shared__ T2 Bs[ZG_BK][ZG_BN];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    T2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = C::make(0, 0);

    for (int k0 = 0; k0 < g.k; k0 += ZG_BK) {
#pragma unroll
        for (int t = 0; t < (ZG_BM * ZG_BK) / 256; ++t) {
            const int i = tid + t * 256;
            const int r = i / ZG_BK, kk = i % ZG_BK;
            const int gr = m0 + r, gk = k0 + kk;
            As[kk][r] = (gr < g.m && gk < g.k) ? A[(long)gr * g.lda + gk] : C::make(0, 0);
        }
#pragma unroll
        for (int t = 0; t < (ZG_BK * ZG_BN) / 256; ++t) {
            const int i = tid + t * 256;
            const int kk = i / ZG_BN, c = i % ZG_BN;
            const int gk = k0 + kk, gc = n0 + c;
            Bs[kk][c] = (gk < g.k && gc < g.n) ? B[(long)gk * g.ldb + gc] : C::make(0, 0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < ZG_BK; ++kk) {
            T2 a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], bb[j]);
        }
        __syncthreads();
    }
    const T2* Cin = g.Cin ? g.Cin + (long)bi * g.sCin : nullptr;
    T2* Cp = g.C + (long)bi * g.sC;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = m0 + ty + 16 * i;
        if (r >= g.m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = n0 + tx + 16 * j;
            if (c >= g.n || (c >= g.skip0 && c < g.skip1)) continue;
            T2 v = cmul(g.alpha, acc[i][j]);
            if (Cin) v = cadd(v, cmul(g.beta, Cin[(long)r * g.ldcin + c]));
            Cp[(long)r * g.ldc + c] = v;
        }
    }
}

template <typename T2>
rgf_status zgemm_t(const GemmArgs<T2>& g, cudaStream_t st) {
    if (g.batch <= 0 || g.m <= 0 || g.n <= 0) return RGF_OK;
    if (g.batch > 65535) {
        set_error("zgemm: batch %d > 65535", g.batch);
        return RGF_E_INVALID;
    }
    dim3 grid(ceil_div(g.n, ZG_BN), ceil_div(g.m, ZG_BM), g.batch);
    k_zgemm<T2><<<grid, 256, 0, st>>>(g);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

// Trailing update of the FP32 Gauss-Jordan inverse: C += A B for one batch
// entry per blockIdx.z, with A m x K (K <= 32, row-major, lda = K), B K x n
// (row-major, ldb = ldc) and columns [skip0, skip1) of C left alone.  K is
// small, so the whole A and B tiles are staged in shared memory at once; a
// CTA owns 128 x 64 complex outputs, a thread 8 x 4 of them.
constexpr int GU_BM = 128, GU_BN = 64, GU_KMAX = 32, GU_AP = GU_KMAX + 1;
constexpr size_t GU_SMEM = (size_t)(GU_BM * GU_AP + GU_KMAX * GU_BN) * sizeof(float2);

static __global__ void __launch_bounds__(256) k_gj_update_f32(int m, int n, int K, const float2* __restrict__ A, long sA,
                                                       const float2* __restrict__ B, long sB, float2* C, long ldc,
                                                       long sC, int skip0, int skip1, const int* active) {
    const int bi = blockIdx.z;
    if (active && !active[bi]) return;
    const int m0 = blockIdx.y * GU_BM, n0 = blockIdx.x * GU_BN;
    if (n0 >= skip0 && n0 + GU_BN <= skip1) return;
    extern __shared__ __align__(16) unsigned char gu_smem[];
    float2* As = reinterpret_cast<float2*>(gu_smem);  // [GU_BM][GU_AP]
    float2* Bs = As + GU_BM * GU_AP;                   // [GU_KMAX][GU_BN]
    const float2* Ab = A + (long)bi * sA;
    const float2* Bb = B + (long)bi * sB;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    float2* Cb = C + (long)bi * sC;
    // The accumulators start from C: its loads are issued first and are in
    // flight while A and B are staged.
    float2 acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = m0 + ty + 16 * i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = n0 + tx + 16 * j;
            acc[i][j] = (r < m && c < n) ? Cb[(long)r * ldc + c] : make_float2(0.f, 0.f);
        }
    }
    for (int i = tid; i < GU_BM * K; i += 256) {
        const int r = i / K, k = i - r * K;
        As[r * GU_AP + k] = (m0 + r < m) ? Ab[(long)(m0 + r) * K + k] : make_float2(0.f, 0.f);
    }
    for (int i = tid; i < K * GU_BN; i += 256) {
        const int k = i / GU_BN, c = i - k * GU_BN;
        Bs[k * GU_BN + c] = (n0 + c < n) ? Bb[(long)k * ldc + n0 + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int k = 0; k < K; ++k) {
        float2 a[8], b[4];
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = As[(ty + 16 * i) * GU_AP + k];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[k * GU_BN + tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = m0 + ty + 16 * i;
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = n0 + tx + 16 * j;
            if (c >= n || (c >= skip0 && c < skip1)) continue;
            Cb[(long)r * ldc + c] = acc[i][j];
        }
    }
}

static rgf_status gj_update_f32(int batch, int m, int n, int K, const float2* A, long sA, const float2* B, long sB,
                                float2* C, long ldc, long sC, int skip0, int skip1, const int* active,
                                cudaStream_t st) {
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        RGF_CUDA_TRY(cudaFuncSetAttribute(k_gj_update_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GU_SMEM));
        attr.store(true);
    }
    dim3 grid(ceil_div(n, GU_BN), ceil_div(m, GU_BM), batch);
    k_gj_update_f32<<<grid, 256, GU_SMEM, st>>>(m, n, K, A, sA, B, sB, C, ldc, sC, skip0, skip1, active);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

// ------------------------------------------------------------------ inverse
// Blocked Gauss-Jordan with partial pivoting, in place.  For each panel of
// nb columns K = [k0, k0+nb):
//  1. panel kernel: unblocked in-place Gauss-Jordan on the b x nb panel
//     (pivot search among the rows not yet used as pivots, row swaps inside
//     the panel), giving [-A_0K A_KK^-1; A_KK^-1; -A_2K A_KK^-1]; it also
//     writes Pbar = that panel minus the identity on the K x K block;
//  2. swap kernel: applies the panel's row swaps to the other columns and
//     copies rows K of those columns into T (nb x b);
//  3. GEMM: A[:, not K] += Pbar T.
// At the end the column interchanges are undone in reverse order.
static inline int gj_nb(int b) { return b <= 320 ? (b < 32 ? b : 32) : 16; }

template <typename T2>
size_t inv_workspace_bytes_t(int batch, int b) {
    // Pbar (b x nb) and T (nb x b) per matrix, plus pivots.
    const int nb = gj_nb(b);
    return (size_t)batch * ((size_t)b * nb * sizeof(T2) * 2 + (size_t)b * sizeof(int)) + 256;
}

template <typename R>
__device__ __forceinline__ void argmax_merge(R& v, int& i, R v2, int i2) {
    if (v2 > v || (v2 == v && i2 < i)) {
        v = v2;
        i = i2;
    }
}

template <typename T2>
__device__ __forceinline__ T2 shfl_c(T2 v, int src) {
    v.x = __shfl_sync(0xffffffffu, v.x, src);
    v.y = __shfl_sync(0xffffffffu, v.y, src);
    return v;
}

// Panel kernel: 256 threads; lane = panel column (NB <= 32), warp w owns
// rows w, w + 8, ...  The panel lives in shared memory with a row pitch of
// NB + 1 elements; the pivot column is copied to a separate array (fcol) so
// that the rank-1 update reads and writes never alias and can be pipelined.
// One pivot step: all threads merge the warps' pivot candidates; warp 0
// swaps and scales the pivot row while the other warps copy their part of
// the pivot column; barrier; rank-1 update without branches between lanes;
// barrier; search of the next column by all 256 threads; barrier.
constexpr int GJ_WARPS = 8;
template <typename T2, int NB>
__global__ void __launch_bounds__(256) k_gj_panel(int b, int k0, int nbk, T2* A, long sA, T2* Pbar,
                                                  __nv_bfloat16* Ps, int* piv, int* flags, const int* active) {
    using C = CT<T2>;
    using R = typename C::R;
    constexpr int P = NB + 1, NW = GJ_WARPS;
    const int bi = blockIdx.x;
    if (active && !active[bi]) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* pan = reinterpret_cast<T2*>(smem_raw);  // b x P
    T2* fcol = pan + (long)b * P;                // b
    __shared__ R red_v[2][NW];
    __shared__ int red_i[2][NW];
    T2* Ab = A + (long)bi * sA;
    int* pv = piv + (long)bi * b;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool col_ok = lane < nbk;
    const T2 zero = C::make(0, 0);

    for (int r = wid; r < b; r += NW)
        if (col_ok) pan[r * P + lane] = Ab[(long)r * b + k0 + lane];
    __syncthreads();
    {
        // Candidates of the first column: rows k0 .. b-1.
        R bv = -1;
        int bix = b;
        for (int r = k0 + tid; r < b; r += 32 * NW) argmax_merge<R>(bv, bix, cabs2(pan[r * P]), r);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const R ov = __shfl_down_sync(0xffffffffu, bv, off);
            const int oi = __shfl_down_sync(0xffffffffu, bix, off);
            argmax_merge<R>(bv, bix, ov, oi);
        }
        if (lane == 0) {
            red_v[0][wid] = bv;
            red_i[0][wid] = bix;
        }
    }
    __syncthreads();

    for (int jj = 0; jj < nbk; ++jj) {
        const int j = k0 + jj, buf = jj & 1;
        R v = red_v[buf][0];
        int p = red_i[buf][0];
#pragma unroll
        for (int w = 1; w < NW; ++w) argmax_merge<R>(v, p, red_v[buf][w], red_i[buf][w]);
        if (p >= b) p = j;
        if (!RGF_DCHECK(p >= j && p < b, RGF_DBG_PIVOT)) p = j;
        if (tid == 0) {
            pv[j] = p;
            if (!(v > 0) && flags) atomicOr(&flags[bi], RGF_FLAG_SINGULAR);
        }
        // Pivot column of the rows other than j and p (unchanged by the swap).
        for (int r = wid + 32 * 0 + lane * NW; r < b; r += 32 * NW)
            if (r != j && r != p) fcol[r] = pan[r * P + jj];
        if (wid == 0) {
            // Row p becomes the pivot row j, scaled by the inverse pivot;
            // the old row j moves to position p.
            const T2 rj = col_ok ? pan[j * P + lane] : zero;
            const T2 rp = col_ok ? pan[p * P + lane] : zero;
            const T2 inv_d = cinv(shfl_c(rp, jj));
            const T2 rj_jj = shfl_c(rj, jj);
            if (col_ok) {
                pan[j * P + lane] = (lane == jj) ? inv_d : cmul(rp, inv_d);
                if (p != j) pan[p * P + lane] = rj;
            }
            if (lane == 0 && p != j) fcol[p] = rj_jj;
        }
        __syncthreads();
        const T2 pj = col_ok ? pan[j * P + lane] : zero;
        const T2 inv_d = pan[j * P + jj];
        if (col_ok) {
            // Branch-free over lanes: lane jj takes -f / pivot, the others
            // x - f p_j.
            const T2 mid = C::make(-inv_d.x, -inv_d.y);
#pragma unroll 8
            for (int r = wid; r < b; r += NW) {
                const T2 f = fcol[r];
                const T2 x = pan[r * P + lane];
                T2 y;
                y.x = x.x - (f.x * pj.x - f.y * pj.y);
                y.y = x.y - (f.x * pj.y + f.y * pj.x);
                const T2 out = (lane == jj) ? cmul(f, mid) : y;
                if (r != j) pan[r * P + lane] = out;
            }
        }
        __syncthreads();
        if (jj + 1 < nbk) {
            // Candidates of the next column: rows j+1 .. b-1.
            const int c = jj + 1;
            R bv = -1;
            int bix = b;
            for (int r = j + 1 + tid; r < b; r += 32 * NW) argmax_merge<R>(bv, bix, cabs2(pan[r * P + c]), r);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const R ov = __shfl_down_sync(0xffffffffu, bv, off);
                const int oi = __shfl_down_sync(0xffffffffu, bix, off);
                argmax_merge<R>(bv, bix, ov, oi);
            }
            if (lane == 0) {
                red_v[buf ^ 1][wid] = bv;
                red_i[buf ^ 1][wid] = bix;
            }
            __syncthreads();
        }
    }
    if constexpr (std::is_same<T2, float2>::value) {
        if (Ps) {
            // Tensor-core update: Pbar as BF16 splits (zero beyond nbk).
            __nv_bfloat16* Pq = Ps + (long)bi * kGjSplits * b * kGjKp;
            for (int r = wid; r < b; r += NW) {
                float2 v = make_float2(0.f, 0.f);
                if (col_ok) {
                    v = pan[r * P + lane];
                    Ab[(long)r * b + k0 + lane] = v;
                    if (r == k0 + lane) v.x -= 1.0f;
                }
                __nv_bfloat16 re[kGjSplits], im[kGjSplits];
                split3_bf16(v.x, re);
                split3_bf16(v.y, im);
#pragma unroll
                for (int s = 0; s < kGjSplits; ++s) store_bf2(Pq + ((long)s * b + r) * kGjKp + 2 * lane, re[s], im[s]);
            }
            return;
        }
    }
    T2* Pb = Pbar + (long)bi * b * nbk;
    if (col_ok) {
        for (int r = wid; r < b; r += NW) {
            T2 v = pan[r * P + lane];
            Ab[(long)r * b + k0 + lane] = v;
            if (r == k0 + lane) v.x -= 1;
            Pb[(long)r * nbk + lane] = v;
        }
    }
}

// Row interchanges of one panel applied to the other columns, and T = rows
// K of those columns after the interchanges.  A CTA owns 32 columns of one
// matrix: it stages the (at most 2 nb) rows that the panel's interchanges
// touch in shared memory, applies the interchanges there, and writes the
// rows back, so the global accesses are coalesced and independent.
template <typename T2>
__global__ void __launch_bounds__(256) k_gj_swap(int b, int k0, int nbk, T2* A, long sA, const int* piv, T2* T,
                                                 __nv_bfloat16* Ts, const int* active) {
    const int bi = blockIdx.y;
    if (active && !active[bi]) return;
    __shared__ int rows[64];
    __shared__ int slot_p[32];
    __shared__ int n_rows;
    __shared__ T2 tile[64][33];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int c = blockIdx.x * 32 + lane;
    T2* Ab = A + (long)bi * sA;
    T2* Tb = T + (long)bi * nbk * b;
    const int* pv = piv + (long)bi * b;
    if (tid == 0) {
        // Slots 0..nbk-1 are rows k0..k0+nbk-1; pivot rows beyond the panel
        // get the next slots (each once).
        int n = nbk;
        for (int jj = 0; jj < nbk; ++jj) rows[jj] = k0 + jj;
        for (int jj = 0; jj < nbk; ++jj) {
            int p = pv[k0 + jj];
            if (!RGF_DCHECK(p >= k0 + jj && p < b, RGF_DBG_PIVOT)) p = k0 + jj;
            int sp = -1;
            if (p < k0 + nbk) {
                sp = p - k0;
            } else {
                for (int q = nbk; q < n; ++q)
                    if (rows[q] == p) sp = q;
                if (sp < 0) {
                    sp = n;
                    rows[n++] = p;
                }
            }
            slot_p[jj] = sp;
        }
        n_rows = n;
    }
    __syncthreads();
    const int n = n_rows;
    const bool in_panel = c >= k0 && c < k0 + nbk;
    const bool ok = c < b && !in_panel;
    for (int q = wid; q < n; q += 8) tile[q][lane] = ok ? Ab[(long)rows[q] * b + c] : CT<T2>::make(0, 0);
    __syncthreads();
    if (wid == 0 && ok) {
        for (int jj = 0; jj < nbk; ++jj) {
            const int sp = slot_p[jj];
            if (sp != jj) {
                const T2 t = tile[jj][lane];
                tile[jj][lane] = tile[sp][lane];
                tile[sp][lane] = t;
            }
        }
    }
    __syncthreads();
    if constexpr (std::is_same<T2, float2>::value) {
        if (Ts) {
            if (ok)
                for (int q = wid; q < n; q += 8) Ab[(long)rows[q] * b + c] = tile[q][lane];
            // T as BF16 splits in the B layout of the K-interleaved complex
            // product (zero in the panel's columns and beyond nbk): a warp
            // per column, lane = row of T, so each warp store is 128
            // contiguous bytes of one output row.
            __nv_bfloat16* Tq = Ts + (long)bi * kGjSplits * 2 * b * kGjKp;
            for (int cl = wid; cl < 32; cl += 8) {
                const int cc = blockIdx.x * 32 + cl;
                if (cc >= b) break;
                const bool pc = cc >= k0 && cc < k0 + nbk;
                const float2 t = (!pc && lane < nbk) ? tile[lane][cl] : make_float2(0.f, 0.f);
                __nv_bfloat16 re[kGjSplits], im[kGjSplits];
                split3_bf16(t.x, re);
                split3_bf16(t.y, im);
#pragma unroll
                for (int s = 0; s < kGjSplits; ++s) {
                    __nv_bfloat16* o = Tq + ((long)s * 2 * b + 2 * cc) * kGjKp + 2 * lane;
                    store_bf2(o, re[s], __hneg(im[s]));
                    store_bf2(o + kGjKp, im[s], re[s]);
                }
            }
            return;
        }
    }
    if (c >= b) return;
    if (in_panel) {
        for (int jj = wid; jj < nbk; jj += 8) Tb[(long)jj * b + c] = CT<T2>::make(0, 0);
        return;
    }
    for (int q = wid; q < n; q += 8) Ab[(long)rows[q] * b + c] = tile[q][lane];
    for (int jj = wid; jj < nbk; jj += 8) Tb[(long)jj * b + c] = tile[jj][lane];
}

// Undo the column interchanges: column c of the result is stored column
// src[c], where src is the identity with the swaps (j, piv[j]) applied for
// j = b-1 down to 0.  One CTA per (32-row block, matrix); rows go through
// shared memory so that reads and writes are coalesced.
template <typename T2>
__global__ void __launch_bounds__(256) k_gj_unpermute(int b, T2* A, long sA, const int* piv, const int* active) {
    const int bi = blockIdx.y;
    if (active && !active[bi]) return;
    extern __shared__ __align__(16) unsigned char smem_up[];
    int* src = reinterpret_cast<int*>(smem_up);
    T2* row = reinterpret_cast<T2*>(smem_up + ((b * sizeof(int) + 15) & ~size_t(15)));
    const int* pv = piv + (long)bi * b;
    if (threadIdx.x == 0) {
        for (int c = 0; c < b; ++c) src[c] = c;
        for (int j = b - 1; j >= 0; --j) {
            int p = pv[j];
            if (!RGF_DCHECK(p >= j && p < b, RGF_DBG_PIVOT)) p = j;
            const int t = src[j];
            src[j] = src[p];
            src[p] = t;
        }
    }
    __syncthreads();
    T2* Ab = A + (long)bi * sA;
    const int r1 = min(b, (int)(blockIdx.x + 1) * 32);
    for (int r = blockIdx.x * 32; r < r1; ++r) {
        for (int c = threadIdx.x; c < b; c += blockDim.x) row[c] = Ab[(long)r * b + c];
        __syncthreads();
        for (int c = threadIdx.x; c < b; c += blockDim.x) Ab[(long)r * b + c] = row[src[c]];
        __syncthreads();
    }
}

// The same column interchanges undone while converting the complex64
// inverse to the caller's format: out[r][c] = A[r][src[c]] as double-float
// complex (float4: hi = value, lo = 0) or complex128; A is left as it is.
// The pivots are staged in shared memory and one thread composes src; a CTA
// handles 64 rows of one matrix.
__device__ __forceinline__ void gj_store_as(float4* o, float2 v) { *o = make_float4(v.x, 0.f, v.y, 0.f); }
__device__ __forceinline__ void gj_store_as(double2* o, float2 v) { *o = make_double2((double)v.x, (double)v.y); }
constexpr int GJ_UNPERM_ROWS = 64;
template <typename TO>
__global__ void __launch_bounds__(256) k_gj_unpermute_to(int b, const float2* __restrict__ A, long sA,
                                                         const int* __restrict__ piv, TO* __restrict__ out,
                                                         const int* active) {
    const int bi = blockIdx.y;
    if (active && !active[bi]) return;
    extern __shared__ int gj_perm[];  // src[b], then the pivots[b]
    int* src = gj_perm;
    int* pvs = gj_perm + b;
    const int* pv = piv + (long)bi * b;
    for (int c = threadIdx.x; c < b; c += blockDim.x) {
        src[c] = c;
        pvs[c] = pv[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = b - 1; j >= 0; --j) {
            int p = pvs[j];
            if (!RGF_DCHECK(p >= j && p < b, RGF_DBG_PIVOT)) p = j;
            const int t = src[j];
            src[j] = src[p];
            src[p] = t;
        }
    }
    __syncthreads();
    const float2* Ab = A + (long)bi * sA;
    TO* Ob = out + (long)bi * b * b;
    const int r1 = min(b, (int)(blockIdx.x + 1) * GJ_UNPERM_ROWS);
    for (int r = blockIdx.x * GJ_UNPERM_ROWS; r < r1; ++r)
        for (int c = threadIdx.x; c < b; c += blockDim.x) gj_store_as(Ob + (long)r * b + c, Ab[(long)r * b + src[c]]);
}

// nb_override (16, or 32 where that is the default) replaces the default
// panel width for b >= 64; 0 keeps it.  The workspace is sized for the
// default, which is never narrower.
// tc_status (complex64 only): non-null selects the tensor-core trailing
// update (gj_update_tc; ws laid out as Pbar splits, T splits, pivots).
// out_df / out_c128 (complex64 only, at most one non-null): write the
// inverse there (contiguous b x b per entry) in that format instead of
// undoing the column interchanges in A.
template <typename T2>
rgf_status inv_t(int batch, int b, T2* A, long sA, void* ws, int* flags, const int* active, cudaStream_t st,
                 int nb_override = 0, int* tc_status = nullptr, float4* out_df = nullptr,
                 double2* out_c128 = nullptr) {
    if (batch <= 0) return RGF_OK;
    int nb = gj_nb(b);
    if (b >= 64 && (nb_override == 16 || (nb_override == 32 && nb == 32))) nb = nb_override;
    const bool tc = std::is_same<T2, float2>::value && tc_status != nullptr;
    T2* Pbar = (T2*)ws;
    T2* T = Pbar + (size_t)batch * b * nb;
    int* piv = (int*)(T + (size_t)batch * b * nb);
    __nv_bfloat16* Ps = nullptr;
    __nv_bfloat16* Ts = nullptr;
    if (tc) {
        Ps = (__nv_bfloat16*)ws;
        Ts = Ps + (size_t)batch * kGjSplits * b * kGjKp;
        piv = (int*)(Ts + (size_t)batch * kGjSplits * 2 * b * kGjKp);
    }
    const size_t smem = ((size_t)b * (nb + 1) + b) * sizeof(T2);
    if (smem > 200 * 1024) {
        set_error("inverse: b = %d needs %zu bytes of shared memory", b, smem);
        return RGF_E_INVALID;
    }
    auto panel = (nb == 32) ? k_gj_panel<T2, 32> : k_gj_panel<T2, 16>;
    if (nb != 32 && nb != 16 && b >= 32) {
        set_error("inverse: unsupported panel width %d", nb);
        return RGF_E_INVALID;
    }
    if (b < 32) panel = k_gj_panel<T2, 32>;  // nb = b < 32 columns of a 32-lane panel
    // One fixed limit for every block size (host threads inverting
    // different sizes share the function).
    if (smem > 48 * 1024) RGF_TRY(smem_limit_once(reinterpret_cast<const void*>(panel), 200 * 1024));
    const int pitch_nb = (panel == k_gj_panel<T2, 16>) ? 16 : 32;
    for (int k0 = 0; k0 < b; k0 += nb) {
        const int nbk = (b - k0) < nb ? (b - k0) : nb;
        const size_t sm = ((size_t)b * (pitch_nb + 1) + b) * sizeof(T2);
        panel<<<batch, 256, sm, st>>>(b, k0, nbk, A, sA, Pbar, Ps, piv, flags, active);
        RGF_LAUNCH_CHECK();
        if (nbk < b) {
            dim3 g2(ceil_div(b, 32), batch);
            k_gj_swap<T2><<<g2, 256, 0, st>>>(b, k0, nbk, A, sA, piv, T, Ts, active);
            RGF_LAUNCH_CHECK();
            if constexpr (std::is_same<T2, float2>::value) {
                if (tc) {
                    RGF_TRY(gj_update_tc(batch, b, nbk, Ps, Ts, A, sA, k0, k0 + nbk, active, tc_status, st));
                    continue;
                }
                RGF_TRY(gj_update_f32(batch, b, b, nbk, Pbar, (long)b * nbk, T, (long)nbk * b, A, b, sA, k0,
                                      k0 + nbk, active, st));
                continue;
            }
            GemmArgs<T2> g{};
            g.batch = batch;
            g.m = b;
            g.n = b;
            g.k = nbk;
            g.alpha = CT<T2>::make(1, 0);
            g.beta = CT<T2>::make(1, 0);
            g.A = Pbar;
            g.lda = nbk;
            g.sA = (long)b * nbk;
            g.B = T;
            g.ldb = b;
            g.sB = (long)nbk * b;
            g.Cin = A;
            g.ldcin = b;
            g.sCin = sA;
            g.C = A;
            g.ldc = b;
            g.sC = sA;
            g.active = active;
            g.skip0 = k0;
            g.skip1 = k0 + nbk;
            RGF_TRY(zgemm_t<T2>(g, st));
        }
    }
    if constexpr (std::is_same<T2, float2>::value) {
        if (out_df || out_c128) {
            dim3 g4(ceil_div(b, GJ_UNPERM_ROWS), batch);
            const size_t smp = 2 * (size_t)b * sizeof(int);
            if (out_df)
                k_gj_unpermute_to<float4><<<g4, 256, smp, st>>>(b, A, sA, piv, out_df, active);
            else
                k_gj_unpermute_to<double2><<<g4, 256, smp, st>>>(b, A, sA, piv, out_c128, active);
            RGF_LAUNCH_CHECK();
            return RGF_OK;
        }
    }
    dim3 g3(ceil_div(b, 32), batch);
    const size_t smu = ((b * sizeof(int) + 15) & ~size_t(15)) + (size_t)b * sizeof(T2);
    k_gj_unpermute<T2><<<g3, 256, smu, st>>>(b, A, sA, piv, active);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

}  // namespace rgf
