// Slice-product complex GEMM on the Blackwell tensor cores (sm_103a).
//
// One CTA computes a 128 x BN tile of the real output (128 rows, BN/2
// complex columns as interleaved re/im pairs; BN = 64, 80 or 96 for the
// double-float variant, 80 for the FP64 variant) of one batch entry:
//   * TMA (cp.async.bulk.tensor, 64-byte swizzle) brings, per 32-element K
//     chunk, the six BF16 slices of the A rows and of the B columns into
//     shared memory; two stages (84 KB each at BN = 96);
//   * one thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32,
//     M = 128, N = BN, K = 16) for the 21 slice pairs (i, j), i + j <= 5,
//     accumulating pair (i, j) in TMEM accumulator min(i + j, 4) (five
//     accumulators x BN columns of the 512 allocated);
//   * eight warps (two per TMEM lane quarter, alternating 16-column chunks)
//     read the accumulators back with tcgen05.ld and combine
//     the groups with exact FP32 TwoSums into double-float results (or, for
//     the FP64 variant, into an FP32 expansion rounded once to FP64), apply
//     the epilogue (sign, addend, identity) and store.
// Every wait on an mbarrier is bounded (2 s); a timeout sets a status bit
// that the host turns into an error, and the CTA still releases its TMEM.
#include <atomic>
#include <cstdlib>
#include <cuda.h>
#include <cudaTypedefs.h>

#include "df.cuh"
#include "metrics.h"
#include "mixed.h"

namespace rgf {

namespace {
constexpr int TC_BM = 128;
constexpr uint32_t TC_TMEM_COLS = 512;
// Per-epilogue-warp transpose buffer of the FP32 update (kOutC32): 32 rows
// of 16 floats, pitch 18 (8-byte aligned float2 accesses), after the
// barriers; eight epilogue warps.
constexpr int kC32Pitch = 18;
constexpr int kC32Warp = 32 * kC32Pitch;
constexpr int kC32Smem = 8 * kC32Warp * 4;

// Tile configuration of one kernel variant: NSL slices per operand, NGRP
// TMEM accumulators (groups 0..NGRP-2 exact, the last one the tail), BN real
// output columns per CTA (NGRP * BN <= 512 TMEM columns), BK BF16 elements
// of K per pipeline stage: 32 (64-byte rows, 64-byte swizzle, two stages)
// or 16 (32-byte rows, 32-byte swizzle, four stages of half the size).
template <int NSL, int NGRP, int BN, int BK>
struct TcCfg {
    static constexpr int STAGES = BK == 32 ? 2 : 4;
    static constexpr int ATILE = TC_BM * BK * 2;   // A slice tile
    static constexpr int BTILE = BN * BK * 2;      // BN rows of 2 BK bytes
    static constexpr int STAGE = NSL * (ATILE + BTILE);
    static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
    // Instruction descriptor: D = F32, A = B = BF16, both K-major, N = BN, M = 128.
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(TC_BM >> 4) << 24);
    // Shared-memory descriptor: layout type (4 = 64-byte swizzle, 6 = 32-byte
    // swizzle) and the byte distance between 8-row groups.
    static constexpr uint64_t SWZ = BK == 32 ? 4 : 6;
    static constexpr uint32_t SBO = 8 * BK * 2;
    static_assert(BK == 16 || BK == 32, "K per stage is 16 or 32 BF16 elements");
    static_assert(NGRP * BN <= 512, "accumulators exceed TMEM");
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "invalid N for M = 128");
    // Tiles start on their swizzle atom (8 rows): 1024 bytes kept for the
    // 64-byte swizzle, 256 bytes (one atom) for the 32-byte swizzle.
    static_assert(BTILE % (BK == 32 ? 1024 : 256) == 0, "B tiles must keep swizzle-atom alignment");
};
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: true when the phase completed, false (and status |= code)
// after limit_ns nanoseconds.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* status, int code,
                                          unsigned long long limit_ns) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (unsigned it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 0 && globaltimer() - t0 > limit_ns) {
            atomicOr(status, code);
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
// Shared-memory matrix descriptor: K-major tile with swizzled rows (layout
// type swz), 8-row groups sbo bytes apart.
__device__ __forceinline__ uint64_t desc_sw(uint32_t saddr, uint64_t swz, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(sbo >> 4) << 32;     // stride byte offset
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= swz << 61;
    return d;
}
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Exact FP32 -> FP64 widening on the integer pipe for normal numbers,
// infinities and NaNs (rebias the exponent, shift the mantissa); zeros and
// subnormals take the hardware conversion.  The FP64 pipe of this GPU is
// narrow and the seven-slice epilogue is bound by it.
__device__ __forceinline__ double f2d(float x) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t e = (u >> 23) & 0xffu;
    if (e == 0) return (double)x;
    const uint64_t sign = (uint64_t)(u >> 31) << 63;
    const uint64_t exp = (e == 0xffu) ? 0x7ffull : (uint64_t)(e + 896u);
    const uint64_t man = (uint64_t)(u & 0x7fffffu) << 29;
    return __longlong_as_double((long long)(sign | (exp << 52) | man));
}

// FP64 value of the sum of NGRP group values: a TwoSum cascade in FP32
// leaves the rounded sum s and the exact errors e_1..e_{NGRP-1}; those are
// summed again with TwoSum into t and a last correction f, and only
// s + (t + f) is formed in FP64 (three widenings, done on the integer pipe,
// and two FP64 additions per output instead of a conversion and an addition
// per group: the FP64 pipe is narrow).
template <int NGRP>
__device__ __forceinline__ double sum_groups_f64(const float (&v)[NGRP][16], int idx) {
    float s = v[0][idx];
    float e[NGRP - 1];
#pragma unroll
    for (int gq = 1; gq < NGRP; ++gq) {
        const float2 r = two_sum(s, v[gq][idx]);
        s = r.x;
        e[gq - 1] = r.y;
    }
    float t = e[0], f = 0.0f;
#pragma unroll
    for (int k = 1; k < NGRP - 1; ++k) {
        const float2 r = two_sum(t, e[k]);
        t = r.x;
        f += r.y;
    }
    return f2d(s) + (f2d(t) + f2d(f));
}

// Double-float value of the group sums: groups 0..NGRP-2 through exact
// TwoSums, the last (tail) group into the low word.
template <int NGRP>
__device__ __forceinline__ float2 combine_df(const float (&v)[NGRP][16], int idx) {
    float hi = v[0][idx], lo = 0.0f;
#pragma unroll
    for (int gq = 1; gq < NGRP - 1; ++gq) {
        const float2 r = two_sum(hi, v[gq][idx]);
        hi = r.x;
        lo += r.y;
    }
    lo += v[NGRP - 1][idx];
    return fast_two_sum(hi, lo);
}
}  // namespace

// Arguments of one launch; C and D are float4 (double-float complex) for
// the double-float variant and double2 for the FP64 variant.
struct TcArgs {
    int batch, m, n, k;
    const __nv_bfloat16* As;
    const __nv_bfloat16* Bs;
    int Kp;
    float alpha;
    const void* D;
    long sD;
    int add_identity;
    void* C;
    long sC;
    const int* active;
    int* status;
    // Failure-path test hooks: wait limit, and a producer that skips the
    // loads of the first K chunk so that the pipeline's waits run out.
    unsigned long long wait_ns;
    int skip_first_chunk;
    int skip0, skip1;  // complex columns left alone (kOutC32)
    float2* C2;        // kOutDF: C rounded to complex64 as well (optional)
    // kOutDF (optional): residual statistics of the result per block of 32
    // rows x 8 complex columns (slot (bi * ceil(m/32) + r/32) * ceil(n/8) +
    // c/8, written by the one warp that stores the block): the sum of the
    // squared high words of Re and Im, and of the diagonal entries.
    float* rsq;
    double2* rtr;
};

// Output modes: double-float complex (float4), FP64 complex (double2), or
// FP32 complex (float2; one accumulator, for the FP32 seed inverse's
// trailing updates, which also skip the columns [skip0, skip1)).
constexpr int kOutDF = 0, kOutF64 = 1, kOutC32 = 2;
template <int OM> struct OutSel { using T = float4; };
template <> struct OutSel<kOutF64> { using T = double2; };
template <> struct OutSel<kOutC32> { using T = float2; };
template <int OM>
using OutT = typename OutSel<OM>::T;

// The 8 complex values (16 real accumulator columns) one lane holds for one
// row: group sums combined, sign applied.
template <int NGRP, int OM>
__device__ __forceinline__ void combine_chunk(const TcArgs& g, const float (&v)[NGRP][16], OutT<OM> (&res)[8]) {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        if constexpr (OM == kOutC32) {
            const float sg = g.alpha < 0.0f ? -1.0f : 1.0f;
            res[t] = make_float2(sg * v[0][2 * t], sg * v[0][2 * t + 1]);
        } else if constexpr (OM == kOutF64) {
            double re = sum_groups_f64<NGRP>(v, 2 * t);
            double im = sum_groups_f64<NGRP>(v, 2 * t + 1);
            if (g.alpha < 0.0f) {
                re = -re;
                im = -im;
            }
            res[t] = make_double2(re, im);
        } else {
            float2 re = combine_df<NGRP>(v, 2 * t);
            float2 im = combine_df<NGRP>(v, 2 * t + 1);
            if (g.alpha < 0.0f) {
                re = df_neg(re);
                im = df_neg(im);
            }
            res[t] = cdf(re, im);
        }
    }
}

// Addend and identity of those values and their store: row r, columns from cb.
// Called by whole warps (lanes: consecutive rows r, one 8-column block cb).
template <int OM>
__device__ __forceinline__ void finish_chunk(const TcArgs& g, const OutT<OM> (&res)[8], int bi, int r, int cb) {
    const bool rok = r < g.m;
    float sq = 0.0f;
    double tre = 0.0, tim = 0.0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int c = cb + t;
        if (!rok || c >= g.n) continue;
        const long o = (long)bi * g.sC + (long)r * g.n + c;
        if constexpr (OM == kOutC32) {
            if (c >= g.skip0 && c < g.skip1) continue;
            float2 x = res[t];
            if (g.D) {
                const float2 d = reinterpret_cast<const float2*>(g.D)[(long)bi * g.sD + (long)r * g.n + c];
                x.x += d.x;
                x.y += d.y;
            }
            reinterpret_cast<float2*>(g.C)[o] = x;
        } else if constexpr (OM == kOutF64) {
            double re = res[t].x, im = res[t].y;
            if (g.D) {
                const double2 d = reinterpret_cast<const double2*>(g.D)[(long)bi * g.sD + (long)r * g.n + c];
                re += d.x;
                im += d.y;
            }
            if (g.add_identity && r == c) re += 1.0;
            reinterpret_cast<double2*>(g.C)[o] = make_double2(re, im);
        } else {
            float2 re = re_of(res[t]), im = im_of(res[t]);
            if (g.D) {
                const float4 d = reinterpret_cast<const float4*>(g.D)[(long)bi * g.sD + (long)r * g.n + c];
                re = df_add(re, re_of(d));
                im = df_add(im, im_of(d));
            }
            if (g.add_identity && r == c) re = df_add(re, make_float2(1.0f, 0.0f));
            reinterpret_cast<float4*>(g.C)[o] = cdf(re, im);
            if (g.C2) g.C2[o] = make_float2(re.x + re.y, im.x + im.y);
            if (g.rsq) {
                sq = fmaf(re.x, re.x, fmaf(im.x, im.x, sq));
                if (r == c) {
                    tre = (double)re.x + (double)re.y;
                    tim = (double)im.x + (double)im.y;
                }
            }
        }
    }
    if constexpr (OM == kOutDF) {
        if (g.rsq) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                sq += __shfl_xor_sync(0xffffffffu, sq, off);
                tre += __shfl_xor_sync(0xffffffffu, tre, off);
                tim += __shfl_xor_sync(0xffffffffu, tim, off);
            }
            // Lane 0 holds the block's first row; blocks past the matrix
            // (the ragged last column tile, row tiles past m) have no slot.
            if ((threadIdx.x & 31) == 0 && r < g.m && cb < g.n) {
                const long slot = ((long)bi * ((g.m + 31) >> 5) + (r >> 5)) * ((g.n + 7) >> 3) + (cb >> 3);
                g.rsq[slot] = sq;
                if (g.rtr) g.rtr[slot] = make_double2(tre, tim);
            }
        }
    }
}

template <int NGRP, int OM>
__device__ __forceinline__ void store_chunk(const TcArgs& g, const float (&v)[NGRP][16], int bi, int r, int cb) {
    OutT<OM> res[8];
    combine_chunk<NGRP, OM>(g, v, res);
    finish_chunk<OM>(g, res, bi, r, cb);
}

// MMAs of one K chunk in stage buffer st: the slice pairs (i, j), i + j <=
// NSL - 1, into accumulator min(i + j, NGRP - 1).  first: the tile's first
// chunk (each accumulator is overwritten by its first product).
template <int NSL, int NGRP, int BN, int BK>
__device__ __forceinline__ void mma_chunk(const unsigned char* st, uint32_t taddr, bool first) {
    using Cfg = TcCfg<NSL, NGRP, BN, BK>;
    // Descriptors of the stage's first A and B tiles; a tile at byte offset
    // o from them has the descriptor + o / 16 (the start-address field is
    // the low 14 bits of address / 16, and shared addresses stay below
    // 256 KB, so the addition never carries out of it).
    const uint64_t da = desc_sw(smem_u32(st), Cfg::SWZ, Cfg::SBO);
    const uint64_t db = desc_sw(smem_u32(st + NSL * Cfg::ATILE), Cfg::SWZ, Cfg::SBO);
    uint32_t started = 0;
#pragma unroll
    for (int i = 0; i < NSL; ++i) {
#pragma unroll
        for (int j = 0; j < NSL; ++j) {
            if (i + j > NSL - 1) continue;
            const int grp = (i + j) < (NGRP - 1) ? (i + j) : (NGRP - 1);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t ad = da + (uint64_t)((i * Cfg::ATILE + kk * 32) >> 4);
                const uint64_t bd = db + (uint64_t)((j * Cfg::BTILE + kk * 32) >> 4);
                const uint32_t acc = (!first || (started >> grp) & 1u) ? 1u : 0u;
                umma(taddr + (uint32_t)(grp * BN), ad, bd, Cfg::IDESC, acc);
                started |= 1u << grp;
            }
        }
    }
}

template <int NSL, int NGRP, int BN, int OM, int BK, int PL>
__global__ void __launch_bounds__(256, 1)
    k_oz_tc(TcArgs g, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB) {
    using Cfg = TcCfg<NSL, NGRP, BN, BK>;
    constexpr int S = Cfg::STAGES;
    const int bi = blockIdx.z;
    if (g.active && !g.active[bi]) return;
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_tc + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + S * Cfg::STAGE);
    // bars[0..S-1] full, bars[S..2S-1] empty, bars[2S] done; slot after them
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * BN;
    const int nk = g.Kp / BK;
    int* status = g.status;

    if (tid == 0) {
        for (int i = 0; i < 2 * S + 1; ++i) mbar_init(smem_u32(&bars[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tmem_slot;

    if (tid == 0) {
        // ---------------- TMA producer
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % S;
            if (kc >= S) {
                if (!mbar_wait(smem_u32(&bars[S + s]), ((kc / S) - 1) & 1, status, 0x1, g.wait_ns)) break;
            }
            if (kc == 0 && g.skip_first_chunk) continue;
            const uint32_t fb = smem_u32(&bars[s]);
            mbar_expect_tx(fb, Cfg::STAGE);
            unsigned char* st = base + s * Cfg::STAGE;
#pragma unroll
            for (int sl = 0; sl < NSL; ++sl) {
                tma_load_3d(smem_u32(st + sl * Cfg::ATILE), &tmA, kc * BK, m0, bi * PL + sl, fb);
                tma_load_3d(smem_u32(st + NSL * Cfg::ATILE + sl * Cfg::BTILE), &tmB, kc * BK, n0, bi * PL + sl,
                            fb);
            }
        }
    } else if (tid == 32) {
        // ---------------- MMA issuer
        bool ok = true;
        for (int kc = 0; kc < nk && ok; ++kc) {
            const int s = kc % S;
            if (!mbar_wait(smem_u32(&bars[s]), (kc / S) & 1, status, 0x2, g.wait_ns)) {
                ok = false;
                break;
            }
            tc_fence_after();
            mma_chunk<NSL, NGRP, BN, BK>(base + s * Cfg::STAGE, taddr, kc == 0);
            umma_commit(smem_u32(&bars[S + s]));
        }
        umma_commit(smem_u32(&bars[2 * S]));
    }
    __syncwarp();

    // ---------------- epilogue: TMEM -> registers -> result -> global
    // One lane per warp waits; the outcome is made warp-uniform because the
    // TMEM loads below are warp-collective.
    int done_i = 0;
    if (lane == 0) done_i = mbar_wait(smem_u32(&bars[2 * S]), 0, status, 0x4, g.wait_ns) ? 1 : 0;
    const bool done = __shfl_sync(0xffffffffu, done_i, 0) != 0;
    __syncwarp();
    tc_fence_after();
    if (done) {
        // Eight warps: warp w reads TMEM lanes 32 (w % 4) .. +31 (its row
        // quarter) and takes every other 16-column chunk, starting at w / 4.
        const int quad = warp & 3;
        const int r = m0 + quad * 32 + lane;
        const uint32_t trow = taddr + ((uint32_t)(quad * 32) << 16);
#pragma unroll 1
        for (int q = warp >> 2; q < BN / 16; q += 2) {
            float v[NGRP][16];
#pragma unroll
            for (int gq = 0; gq < NGRP; ++gq) tmem_ld16(trow + gq * BN + q * 16, v[gq]);
            tmem_ld_wait();
            store_chunk<NGRP, OM>(g, v, bi, r, (n0 + q * 16) >> 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (!done && tid == 0) {
        // Drain TMA copies that may still be in flight before the CTA exits.
        for (int s = 0; s < S; ++s) mbar_wait(smem_u32(&bars[s]), 0, status, 0x8, g.wait_ns);
    }
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

// Persistent form: one CTA per SM walks the tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... (same tile order as the one-tile grid), with
// warp 0 the TMA producer, warp 1 the MMA issuer and warps 2..9 the
// epilogue (TMEM lane quarter warp % 4, alternate 16-column chunks).  The
// stage ring and its phases run on across tiles, so the producer loads the
// next tile's first chunks while the epilogue drains the accumulators, and
// the MMA issuer starts the next tile as soon as every epilogue warp has
// read and combined its chunks (the accumulators are single-buffered:
// NGRP * BN of the 512 columns); addends and stores follow.
template <int NSL, int NGRP, int BN, int OM, int BK, int PL>
__global__ void __launch_bounds__(320, 1)
    k_oz_tc_p(TcArgs g, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB) {
    using Cfg = TcCfg<NSL, NGRP, BN, BK>;
    constexpr int S = Cfg::STAGES;
    constexpr int NQ = BN / 16;      // 16-column chunks of the tile
    constexpr int NCH = (NQ + 1) / 2;  // chunks per epilogue warp (at most)
    // Results of all chunks held in registers until the accumulators are
    // released: only where they fit in the 168 registers a thread of a
    // ten-warp CTA gets (the double-float tiles of width 64 and 96).
    constexpr bool kDefer = OM == kOutDF && BN != 80;
    static_assert(NQ >= 2, "every epilogue warp needs a chunk");
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_tc + 1023) & ~(uintptr_t)1023);
    // bars[0..S-1] full, bars[S..2S-1] empty, bars[2S] accumulators full,
    // bars[2S+1] accumulators empty; then the TMEM slot and three words.
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + S * Cfg::STAGE);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 2);
    volatile int* s_fail = reinterpret_cast<volatile int*>(tmem_slot + 1);  // a role gave up on a wait
    volatile int* s_issued = s_fail + 1;    // chunks whose loads were issued
    volatile int* s_consumed = s_fail + 2;  // chunks the MMA issuer received
    const uint32_t acc_full = smem_u32(&bars[2 * S]), acc_empty = smem_u32(&bars[2 * S + 1]);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = (2 * g.n + BN - 1) / BN, nty = (g.m + TC_BM - 1) / TC_BM;
    const int ntiles = ntx * nty * g.batch;
    const int nk = g.Kp / BK;
    int* status = g.status;

    if (tid == 0) {
        for (int i = 0; i < 2 * S + 1; ++i) mbar_init(smem_u32(&bars[i]), 1);
        mbar_init(acc_empty, 8);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_fail = 0;
        *s_issued = 0;
        *s_consumed = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            int gc = 0;
            for (int t = blockIdx.x; t < ntiles && !*s_fail; t += gridDim.x) {
                const int bx = t % ntx, by = (t / ntx) % nty, bi = t / (ntx * nty);
                if (g.active && !g.active[bi]) continue;
                bool ok = true;
                for (int kc = 0; kc < nk; ++kc, ++gc) {
                    const int s = gc % S;
                    if (gc >= S && !mbar_wait(smem_u32(&bars[S + s]), ((gc / S) - 1) & 1, status, 0x1, g.wait_ns)) {
                        ok = false;
                        break;
                    }
                    *s_issued = gc + 1;
                    if (gc == 0 && g.skip_first_chunk) continue;
                    const uint32_t fb = smem_u32(&bars[s]);
                    mbar_expect_tx(fb, Cfg::STAGE);
                    unsigned char* st = base + s * Cfg::STAGE;
#pragma unroll
                    for (int sl = 0; sl < NSL; ++sl) {
                        tma_load_3d(smem_u32(st + sl * Cfg::ATILE), &tmA, kc * BK, by * TC_BM, bi * PL + sl, fb);
                        tma_load_3d(smem_u32(st + NSL * Cfg::ATILE + sl * Cfg::BTILE), &tmB, kc * BK, bx * BN,
                                    bi * PL + sl, fb);
                    }
                }
                if (!ok) {
                    *s_fail = 1;
                    break;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            int gc = 0, lt = 0;
            for (int t = blockIdx.x; t < ntiles && !*s_fail; t += gridDim.x) {
                const int bi = t / (ntx * nty);
                if (g.active && !g.active[bi]) continue;
                if (lt > 0 && !mbar_wait(acc_empty, (lt - 1) & 1, status, 0x2, g.wait_ns)) {
                    *s_fail = 1;
                    break;
                }
                tc_fence_after();
                bool ok = true;
                for (int kc = 0; kc < nk; ++kc, ++gc) {
                    const int s = gc % S;
                    if (!mbar_wait(smem_u32(&bars[s]), (gc / S) & 1, status, 0x2, g.wait_ns)) {
                        ok = false;
                        break;
                    }
                    *s_consumed = gc + 1;
                    tc_fence_after();
                    mma_chunk<NSL, NGRP, BN, BK>(base + s * Cfg::STAGE, taddr, kc == 0);
                    umma_commit(smem_u32(&bars[S + s]));
                }
                if (!ok) *s_fail = 1;
                // Committed also after a failure, so that the epilogue's wait ends.
                umma_commit(acc_full);
                if (!ok) break;
                ++lt;
            }
        }
    } else {
        // ---------------- epilogue: TMEM -> registers -> result -> global
        const int quad = warp & 3;
        const int half = (warp - 2) >> 2;
        const uint32_t trow = taddr + ((uint32_t)(quad * 32) << 16);
        int lt = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const int bx = t % ntx, by = (t / ntx) % nty, bi = t / (ntx * nty);
            if (g.active && !g.active[bi]) continue;
            const int r = by * TC_BM + quad * 32 + lane;
            if constexpr (OM == kOutC32) {
                // In-place FP32 update C += A B.  A lane holds one row of a
                // 16-column chunk; the chunk goes through a per-warp
                // shared-memory transpose so that each access covers four rows
                // of 64 contiguous bytes (lane: row sub + 4 s, complex column
                // col8), i.e. whole sectors.  The addends do not depend on the
                // MMAs and are loaded before the wait for the accumulators.
                const int row0 = by * TC_BM + quad * 32;
                const int sub = lane >> 3, col8 = lane & 7;
                float* tb = reinterpret_cast<float*>(base + S * Cfg::STAGE + 256) + (warp - 2) * kC32Warp;
                float2 dv[NCH][8];
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    const int c = ((bx * BN + (half + 2 * k) * 16) >> 1) + col8;
#pragma unroll
                    for (int s8 = 0; s8 < 8; ++s8) {
                        const int rr = row0 + sub + 4 * s8;
                        const bool in = g.D && half + 2 * k < NQ && rr < g.m && c < g.n;
                        dv[k][s8] = in ? reinterpret_cast<const float2*>(g.D)[(long)bi * g.sD + (long)rr * g.n + c]
                                       : make_float2(0.f, 0.f);
                    }
                }
                int ok_c = 0;
                if (lane == 0) ok_c = (mbar_wait(acc_full, lt & 1, status, 0x4, g.wait_ns) && !*s_fail) ? 1 : 0;
                if (__shfl_sync(0xffffffffu, ok_c, 0) == 0) break;
                tc_fence_after();
                const float sg = g.alpha < 0.0f ? -1.0f : 1.0f;
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    const int q = half + 2 * k;
                    if (q >= NQ) continue;
                    float v[16];
                    tmem_ld16(trow + q * 16, v);
                    tmem_ld_wait();
                    if (q + 2 >= NQ) {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(acc_empty);
                    }
#pragma unroll
                    for (int t = 0; t < 8; ++t)
                        *reinterpret_cast<float2*>(tb + lane * kC32Pitch + 2 * t) =
                            make_float2(sg * v[2 * t], sg * v[2 * t + 1]);
                    __syncwarp();
                    const int c = ((bx * BN + q * 16) >> 1) + col8;
                    const bool c_ok = c < g.n && !(c >= g.skip0 && c < g.skip1);
#pragma unroll
                    for (int s8 = 0; s8 < 8; ++s8) {
                        const int rr = row0 + sub + 4 * s8;
                        const float2 x = *reinterpret_cast<const float2*>(tb + (sub + 4 * s8) * kC32Pitch + 2 * col8);
                        if (c_ok && rr < g.m)
                            reinterpret_cast<float2*>(g.C)[(long)bi * g.sC + (long)rr * g.n + c] =
                                make_float2(x.x + dv[k][s8].x, x.y + dv[k][s8].y);
                    }
                    __syncwarp();
                }
                ++lt;
                continue;
            }
            // One lane waits; the outcome is made warp-uniform because the
            // TMEM loads below are warp-collective.
            int ok_i = 0;
            if (lane == 0) ok_i = (mbar_wait(acc_full, lt & 1, status, 0x4, g.wait_ns) && !*s_fail) ? 1 : 0;
            if (__shfl_sync(0xffffffffu, ok_i, 0) == 0) break;
            tc_fence_after();
            if constexpr (!kDefer) {
#pragma unroll 1
                for (int q = half; q < NQ; q += 2) {
                    float v[NGRP][16];
#pragma unroll
                    for (int gq = 0; gq < NGRP; ++gq) tmem_ld16(trow + gq * BN + q * 16, v[gq]);
                    tmem_ld_wait();
                    if (q + 2 >= NQ) {
                        // This warp's last chunk is in registers: release
                        // the accumulators to the next tile's MMAs.
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(acc_empty);
                    }
                    store_chunk<NGRP, OM>(g, v, bi, r, (bx * BN + q * 16) >> 1);
                }
                ++lt;
                continue;
            }
            // All of this warp's chunks are read and combined into registers
            // before the accumulators are released; the addends are read and
            // the results stored while the next tile's MMAs run.
            OutT<OM> res[NCH][8];
#pragma unroll
            for (int k = 0; k < NCH; ++k) {
                const int q = half + 2 * k;
                if (q < NQ) {
                    float v[NGRP][16];
#pragma unroll
                    for (int gq = 0; gq < NGRP; ++gq) tmem_ld16(trow + gq * BN + q * 16, v[gq]);
                    tmem_ld_wait();
                    if (q + 2 >= NQ) {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(acc_empty);
                    }
                    combine_chunk<NGRP, OM>(g, v, res[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < NCH; ++k) {
                const int q = half + 2 * k;
                if (q < NQ) finish_chunk<OM>(g, res[k], bi, r, (bx * BN + q * 16) >> 1);
            }
            ++lt;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *s_fail) {
        // Drain TMA copies that may still be in flight before the CTA exits:
        // the chunks issued but not received by the MMA issuer (at most S,
        // on distinct stages).
        for (int c = *s_consumed; c < *s_issued; ++c)
            mbar_wait(smem_u32(&bars[c % S]), (c / S) & 1, status, 0x8, g.wait_ns);
    }
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------- CTA pair
// Two-SM form for row tiles of 256 (M = 256 per MMA, tcgen05 cta_group::2):
// a cluster of two CTAs computes a 256 x BN tile.  Each CTA stages its own
// 128 rows of the A slices and half (BN / 2 rows) of the B slices; the
// leader CTA (cluster rank 0) issues the MMAs, which read both CTAs' tiles,
// and each CTA's TMEM receives its 128 rows of the BN accumulator columns.
// Per SM this halves the B operand's shared-memory reads (A 4 KB + B 1.5 KB
// per 128 x BN x 16 MMA instead of 4 + 3 KB) and halves the stage, so three
// stages fit.  Synchronisation: the peer's TMA copies complete on the
// leader's full barrier (which the leader's producer arms for both CTAs'
// bytes); the leader's commits arrive on the empty and accumulator-full
// barriers of both CTAs (multicast); both CTAs' epilogue warps release the
// accumulators on the leader's accumulator-empty barrier.  Every wait is
// bounded as in the one-SM form; both CTAs meet at a cluster barrier before
// the TMEM is released.
template <int NSL, int NGRP, int BN>
struct TcCfg2 {
    static constexpr int BK = 32, STAGES = 3;
    static constexpr int ATILE = TC_BM * BK * 2;     // this CTA's 128 rows of one A slice
    static constexpr int BTILE = (BN / 2) * BK * 2;  // this CTA's BN / 2 rows of one B slice
    static constexpr int STAGE = NSL * (ATILE + BTILE);
    static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
    // D = F32, A = B = BF16, K-major, N = BN, M = 256 (the pair).
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(256 >> 4) << 24);
    static constexpr uint64_t SWZ = 4;
    static constexpr uint32_t SBO = 8 * BK * 2;
    static_assert(NGRP * BN <= 512, "accumulators exceed TMEM");
    static_assert(BTILE % 1024 == 0, "B half tiles must keep swizzle-atom alignment");
    static_assert(SMEM <= 227 * 1024, "stages exceed shared memory");
};

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// Shared::cluster address of the object at this CTA's shared address a in
// the CTA of the given cluster rank.
__device__ __forceinline__ uint32_t mapa_rank(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// TMA load into this CTA's shared memory whose completion is signalled on
// the mbarrier at a shared::cluster address (the leader's for both CTAs).
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                                 uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void umma_pair(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}
// Completion of the leader's MMAs arrives on the barrier at this shared
// offset in both CTAs of the pair.
__device__ __forceinline__ void umma_pair_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"((unsigned short)0x3)
        : "memory");
}

template <int NSL, int NGRP, int BN>
__device__ __forceinline__ void mma_chunk_pair(const unsigned char* st, uint32_t taddr, bool first) {
    using Cfg = TcCfg2<NSL, NGRP, BN>;
    const uint64_t da = desc_sw(smem_u32(st), Cfg::SWZ, Cfg::SBO);
    const uint64_t db = desc_sw(smem_u32(st + NSL * Cfg::ATILE), Cfg::SWZ, Cfg::SBO);
    uint32_t started = 0;
#pragma unroll
    for (int i = 0; i < NSL; ++i) {
#pragma unroll
        for (int j = 0; j < NSL; ++j) {
            if (i + j > NSL - 1) continue;
            const int grp = (i + j) < (NGRP - 1) ? (i + j) : (NGRP - 1);
#pragma unroll
            for (int kk = 0; kk < Cfg::BK / 16; ++kk) {
                const uint64_t ad = da + (uint64_t)((i * Cfg::ATILE + kk * 32) >> 4);
                const uint64_t bd = db + (uint64_t)((j * Cfg::BTILE + kk * 32) >> 4);
                const uint32_t acc = (!first || (started >> grp) & 1u) ? 1u : 0u;
                umma_pair(taddr + (uint32_t)(grp * BN), ad, bd, Cfg::IDESC, acc);
                started |= 1u << grp;
            }
        }
    }
}

template <int NSL, int NGRP, int BN, int PL>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(320, 1)
    k_oz_tc_pair(TcArgs g, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB) {
    using Cfg = TcCfg2<NSL, NGRP, BN>;
    constexpr int S = Cfg::STAGES;
    constexpr int NQ = BN / 16;
    constexpr int NCH = (NQ + 1) / 2;
    static_assert(BN == 64 || BN == 96, "the deferred epilogue holds the chunks of a 64 or 96 wide tile");
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_tc + 1023) & ~(uintptr_t)1023);
    // bars[0..S-1] full, bars[S..2S-1] empty, bars[2S] accumulators full,
    // bars[2S+1] accumulators empty (the leader's counts both CTAs' warps).
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + S * Cfg::STAGE);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 2);
    volatile int* s_fail = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* s_issued = s_fail + 1;
    volatile int* s_consumed = s_fail + 2;
    const uint32_t acc_full = smem_u32(&bars[2 * S]), acc_empty = smem_u32(&bars[2 * S + 1]);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = cluster_ctarank();
    const bool leader = rank == 0;
    const int cl = (int)cluster_id_x(), ncl = (int)cluster_count_x();
    const int ntx = (2 * g.n + BN - 1) / BN, nty = (g.m + 255) / 256;
    const int ntiles = ntx * nty * g.batch;
    const int nk = g.Kp / Cfg::BK;
    int* status = g.status;

    if (tid == 0) {
        for (int i = 0; i < 2 * S + 1; ++i) mbar_init(smem_u32(&bars[i]), 1);
        mbar_init(acc_empty, 16);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_fail = 0;
        *s_issued = 0;
        *s_consumed = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    // Both CTAs' barriers are initialised and their TMEM allocated before
    // either signals the other.
    cluster_sync_all();
    tc_fence_after();
    const uint32_t taddr = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (both CTAs)
            int gc = 0;
            for (int t = cl; t < ntiles && !*s_fail; t += ncl) {
                const int bx = t % ntx, by = (t / ntx) % nty, bi = t / (ntx * nty);
                if (g.active && !g.active[bi]) continue;
                bool ok = true;
                for (int kc = 0; kc < nk; ++kc, ++gc) {
                    const int s = gc % S;
                    if (gc >= S && !mbar_wait(smem_u32(&bars[S + s]), ((gc / S) - 1) & 1, status, 0x1, g.wait_ns)) {
                        ok = false;
                        break;
                    }
                    *s_issued = gc + 1;
                    const uint32_t fb_local = smem_u32(&bars[s]);
                    if (leader) mbar_expect_tx(fb_local, 2 * Cfg::STAGE);
                    const uint32_t fb = mapa_rank(fb_local, 0);
                    unsigned char* st = base + s * Cfg::STAGE;
#pragma unroll
                    for (int sl = 0; sl < NSL; ++sl) {
                        tma_load_3d_pair(smem_u32(st + sl * Cfg::ATILE), &tmA, kc * Cfg::BK, by * 256 + (int)rank * TC_BM,
                                         bi * PL + sl, fb);
                        tma_load_3d_pair(smem_u32(st + NSL * Cfg::ATILE + sl * Cfg::BTILE), &tmB, kc * Cfg::BK,
                                         bx * BN + (int)rank * (BN / 2), bi * PL + sl, fb);
                    }
                }
                if (!ok) {
                    *s_fail = 1;
                    break;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            // ---------------- MMA issuer (leader CTA)
            int gc = 0, lt = 0;
            for (int t = cl; t < ntiles && !*s_fail; t += ncl) {
                const int bi = t / (ntx * nty);
                if (g.active && !g.active[bi]) continue;
                if (lt > 0 && !mbar_wait(acc_empty, (lt - 1) & 1, status, 0x2, g.wait_ns)) {
                    *s_fail = 1;
                    break;
                }
                tc_fence_after();
                bool ok = true;
                for (int kc = 0; kc < nk; ++kc, ++gc) {
                    const int s = gc % S;
                    if (!mbar_wait(smem_u32(&bars[s]), (gc / S) & 1, status, 0x2, g.wait_ns)) {
                        ok = false;
                        break;
                    }
                    *s_consumed = gc + 1;
                    tc_fence_after();
                    mma_chunk_pair<NSL, NGRP, BN>(base + s * Cfg::STAGE, taddr, kc == 0);
                    umma_pair_commit(smem_u32(&bars[S + s]));
                }
                if (!ok) *s_fail = 1;
                // Committed also after a failure, so that the epilogues' waits end.
                umma_pair_commit(acc_full);
                if (!ok) break;
                ++lt;
            }
        }
    } else {
        // ---------------- epilogue (both CTAs): this CTA's 128 rows
        const int quad = warp & 3;
        const int half = (warp - 2) >> 2;
        const uint32_t trow = taddr + ((uint32_t)(quad * 32) << 16);
        const uint32_t release = mapa_rank(acc_empty, 0);
        int lt = 0;
        for (int t = cl; t < ntiles; t += ncl) {
            const int bx = t % ntx, by = (t / ntx) % nty, bi = t / (ntx * nty);
            if (g.active && !g.active[bi]) continue;
            int ok_i = 0;
            if (lane == 0) ok_i = (mbar_wait(acc_full, lt & 1, status, 0x4, g.wait_ns) && !*s_fail) ? 1 : 0;
            if (__shfl_sync(0xffffffffu, ok_i, 0) == 0) break;
            tc_fence_after();
            const int r = by * 256 + (int)rank * TC_BM + quad * 32 + lane;
            float4 res[NCH][8];
#pragma unroll
            for (int k = 0; k < NCH; ++k) {
                const int q = half + 2 * k;
                if (q < NQ) {
                    float v[NGRP][16];
#pragma unroll
                    for (int gq = 0; gq < NGRP; ++gq) tmem_ld16(trow + gq * BN + q * 16, v[gq]);
                    tmem_ld_wait();
                    if (q + 2 >= NQ) {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive_remote(release);
                    }
                    combine_chunk<NGRP, kOutDF>(g, v, res[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < NCH; ++k) {
                const int q = half + 2 * k;
                if (q < NQ) finish_chunk<kOutDF>(g, res[k], bi, r, (bx * BN + q * 16) >> 1);
            }
            ++lt;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && leader && *s_fail) {
        // Copies issued but not received by the MMA issuer complete on the
        // leader's full barriers (both CTAs' bytes).
        for (int c = *s_consumed; c < *s_issued; ++c)
            mbar_wait(smem_u32(&bars[c % S]), (c / S) & 1, status, 0x8, g.wait_ns);
    }
    __syncthreads();
    // Neither CTA releases its TMEM or exits while its peer may still
    // signal its barriers or read its tiles.
    cluster_sync_all();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

// The driver's tensor-map encoder, looked up at run time so that the library
// loads (and its host-only entry points work) on machines without a driver.
static PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    // Initialised once, thread-safely, on first use.
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
        return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }();
    return fn;
}

static rgf_status encode_slices(CUtensorMap* map, const __nv_bfloat16* ptr, int Kp, long rows, long planes,
                                int box_rows, int bk) {
    cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)rows * Kp * 2};
    cuuint32_t box[3] = {(cuuint32_t)bk, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return RGF_E_CUDA;
    }
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)ptr, dims, strides, box, estr,
                                        CU_TENSOR_MAP_INTERLEAVE_NONE,
                                        bk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return RGF_E_CUDA;
    }
    return RGF_OK;
}

// PL: slice planes per batch entry in the buffers (>= NSL; the kernel reads
// the NSL most significant).
// Shared memory of a persistent CTA: at least 116 KB, so that no two CTAs
// that allocate the whole TMEM share an SM (one would wait in tcgen05.alloc
// until the other has finished all its tiles).
template <int SMEM>
constexpr int kPersistSmem = SMEM > 116 * 1024 ? SMEM : 116 * 1024;
// The FP32 update's persistent CTA also holds the epilogue transpose buffers.
template <int SMEM, int OM>
constexpr int kPersistSmemOf = kPersistSmem<SMEM + (OM == kOutC32 ? kC32Smem : 0)>;

// Persistent tile loop (default) or one CTA per tile with
// RGF_TC_PERSIST=0 in the environment (read once).
static bool tc_persistent() {
    static const bool on = [] {
        const char* e = getenv("RGF_TC_PERSIST");
        return !(e && e[0] == '0');
    }();
    return on;
}

template <int NSL, int NGRP, int BN, int OM, int BK, int PL = NSL>
static rgf_status launch_tc(const TcArgs& g, cudaStream_t st, bool count_work = true) {
    using Cfg = TcCfg<NSL, NGRP, BN, BK>;
    if (g.batch <= 0) return RGF_OK;
    if (g.Kp % BK != 0 || ((uintptr_t)g.As & 15) || ((uintptr_t)g.Bs & 15) || !g.status) {
        set_error("oz_gemm_tc: bad slice layout");
        return RGF_E_INVALID;
    }
    if (g.batch > 65535 || (long)g.batch * PL > 0x7fffffffL) {
        set_error("oz_gemm_tc: batch too large");
        return RGF_E_INVALID;
    }
    CUtensorMap ta, tb;
    RGF_TRY(encode_slices(&ta, g.As, g.Kp, g.m, (long)g.batch * PL, TC_BM, BK));
    RGF_TRY(encode_slices(&tb, g.Bs, g.Kp, 2L * g.n, (long)g.batch * PL, BN, BK));
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        // Idempotent: threads that race here all set the same value.
        RGF_CUDA_TRY(cudaFuncSetAttribute(k_oz_tc<NSL, NGRP, BN, OM, BK, PL>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
        RGF_CUDA_TRY(cudaFuncSetAttribute(k_oz_tc_p<NSL, NGRP, BN, OM, BK, PL>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, kPersistSmemOf<Cfg::SMEM, OM>));
        attr.store(true);
    }
    dim3 grid(ceil_div(2L * g.n, BN), ceil_div(g.m, TC_BM), g.batch);
    const long ntiles = (long)grid.x * grid.y * grid.z;
    int dev = 0, nsm = 0;
    RGF_CUDA_TRY(cudaGetDevice(&dev));
    RGF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const bool persistent = tc_persistent() && ntiles < 0x7fffffffL;
    // Only unmasked launches are timed: their work is exactly known.
    const bool timed = count_work && gemm_timing_enabled() && g.active == nullptr;
    cudaEvent_t ev = nullptr;
    if (timed) gemm_timing_before(st, &ev);
    if (persistent) {
        const int nblk = (int)(ntiles < nsm ? ntiles : nsm);
        k_oz_tc_p<NSL, NGRP, BN, OM, BK, PL><<<nblk, 320, kPersistSmemOf<Cfg::SMEM, OM>, st>>>(g, ta, tb);
    } else {
        k_oz_tc<NSL, NGRP, BN, OM, BK, PL><<<grid, 256, Cfg::SMEM, st>>>(g, ta, tb);
    }
    RGF_LAUNCH_CHECK();
    if (timed) {
        // NSL(NSL+1)/2 slice-pair real products of M = m, N = 2n, K = 2k per batch entry.
        const double pairs = (double)(NSL * (NSL + 1) / 2);
        gemm_timing_after(st, ev, pairs * 2.0 * g.m * (2.0 * g.n) * (2.0 * g.k) * g.batch);
    }
    return RGF_OK;
}

// Two-SM tiles for row counts that are multiples of 256 with RGF_TC_PAIR=1
// in the environment (read once).  Off by default: at b = 256 (296 entries)
// the pair took 711 us per product against 693 us for the one-SM kernel,
// both with the tensor pipe about 60% active, so neither the B operand's
// shared-memory reads nor the stage depth is what limits this GEMM.
static bool tc_pair_enabled() {
    static const bool on = [] {
        const char* e = getenv("RGF_TC_PAIR");
        return e && e[0] == '1';
    }();
    return on;
}

template <int NSL, int NGRP, int BN, int PL>
static rgf_status launch_tc_pair(const TcArgs& g, cudaStream_t st) {
    using Cfg = TcCfg2<NSL, NGRP, BN>;
    if (g.batch <= 0) return RGF_OK;
    if (g.Kp % Cfg::BK != 0 || ((uintptr_t)g.As & 15) || ((uintptr_t)g.Bs & 15) || !g.status || g.m % 256 != 0) {
        set_error("oz_gemm_tc (pair): bad slice layout");
        return RGF_E_INVALID;
    }
    if ((long)g.batch * PL > 0x7fffffffL) {
        set_error("oz_gemm_tc (pair): batch too large");
        return RGF_E_INVALID;
    }
    CUtensorMap ta, tb;
    RGF_TRY(encode_slices(&ta, g.As, g.Kp, g.m, (long)g.batch * PL, TC_BM, Cfg::BK));
    RGF_TRY(encode_slices(&tb, g.Bs, g.Kp, 2L * g.n, (long)g.batch * PL, BN / 2, Cfg::BK));
    // Resident clusters of this kernel (one CTA per SM), found once.
    static std::atomic<int> max_clusters{0};
    if (max_clusters.load() == 0) {
        RGF_CUDA_TRY(cudaFuncSetAttribute(k_oz_tc_pair<NSL, NGRP, BN, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          Cfg::SMEM));
        int dev = 0, nsm = 0;
        RGF_CUDA_TRY(cudaGetDevice(&dev));
        RGF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(nsm & ~1), 1, 1);
        cfg.blockDim = dim3(320, 1, 1);
        cfg.dynamicSmemBytes = Cfg::SMEM;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        RGF_CUDA_TRY(cudaOccupancyMaxActiveClusters(&n, (const void*)k_oz_tc_pair<NSL, NGRP, BN, PL>, &cfg));
        if (n < 1) {
            set_error("oz_gemm_tc (pair): no CTA pair of %d bytes of shared memory fits", Cfg::SMEM);
            return RGF_E_CUDA;
        }
        max_clusters.store(n);
    }
    const long ntiles = (long)ceil_div(2L * g.n, BN) * (g.m / 256) * g.batch;
    const int ncl = (int)(ntiles < max_clusters.load() ? ntiles : max_clusters.load());
    const bool timed = gemm_timing_enabled() && g.active == nullptr;
    cudaEvent_t ev = nullptr;
    if (timed) gemm_timing_before(st, &ev);
    k_oz_tc_pair<NSL, NGRP, BN, PL><<<2 * ncl, 320, Cfg::SMEM, st>>>(g, ta, tb);
    RGF_LAUNCH_CHECK();
    if (timed) {
        const double pairs = (double)(NSL * (NSL + 1) / 2);
        gemm_timing_after(st, ev, pairs * 2.0 * g.m * (2.0 * g.n) * (2.0 * g.k) * g.batch);
    }
    return RGF_OK;
}

// K per pipeline stage of the tensor-core cores: 32 (default) or 16 with
// RGF_TC_BK=16 in the environment (read once).
static int tc_bk() {
    static const int bk = [] {
        const char* e = getenv("RGF_TC_BK");
        return (e && e[0] == '1' && e[1] == '6') ? 16 : 32;
    }();
    return bk;
}

rgf_status oz_gemm_tc(const OzGemm& g, cudaStream_t st) {
    TcArgs a{g.batch, g.m, g.n, g.k, g.As, g.Bs, g.Kp, g.alpha, g.D, g.sD, g.add_identity, g.C, g.sC, g.active,
             g.status, TC_WAIT_NS, 0, 0, 0, g.C2, g.rsq, g.rtr};
    if (g.test_wait_ns) {
        a.wait_ns = g.test_wait_ns;
        a.skip_first_chunk = 1;
    }
    if (g.m % 256 == 0 && !g.test_wait_ns && tc_persistent() && tc_pair_enabled() && tc_bk() == 32 &&
        (g.bn == 0 || g.bn == 96)) {
        if (g.nsl == 4) return launch_tc_pair<4, 4, 96, kSlices>(a, st);
        if (g.nsl == 0 || g.nsl == kSlices) return launch_tc_pair<kSlices, kGroups, 96, kSlices>(a, st);
    }
    if (g.nsl == 4) {
        // Four of the six slices (ten pairs, four exact groups): for
        // products whose result is a small correction (see OzGemm::nsl).
        switch (g.bn) {
            case 64: return launch_tc<4, 4, 64, kOutDF, 32, kSlices>(a, st);
            case 80: return launch_tc<4, 4, 80, kOutDF, 32, kSlices>(a, st);
            case 0:
            case 96: return launch_tc<4, 4, 96, kOutDF, 32, kSlices>(a, st);
            default: break;
        }
    } else if (g.nsl == 5) {
        // Five of the six slices (15 pairs, one accumulator per group; see
        // OzGemm::nsl): reached through the kernel-level entry point.
        switch (g.bn) {
            case 64: return launch_tc<5, 5, 64, kOutDF, 32, kSlices>(a, st);
            case 80: return launch_tc<5, 5, 80, kOutDF, 32, kSlices>(a, st);
            case 0:
            case 96: return launch_tc<5, 5, 96, kOutDF, 32, kSlices>(a, st);
            default: break;
        }
    } else if (tc_bk() == 16) {
        switch (g.bn) {
            case 64: return launch_tc<kSlices, kGroups, 64, kOutDF, 16>(a, st);
            case 80: return launch_tc<kSlices, kGroups, 80, kOutDF, 16>(a, st);
            case 0:
            case 96: return launch_tc<kSlices, kGroups, 96, kOutDF, 16>(a, st);
            default: break;
        }
    } else {
        switch (g.bn) {
            case 64: return launch_tc<kSlices, kGroups, 64, kOutDF, 32>(a, st);
            case 80: return launch_tc<kSlices, kGroups, 80, kOutDF, 32>(a, st);
            case 0:
            case 96: return launch_tc<kSlices, kGroups, 96, kOutDF, 32>(a, st);
            default: break;
        }
    }
    set_error("oz_gemm_tc: unsupported tile width %d", g.bn);
    return RGF_E_INVALID;
}

rgf_status gj_update_tc(int batch, int b, int nbk, const __nv_bfloat16* Ps, const __nv_bfloat16* Ts, float2* C,
                        long sC, int skip0, int skip1, const int* active, int* status, cudaStream_t st) {
    // C (b x b, row stride b) += Pbar T: M = b, N = 2b real columns, K =
    // 2 nbk reals padded to kGjKp; three splits per operand, the six pairs
    // i + j <= 2 in one FP32 accumulator.  Not counted in the slice-product
    // GEMM timing (a different product).
    TcArgs a{batch, b, b, nbk, Ps, Ts, kGjKp, 1.0f, C, sC, 0, C, sC, active, status, TC_WAIT_NS, 0, skip0, skip1};
    return launch_tc<kGjSplits, 1, 128, kOutC32, 32, kGjSplits>(a, st, false);
}

rgf_status oz_gemm_hp(const OzGemmHP& g, cudaStream_t st) {
    TcArgs a{g.batch, g.m, g.n, g.k, g.As, g.Bs, g.Kp, g.alpha, g.D, g.sD, g.add_identity, g.C, g.sC, g.active,
             g.status, TC_WAIT_NS, 0};
    // Tiles 64 wide: 2n = 512 real columns in eight whole tiles (80 wide
    // needs seven, the last 32 wide, and measured 3% slower in the lead
    // decimation); RGF_HP_BN=80 in the environment (read once) selects 80.
    static const bool bn64 = [] {
        const char* e = getenv("RGF_HP_BN");
        return !(e && e[0] == '8' && e[1] == '0');
    }();
    if (g.nsl == 5) {
        if (bn64) return launch_tc<5, 5, 64, kOutF64, 32, kSlicesHP>(a, st);
        return launch_tc<5, 5, 80, kOutF64, 32, kSlicesHP>(a, st);
    }
    if (g.nsl != 0 && g.nsl != kSlicesHP) {
        set_error("oz_gemm_hp: unsupported slice count %d", g.nsl);
        return RGF_E_INVALID;
    }
    if (tc_bk() == 16) return launch_tc<kSlicesHP, kGroupsHP, 80, kOutF64, 16>(a, st);
    if (bn64) return launch_tc<kSlicesHP, kGroupsHP, 64, kOutF64, 32>(a, st);
    return launch_tc<kSlicesHP, kGroupsHP, 80, kOutF64, 32>(a, st);
}

}  // namespace rgf
