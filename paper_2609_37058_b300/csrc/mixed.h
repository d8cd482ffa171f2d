// Mixed-precision building blocks: double-float complex matrices (float4
// per element: re_hi, re_lo, im_hi, im_lo), their BF16 slice expansions and
// the exact slice-product complex GEMM.
#pragma once

#include <cuda_bf16.h>

#include "kernels.h"

namespace rgf {

// Number of BF16 slices per operand.  A value x in a row (or column) whose
// largest entry is below 2^e is written as x = 2^e * sum_s q_s 2^(-7-8s),
// s = 0..5, with integers |q_s| <= 128 (8 significant bits, exact in BF16).
constexpr int kSlices = 6;

// Products kept: slice pairs (i, j) with i + j <= kSlices - 1 (21 pairs).
// Pair (i, j) lands in accumulator min(i + j, kGroups - 1).  Every partial
// sum of group g = i + j is an integer multiple of that group's unit
// 2^(-14-8g) sigma_row sigma_col, at most (g+1) 2^14 K units, so the FP32
// accumulation of groups 0..3 is exact (worst case: all slices at full
// magnitude with equal signs) up to K = 1024, 512, 341 and 256 real terms,
// and in practice far beyond.  The last accumulator collects the tail
// g = 4, 5, whose products are not all integers in one unit: the tensor
// core truncates their low bits, an error of order K * 11 * 2^-56 of the
// leading term.  (Folding g = 3 into the tail as well would cost ~2^-35 at
// K = 512, which is why five accumulators are kept.)
constexpr int kGroups = 5;

// High-precision variant for FP64 operands: seven balanced 8-bit digits
// x = 2^e sum_{s=0..6} d_s 2^(-7-8s), |d_s| <= 128 (56 bits), 28 slice pairs,
// groups 0..4 exact and the tail g = 5, 6 in a sixth accumulator (its
// truncation is of order K * 13 * 2^-64 of the leading term); FP64 result.
constexpr int kSlicesHP = 7;
constexpr int kGroupsHP = 6;

// Row pitch of a slice matrix in BF16 elements: real K = 2 k (re/im
// interleaved) rounded up to a multiple of 64 so every 64-element chunk is
// full; the padding is zero.
inline int slice_pitch(int k) { return ((2 * k + 63) / 64) * 64; }

// Slices of the left operand A (m x k complex, df):
//   out[((bi*kSlices + s)*m + r)*Kp + 2j + {0,1}] = slice s of (Re, Im) A[r][j]
// planes: how many of the slices (the most significant) are written; a
// product that reads fewer slices (OzGemm::nsl) needs only those.
rgf_status slice_rows(int batch, int m, int k, const float4* A, long sA, __nv_bfloat16* out, int Kp,
                      const int* active, cudaStream_t st, int planes = kSlices);
// Slices of the right operand B (k x n complex, df) in transposed,
// complex-expanded form (2n rows of Kp):
//   row 2c  : (Re B[j][c], -Im B[j][c]) at K positions (2j, 2j+1)
//   row 2c+1: (Im B[j][c],  Re B[j][c])
// so that one real GEMM gives Re C in real column 2c and Im C in 2c+1.
rgf_status slice_cols(int batch, int k, int n, const float4* B, long sB, __nv_bfloat16* out, int Kp,
                      const int* active, cudaStream_t st, int planes = kSlices);

// Slices of the coupling blocks formed on the fly for W energies (entry =
// energy, z = E[e] + i eta; S, H one b x b df block each):
//   form_slice_rows:     A-operand slices of tau  = z S - H;
//   form_slice_cols_dag: B-operand slices of tau' = z S^dagger - H^dagger.
rgf_status form_slice_rows(int W, int b, const double* E, double eta, const float4* S, const float4* H,
                           __nv_bfloat16* out, int Kp, cudaStream_t st);
rgf_status form_slice_cols_dag(int W, int b, const double* E, double eta, const float4* S, const float4* H,
                               __nv_bfloat16* out, int Kp, cudaStream_t st);

struct OzGemm {
    int batch, m, n, k;          // complex sizes: C (m x n) = A (m x k) B (k x n)
    const __nv_bfloat16* As;     // [batch][kSlices][m][Kp]
    const __nv_bfloat16* Bs;     // [batch][kSlices][2n][Kp]
    int Kp;
    float alpha;                 // +1 or -1
    const float4* D; long sD;    // optional addend (may alias C)
    int add_identity;            // C += I
    float4* C; long sC;
    float2* C2;                  // optional: C rounded to complex64 as well (same layout)
    // Optional residual statistics per 32-row x 8-column block (tcgen05
    // core): sum of squared high words (rsq) and of diagonal entries (rtr);
    // see ns_check.
    float* rsq;
    double2* rtr;
    const int* active;
    int* status;                 // device word, nonzero after a pipeline timeout
    // Test hook (0 in normal use): nonzero makes the tcgen05 core skip the
    // loads of the first K chunk and use this wait limit in nanoseconds, so
    // that its bounded waits run out and report through *status.
    unsigned long long test_wait_ns;
    // Real output columns per CTA of the tcgen05 core: 64, 80 or 96 (0 = 96).
    int bn;
    // Slices of each operand that take part: 6 (0 = 6, full double-float
    // product); 5 (15 pairs, relative error ~k 2^-39 of row-max x column-max;
    // kernel-level entry point only: used for the running product Q_i =
    // Q_{i-1} P_i of the sweep it moved well-conditioned T by up to 1.3e-6 at
    // b = 256, N = 500, because the entries that carry T are far below the
    // row and column maxima the error is relative to); or 4 (ten pairs,
    // relative error ~2^-30 of |A| |B|; enough for a Newton-Schulz correction
    // X R, whose size is |X| |R| with R small and whose error the next
    // residual, computed in full, measures again).
    int nsl;
};

struct OzGemmHP {
    int batch, m, n, k;          // complex sizes: C (m x n) = A (m x k) B (k x n)
    const __nv_bfloat16* As;     // [batch][kSlicesHP][m][Kp]
    const __nv_bfloat16* Bs;     // [batch][kSlicesHP][2n][Kp]
    int Kp;
    float alpha;                 // +1 or -1
    const double2* D; long sD;   // optional FP64 addend (may alias C)
    int add_identity;
    double2* C; long sC;
    const int* active;
    int* status;
    // Slices of each operand that take part: 7 (0 = 7), or 5 for products
    // whose result is a small correction (15 pairs in five accumulators, one
    // per group; group g is exact for K <= 1024 / (g + 1) real terms in the
    // worst case, beyond that FP32-rounded at ~2^-24 of its own size, i.e.
    // ~2^-(40 + 8 (g - 2)) of the leading term; relative error ~k 2^-39 of
    // row-max x column-max in all).
    int nsl;
};
rgf_status oz_gemm_hp(const OzGemmHP& g, cudaStream_t st);
// Seven-digit slicing of FP64 complex operands (layouts as slice_rows /
// slice_cols with kSlicesHP planes); digits come from the FP64 bit pattern
// by integer arithmetic.
rgf_status slice_rows_f64(int batch, int m, int k, const double2* A, long sA, __nv_bfloat16* out, int Kp,
                          const int* active, cudaStream_t st);
rgf_status slice_cols_f64(int batch, int k, int n, const double2* B, long sB, __nv_bfloat16* out, int Kp,
                          const int* active, cudaStream_t st);

// Reference core on the legacy warp-level tensor path (mma.sync BF16).
rgf_status oz_gemm_mma(const OzGemm& g, cudaStream_t st);
// Blackwell core: TMA -> shared memory -> tcgen05.mma -> TMEM accumulators.
rgf_status oz_gemm_tc(const OzGemm& g, cudaStream_t st);
// Which core oz_gemm uses (0 = tcgen05, 1 = mma.sync); set by the plan.
rgf_status oz_gemm(const OzGemm& g, int core, cudaStream_t st);

// Elementwise df kernels (batch of b x b matrices, stride b*b unless noted).
rgf_status to_dfc(long n, const double2* src, float4* dst, cudaStream_t st);
// out[s*W+e] = z_e S' - H' - sub[s*W+e] in df arithmetic; S, H df blocks.
struct FormSrcDf {
    const float4* S[2];
    const float4* H[2];
    int trans[2];
};
rgf_status form_dfc(int W, int nsrc, int b, const double* E, double eta, const FormSrcDf& src, float4* out,
                    const float4* sub, const int* active, cudaStream_t st);
rgf_status dfc_hi_to_c64(int batch, int b, const float4* X, float2* Y, const int* active, cudaStream_t st);
rgf_status c64_to_dfc(int batch, int b, const float2* X, float4* Y, const int* active, cudaStream_t st);
rgf_status copy_dfc(int batch, int b, float4* dst, const float4* src, const int* active, cudaStream_t st);
rgf_status set_identity_dfc(int batch, int b, float4* A, cudaStream_t st);
rgf_status dec_update_dfc(int batch, int b, float4* eps_s, float4* eps, const float4* agb, const float4* bga,
                          const int* active, cudaStream_t st);
rgf_status dec_check_dfc(int batch, int b, const float4* alpha, const float4* beta, const double* anorm, double tol,
                         int it, int* active, int* iters, int* remaining, cudaStream_t st);
rgf_status fro_norm_dfc(int batch, int b, const float4* A, double* out, cudaStream_t st);
rgf_status gamma_dfc(int batch, int b, const float4* sigma, float4* gamma, cudaStream_t st);
rgf_status axpy_dfc(int batch, int b, float alpha, const float4* X, float4* Y, cudaStream_t st);
// A double-float inverse is done once |I - M X|_F <= kNsTol: after that
// step's correction its residual is about |I - M X|_F^2 <= 1e-12.  (3e-7,
// i.e. 1e-13, moved T by at most 5e-8 on the stored oracle grids at b = 128
// and 256, against 1e-6 allowed; 1e-6 spares most inverses a third step.)
// The FP64-class inverses of the lead decimation keep 3e-7.
constexpr double kNsTol = 1e-6;
// The FP64-class inverses of the lead decimation take an FP32 seed with
// |I - M X0|_F < kHpBad and refine it, with up to kHpSteps Newton-Schulz
// steps: any |R|_F < 1 bounds the spectral radius below one, so the
// iteration converges (from 0.9 in about nine steps, each a masked pair of
// slice products for the few such entries); seeds at or above it are
// replaced (the previous decimation iteration's inverse, else the FP64
// Gauss-Jordan inverse, which runs one matrix per SM on the narrow FP64
// pipe: about 13 ms per event at b = 256).
constexpr double kHpBad = 0.98;
constexpr int kHpSteps = 12;

// Newton-Schulz bookkeeping for step s of at most max_steps on batch
// entries i (energy e = i mod W), given R = I - M X:
//   step 0: theta[i] = 1 / (1 - tr R_i) for a finite residual with
//     |R_i|_F >= 0.5 (Sherman-Morrison scale of the first correction for a
//     seed whose error is one near-singular direction), else 1;
//   step 1: entries with |R_i|_F >= 0.5 (or not finite) get bad[i] = 1,
//     are counted in *bad_count and flagged RGF_FLAG_REFINE; the caller
//     reseeds them with an FP64 inverse;
//   next_act[i] = act[i] && |R_i|_F > kNsTol (after this step's correction
//     the residual is below |R_i|^2 <= 1e-12, so the entry is done);
//   err[e] = max(err[e], estimated final residual); an entry still above
//     kNsTol on the last step is flagged RGF_FLAG_REFINE.
// more_count (may be null) counts the entries with next_act = 1.
// rsq / rtr (may be null): the residual GEMM's per-block statistics (see
// OzGemm); then |R|_F and tr R come from them instead of reading R.
rgf_status ns_check(int batch, int W, int b, const float4* R, double* err, int* flags, int step, int max_steps,
                    const int* act, int* next_act, int* bad, int* bad_count, double2* theta, cudaStream_t st,
                    int* more_count = nullptr, const float* rsq = nullptr, const double2* rtr = nullptr);
// Slots of those statistics per batch entry.
__host__ __device__ inline int rstat_slots(int b) { return ((b + 31) / 32) * ((b + 7) / 8); }
// R[i] *= theta[i] (complex) where theta[i] != 1.
rgf_status scale_theta(int batch, int b, float4* R, const double2* theta, const int* act, cudaStream_t st);
rgf_status ns_check_f64(int batch, int W, int b, const double2* R, double* err, int* flags, int step, int max_steps,
                        const int* act, int* next_act, int* bad, int* bad_count, cudaStream_t st,
                        int* more_count = nullptr);
rgf_status c128_to_c64(int batch, int b, const double2* X, float2* Y, const int* mask, cudaStream_t st);
rgf_status c64_to_c128(int batch, int b, const float2* X, double2* Y, const int* mask, cudaStream_t st);
// Masked conversions between df and FP64 complex (entries with mask[i]).
rgf_status dfc_to_c128(int batch, int b, const float4* X, double2* Y, const int* mask, cudaStream_t st);
rgf_status c128_to_dfc(int batch, int b, const double2* X, float4* Y, const int* mask, cudaStream_t st);
// out[i] = act ? act[i] : 1
rgf_status mask_init(int batch, const int* act, int* out, cudaStream_t st);
// For FP64 inverses reseeded from a nearby inverse (mask): still_bad where
// |I - M X|_F >= kHpBad (counted), next_act = |R|_F > 3e-7 for the mask entries.
rgf_status recheck_f64(int batch, int b, const double2* R, const int* mask, int* still_bad, int* count,
                       int* next_act, cudaStream_t st);
// *acc += *count (one thread)
rgf_status accumulate_count(long long* acc, const int* count, cudaStream_t st);
// T[i] = Re sum X_jk conj(Y_jk) reduced in FP64 from df inputs.
rgf_status trace_dfc(int batch, int b, const float4* X, const float4* Y, double* T, double* Ti, cudaStream_t st);

}  // namespace rgf
