// Kernel launch wrappers of the RGF library (host-callable, stream-ordered).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace rgf {

// Source blocks of a batched "z S - H" formation.  Batch entry be = s*W + e
// (s = side/source index < nsrc, e = energy index < W) reads S[s], H[s]
// (b x b, row-major complex128) and, when trans[s] != 0, their conjugate
// transposes.  S[s] == nullptr means S = 0.
struct FormSrc {
    const double2* S[2];
    const double2* H[2];
    int trans[2];
};

// out[be] = (E[e] + i eta) S' - H' - sub_coef * sub[be]   (sub may be null)
rgf_status form_f64(int W, int nsrc, int b, const double* E, double eta, const FormSrc& src,
                    double2* out, const double2* sub, double sub_coef, const int* active,
                    cudaStream_t st);

// Batched complex GEMM in FP64:  C[i] = alpha * A[i] B[i] + beta * Cin[i]
// for i < batch, A m x k (lda), B k x n (ldb), C m x n (ldc); batch strides
// in elements (0 = shared operand).  Columns [skip0, skip1) of C are not
// written.  active (may be null) masks batch entries.  Cin may alias C.
template <typename T2>
struct GemmArgs {
    int batch, m, n, k;
    T2 alpha, beta;
    const T2* A; long lda, sA;
    const T2* B; long ldb, sB;
    const T2* Cin; long ldcin, sCin;
    T2* C; long ldc, sC;
    const int* active;
    int skip0, skip1;
};
using ZGemm = GemmArgs<double2>;
rgf_status zgemm_f64(const ZGemm& g, cudaStream_t st);

// In-place batched inverse of b x b complex128 matrices by blocked
// Gauss-Jordan elimination with partial (row) pivoting.  ws must hold
// inv_f64_workspace_bytes(batch, b) bytes.  flags[i] |= RGF_FLAG_SINGULAR on
// an exactly zero pivot (flags may be null).
size_t inv_f64_workspace_bytes(int batch, int b);
rgf_status inv_f64(int batch, int b, double2* A, long sA, void* ws, int* flags,
                   const int* active, cudaStream_t st);

// In-place batched inverse of b x b complex64 matrices (the mixed path's
// seed): the same blocked Gauss-Jordan elimination, with each trailing
// update C += Pbar T on the tensor cores.  Every FP32 value x of Pbar and
// T is split into three BF16 values x0 = bf16(x), x1 = bf16(x - x0), x2 =
// bf16(x - x0 - x1) (x = x0 + x1 + x2 within 2^-24 |x|); the six split
// pairs i + j <= 2 are accumulated in FP32 (the dropped pairs are below
// 2^-23 of the product), i.e. the update is FP32-accurate.  Layouts, per
// batch entry and split, kGjKp BF16 per row, K index 2 j + (0 re, 1 im):
//   Pbar splits [split][b rows][kGjKp]: (Re, Im) of Pbar[r][j];
//   T splits [split][2b rows][kGjKp]: row 2c = (Re T[j][c], -Im T[j][c]),
//   row 2c + 1 = (Im T[j][c], Re T[j][c]).
// status: the tensor-core pipeline's wait-timeout word (bits set on a
// timeout); null selects the CUDA-core update.  RGF_GJ_TC=0 in the
// environment (read once) selects it too.
constexpr int kGjSplits = 3;
constexpr int kGjKp = 64;
size_t inv_c32_workspace_bytes(int batch, int b);
rgf_status inv_c32(int batch, int b, float2* A, long sA, void* ws, int* flags, const int* active, int* status,
                   cudaStream_t st, int nb_override = 0);
// The same, with the inverse written to out (contiguous b x b per entry) as
// double-float complex (hi = the FP32 value, lo = 0) or as complex128,
// instead of back to A (A keeps the inverse with its columns interchanged).
rgf_status inv_c32_to(int batch, int b, float2* A, long sA, void* ws, int* flags, const int* active, int* status,
                      cudaStream_t st, int nb_override, float4* out_df, double2* out_c128);
// One trailing update: C[:, not in [skip0, skip1)] += Pbar T from the splits
// (nbk <= 32 columns of Pbar; K padded with zeros to kGjKp).
rgf_status gj_update_tc(int batch, int b, int nbk, const __nv_bfloat16* Ps, const __nv_bfloat16* Ts, float2* C,
                        long sC, int skip0, int skip1, const int* active, int* status, cudaStream_t st);

// Elementwise helpers (batch of b x b matrices, stride b*b).
rgf_status set_identity_f64(int batch, int b, double2* A, cudaStream_t st);
// eps_s -= agb ; eps -= agb + bga   (decimation update)
rgf_status dec_update_f64(int batch, int b, double2* eps_s, double2* eps, const double2* agb,
                          const double2* bga, const int* active, cudaStream_t st);
// gamma = i (sigma - sigma^dagger)
rgf_status gamma_f64(int batch, int b, const double2* sigma, double2* gamma, cudaStream_t st);
// Decimation convergence: for active i, if max(|alpha_i|_F, |beta_i|_F) <=
// tol * anorm[i] then active[i] = 0; iters[i] = it while active; counts the
// entries still active into *remaining (zeroed by the caller).
rgf_status dec_check_f64(int batch, int b, const double2* alpha, const double2* beta,
                         const double* anorm, double tol, int it, int* active, int* iters,
                         int* remaining, cudaStream_t st);
// anorm[i] = |A_i|_F
rgf_status fro_norm_f64(int batch, int b, const double2* A, double* out, cudaStream_t st);
// T[i] = Re sum_jk X_jk conj(Y_jk); Timag[i] = Im of the same sum.
rgf_status trace_xy_f64(int batch, int b, const double2* X, const double2* Y, double* T,
                        double* Timag, cudaStream_t st);
// Copy with batch masks: dst[i] = src[i] for active i.
rgf_status copy_f64(int batch, int b, double2* dst, const double2* src, const int* active,
                    cudaStream_t st);

// Y[i] += alpha * X[i]  (real alpha)
rgf_status axpy_f64(int batch, int b, double alpha, const double2* X, double2* Y, cudaStream_t st);
// Newton refinement of the lead surface Green's functions (the retarded
// fixed point of g = (a - alpha g beta)^-1; Sancho-Rubio's recursion loses
// digits at some energies):
// out[i] = (mask ? mask[i] : 1) && !dec_active[i]: the converged entries.
rgf_status newton_mask(int n, const int* mask, const int* dec_active, int* out, cudaStream_t st);
// Doubling of the Stein equation: for active i, p = |A_i|_F |B_i|_F (p0[i]
// records p on the first call, first != 0); p <= tol: converged
// (status[i] = 1, active[i] = 0); p not finite or > growth p0[i]: diverged
// (status[i] = 2, active[i] = 0); else *remaining += 1 (zeroed by the caller).
rgf_status stein_check_f64(int batch, int b, const double2* A, const double2* B, double tol, double growth,
                           int first, double* p0, int* status, int* active, int* remaining, cudaStream_t st);
// End of one Newton step for the entries of mask: converged (status 1):
// g += X, and next[i] = |X|_F > again |g|_F (another step is worth taking);
// otherwise g is kept, next[i] = 0 and flags[i] |= RGF_FLAG_LEAD_NEWTON.
// Counts the next[] entries into *remaining (zeroed by the caller).
rgf_status newton_finish_f64(int batch, int b, const double2* X, double2* g, const int* mask, const int* status,
                             double again, int* next, int* flags, int* remaining, cudaStream_t st);
// C[i] = A[i] - B[i] and Y[i] += alpha X[i] for active i (masks may be null).
rgf_status sub_f64(int batch, int b, const double2* A, const double2* B, double2* C, const int* active,
                   cudaStream_t st);
rgf_status axpy_masked_f64(int batch, int b, double alpha, const double2* X, double2* Y, const int* active,
                           cudaStream_t st);
// A[i] += s I for active i.
rgf_status add_identity_f64(int batch, int b, double s, double2* A, const int* active, cudaStream_t st);

// flags[e] |= dec_flags[e] | dec_flags[W+e] | NOCONV bits from the
// decimation active masks (still active after the last iteration).
rgf_status merge_dec_flags(int W, const int* dec_flags, const int* dec_active, int* flags,
                           cudaStream_t st);

}  // namespace rgf
