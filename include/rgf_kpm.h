/*
 * rgf_kpm.h - non-orthogonal kernel polynomial method (KPM) for the Fermi
 * level of a block-tridiagonal device.
 *
 * The paper determines the Fermi level without diagonalization (Results:
 * the generalized problem H c = eps S c in a nonorthogonal basis; the
 * rescaled operator A~ = S^-1 (H - beta S) / alpha expanded in Chebyshev
 * polynomials, its action on a vector evaluated by solving linear systems
 * with S rather than forming S^-1; the Chebyshev moments reconstruct the
 * density of states, which fixes E_F through the electron count; the cost
 * paragraph: O(N_mom N_rand N)).  The paper calls the scale and shift a and
 * b; here they are alpha and beta (b is the block size).
 *
 * Computation (FP64 on the CUDA cores):
 *   - S = L D L^dag, block LDL of the block-tridiagonal overlap, once per
 *     context: D_0 = S_00, F_i = S_{i,i-1} D_{i-1}^-1,
 *     D_i = S_ii - F_i S_{i,i-1}^dag; D_i^-1 and F_i are kept;
 *   - per Chebyshev step and random vector: t = H v, then S x = t by the
 *     forward substitution w_i = t_i - F_i w_{i-1} and the backward one
 *     x_i = D_i^-1 w_i - F_{i+1}^dag x_{i+1}; A~ v = (x - beta v) / alpha;
 *     v_{n+1} = 2 A~ v_n - v_{n-1} (v_1 = A~ v_0, v_0 = r);
 *   - moments mu_n = (1/R) sum_r Re(r^dag v_n);
 *   - Jackson kernel g_n, integrated density of states
 *     N(x) = g_0 mu_0 (pi - theta)/pi - (2/pi) sum_{n>=1} g_n mu_n sin(n theta)/n,
 *     theta = arccos x, and E_F with spin * N((E_F - beta)/alpha) = n_electrons
 *     by bisection.
 * Layouts: blocks as rgf.h (complex128, row-major, lower off-diagonal
 * blocks).  Random vectors: n_rand vectors of n_layers * b complex128
 * entries each, vector-major (vector c, layer i, row r at
 * (c * n_layers + i) * b + r).
 */
#ifndef RGF_KPM_H
#define RGF_KPM_H

#include "rgf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rgf_kpm_s* rgf_kpm_t;

/* Copy H and S (n_layers >= 1 blocks of size 1 <= b <= 512; lower blocks may
 * be NULL when n_layers == 1; memory space mem) into a new context on the
 * current device and factor S.  Work is ordered on cuda_stream (NULL =
 * legacy default stream); returns when the factorization is done.
 * RGF_E_INVALID for bad sizes or pointers, or when a pivot of the
 * factorization is exactly zero (S singular). */
rgf_status rgf_kpm_create(rgf_kpm_t* kpm, int n_layers, int b, const double* H_diag, const double* S_diag,
                          const double* H_lower, const double* S_lower, int mem, void* cuda_stream);

/* Spectral scale by power iteration on S^-1 H (the paper does not say how
 * a and b are chosen): starting from x0 (device, n_layers * b complex128),
 * iters steps v <- S^-1 H v / |S^-1 H v| with the same passes as the
 * moments; the last ratio rho estimates the largest |eps| from below, and
 * *alpha = (1 + margin) rho, *beta = 0 (host outputs).  Choose the margin
 * for the iteration count (0.05 after ~100 steps on the synthetic
 * junctions); rgf_kpm_moments rejects a scale that leaves the spectrum
 * outside [-1, 1].  Blocking. */
rgf_status rgf_kpm_scale(rgf_kpm_t kpm, const double* x0, int iters, double margin, double* alpha, double* beta);

/* mu[n], n < n_mom (n_mom >= 2), from n_rand >= 1 random vectors R (device
 * memory, layout above); mu is device memory.  Blocking.  The spectrum of
 * (H - beta S)/alpha relative to S must lie in [-1, 1] (the recursion
 * diverges otherwise; use rgf_kpm_scale): a moment above 10 mu_0 in
 * magnitude returns RGF_E_INVALID.  Allocates n_rand * 3 vectors of
 * workspace for the call. */
rgf_status rgf_kpm_moments(rgf_kpm_t kpm, double alpha, double beta, int n_rand, const double* R, int n_mom,
                           double* mu);

/* E_F (one double, device memory) from the moments mu (device, n_mom):
 * spin * N((E_F - beta) / alpha) = n_electrons, bisection to the last bit.
 * Stream-ordered on cuda_stream; returns at once. */
rgf_status rgf_kpm_fermi(int n_mom, const double* mu, double alpha, double beta, double n_electrons, double spin,
                         double* E_F, void* cuda_stream);

/* Release the context (NULL is a no-op). */
rgf_status rgf_kpm_destroy(rgf_kpm_t kpm);

#ifdef __cplusplus
}
#endif

#endif /* RGF_KPM_H */
