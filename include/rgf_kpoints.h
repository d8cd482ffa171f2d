/*
 * rgf_kpoints.h - transverse k-point Bloch sums for the transmission path.
 *
 * The paper states the RGF cost per energy point and per transverse k-point
 * (Results, the scaling paragraph) and samples transverse Brillouin zones
 * with Monkhorst-Pack meshes (Methods, transport paragraph).  For a device
 * that is periodic in the transverse directions, every block of H and S is
 * a lattice sum over transverse cell vectors R:
 *
 *   X(k) = sum_R exp(2 pi i (k1 R1 + k2 R2)) X(R),
 *
 * with k in fractional reciprocal coordinates and R in integer lattice
 * coordinates.  The k-resolved blocks then go through rgf_transmission or
 * rgf_server_submit like any other device, and the transmission per unit
 * cell is the weighted mean of T(E, k) over the mesh.  The upper blocks are
 * the conjugate transposes of the lower blocks at the same k, which is the
 * Bloch sum of the R -> -R upper blocks, so only lower blocks are summed.
 */
#ifndef RGF_KPOINTS_H
#define RGF_KPOINTS_H

#include "rgf.h"

#ifdef __cplusplus
extern "C" {
#endif

/* X_k[i] = sum_r phase_r X_R[r][i] for the n_blocks blocks of size b x b
 * (complex128, row-major, block-major), phase_r = exp(2 pi i k.R_r).
 *   R      host, n_R x 2 ints (R1, R2) per lattice vector;
 *   kfrac  host, 2 doubles (k1, k2);
 *   X_R    device, n_R x n_blocks x b x b complex128 (r-major);
 *   X_k    device, n_blocks x b x b complex128 (must not overlap X_R).
 * Stream-ordered on cuda_stream (NULL = legacy default stream); returns at
 * once.  RGF_E_INVALID unless 1 <= n_R <= 64, n_blocks >= 1, b >= 1 and the
 * pointers are non-null. */
rgf_status rgf_bloch_sum(int n_R, const int* R, const double* kfrac, int n_blocks, int b, const double* X_R,
                         double* X_k, void* cuda_stream);

/* T[e] = sum_k w[k] T_k[k][e] for e < n_E (the mesh average of T(E, k)).
 * T_k (n_k x n_E), w (n_k) and T (n_E) are device arrays of doubles.
 * Stream-ordered; RGF_E_INVALID for n_k < 1, n_E < 1 or null pointers. */
rgf_status rgf_kmesh_mean(int n_k, int n_E, const double* T_k, const double* w, double* T, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* RGF_KPOINTS_H */
