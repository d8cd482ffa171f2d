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
#include "rgf_server.h"

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

/* A transverse-periodic device: every block given per lattice vector R. */
typedef struct {
    int n_R;               /* 1..64 lattice vectors */
    const int* R;          /* host, n_R x 2 ints */
    int n_layers;          /* >= 1 */
    int b;                 /* 1..512 */
    const double* H_diag;  /* device, n_R x n_layers x b x b complex128 (r-major) */
    const double* S_diag;
    const double* H_lower; /* device, n_R x (n_layers - 1) x b x b; NULL when n_layers == 1 */
    const double* S_lower;
    const double* lead[2]; /* device, n_R x 6 x b x b per side: H00, S00, H10, S10, Hc, Sc */
} rgf_kdevice;

/* T(E) per unit transverse cell, averaged over a k mesh (the transmission
 * "per transverse k-point" of the Results' cost paragraph, summed with the
 * mesh weights of the Methods' Monkhorst-Pack sampling).  For each k-point:
 * the Bloch sums of every device and lead block (rgf_bloch_sum) into
 * library-owned device memory, one request to `server`, its T(E, k) into
 * row k of T_k; then T = sum_k w[k] T_k[k] (rgf_kmesh_mean).  `group`
 * k-points (1..64) are in flight in the server at once, so their sweeps
 * share launches.
 *   kfrac  host, n_k x 2 doubles (fractional reciprocal coordinates);
 *   w      host, n_k weights;
 *   E      host, n_E energies; eta > 0 as rgf_server's requests;
 *   T      device, n_E doubles (output);
 *   T_k    device, n_k x n_E doubles (output; may be NULL).
 * Blocking: returns when T is written (on cuda_stream, NULL = legacy
 * default stream) or at the first failure (a request's error is returned,
 * its message in rgf_last_error).  Allocates group x (blocks of one
 * device) of device memory for the Bloch-summed blocks, freed on return.
 * RGF_E_INVALID for sizes out of range or null pointers. */
rgf_status rgf_kmesh_transmission(rgf_server_t server, const rgf_kdevice* dev, int n_k, const double* kfrac,
                                  const double* w, const double* E, int n_E, double eta, int group, double* T,
                                  double* T_k, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* RGF_KPOINTS_H */
