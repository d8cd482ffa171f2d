/*
 * rgf_observables.h - quantities derived from the transmission spectrum.
 *
 * Landauer current (the paper's Eq. 1, with the electrode chemical
 * potentials shifted by the bias and the Hamiltonian kept at zero bias, as
 * in its finite-bias discussion of the electrode potentials):
 *
 *   I(V) = G0 * integral T(E) [f(E - mu_L) - f(E - mu_R)] dE,
 *   mu_L = E_F + V/2,  mu_R = E_F - V/2,  f(x) = 1 / (1 + exp(x / kT)),
 *
 * with E, V, E_F and kT in eV, G0 = 2 e^2 / h = 7.748091729863649e-5 S and
 * I in ampere.  The integral is the trapezoidal rule on the caller's energy
 * grid (the paper names no quadrature); the grid must cover the bias window
 * plus several kT.  At kT = 0, f is the step function with f(0) = 1/2.
 */
#ifndef RGF_OBSERVABLES_H
#define RGF_OBSERVABLES_H

#include "rgf.h"

#ifdef __cplusplus
extern "C" {
#endif

/* I[v] for the n_V biases V[v].  E (ascending), T (n_E), V (n_V) and I
 * (n_V) are device arrays of doubles.  Stream-ordered on cuda_stream.
 * RGF_E_INVALID for n_E < 2, n_V < 1, kT < 0 or null pointers. */
rgf_status rgf_current(int n_E, const double* E, const double* T, int n_V, const double* V, double E_F, double kT,
                       double* I, void* cuda_stream);

/* Layer-resolved density of states of a mixed-precision plan (blocks and
 * leads set):
 *
 *   D[k][i] = -(1/pi) Im Tr[(G S)_ii],  (G S)_ii = sum_j G_ij S_ji,
 *
 * the Mulliken partition of the device DOS over the principal layers, with G
 * the retarded device Green's function at z = E_k + i eta (lead self-energies
 * included) and j over the device layers.  The paper shows spatially
 * resolved LDOS of its finite-bias runs without a formula; this is the
 * reading used here.  Computed with a forward sweep that keeps every
 * left-connected g_i and the backward recursion
 *   G_ii = g_i + g_i M_{i,i+1} G_{i+1,i+1} M_{i+1,i} g_i,
 *   G_{i,i+1} = -g_i M_{i,i+1} G_{i+1,i+1},  G_{i+1,i} = -G_{i+1,i+1} M_{i+1,i} g_i,
 * in the mixed-precision arithmetic of RGF_MIXED.  E (n_E) and D (n_E x
 * n_layers, row-major) are in memory space `mem`.  The call allocates the
 * stored inverses (n_layers x b x b double-float per energy of a wave) and
 * shrinks the wave to fit 60% of free memory; RGF_E_OOM if one energy does
 * not fit, RGF_E_STATE for an FP64 plan or missing blocks. */
rgf_status rgf_ldos(rgf_plan_t plan, const double* E, int n_E, double* D, int mem);

#ifdef __cplusplus
}
#endif

#endif /* RGF_OBSERVABLES_H */
