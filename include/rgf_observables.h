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

#ifdef __cplusplus
}
#endif

#endif /* RGF_OBSERVABLES_H */
