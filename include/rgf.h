/*
 * rgf.h - C ABI of the B300 recursive-Green's-function transmission library.
 *
 * The library computes the zero-bias transmission spectrum T(E) of a
 * two-terminal device whose Hamiltonian H and overlap S are block
 * tridiagonal in a nonorthogonal basis, connected to two semi-infinite
 * periodic leads.  This is the transport step of the paper's workflow
 * (Results: the RGF step costs O(N_z M_b^3) per energy point; Methods:
 * the device Hamiltonian is combined with electrode self-energies and the
 * zero-bias transmission is evaluated; Results: the generalized problem
 * H c = eps S c in a nonorthogonal basis).  For every energy E, with
 * z = E + i*eta applied to S everywhere:
 *
 *   g_L, g_R   lead surface Green's functions by Sancho-Rubio decimation
 *   Sigma_L    = M_{0,-1} g_L M_{-1,0},  Sigma_R = M_{N-1,N} g_R M_{N,N-1}
 *   Gamma      = i (Sigma - Sigma^dagger)
 *   g_0        = (A_0 - Sigma_L)^-1,  A_i = z S_ii - H_ii
 *   g_i        = (A_i - tau_i g_{i-1} tau'_i [- Sigma_R at i = N-1])^-1
 *   G_{0,N-1}  = (-1)^{N-1} g_0 tau'_1 g_1 ... tau'_{N-1} g_{N-1}
 *   T(E)       = Re Tr[Gamma_L G_{0,N-1} Gamma_R G_{0,N-1}^dagger]
 *
 * where M = zS - H, tau_i = M_{i,i-1} = z S_{i,i-1} - H_{i,i-1} and
 * tau'_i = M_{i-1,i} = z S_{i,i-1}^dagger - H_{i,i-1}^dagger.
 *
 * Data layout (all calls): a complex matrix is b*b pairs of doubles
 * (re, im), row-major.  Arrays of blocks are block-major and contiguous.
 * Orientation: every off-diagonal block passed in is the LOWER block, the
 * one whose row cell is to the right of its column cell:
 *   H_lower[i-1] = H_{i,i-1}, i = 1..N-1;
 *   lead H10 = H_{j+1,j} between consecutive lead cells;
 *   lead Hc  = H_{0,-1} for the left lead, H_{N,N-1} for the right lead.
 * Upper blocks are their conjugate transposes.
 *
 * Memory: `mem` selects RGF_MEM_HOST (pageable or pinned host memory) or
 * RGF_MEM_DEVICE (device pointers on the plan's GPU, e.g. a torch tensor's
 * data_ptr()).  Input blocks are copied into plan-owned device memory; the
 * caller keeps ownership of every pointer it passes and may free it once
 * the call returns.  Outputs are written into caller-owned arrays.
 *
 * Errors: every call returns an rgf_status; no exception crosses the ABI.
 * A call that fails leaves a message for rgf_last_error() (thread-local).
 * Per-energy numerical trouble (a decimation that did not converge, a
 * singular pivot, a mixed-precision inverse whose refinement did not
 * contract) does not fail the call: it sets bits in flags[k] and the
 * energy's T is NaN when the result is unusable.
 */
#ifndef RGF_H
#define RGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rgf_plan_s* rgf_plan_t;
typedef uint64_t rgf_ticket_t;

typedef enum {
    RGF_OK = 0,
    RGF_E_INVALID = 1,   /* bad argument (null pointer, size out of range, ...) */
    RGF_E_OOM = 2,       /* device allocation failed */
    RGF_E_CUDA = 3,      /* a CUDA runtime call failed */
    RGF_E_NOT_READY = 4, /* rgf_poll: the ticket has not finished yet */
    RGF_E_NOCONV = 5,    /* reserved: per-energy non-convergence goes to flags */
    RGF_E_TIMEOUT = 6,   /* rgf_poll: waited timeout_us without completion */
    RGF_E_REJECTED = 7,  /* a request that can never fit the memory cap */
    RGF_E_STATE = 8      /* call out of order (e.g. transmission before blocks) */
} rgf_status;

typedef enum {
    RGF_FP64 = 0,  /* every step in IEEE binary64 on the CUDA cores */
    RGF_MIXED = 1  /* complex GEMMs as exact BF16 slice products on the tensor
                      cores with double-float (2 x FP32) results; FP32
                      inverse refined by Newton-Schulz to double-float */
} rgf_precision;

typedef enum { RGF_MEM_HOST = 0, RGF_MEM_DEVICE = 1 } rgf_memspace;

typedef enum { RGF_LEAD_LEFT = 0, RGF_LEAD_RIGHT = 1 } rgf_side;

/* Per-energy flag bits written to flags[k]. */
#define RGF_FLAG_NOCONV_L   0x1  /* left-lead decimation hit dec_max_iter  */
#define RGF_FLAG_NOCONV_R   0x2  /* right-lead decimation hit dec_max_iter */
#define RGF_FLAG_SINGULAR   0x4  /* an exactly zero pivot in an inverse     */
#define RGF_FLAG_REFINE     0x8  /* mixed path: an FP32 inverse seed had
                                    ||I - M X||_F >= 0.5 and was replaced by
                                    an FP64 seed (in the lead decimation
                                    first by the previous iteration's
                                    inverse), or the last Newton-Schulz step
                                    left ||I - M X||_F above 1e-6 (3e-7 in
                                    the lead decimation)                    */
#define RGF_FLAG_LEAD_NEWTON 0x10 /* a lead's surface Green's function kept
                                    its decimation value: the Newton step
                                    that refines it diverged (its Stein
                                    doubling grew instead of converging;
                                    near band edges at small eta)          */

typedef struct {
    int precision;     /* rgf_precision; default RGF_FP64 */
    double eta;        /* broadening added to E; default 1e-6 */
    double dec_tol;    /* decimation stops when max(|alpha|_F,|beta|_F) <=
                          dec_tol * |a|_F; default 1e-14 */
    int dec_max_iter;  /* default 100 */
    int ns_steps;      /* most Newton-Schulz steps per mixed inverse; each
                          matrix stops once its residual predicts
                          convergence (usually after 2); default 6 */
    int energy_wave;   /* energies per device pass; 0 = chosen from b and
                          free memory */
} rgf_options;

/* Fill *opt with the defaults listed above. */
void rgf_options_default(rgf_options* opt);

/* Create a plan for devices with n_layers >= 1 principal layers of block
 * size 1 <= b <= 512 (the paper's N_z principal layers of size M_b, Results,
 * the paragraph on the cost of each part of the workflow).  opt may be NULL (defaults).  cuda_stream is a
 * cudaStream_t (NULL = the legacy default stream); all work of the plan is
 * ordered on it.  The plan owns its device memory until rgf_plan_destroy. */
rgf_status rgf_plan_create(rgf_plan_t* plan, int n_layers, int b, const rgf_options* opt,
                           void* cuda_stream);

/* Copy the device Hamiltonian and overlap into the plan (the static device
 * Hamiltonian in a nonorthogonal localized basis, block tridiagonal in
 * principal layers: Results, generalized eigenproblem paragraph, and the
 * cost paragraph).  Hermiticity of the diagonal blocks is checked on the
 * host (RGF_E_INVALID otherwise).
 * H_diag, S_diag: n_layers blocks; H_lower, S_lower: n_layers-1 blocks
 * (may be NULL when n_layers == 1). */
rgf_status rgf_set_device_blocks(rgf_plan_t plan, const double* H_diag, const double* S_diag,
                                 const double* H_lower, const double* S_lower, int mem);

/* Copy one lead (the semi-infinite electrodes whose self-energies are
 * combined with the device Hamiltonian: Methods, transport paragraph):
 * H00/S00 on-site blocks of a lead cell, H10/S10 the
 * coupling between consecutive lead cells, Hc/Sc the lead-device coupling
 * (orientation as stated at the top of this file). */
rgf_status rgf_set_leads(rgf_plan_t plan, int side, const double* H00, const double* S00,
                         const double* H10, const double* S10, const double* Hc,
                         const double* Sc, int mem);

/* T(E_k) for k < n_E, synchronous: the zero-bias transmission of the
 * Methods' transport paragraph, evaluated per energy point by the recursive
 * sweep whose cost the Results' cost paragraph states as O(N_z M_b^3) per
 * energy point (formulas at the top of this file).  E, T, err and flags are all in memory
 * space `mem`.  err[k] (may be NULL) receives, for the mixed path, the
 * largest estimated residual ||I - M X||_F of the energy's refined inverses
 * (|R|^2 of the last Newton-Schulz residual R before its correction), and 0
 * for the FP64 path; flags[k] (may be NULL) receives RGF_FLAG_* bits.
 * n_E = 0 is allowed and does nothing. */
rgf_status rgf_transmission(rgf_plan_t plan, const double* E, int n_E, double* T, double* err,
                            int* flags, int mem);

/* Asynchronous form of rgf_transmission (no counterpart in the paper, which
 * ran its transport on CPUs): copy n_E host energies, enqueue the work on the plan's
 * stream and return a ticket at once.  The plan must not be modified or
 * destroyed until the ticket has been polled to completion. */
rgf_status rgf_submit(rgf_plan_t plan, const double* E, int n_E, rgf_ticket_t* ticket);

/* Collect a submitted result into host arrays T[n_E], err[n_E], flags[n_E]
 * (err/flags may be NULL).  timeout_us = 0 polls without blocking
 * (RGF_E_NOT_READY if still running); timeout_us < 0 waits indefinitely;
 * otherwise waits up to timeout_us and returns RGF_E_TIMEOUT.  A ticket is
 * released by the first call that returns RGF_OK. */
rgf_status rgf_poll(rgf_ticket_t ticket, double* T, double* err, int* flags, int timeout_us);

/* Counters of a plan since its creation (each output may be NULL): waves
 * run, and mixed-path inverses whose FP32 seed was replaced by an FP64 seed. */
rgf_status rgf_plan_stats(rgf_plan_t plan, long long* waves, long long* fp64_reseeds);

/* Device time (ms, CUDA events on the plan's stream) spent by the mixed path
 * since the plan's creation in its two phases: lead decimation with the
 * self-energies, and the layer sweep with the trace (0 for FP64 plans). */
rgf_status rgf_plan_phase_ms(rgf_plan_t plan, double* lead_ms, double* sweep_ms);

/* Device bytes the plan holds (blocks + workspace for one energy wave). */
rgf_status rgf_plan_device_bytes(rgf_plan_t plan, size_t* bytes);

/* Energies processed per device pass. */
rgf_status rgf_plan_energy_wave(rgf_plan_t plan, int* energy_wave);

/* Release the plan and its device memory (NULL is a no-op). */
rgf_status rgf_plan_destroy(rgf_plan_t plan);

/* Message of the last failed call on this thread ("" if none). */
const char* rgf_last_error(void);

/* Library version string. */
const char* rgf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RGF_H */
