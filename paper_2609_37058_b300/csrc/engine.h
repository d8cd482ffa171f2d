// Table-driven kernels of the multi-device engine: every batch entry (an
// energy slot or a decimation item) reads its own blocks through a table
// that the host rebuilds before each launch sequence.
#pragma once

#include "mixed.h"

namespace rgf {

// One energy slot for one sweep step (layer l of its device).
struct SlotTab {
    const float4* Sii;  // S_ll, H_ll (df, bc x bc)
    const float4* Hii;
    const float4* Sl;   // S_{l,l-1}, H_{l,l-1}; null at the first layer
    const float4* Hl;
    double E, eta;
    double* outT;       // where the item's results go (set on its last layer)
    double* outErr;
    int* outFlags;
    int ready;          // index in the ready buffer when the slot is refilled now
    int ready_D;        // items of the decimation batch that filled the ready buffer
};

// Masks that accompany a table of S slots (each an int[S] array).
struct SlotMasks {
    const int* act;    // slot active this step
    const int* nf;     // active and not on its first layer (may be null)
    const int* first;  // active and on its first layer
    const int* last;   // active and on its last layer
    const int* refill; // slot starts a new item this step
};

// One decimation item: lead blocks [side][H00, S00, H10, S10, Hc, Sc] (FP64,
// bc x bc each, contiguous) and its energy.
struct DecTab {
    const double2* lead;
    double E, eta;
};

// dst (bc x bc per block) = src (b x b per block) padded with zeros, and
// diag_fill on the padded part of the diagonal.
rgf_status pad_to_dfc(int nblk, int b, int bc, const double2* src, float4* dst, double diag_fill, cudaStream_t st);
rgf_status pad_f64(int nblk, int b, int bc, const double2* src, double2* dst, double diag_fill, cudaStream_t st);

// Refilled slots: copy the item's Sigma_L, Sigma_R, Gamma_L, Gamma_R (ready
// buffer, entries r, D + r for Sigma and 2D + r, 3D + r for Gamma, with
// r = tab[s].ready and D = tab[s].ready_D) into the slot store (entries s,
// S + s, 2S + s, 3S + s) and reset err/flags from the item's decimation
// results.
rgf_status engine_refill(int S, int bc, const SlotTab* tab, const int* refill, const float4* ready,
                         float4* store, const double* dec_err, const int* dec_flags, double* slot_err,
                         int* slot_flags, cudaStream_t st);
// BF16 slices of the slots' coupling blocks, formed on the fly from the
// table (mask: slots past their first layer):
//   form_slice_rows_tab:     A operand tau  = z S_{l,l-1} - H_{l,l-1};
//   form_slice_cols_dag_tab: B operand tau' = z S_{l,l-1}^dagger - H_{l,l-1}^dagger.
rgf_status form_slice_rows_tab(int S, int b, const SlotTab* tab, const int* mask, __nv_bfloat16* out, int Kp,
                               cudaStream_t st);
rgf_status form_slice_cols_dag_tab(int S, int b, const SlotTab* tab, const int* mask, __nv_bfloat16* out, int Kp,
                                   cudaStream_t st);
// M = z S_ll - H_ll - [first] Sigma_L - [last] Sigma_R for active slots;
// Ut = z S_{l,l-1}^dagger - H_{l,l-1}^dagger, Lt = z S_{l,l-1} - H_{l,l-1}
// for slots past their first layer (skipped when mk.nf is null).
rgf_status engine_form_step(int S, int bc, const SlotTab* tab, SlotMasks mk, const float4* sigL, const float4* sigR,
                            float4* M, float4* Ut, float4* Lt, cudaStream_t st);
rgf_status set_identity_masked_dfc(int S, int bc, float4* A, const int* mask, cudaStream_t st);
// T[s] = Re sum X_jk conj(Y_jk) for masked slots.
rgf_status trace_masked_dfc(int S, int bc, const float4* X, const float4* Y, const int* mask, double* T,
                            cudaStream_t st);
// Write the results of slots on their last layer to their items' outputs.
rgf_status engine_finish(int S, const SlotTab* tab, const int* last, const double* slot_T, const double* slot_err,
                         const int* slot_flags, cudaStream_t st);
// Decimation inputs for D items (entries s*D + j): eps = eps_s = z S00 - H00,
// alpha = outward coupling, beta = inward coupling of side s (FP64).
rgf_status engine_form_dec(int D, int bc, const DecTab* tab, double2* eps_s, double2* eps, double2* alpha,
                           double2* beta, cudaStream_t st);
// Lead-device couplings: x1 = M_{0,-1} (left) / M_{N-1,N} (right),
// x2 = M_{-1,0} (left) / M_{N,N-1} (right), so that Sigma = x1 g x2.
rgf_status engine_form_coupling(int D, int bc, const DecTab* tab, double2* x1, double2* x2, cudaStream_t st);

}  // namespace rgf
