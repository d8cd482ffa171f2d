// Mixed-precision workspace and the composite operations built on the
// slice-product GEMMs: refined inverses and Sancho-Rubio decimation.  Used by
// the single-device plan and by the multi-device server.
#pragma once

#include "mixed.h"

namespace rgf {

constexpr int kPoolUnits = 20;  // df matrices, in units of W
constexpr int kDecUnits = 32;   // FP64 decimation matrices, in units of W (26 + 6 kept for the Newton step)

// Workspace of W energies of block size b, with lead decimation for Wd
// energies (2 Wd lead entries) at a time.
struct MixedState {
    int b = 0, W = 0, Wd = 0, Kp = 0;
    int slice_entries = 0;   // batch entries the df slice buffers hold (W or 2W)
    int inv_entries = 0;     // batch entries of the inverse workspaces
    float4* pool = nullptr;  // kPoolUnits * W df matrices
    __nv_bfloat16* sa[2] = {};
    __nv_bfloat16* sb[2] = {};
    float2* c64 = nullptr;
    void* inv_ws = nullptr;
    int* status = nullptr;   // tcgen05 pipeline timeout word
    long long* reseed_acc = nullptr;  // FP64 reseeds counted on the device (graph mode)
    int* nsact[2] = {};
    int* bad = nullptr;
    int* bad2 = nullptr;     // entries still bad after a reseed from a nearby inverse
    int* bad_count = nullptr;
    int* more_count = nullptr;  // entries that need another Newton-Schulz step
    int* h_more = nullptr;      // pinned
    float* r_sumsq = nullptr;   // residual statistics (rstat_slots(b) per inverse entry)
    double2* r_trace = nullptr;
    int* h_bad = nullptr;    // pinned
    double2* c128 = nullptr;
    void* inv64_ws = nullptr;
    double2* theta = nullptr;  // 2W
    // High-precision lead decimation: FP64 matrices and seven-slice buffers.
    double2* dec_pool = nullptr;  // kDecUnits * W matrices
    __nv_bfloat16* hsa[2] = {};
    __nv_bfloat16* hsb[2] = {};
    // Decimation bookkeeping (2W entries each).
    int* dec_active = nullptr;
    int* dec_iters = nullptr;
    int* dec_flags = nullptr;
    double* dec_anorm = nullptr;
    int* dec_remaining = nullptr;
    int* dec_newton = nullptr;  // 2Wd: converged entries (Newton-refined)
    int* dec_smask = nullptr;   // 2Wd: the Newton step's doubling mask
    int* dec_next = nullptr;    // 2Wd: entries that take a second Newton step
    int* dec_status = nullptr;  // 2Wd: doubling outcome (1 converged, 2 diverged)
    double* dec_p0 = nullptr;   // 2Wd: first doubling's |A| |B|
    int* h_remaining = nullptr;  // pinned
    int core = 0;                // 0 = tcgen05, 1 = mma.sync reference core
    int bn = 96;                 // tcgen05 tile width of the double-float GEMM (64, 80, 96)
    int gj_nb = 0;               // panel width of the FP32 seed inverse (0 = default, 16 or 32)
    void* own = nullptr;         // allocation owned by the state (when ws was not given)
    void* dec_own = nullptr;
};

// Bytes of the carved workspace (without the decimation pool) for W energies
// whose df slice buffers hold slice_entries (W or 2W) batch entries and
// whose inverse workspaces hold inv_entries.  The two-argument form is the
// single-device plan's (slice and inverse buffers for 2W entries).
size_t mixed_workspace_bytes(int W, int b, int slice_entries, int inv_entries);
size_t mixed_workspace_bytes(int W, int b);
// Bytes of the decimation pool and its slice buffers for Wd energies.
size_t mixed_dec_bytes(int Wd, int b);
// Set up m for W energies of block size b and decimation batches of Wd
// energies (Wd <= W; 0 = W).  slice_entries: W when only W-entry products
// are sliced in double-float (the server's engines), 2W for the plan.  ws
// (mixed_workspace_bytes) may be null, in which case the state allocates it.
// The decimation pool and the small buffers are always allocated by the state.
rgf_status mixed_state_init(MixedState* m, int b, int W, void* ws, cudaStream_t st, int Wd = 0,
                            int slice_entries = 0);
void mixed_state_free(MixedState* m);

// What one batch of refined inverses writes besides X.
struct Ctx {
    MixedState* m;
    cudaStream_t st;
    long nn;
    int b;
    int ns_steps;
    double* err;           // per energy (entry i -> energy i mod W)
    int* flags;            // per energy
    long long* n_reseeds;  // host counter
    // Graph mode: no host synchronisation inside; the FP64 reseed path is
    // always launched, masked by the entries that need it, and reseeds are
    // counted in MixedState::reseed_acc.
    bool graph = false;
};

// Slice A by rows into sa[ia], B by columns into sb[ib] (the most
// significant `planes` slices); C = alpha A B (+ D) (+ I).
rgf_status sliceA(const Ctx& c, int cnt, int ia, const float4* A, const int* act, int planes = kSlices);
rgf_status sliceB(const Ctx& c, int cnt, int ib, const float4* B, const int* act, int planes = kSlices);
rgf_status mm(const Ctx& c, int cnt, int ia, int ib, float alpha, const float4* D, int addI, float4* C,
              const int* act, float2* C2 = nullptr, float* rsq = nullptr, double2* rtr = nullptr);
// C = A B + D from the four most significant slices of each operand.
rgf_status mm4(const Ctx& c, int cnt, int ia, int ib, const float4* D, float4* C, const int* act);
// Seven-slice (FP64-class) counterparts for FP64 matrices.
rgf_status hsliceA(const Ctx& c, int cnt, int ia, const double2* A, const int* act);
rgf_status hsliceB(const Ctx& c, int cnt, int ib, const double2* B, const int* act);
// nsl: slices of each operand in the product (0 = all seven, 5 for corrections).
rgf_status hmm(const Ctx& c, int cnt, int ia, int ib, float alpha, const double2* D, int addI, double2* C,
               const int* act, int nsl = 0);

// X = M^-1 (df) for cnt entries: FP32 seed, Newton-Schulz refinement with a
// Sherman-Morrison-scaled first step, FP64 reseed of entries that do not
// contract.  R is df scratch of cnt matrices.
// m64_ready: MixedState::c64 already holds M rounded to complex64 (written
// by the GEMM that produced M).
rgf_status inv_mixed(const Ctx& c, int cnt, int W, const float4* M, float4* X, float4* R, const int* act,
                     int* gj_flags, bool m64_ready = false);
// The same in parts: the seed (when s_begin == 0) and Newton-Schulz steps
// s_begin .. s_end-1.  From step 1 on, MixedState::more_count holds the
// number of entries that need another step.
rgf_status inv_mixed_steps(const Ctx& c, int cnt, int W, const float4* M, float4* X, float4* R, const int* act,
                           int* gj_flags, int s_begin, int s_end, bool m64_ready = false);
// The same for FP64 matrices with seven-slice products.
// X_prev (optional): inverses of nearby matrices (the previous decimation
// iteration's); entries whose FP32 seed does not contract try X_prev before
// the FP64 Gauss-Jordan inverse.
rgf_status inv_hp(const Ctx& c, int cnt, int W, const double2* M, double2* X, double2* R, const int* act,
                  int* gj_flags, const double2* X_prev = nullptr);


// Decimation pool unit u (u*W matrices in).  Units 0, 2, 4, 6 hold eps_s,
// eps, alpha, beta of the 2W entries (s*W + e, s = side) on entry to
// hp_decimate_run; units 8..25 are its scratch.
inline double2* dec_unit(const MixedState* m, int W, int u) { return m->dec_pool + (long)u * W * m->b * m->b; }
// Sancho-Rubio decimation of the 2W lead entries already formed in units
// 0, 2, 4, 6 (FP64 storage, seven-slice products).  *g_out receives the 2W
// surface Green's functions; per-energy flags (c.flags) get the decimation's
// NOCONV and SINGULAR bits.
rgf_status hp_decimate_run(const Ctx& c, int W, double tol, int max_iter, double2** g_out);

// Device Hamiltonian of a mixed-precision plan in double-float, plus its
// workspace (rgf_plan_s::mixed).
struct PlanMixed {
    MixedState ms;
    float4* H_diag = nullptr;
    float4* S_diag = nullptr;
    float4* H_lower = nullptr;
    float4* S_lower = nullptr;
    float4* lead[2][6] = {};
};

}  // namespace rgf

struct rgf_plan_s;
namespace rgf {
// Lead decimation, Sigma and Gamma of a plan's W energies (p->d_E) into pool
// units 0 (Sigma_L, Sigma_R) and 2 (Gamma_L, Gamma_R); resets p->d_flags and
// p->d_err.
rgf_status mixed_leads(rgf_plan_s* p, int W, const Ctx& c);
}  // namespace rgf
