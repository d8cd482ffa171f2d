// Plan object behind the rgf_plan_t handle.
#pragma once

#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

struct rgf_plan_s {
    int N = 0, b = 0;
    rgf_options opt{};
    cudaStream_t stream = nullptr;
    int W = 0;  // energies per wave

    // Device Hamiltonian / overlap (complex128, row-major blocks).
    double2* H_diag = nullptr;
    double2* S_diag = nullptr;
    double2* H_lower = nullptr;  // N-1 blocks (null when N == 1)
    double2* S_lower = nullptr;
    // Leads: [side][H00, S00, H10, S10, Hc, Sc]
    double2* lead[2][6] = {};
    bool blocks_set = false;
    bool lead_set[2] = {false, false};

    // Workspace of one wave (FP64 path or mixed path).
    void* ws = nullptr;
    size_t ws_bytes = 0;
    size_t block_bytes = 0;

    // Per-wave small arrays.
    double* d_E = nullptr;
    double* d_T = nullptr;
    double* d_Ti = nullptr;
    double* d_err = nullptr;
    int* d_flags = nullptr;
    int* d_dec_flags = nullptr;  // 2W
    int* d_active = nullptr;     // 2W
    int* d_iters = nullptr;      // 2W
    int* d_nmask = nullptr;      // 2W: entries refined by Newton steps, then the doubling's active mask
    int* d_smask = nullptr;      // 2W
    int* d_nnext = nullptr;      // 2W: entries that take a second Newton step
    int* d_status = nullptr;     // 2W: doubling outcome (1 converged, 2 diverged)
    double* d_p0 = nullptr;      // 2W: first doubling's |A| |B|
    int* d_remaining = nullptr;
    double* d_anorm = nullptr;   // 2W
    int* h_remaining = nullptr;  // pinned

    // Counters.
    long long n_waves = 0;
    long long n_reseeds = 0;
    // Device time of the mixed path's phases (CUDA events on the plan's
    // stream, accumulated over waves): lead decimation with Sigma/Gamma, and
    // the layer sweep with the trace.
    double lead_ms = 0.0, sweep_ms = 0.0;

    // Mixed-path state (allocated only for RGF_MIXED).
    void* mixed = nullptr;

    // Asynchronous submissions run one at a time on a worker thread.
    std::mutex mu;       // guards queue / stop
    std::mutex exec_mu;  // serialises work on the plan's workspace
    std::condition_variable cv;
    std::deque<struct rgf_job*> queue;
    std::thread worker;
    bool stop = false;
    bool worker_started = false;
};

namespace rgf {
// Runs every wave of one transmission request on the plan's stream.  E (host
// or device per mem) has n_E entries; outputs likewise.
rgf_status run_transmission(rgf_plan_s* p, const double* E, int n_E, double* T, double* err,
                            int* flags, int mem);
// One wave, energies already in p->d_E[0..Wc); writes p->d_T, d_err, d_flags.
rgf_status fp64_wave(rgf_plan_s* p, int Wc);
// FP64 Sancho-Rubio for the masked (energy, lead) entries of one wave.
rgf_status fp64_decimate(rgf_plan_s* p, int W, const int* mask, double2* pool, void* inv_ws, int* dec_active,
                         double2** g_out);
constexpr int kDecMats = 22;  // FP64 decimation matrices, in units of W
rgf_status mixed_wave(rgf_plan_s* p, int Wc);
size_t fp64_workspace_bytes(int W, int b);
size_t mixed_workspace_bytes(int W, int b);
rgf_status mixed_init(rgf_plan_s* p);
rgf_status mixed_on_blocks(rgf_plan_s* p);
rgf_status mixed_on_lead(rgf_plan_s* p, int side);
void mixed_free(rgf_plan_s* p);
}  // namespace rgf
