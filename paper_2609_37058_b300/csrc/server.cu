// Multi-device transmission server: admission by resident bytes, one engine
// per padded block size, energy slots refilled from lead-decimated items
// (continuous batching across devices of different lengths).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <string>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <utility>
#include <vector>

#include "../../include/rgf_server.h"
#include "engine.h"
#include "mixed_ops.h"

namespace rgf {
namespace {

using Clock = std::chrono::steady_clock;

struct Server;

struct Request {
    rgf_ticket_t ticket = 0;
    rgf_request in{};
    int bc = 0;
    size_t block_bytes = 0, out_bytes = 0;
    float4* blk = nullptr;     // H_diag[N], S_diag[N], H_lower[N-1], S_lower[N-1] (df, bc x bc)
    double2* lead = nullptr;   // [side][H00, S00, H10, S10, Hc, Sc] (FP64, bc x bc)
    double* out = nullptr;     // T[n_E], err[n_E], then flags (int) [n_E]
    std::vector<double> E;     // host copy of the energies
    cudaEvent_t ready_ev = nullptr;
    bool waited = false;
    int next = 0;              // next energy to hand to a decimation batch
    int done = 0;              // energies finished
    bool complete = false;
    rgf_status status = RGF_OK;
    std::string msg;  // error message of a failed request
    Clock::time_point t_submit, t_done;

    const float4* Hd(int l) const { return blk + (long)l * bc * bc; }
    const float4* Sd(int l) const { return blk + (long)(in.n_layers + l) * bc * bc; }
    const float4* Hl(int l) const { return blk + (long)(2 * in.n_layers + l - 1) * bc * bc; }
    const float4* Sl(int l) const { return blk + (long)(3 * in.n_layers - 1 + l - 1) * bc * bc; }
    double* T() const { return out; }
    double* Err() const { return out + in.n_E; }
    int* Flags() const { return (int*)(out + 2 * (long)in.n_E); }
};

struct Engine {
    Server* sv = nullptr;
    int bc = 0, W = 0, Wd = 0;  // slots, decimation batch
    cudaStream_t st = nullptr;
    MixedState ms;
    std::thread th;
    std::deque<Request*> incoming;  // guarded by Server::mu
    std::condition_variable cv;
    std::vector<Request*> reqs;     // engine thread only
    struct Slot {
        Request* r = nullptr;
        int k = -1;
        int layer = 0;
    };
    std::vector<Slot> slots;
    std::vector<std::pair<Request*, int>> ready;  // decimated items not yet in a slot
    size_t ready_pos = 0;
    int ready_D = 0;
    SlotTab* d_tab = nullptr;
    int* d_masks = nullptr;  // act, nf, first, last, refill (W each)
    DecTab* d_dtab = nullptr;
    double* slot_T = nullptr;
    double* slot_err = nullptr;
    int* slot_flags = nullptr;
    double* dec_err = nullptr;
    int* dec_flags = nullptr;
    SlotTab* h_tab = nullptr;  // pinned
    int* h_masks = nullptr;    // pinned
    DecTab* h_dtab = nullptr;  // pinned
    bool graphs = true;             // replay each step as a CUDA graph
    cudaGraphExec_t gx[2] = {};      // step front, one per Q/Qn parity
    cudaGraphExec_t gx_back[2] = {}; // step back (G, trace, results), per parity
    cudaGraphExec_t gx_tail = nullptr;  // Newton-Schulz steps beyond the second
    int parity = 0;                 // 0: Q = unit 9, 1: Q = unit 10
    std::atomic<long long> steps{0}, decs{0};
    long long reseeds = 0;  // engine thread; copied to reseeds_seen after each step
    std::atomic<long long> reseeds_seen{0};
    size_t ws_bytes = 0;
    rgf_status failed = RGF_OK;

    float4* U(int u) const { return ms.pool + (long)u * W * bc * bc; }
};

struct ClassCfg {
    int slots = 0, tile_n = 0, panel = 0;
};

struct Server {
    rgf_server_options opt{};
    std::map<int, ClassCfg> class_cfg;  // guarded by mu
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_admit;  // queue or resident bytes changed
    std::condition_variable cv_done;   // a request completed
    std::deque<Request*> queue;        // submitted, not yet admitted
    std::map<rgf_ticket_t, Request*> tickets;
    std::map<int, std::unique_ptr<Engine>> engines;
    std::thread admit_th;
    bool stop = false;
    rgf_ticket_t next_ticket = 1;
    size_t capacity = 0, resident = 0, peak_resident = 0, workspace = 0;
    cudaStream_t upload_st = nullptr, io_st = nullptr;
    void* staging = nullptr;
    size_t staging_bytes = 0;
    std::mutex io_mu;
    // statistics
    long long submitted = 0, completed = 0, rejected = 0, energies_done = 0;
    std::vector<double> latencies_ms;
    bool any_submit = false;
    Clock::time_point t_first, t_last;
};

size_t block_bytes_of(const rgf_request& r, int bc) {
    const size_t nn = (size_t)bc * bc;
    return (size_t)(4 * r.n_layers - 2) * nn * sizeof(float4) + 12 * nn * sizeof(double2);
}

int class_of(int b, int step) { return ((b + step - 1) / step) * step; }

// ---------------------------------------------------------------- engine
rgf_status engine_init(Engine* e) {
    Server* sv = e->sv;
    RGF_CUDA_TRY(cudaStreamCreateWithFlags(&e->st, cudaStreamNonBlocking));
    const int W = e->W;
    // Decimation batches of at most 148 items (one per SM): more slots do not
    // need a larger decimation pool.
    e->Wd = std::min(W, 148);
    RGF_TRY(mixed_state_init(&e->ms, e->bc, W, nullptr, e->st, e->Wd, W));
    e->ws_bytes = mixed_workspace_bytes(W, e->bc, W, std::max(W, 2 * e->Wd)) + mixed_dec_bytes(e->Wd, e->bc);
    auto dal = [&](void** p, size_t n) -> rgf_status {
        if (cudaMalloc(p, n) != cudaSuccess) {
            cudaGetLastError();
            set_error("server engine: cudaMalloc(%zu) failed", n);
            return RGF_E_OOM;
        }
        return RGF_OK;
    };
    RGF_TRY(dal((void**)&e->d_tab, sizeof(SlotTab) * W));
    RGF_TRY(dal((void**)&e->d_masks, sizeof(int) * 5 * W));
    RGF_TRY(dal((void**)&e->d_dtab, sizeof(DecTab) * e->Wd));
    RGF_TRY(dal((void**)&e->slot_T, sizeof(double) * W));
    RGF_TRY(dal((void**)&e->slot_err, sizeof(double) * W));
    RGF_TRY(dal((void**)&e->slot_flags, sizeof(int) * W));
    RGF_TRY(dal((void**)&e->dec_err, sizeof(double) * e->Wd));
    RGF_TRY(dal((void**)&e->dec_flags, sizeof(int) * e->Wd));
    RGF_CUDA_TRY(cudaMallocHost((void**)&e->h_tab, sizeof(SlotTab) * W));
    RGF_CUDA_TRY(cudaMallocHost((void**)&e->h_masks, sizeof(int) * 5 * W));
    RGF_CUDA_TRY(cudaMallocHost((void**)&e->h_dtab, sizeof(DecTab) * e->Wd));
    e->slots.assign(W, Engine::Slot{});
    const char* ng = getenv("RGF_NO_GRAPHS");
    e->graphs = !(ng && ng[0] == '1');
    (void)sv;
    return RGF_OK;
}

void engine_free(Engine* e) {
    cudaFree(e->d_tab);
    cudaFree(e->d_masks);
    cudaFree(e->d_dtab);
    cudaFree(e->slot_T);
    cudaFree(e->slot_err);
    cudaFree(e->slot_flags);
    cudaFree(e->dec_err);
    cudaFree(e->dec_flags);
    if (e->h_tab) cudaFreeHost(e->h_tab);
    if (e->h_masks) cudaFreeHost(e->h_masks);
    if (e->h_dtab) cudaFreeHost(e->h_dtab);
    for (auto& g : e->gx)
        if (g) cudaGraphExecDestroy(g);
    for (auto& g : e->gx_back)
        if (g) cudaGraphExecDestroy(g);
    if (e->gx_tail) cudaGraphExecDestroy(e->gx_tail);
    mixed_state_free(&e->ms);
    if (e->st) cudaStreamDestroy(e->st);
}

Ctx engine_ctx(Engine* e, double* err, int* flags) {
    return Ctx{&e->ms, e->st, (long)e->bc * e->bc, e->bc, e->sv->opt.ns_steps, err, flags, &e->reseeds};
}

rgf_status check_status(Engine* e) {
    int h = 0;
    RGF_CUDA_TRY(cudaMemcpyAsync(&h, e->ms.status, sizeof(int), cudaMemcpyDeviceToHost, e->st));
    RGF_CUDA_TRY(cudaStreamSynchronize(e->st));
    if (h != 0) {
        set_error("tensor-core GEMM pipeline timed out (status 0x%x)", h);
        return RGF_E_CUDA;
    }
    return RGF_OK;
}

void wait_ready(Engine* e, Request* r) {
    if (!r->waited) {
        cudaStreamWaitEvent(e->st, r->ready_ev, 0);
        r->waited = true;
    }
}

// Lead decimation, self-energies and broadening matrices of n items into the
// ready buffer (pool units 16..19).
rgf_status engine_decimate(Engine* e, const std::vector<std::pair<Request*, int>>& items) {
    NvtxRange nvtx_range("rgf server decimation batch");
    const int n = (int)items.size();
    const int bc = e->bc;
    MixedState* m = &e->ms;
    cudaStream_t st = e->st;
    for (int j = 0; j < n; ++j) {
        Request* r = items[j].first;
        wait_ready(e, r);
        e->h_dtab[j] = DecTab{r->lead, r->E[items[j].second], r->in.eta};
    }
    RGF_CUDA_TRY(cudaMemcpyAsync(e->d_dtab, e->h_dtab, sizeof(DecTab) * n, cudaMemcpyHostToDevice, st));
    RGF_CUDA_TRY(cudaMemsetAsync(e->dec_err, 0, sizeof(double) * n, st));
    RGF_CUDA_TRY(cudaMemsetAsync(e->dec_flags, 0, sizeof(int) * n, st));
    RGF_CUDA_TRY(cudaMemsetAsync(m->status, 0, sizeof(int), st));
    Ctx c = engine_ctx(e, e->dec_err, e->dec_flags);
    auto D = [&](int u) { return dec_unit(m, n, u); };
    RGF_TRY(engine_form_dec(n, bc, e->d_dtab, D(0), D(2), D(4), D(6), st));
    double2* g = nullptr;
    RGF_TRY(hp_decimate_run(c, n, e->sv->opt.dec_tol, e->sv->opt.dec_max_iter, &g));
    // Sigma = x1 g x2 with FP64-class products, then df Sigma and Gamma.
    RGF_TRY(engine_form_coupling(n, bc, e->d_dtab, D(0), D(2), st));
    const int n2 = 2 * n;
    RGF_TRY(hsliceA(c, n2, 0, D(0), nullptr));
    RGF_TRY(hsliceB(c, n2, 0, g, nullptr));
    RGF_TRY(hmm(c, n2, 0, 0, 1.0f, nullptr, 0, D(4), nullptr));
    RGF_TRY(hsliceA(c, n2, 0, D(4), nullptr));
    RGF_TRY(hsliceB(c, n2, 0, D(2), nullptr));
    RGF_TRY(hmm(c, n2, 0, 0, 1.0f, nullptr, 0, D(6), nullptr));
    float4* sig = e->U(16);
    float4* gam = sig + (long)n2 * bc * bc;
    RGF_TRY(c128_to_dfc(n2, bc, D(6), sig, nullptr, st));
    RGF_TRY(gamma_dfc(n2, bc, sig, gam, st));
    RGF_TRY(check_status(e));
    e->ready = items;
    e->ready_pos = 0;
    e->ready_D = n;
    ++e->decs;
    return RGF_OK;
}

// Kernels of one layer for every active slot, in three parts so that the
// Newton-Schulz steps beyond the second (rarely needed) can be skipped:
//   front: table copy, refills, block formation, the P / M / Q products,
//          the inverse's seed and Newton-Schulz steps 0 and 1 (with the FP64
//          reseed of entries that do not contract), and the read-back of how
//          many entries need a further step;
//   tail:  Newton-Schulz steps 2 .. ns_steps-1;
//   back:  G = Q g, the trace and the results of slots on their last layer.
// With all = true every kernel is launched (masks select the entries), so
// that each part is the same sequence every step and can be captured as a
// graph; Q/Qn are the buffers of the step's parity.
struct StepCounts {
    int n_nf = 0, n_first = 0, n_last = 0, n_refill = 0;
};

rgf_status engine_front(Engine* e, bool all, const StepCounts& n, float4* Q, float4* Qn) {
    const int W = e->W, bc = e->bc;
    cudaStream_t st = e->st;
    RGF_CUDA_TRY(cudaMemcpyAsync(e->d_tab, e->h_tab, sizeof(SlotTab) * W, cudaMemcpyHostToDevice, st));
    RGF_CUDA_TRY(cudaMemcpyAsync(e->d_masks, e->h_masks, sizeof(int) * 5 * W, cudaMemcpyHostToDevice, st));
    const int* d_act = e->d_masks;
    const int* d_nf = d_act + W;
    const int* d_first = d_act + 2 * W;
    const int* d_last = d_act + 3 * W;
    const int* d_refill = d_act + 4 * W;
    if (all || n.n_refill)
        RGF_TRY(engine_refill(W, bc, e->d_tab, d_refill, e->U(16), e->U(0), e->dec_err, e->dec_flags, e->slot_err,
                              e->slot_flags, st));
    float4 *sigL = e->U(0), *sigR = e->U(1);
    float4 *gi = e->U(4), *P = e->U(5), *M = e->U(6), *Rs = e->U(14);
    // M only (nf = nullptr): tau and tau' go straight to their slices below.
    SlotMasks mk{d_act, nullptr, d_first, d_last, d_refill};
    RGF_TRY(engine_form_step(W, bc, e->d_tab, mk, sigL, sigR, M, nullptr, nullptr, st));
    Ctx c = engine_ctx(e, e->slot_err, e->slot_flags);
    c.graph = all;
    if (all || n.n_nf) {
        RGF_TRY(sliceA(c, W, 0, gi, d_nf));
        RGF_TRY(form_slice_cols_dag_tab(W, bc, e->d_tab, d_nf, e->ms.sb[0], e->ms.Kp, st));
        RGF_TRY(mm(c, W, 0, 0, -1.0f, nullptr, 0, P, d_nf));  // P = -g tau'
        RGF_TRY(form_slice_rows_tab(W, bc, e->d_tab, d_nf, e->ms.sa[0], e->ms.Kp, st));
        RGF_TRY(sliceB(c, W, 0, P, d_nf));
        RGF_TRY(mm(c, W, 0, 0, 1.0f, M, 0, M, d_nf));  // M += tau P
        RGF_TRY(sliceA(c, W, 1, Q, d_nf));
        RGF_TRY(mm(c, W, 1, 0, 1.0f, nullptr, 0, Qn, d_nf));  // Q P, the next step's Q
    }
    // Slots on their first layer start the chain with Q = I in the next
    // step's Q buffer.
    if (all || n.n_first) RGF_TRY(set_identity_masked_dfc(W, bc, Qn, d_first, st));
    RGF_TRY(inv_mixed_steps(c, W, W, M, gi, Rs, d_act, e->slot_flags, 0, 2));
    RGF_CUDA_TRY(cudaMemcpyAsync(e->ms.h_more, e->ms.more_count, sizeof(int), cudaMemcpyDeviceToHost, st));
    return RGF_OK;
}

rgf_status engine_tail(Engine* e, bool all) {
    const int W = e->W;
    Ctx c = engine_ctx(e, e->slot_err, e->slot_flags);
    c.graph = all;
    return inv_mixed_steps(c, W, W, e->U(6), e->U(4), e->U(14), e->d_masks, e->slot_flags, 2, c.ns_steps);
}

rgf_status engine_back(Engine* e, bool all, const StepCounts& n, float4* Qn) {
    const int W = e->W, bc = e->bc;
    cudaStream_t st = e->st;
    if (!(all || n.n_last)) return RGF_OK;
    const int* d_last = e->d_masks + 3 * W;
    float4 *gamL = e->U(2), *gamR = e->U(3), *gi = e->U(4);
    float4 *G = e->U(11), *Xt = e->U(12), *Yt = e->U(13);
    Ctx c = engine_ctx(e, e->slot_err, e->slot_flags);
    c.graph = all;
    RGF_TRY(sliceA(c, W, 0, Qn, d_last));
    RGF_TRY(sliceB(c, W, 0, gi, d_last));
    RGF_TRY(mm(c, W, 0, 0, 1.0f, nullptr, 0, G, d_last));  // G_{0,N-1} = Q g
    RGF_TRY(sliceA(c, W, 0, gamL, d_last));
    RGF_TRY(sliceB(c, W, 0, G, d_last));
    RGF_TRY(mm(c, W, 0, 0, 1.0f, nullptr, 0, Xt, d_last));
    RGF_TRY(sliceA(c, W, 0, G, d_last));
    RGF_TRY(sliceB(c, W, 0, gamR, d_last));
    RGF_TRY(mm(c, W, 0, 0, 1.0f, nullptr, 0, Yt, d_last));
    RGF_TRY(trace_masked_dfc(W, bc, Xt, Yt, d_last, e->slot_T, st));
    RGF_TRY(engine_finish(W, e->d_tab, d_last, e->slot_T, e->slot_err, e->slot_flags, st));
    return RGF_OK;
}

// Capture (once) and launch one part of the step as a graph.
template <typename F>
rgf_status run_graph(Engine* e, cudaGraphExec_t& gx, F issue) {
    cudaStream_t st = e->st;
    if (!gx) {
        RGF_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        rgf_status s = issue();
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(st, &g);
        if (s != RGF_OK || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            if (s == RGF_OK) set_error("step capture failed: %s", cudaGetErrorString(ce));
            return s != RGF_OK ? s : RGF_E_CUDA;
        }
        ce = cudaGraphInstantiate(&gx, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
            gx = nullptr;
            cudaGetLastError();
            set_error("step graph instantiation failed: %s", cudaGetErrorString(ce));
            return RGF_E_CUDA;
        }
    }
    RGF_CUDA_TRY(cudaGraphLaunch(gx, st));
    return RGF_OK;
}

// One layer for every active slot.
rgf_status engine_step(Engine* e) {
    NvtxRange nvtx_range("rgf server engine step");
    const int W = e->W;
    int* act = e->h_masks;
    int* nf = act + W;
    int* first = act + 2 * W;
    int* last = act + 3 * W;
    int* refill = act + 4 * W;
    StepCounts n;
    for (int s = 0; s < W; ++s) {
        const Engine::Slot& sl = e->slots[s];
        SlotTab& t = e->h_tab[s];
        if (!sl.r) {
            act[s] = nf[s] = first[s] = last[s] = 0;
            // refill[] was set by the assignment (0 for empty slots).
            continue;
        }
        Request* r = sl.r;
        const int l = sl.layer, N = r->in.n_layers;
        act[s] = 1;
        first[s] = l == 0;
        nf[s] = l > 0;
        last[s] = l == N - 1;
        n.n_nf += nf[s];
        n.n_first += first[s];
        n.n_last += last[s];
        n.n_refill += refill[s];
        t.Sii = r->Sd(l);
        t.Hii = r->Hd(l);
        t.Sl = l > 0 ? r->Sl(l) : nullptr;
        t.Hl = l > 0 ? r->Hl(l) : nullptr;
        t.E = r->E[sl.k];
        t.eta = r->in.eta;
        t.outT = r->T() + sl.k;
        t.outErr = r->Err() + sl.k;
        t.outFlags = r->Flags() + sl.k;
    }
    cudaStream_t st = e->st;
    RGF_CUDA_TRY(cudaMemsetAsync(e->ms.status, 0, sizeof(int), st));
    float4* Q = e->U(9 + e->parity);
    float4* Qn = e->U(10 - e->parity);
    // The first two steps run directly (one-time set-up calls happen there);
    // later steps replay the captured parts of their parity.
    const bool graph = e->graphs && e->steps >= 2;
    const bool all = e->graphs;
    const int par = e->parity;
    if (graph)
        RGF_TRY(run_graph(e, e->gx[par], [&] { return engine_front(e, true, n, Q, Qn); }));
    else
        RGF_TRY(engine_front(e, all, n, Q, Qn));
    // Newton-Schulz steps beyond the second only when an entry needs them.
    RGF_CUDA_TRY(cudaStreamSynchronize(st));
    if (e->sv->opt.ns_steps > 2 && *e->ms.h_more > 0) {
        if (graph)
            RGF_TRY(run_graph(e, e->gx_tail, [&] { return engine_tail(e, true); }));
        else
            RGF_TRY(engine_tail(e, all));
    }
    if (graph)
        RGF_TRY(run_graph(e, e->gx_back[par], [&] { return engine_back(e, true, n, Qn); }));
    else
        RGF_TRY(engine_back(e, all, n, Qn));
    e->parity ^= 1;
    long long acc = 0;
    RGF_CUDA_TRY(cudaMemcpyAsync(&acc, e->ms.reseed_acc, sizeof(acc), cudaMemcpyDeviceToHost, st));
    RGF_TRY(check_status(e));
    ++e->steps;
    e->reseeds_seen = e->reseeds + acc;
    return RGF_OK;
}

void finish_request(Server* sv, Engine* e, Request* r, rgf_status status) {
    if (r->blk) cudaFreeAsync(r->blk, e ? e->st : sv->upload_st);
    if (r->lead) cudaFreeAsync(r->lead, e ? e->st : sv->upload_st);
    r->blk = nullptr;
    r->lead = nullptr;
    std::lock_guard<std::mutex> lk(sv->mu);
    r->status = status;
    if (status != RGF_OK) r->msg = get_error();
    r->complete = true;
    r->t_done = Clock::now();
    sv->resident -= r->block_bytes;
    if (status == RGF_OK) {
        sv->completed += 1;
        sv->energies_done += r->in.n_E;
        sv->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
        sv->t_last = r->t_done;
    }
    sv->cv_done.notify_all();
    sv->cv_admit.notify_all();
}

void engine_fail(Engine* e, rgf_status s) {
    e->failed = s;
    std::vector<Request*> all = e->reqs;
    for (Request* r : all)
        if (!r->complete) finish_request(e->sv, e, r, s);
    e->reqs.clear();
    for (auto& sl : e->slots) sl = Engine::Slot{};
    e->ready.clear();
    e->ready_pos = 0;
}

void engine_loop(Engine* e) {
    Server* sv = e->sv;
    cudaSetDevice(sv->device);
    const int W = e->W;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            if (sv->stop) break;
            while (!e->incoming.empty()) {
                e->reqs.push_back(e->incoming.front());
                e->incoming.pop_front();
            }
        }
        if (e->failed != RGF_OK) {
            engine_fail(e, e->failed);
            std::unique_lock<std::mutex> lk(sv->mu);
            e->cv.wait_for(lk, std::chrono::milliseconds(20));
            continue;
        }
        // Refill free slots from the ready items.
        int* refill = e->h_masks + 4 * W;
        int n_free = 0, n_active = 0;
        for (int s = 0; s < W; ++s) {
            refill[s] = 0;
            Engine::Slot& sl = e->slots[s];
            if (!sl.r && e->ready_pos < e->ready.size()) {
                const int idx = (int)e->ready_pos++;
                sl.r = e->ready[idx].first;
                sl.k = e->ready[idx].second;
                sl.layer = 0;
                refill[s] = 1;
                e->h_tab[s].ready = idx;
                e->h_tab[s].ready_D = e->ready_D;
            }
            if (sl.r)
                ++n_active;
            else
                ++n_free;
        }
        // Decimate the next items when the ready buffer is used up.
        if (e->ready_pos >= e->ready.size() && n_free > 0) {
            long pending = 0;
            for (Request* r : e->reqs) pending += r->in.n_E - r->next;
            if (pending > 0 && (n_active == 0 || n_free >= W / 4 || pending <= n_free)) {
                // Refilled slots of this pass keep their ready indices only
                // if the buffer is not replaced: run the step first.
                bool pending_refill = false;
                for (int s = 0; s < W; ++s) pending_refill |= refill[s] != 0;
                if (!pending_refill) {
                    std::vector<std::pair<Request*, int>> items;
                    for (Request* r : e->reqs) {
                        while (r->next < r->in.n_E && (int)items.size() < e->Wd) items.emplace_back(r, r->next++);
                        if ((int)items.size() >= e->Wd) break;
                    }
                    rgf_status s = engine_decimate(e, items);
                    if (s != RGF_OK) {
                        e->failed = s;
                        continue;
                    }
                    continue;  // assign the new items to slots
                }
            }
        }
        if (n_active == 0) {
            std::unique_lock<std::mutex> lk(sv->mu);
            if (sv->stop) break;
            if (e->incoming.empty()) e->cv.wait_for(lk, std::chrono::milliseconds(20));
            continue;
        }
        rgf_status s = engine_step(e);
        if (s != RGF_OK) {
            e->failed = s;
            continue;
        }
        // Advance the slots; finished items complete their requests.
        for (int i = 0; i < W; ++i) {
            Engine::Slot& sl = e->slots[i];
            if (!sl.r) continue;
            if (sl.layer == sl.r->in.n_layers - 1) {
                Request* r = sl.r;
                if (++r->done == r->in.n_E) {
                    finish_request(sv, e, r, RGF_OK);
                    e->reqs.erase(std::remove(e->reqs.begin(), e->reqs.end(), r), e->reqs.end());
                }
                sl = Engine::Slot{};
            } else {
                ++sl.layer;
            }
        }
    }
}

// ---------------------------------------------------------------- admission
rgf_status upload(Server* sv, Request* r) {
    const rgf_request& q = r->in;
    const int b = q.b, bc = r->bc, N = q.n_layers;
    const size_t nn = (size_t)bc * bc, bb = (size_t)b * b * sizeof(double2);
    cudaStream_t st = sv->upload_st;
    RGF_CUDA_TRY(cudaMallocAsync((void**)&r->blk, (size_t)(4 * N - 2) * nn * sizeof(float4), st));
    RGF_CUDA_TRY(cudaMallocAsync((void**)&r->lead, 12 * nn * sizeof(double2), st));
    RGF_CUDA_TRY(cudaMallocAsync((void**)&r->out, r->out_bytes, st));
    const size_t per_chunk = std::max<size_t>(1, sv->staging_bytes / bb);
    // Copy nblk blocks (b x b, FP64) from src to dst (bc x bc), through the
    // staging buffer when they are in host memory.
    auto put = [&](const double* src, int nblk, float4* dst_df, double2* dst64, double fill) -> rgf_status {
        for (int i0 = 0; i0 < nblk; i0 += (int)per_chunk) {
            const int cnt = std::min<int>((int)per_chunk, nblk - i0);
            const double2* s = (const double2*)src + (size_t)i0 * b * b;
            if (q.mem == RGF_MEM_HOST) {
                RGF_CUDA_TRY(cudaMemcpyAsync(sv->staging, s, cnt * bb, cudaMemcpyHostToDevice, st));
                s = (const double2*)sv->staging;
            }
            if (dst_df)
                RGF_TRY(pad_to_dfc(cnt, b, bc, s, dst_df + (size_t)i0 * nn, fill, st));
            else
                RGF_TRY(pad_f64(cnt, b, bc, s, dst64 + (size_t)i0 * nn, fill, st));
        }
        return RGF_OK;
    };
    // Padded orbitals: H = -1, S = 0 on the diagonal, so z S - H = 1 there.
    RGF_TRY(put(q.H_diag, N, r->blk, nullptr, -1.0));
    RGF_TRY(put(q.S_diag, N, r->blk + (size_t)N * nn, nullptr, 0.0));
    if (N > 1) {
        RGF_TRY(put(q.H_lower, N - 1, r->blk + (size_t)2 * N * nn, nullptr, 0.0));
        RGF_TRY(put(q.S_lower, N - 1, r->blk + (size_t)(3 * N - 1) * nn, nullptr, 0.0));
    }
    for (int side = 0; side < 2; ++side)
        for (int k = 0; k < 6; ++k)
            RGF_TRY(put(q.lead[side][k], 1, nullptr, r->lead + (size_t)(6 * side + k) * nn, k == 0 ? -1.0 : 0.0));
    RGF_CUDA_TRY(cudaEventCreateWithFlags(&r->ready_ev, cudaEventDisableTiming));
    RGF_CUDA_TRY(cudaEventRecord(r->ready_ev, st));
    // The staging buffer is reused by the next upload: wait for this one.
    if (q.mem == RGF_MEM_HOST) RGF_CUDA_TRY(cudaStreamSynchronize(st));
    return RGF_OK;
}

Engine* engine_for(Server* sv, int bc, rgf_status* st) {
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->engines.find(bc);
        if (it != sv->engines.end()) return it->second.get();
    }
    ClassCfg cfg;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->class_cfg.find(bc);
        if (it != sv->class_cfg.end()) cfg = it->second;
    }
    auto e = std::make_unique<Engine>();
    e->sv = sv;
    e->bc = bc;
    e->W = cfg.slots > 0 ? cfg.slots : sv->opt.slots;
    *st = engine_init(e.get());
    if (*st == RGF_OK) {
        e->ms.bn = cfg.tile_n > 0 ? cfg.tile_n : 96;
        e->ms.gj_nb = cfg.panel;
    }
    if (*st != RGF_OK) {
        engine_free(e.get());
        return nullptr;
    }
    Engine* raw = e.get();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->workspace += raw->ws_bytes;
        sv->engines[bc] = std::move(e);
    }
    raw->th = std::thread(engine_loop, raw);
    return raw;
}

void admit_loop(Server* sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            for (;;) {
                if (sv->stop) return;
                if (!sv->queue.empty()) {
                    Request* h = sv->queue.front();
                    if (sv->resident == 0 || sv->resident + h->block_bytes + h->out_bytes <= sv->capacity) break;
                }
                sv->cv_admit.wait(lk);
            }
            r = sv->queue.front();
            sv->queue.pop_front();
            sv->resident += r->block_bytes;
            sv->peak_resident = std::max(sv->peak_resident, sv->resident);
        }
        rgf_status s = RGF_OK;
        Engine* e = engine_for(sv, r->bc, &s);
        if (s == RGF_OK) s = upload(sv, r);
        if (s != RGF_OK) {
            finish_request(sv, nullptr, r, s);
            continue;
        }
        std::lock_guard<std::mutex> lk(sv->mu);
        e->incoming.push_back(r);
        e->cv.notify_all();
    }
}

bool request_ok(const rgf_request* q) {
    if (!q || q->n_layers < 1 || q->b < 1 || q->b > 512 || q->n_E < 1 || !(q->eta > 0.0)) return false;
    if (q->mem != RGF_MEM_HOST && q->mem != RGF_MEM_DEVICE) return false;
    if (!q->H_diag || !q->S_diag || !q->E) return false;
    if (q->n_layers > 1 && (!q->H_lower || !q->S_lower)) return false;
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < 6; ++k)
            if (!q->lead[s][k]) return false;
    return true;
}

}  // namespace
}  // namespace rgf

using rgf::Clock;
using rgf::Request;
using rgf::Server;

struct rgf_server_s {
    Server s;
};

extern "C" {

void rgf_server_options_default(rgf_server_options* o) {
    if (!o) return;
    o->dec_tol = 1e-14;
    o->dec_max_iter = 100;
    o->ns_steps = 6;
    o->slots = 148;
    o->class_step = 32;
    o->capacity_bytes = 0;
}

rgf_status rgf_server_create(rgf_server_t* out, const rgf_server_options* opt) {
    if (!out) {
        rgf::set_error("rgf_server_create: null output pointer");
        return RGF_E_INVALID;
    }
    *out = nullptr;
    rgf_server_options o;
    rgf_server_options_default(&o);
    if (opt) o = *opt;
    if (o.slots < 1 || o.slots > 4096 || o.class_step < 1 || o.class_step > 512 || o.ns_steps < 0 ||
        o.dec_max_iter < 1 || !(o.dec_tol > 0.0)) {
        rgf::set_error("rgf_server_create: option out of range");
        return RGF_E_INVALID;
    }
    auto* h = new rgf_server_s();
    Server* sv = &h->s;
    sv->opt = o;
    cudaGetDevice(&sv->device);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        rgf::set_error("rgf_server_create: no CUDA device");
        return RGF_E_CUDA;
    }
    sv->capacity = o.capacity_bytes ? o.capacity_bytes : std::min<size_t>((size_t)150e9, (size_t)(0.55 * free_b));
    // Keep freed request memory in the stream-ordered pool of this process.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, sv->device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    if (cudaStreamCreateWithFlags(&sv->upload_st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sv->io_st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        rgf::set_error("rgf_server_create: stream creation failed");
        return RGF_E_CUDA;
    }
    sv->staging_bytes = (size_t)256 << 20;
    if (cudaMalloc(&sv->staging, sv->staging_bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamDestroy(sv->upload_st);
        cudaStreamDestroy(sv->io_st);
        delete h;
        rgf::set_error("rgf_server_create: staging allocation failed");
        return RGF_E_OOM;
    }
    sv->admit_th = std::thread(rgf::admit_loop, sv);
    *out = h;
    return RGF_OK;
}

rgf_status rgf_server_set_class(rgf_server_t h, int block_class, int slots, int tile_n, int panel) {
    if (!h || block_class < 1 || block_class > 512 || slots < 0 || slots > 4096 ||
        (tile_n != 0 && tile_n != 64 && tile_n != 80 && tile_n != 96) || (panel != 0 && panel != 16 && panel != 32)) {
        rgf::set_error("rgf_server_set_class: invalid arguments");
        return RGF_E_INVALID;
    }
    Server* sv = &h->s;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->engines.count(block_class)) {
        rgf::set_error("rgf_server_set_class: class %d already has an engine", block_class);
        return RGF_E_STATE;
    }
    sv->class_cfg[block_class] = rgf::ClassCfg{slots, tile_n, panel};
    return RGF_OK;
}

rgf_status rgf_server_submit(rgf_server_t h, const rgf_request* q, rgf_ticket_t* ticket) {
    if (!h || !ticket || !rgf::request_ok(q)) {
        rgf::set_error("rgf_server_submit: invalid request");
        return RGF_E_INVALID;
    }
    Server* sv = &h->s;
    auto* r = new Request();
    r->in = *q;
    r->bc = rgf::class_of(q->b, sv->opt.class_step);
    if (r->bc > 512) r->bc = 512;
    r->block_bytes = rgf::block_bytes_of(*q, r->bc);
    r->out_bytes = (size_t)q->n_E * (2 * sizeof(double) + sizeof(int)) + 64;
    r->E.resize(q->n_E);
    if (q->mem == RGF_MEM_HOST) {
        std::memcpy(r->E.data(), q->E, sizeof(double) * q->n_E);
    } else if (cudaMemcpy(r->E.data(), q->E, sizeof(double) * q->n_E, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        delete r;
        rgf::set_error("rgf_server_submit: reading the device energies failed");
        return RGF_E_CUDA;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (r->block_bytes + r->out_bytes > sv->capacity) {
        sv->rejected += 1;
        delete r;
        rgf::set_error("rgf_server_submit: request needs more than the capacity");
        return RGF_E_REJECTED;
    }
    r->ticket = sv->next_ticket++;
    r->t_submit = Clock::now();
    if (!sv->any_submit) {
        sv->any_submit = true;
        sv->t_first = r->t_submit;
    }
    sv->submitted += 1;
    sv->tickets[r->ticket] = r;
    sv->queue.push_back(r);
    sv->cv_admit.notify_all();
    *ticket = r->ticket;
    return RGF_OK;
}

rgf_status rgf_server_poll(rgf_server_t h, rgf_ticket_t ticket, double* T, double* err, int* flags,
                           double* latency_ms, int timeout_us) {
    if (!h || !T) {
        rgf::set_error("rgf_server_poll: invalid arguments");
        return RGF_E_INVALID;
    }
    Server* sv = &h->s;
    Request* r = nullptr;
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        auto it = sv->tickets.find(ticket);
        if (it == sv->tickets.end()) {
            rgf::set_error("rgf_server_poll: unknown ticket %llu", (unsigned long long)ticket);
            return RGF_E_INVALID;
        }
        r = it->second;
        auto done = [&] { return r->complete; };
        if (timeout_us == 0) {
            if (!done()) return RGF_E_NOT_READY;
        } else if (timeout_us < 0) {
            sv->cv_done.wait(lk, done);
        } else if (!sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done)) {
            return RGF_E_TIMEOUT;
        }
        sv->tickets.erase(it);
    }
    rgf_status status = r->status;
    if (status == RGF_OK) {
        std::lock_guard<std::mutex> lk(sv->io_mu);
        const int n = r->in.n_E;
        cudaError_t ce = cudaMemcpyAsync(T, r->T(), sizeof(double) * n, cudaMemcpyDefault, sv->io_st);
        if (ce == cudaSuccess && err) ce = cudaMemcpyAsync(err, r->Err(), sizeof(double) * n, cudaMemcpyDefault, sv->io_st);
        if (ce == cudaSuccess && flags)
            ce = cudaMemcpyAsync(flags, r->Flags(), sizeof(int) * n, cudaMemcpyDefault, sv->io_st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(sv->io_st);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            rgf::set_error("rgf_server_poll: copy of the results failed: %s", cudaGetErrorString(ce));
            status = RGF_E_CUDA;
        }
    } else {
        rgf::set_error("rgf_server_poll: request failed: %s", r->msg.c_str());
    }
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    if (r->out) cudaFreeAsync(r->out, sv->io_st);
    if (r->ready_ev) cudaEventDestroy(r->ready_ev);
    delete r;
    return status;
}

rgf_status rgf_server_stats_get(rgf_server_t h, rgf_server_stats* o) {
    if (!h || !o) {
        rgf::set_error("rgf_server_stats_get: invalid arguments");
        return RGF_E_INVALID;
    }
    Server* sv = &h->s;
    std::lock_guard<std::mutex> lk(sv->mu);
    std::memset(o, 0, sizeof(*o));
    o->submitted = sv->submitted;
    o->completed = sv->completed;
    o->rejected = sv->rejected;
    o->energies_done = sv->energies_done;
    for (auto& kv : sv->engines) {
        o->steps += kv.second->steps;
        o->decimations += kv.second->decs;
        o->fp64_reseeds += kv.second->reseeds_seen;
    }
    o->engines = (int)sv->engines.size();
    o->resident_bytes = sv->resident;
    o->peak_resident_bytes = sv->peak_resident;
    o->workspace_bytes = sv->workspace;
    if (sv->completed > 0) o->busy_s = std::chrono::duration<double>(sv->t_last - sv->t_first).count();
    std::vector<double> v = sv->latencies_ms;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            // Nearest-rank percentile.
            size_t k = (size_t)std::ceil(p / 100.0 * v.size());
            k = std::max<size_t>(1, std::min(k, v.size()));
            return v[k - 1];
        };
        o->latency_p50_ms = pct(50);
        o->latency_p99_ms = pct(99);
        o->latency_max_ms = v.back();
    }
    return RGF_OK;
}

rgf_status rgf_server_destroy(rgf_server_t h) {
    if (!h) return RGF_OK;
    Server* sv = &h->s;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv_admit.notify_all();
        for (auto& kv : sv->engines) kv.second->cv.notify_all();
    }
    if (sv->admit_th.joinable()) sv->admit_th.join();
    for (auto& kv : sv->engines)
        if (kv.second->th.joinable()) kv.second->th.join();
    cudaDeviceSynchronize();
    for (auto& kv : sv->tickets) {
        Request* r = kv.second;
        if (r->blk) cudaFreeAsync(r->blk, sv->io_st);
        if (r->lead) cudaFreeAsync(r->lead, sv->io_st);
        if (r->out) cudaFreeAsync(r->out, sv->io_st);
        if (r->ready_ev) cudaEventDestroy(r->ready_ev);
        delete r;
    }
    cudaStreamSynchronize(sv->io_st);
    for (auto& kv : sv->engines) rgf::engine_free(kv.second.get());
    cudaFree(sv->staging);
    // Hand the request memory cached in the stream-ordered pool back.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, sv->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    cudaStreamDestroy(sv->upload_st);
    cudaStreamDestroy(sv->io_st);
    cudaGetLastError();
    delete h;
    return RGF_OK;
}

}  // extern "C"
