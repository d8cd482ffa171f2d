// C ABI entry points of the RGF library (see include/rgf.h).
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>

#include "kernels.h"
#include "plan.h"

using rgf::set_error;

struct rgf_job {
    rgf_ticket_t id = 0;
    rgf_plan_s* plan = nullptr;
    std::vector<double> E, T, err;
    std::vector<int> flags;
    rgf_status status = RGF_OK;
    std::string message;
    bool done = false;
};

namespace {

std::mutex g_jobs_mu;
std::condition_variable g_jobs_cv;
std::map<rgf_ticket_t, std::shared_ptr<rgf_job>> g_jobs;
std::atomic<uint64_t> g_next_ticket{1};

size_t mat_bytes(int b) { return (size_t)b * b * sizeof(double2); }

rgf_status check_plan(rgf_plan_t p) {
    if (!p) {
        set_error("null plan");
        return RGF_E_INVALID;
    }
    return RGF_OK;
}

cudaMemcpyKind kind_in(int mem) {
    return mem == RGF_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind kind_out(int mem) {
    return mem == RGF_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

// Hermiticity of host diagonal blocks: |A - A^dag|_F <= 1e-10 |A|_F.
bool hermitian_host(const double* A, int b) {
    double diff = 0.0, nrm = 0.0;
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) {
            const double* x = A + 2 * ((size_t)r * b + c);
            const double* y = A + 2 * ((size_t)c * b + r);
            const double dr = x[0] - y[0], di = x[1] + y[1];
            diff += dr * dr + di * di;
            nrm += x[0] * x[0] + x[1] * x[1];
        }
    return std::sqrt(diff) <= 1e-10 * std::sqrt(nrm) + 1e-300;
}

void worker_loop(rgf_plan_s* p);

}  // namespace

namespace rgf {

rgf_status run_transmission(rgf_plan_s* p, const double* E, int n_E, double* T, double* err, int* flags,
                            int mem) {
    for (int w0 = 0; w0 < n_E; w0 += p->W) {
        const int Wc = (n_E - w0) < p->W ? (n_E - w0) : p->W;
        RGF_CUDA_TRY(cudaMemcpyAsync(p->d_E, E + w0, sizeof(double) * Wc, kind_in(mem), p->stream));
        if (p->opt.precision == RGF_MIXED) {
            RGF_TRY(mixed_wave(p, Wc));
        } else {
            RGF_TRY(fp64_wave(p, Wc));
        }
        p->n_waves++;
        RGF_CUDA_TRY(cudaMemcpyAsync(T + w0, p->d_T, sizeof(double) * Wc, kind_out(mem), p->stream));
        if (err)
            RGF_CUDA_TRY(cudaMemcpyAsync(err + w0, p->d_err, sizeof(double) * Wc, kind_out(mem), p->stream));
        if (flags)
            RGF_CUDA_TRY(cudaMemcpyAsync(flags + w0, p->d_flags, sizeof(int) * Wc, kind_out(mem), p->stream));
    }
    RGF_CUDA_TRY(cudaStreamSynchronize(p->stream));
    return RGF_OK;
}

}  // namespace rgf

extern "C" {

const char* rgf_version(void) { return "rgf-b300 0.1.0 (sm_103a)"; }

const char* rgf_last_error(void) { return rgf::get_error(); }

void rgf_options_default(rgf_options* opt) {
    if (!opt) return;
    opt->precision = RGF_FP64;
    opt->eta = 1e-6;
    opt->dec_tol = 1e-14;
    opt->dec_max_iter = 100;
    opt->ns_steps = 6;
    opt->energy_wave = 0;
}

rgf_status rgf_plan_destroy(rgf_plan_t p) {
    if (!p) return RGF_OK;
    if (p->worker_started) {
        {
            std::lock_guard<std::mutex> lk(p->mu);
            p->stop = true;
        }
        p->cv.notify_all();
        p->worker.join();
    }
    if (p->stream) cudaStreamSynchronize(p->stream);
    rgf::mixed_free(p);
    cudaFree(p->H_diag);
    cudaFree(p->S_diag);
    cudaFree(p->H_lower);
    cudaFree(p->S_lower);
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < 6; ++k) cudaFree(p->lead[s][k]);
    cudaFree(p->ws);
    cudaFree(p->d_E);
    cudaFree(p->d_T);
    cudaFree(p->d_Ti);
    cudaFree(p->d_err);
    cudaFree(p->d_flags);
    cudaFree(p->d_dec_flags);
    cudaFree(p->d_active);
    cudaFree(p->d_iters);
    cudaFree(p->d_nmask);
    cudaFree(p->d_smask);
    cudaFree(p->d_nnext);
    cudaFree(p->d_status);
    cudaFree(p->d_p0);
    cudaFree(p->d_remaining);
    cudaFree(p->d_anorm);
    if (p->h_remaining) cudaFreeHost(p->h_remaining);
    delete p;
    return RGF_OK;
}

rgf_status rgf_plan_create(rgf_plan_t* out, int n_layers, int b, const rgf_options* opt, void* cuda_stream) {
    if (!out) {
        set_error("rgf_plan_create: null output handle");
        return RGF_E_INVALID;
    }
    *out = nullptr;
    if (n_layers < 1 || b < 1 || b > 512) {
        set_error("rgf_plan_create: need n_layers >= 1 and 1 <= b <= 512 (got %d, %d)", n_layers, b);
        return RGF_E_INVALID;
    }
    rgf_options o;
    rgf_options_default(&o);
    if (opt) o = *opt;
    if (o.precision != RGF_FP64 && o.precision != RGF_MIXED) {
        set_error("rgf_plan_create: unknown precision %d", o.precision);
        return RGF_E_INVALID;
    }
    if (!(o.eta >= 0.0) || !(o.dec_tol > 0.0) || o.dec_max_iter < 1 || o.ns_steps < 0 || o.ns_steps > 8 ||
        o.energy_wave < 0) {
        set_error("rgf_plan_create: invalid options");
        return RGF_E_INVALID;
    }
    auto* p = new rgf_plan_s();
    p->N = n_layers;
    p->b = b;
    p->opt = o;
    p->stream = (cudaStream_t)cuda_stream;
    const size_t mb = mat_bytes(b);

    auto fail = [&](rgf_status s) {
        rgf_plan_destroy(p);
        return s;
    };
#define ALLOC(ptr, bytes)                                                             \
    do {                                                                              \
        cudaError_t _e = cudaMalloc((void**)&(ptr), (bytes) ? (bytes) : 16);          \
        if (_e != cudaSuccess) {                                                      \
            cudaGetLastError();                                                       \
            set_error("rgf_plan_create: cudaMalloc(%zu) failed: %s", (size_t)(bytes), \
                      cudaGetErrorString(_e));                                        \
            return fail(RGF_E_OOM);                                                   \
        }                                                                             \
    } while (0)

    ALLOC(p->H_diag, mb * n_layers);
    ALLOC(p->S_diag, mb * n_layers);
    if (n_layers > 1) {
        ALLOC(p->H_lower, mb * (n_layers - 1));
        ALLOC(p->S_lower, mb * (n_layers - 1));
    }
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < 6; ++k) ALLOC(p->lead[s][k], mb);
    p->block_bytes = mb * (2 * n_layers + 2 * (n_layers - 1) + 12);

    // Energy wave: requested, else as many energies as fit in 40% of the free
    // memory, at most 2 per SM-pair of the B300's 148 SMs.
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    auto ws_for = [&](int W) {
        return o.precision == RGF_MIXED ? rgf::mixed_workspace_bytes(W, b) : rgf::fp64_workspace_bytes(W, b);
    };
    int W = o.energy_wave;
    if (W == 0) {
        W = 296;
        while (W > 1 && ws_for(W) > (size_t)(0.4 * (double)free_b)) W = (W * 3) / 4;
    }
    if (W > 32767) W = 32767;
    p->W = W;
    p->ws_bytes = ws_for(W);
    ALLOC(p->ws, p->ws_bytes);
    ALLOC(p->d_E, sizeof(double) * W);
    ALLOC(p->d_T, sizeof(double) * W);
    ALLOC(p->d_Ti, sizeof(double) * W);
    ALLOC(p->d_err, sizeof(double) * W);
    ALLOC(p->d_flags, sizeof(int) * W);
    ALLOC(p->d_dec_flags, sizeof(int) * 2 * W);
    ALLOC(p->d_active, sizeof(int) * 2 * W);
    ALLOC(p->d_iters, sizeof(int) * 2 * W);
    ALLOC(p->d_nmask, sizeof(int) * 2 * W);
    ALLOC(p->d_smask, sizeof(int) * 2 * W);
    ALLOC(p->d_nnext, sizeof(int) * 2 * W);
    ALLOC(p->d_status, sizeof(int) * 2 * W);
    ALLOC(p->d_p0, sizeof(double) * 2 * W);
    ALLOC(p->d_remaining, sizeof(int));
    ALLOC(p->d_anorm, sizeof(double) * 2 * W);
#undef ALLOC
    if (cudaMallocHost((void**)&p->h_remaining, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        set_error("rgf_plan_create: cudaMallocHost failed");
        return fail(RGF_E_OOM);
    }
    if (o.precision == RGF_MIXED) {
        rgf_status s = rgf::mixed_init(p);
        if (s != RGF_OK) return fail(s);
    }
    *out = p;
    return RGF_OK;
}

rgf_status rgf_plan_device_bytes(rgf_plan_t p, size_t* bytes) {
    RGF_TRY(check_plan(p));
    if (!bytes) {
        set_error("null output");
        return RGF_E_INVALID;
    }
    *bytes = p->block_bytes + p->ws_bytes;
    return RGF_OK;
}

rgf_status rgf_plan_stats(rgf_plan_t p, long long* waves, long long* fp64_reseeds) {
    RGF_TRY(check_plan(p));
    if (waves) *waves = p->n_waves;
    if (fp64_reseeds) *fp64_reseeds = p->n_reseeds;
    return RGF_OK;
}

rgf_status rgf_plan_phase_ms(rgf_plan_t p, double* lead_ms, double* sweep_ms) {
    RGF_TRY(check_plan(p));
    if (lead_ms) *lead_ms = p->lead_ms;
    if (sweep_ms) *sweep_ms = p->sweep_ms;
    return RGF_OK;
}

rgf_status rgf_plan_energy_wave(rgf_plan_t p, int* w) {
    RGF_TRY(check_plan(p));
    if (!w) {
        set_error("null output");
        return RGF_E_INVALID;
    }
    *w = p->W;
    return RGF_OK;
}

rgf_status rgf_set_device_blocks(rgf_plan_t p, const double* H_diag, const double* S_diag,
                                 const double* H_lower, const double* S_lower, int mem) {
    RGF_TRY(check_plan(p));
    if (mem != RGF_MEM_HOST && mem != RGF_MEM_DEVICE) {
        set_error("rgf_set_device_blocks: bad memory space %d", mem);
        return RGF_E_INVALID;
    }
    if (!H_diag || !S_diag || (p->N > 1 && (!H_lower || !S_lower))) {
        set_error("rgf_set_device_blocks: null block pointer");
        return RGF_E_INVALID;
    }
    if (mem == RGF_MEM_HOST) {
        for (int i = 0; i < p->N; ++i) {
            if (!hermitian_host(H_diag + 2 * (size_t)i * p->b * p->b, p->b) ||
                !hermitian_host(S_diag + 2 * (size_t)i * p->b * p->b, p->b)) {
                set_error("rgf_set_device_blocks: diagonal block %d of H or S is not Hermitian", i);
                return RGF_E_INVALID;
            }
        }
    }
    const size_t mb = mat_bytes(p->b);
    RGF_CUDA_TRY(cudaMemcpyAsync(p->H_diag, H_diag, mb * p->N, kind_in(mem), p->stream));
    RGF_CUDA_TRY(cudaMemcpyAsync(p->S_diag, S_diag, mb * p->N, kind_in(mem), p->stream));
    if (p->N > 1) {
        RGF_CUDA_TRY(cudaMemcpyAsync(p->H_lower, H_lower, mb * (p->N - 1), kind_in(mem), p->stream));
        RGF_CUDA_TRY(cudaMemcpyAsync(p->S_lower, S_lower, mb * (p->N - 1), kind_in(mem), p->stream));
    }
    RGF_CUDA_TRY(cudaStreamSynchronize(p->stream));
    if (p->opt.precision == RGF_MIXED) RGF_TRY(rgf::mixed_on_blocks(p));
    p->blocks_set = true;
    return RGF_OK;
}

rgf_status rgf_set_leads(rgf_plan_t p, int side, const double* H00, const double* S00, const double* H10,
                         const double* S10, const double* Hc, const double* Sc, int mem) {
    RGF_TRY(check_plan(p));
    if (side != RGF_LEAD_LEFT && side != RGF_LEAD_RIGHT) {
        set_error("rgf_set_leads: bad side %d", side);
        return RGF_E_INVALID;
    }
    if (mem != RGF_MEM_HOST && mem != RGF_MEM_DEVICE) {
        set_error("rgf_set_leads: bad memory space %d", mem);
        return RGF_E_INVALID;
    }
    const double* src[6] = {H00, S00, H10, S10, Hc, Sc};
    for (int k = 0; k < 6; ++k)
        if (!src[k]) {
            set_error("rgf_set_leads: null block pointer");
            return RGF_E_INVALID;
        }
    if (mem == RGF_MEM_HOST && (!hermitian_host(H00, p->b) || !hermitian_host(S00, p->b))) {
        set_error("rgf_set_leads: lead on-site block is not Hermitian");
        return RGF_E_INVALID;
    }
    const size_t mb = mat_bytes(p->b);
    for (int k = 0; k < 6; ++k)
        RGF_CUDA_TRY(cudaMemcpyAsync(p->lead[side][k], src[k], mb, kind_in(mem), p->stream));
    RGF_CUDA_TRY(cudaStreamSynchronize(p->stream));
    if (p->opt.precision == RGF_MIXED) RGF_TRY(rgf::mixed_on_lead(p, side));
    p->lead_set[side] = true;
    return RGF_OK;
}

rgf_status rgf_transmission(rgf_plan_t p, const double* E, int n_E, double* T, double* err, int* flags,
                            int mem) {
    RGF_TRY(check_plan(p));
    if (n_E < 0 || (n_E > 0 && (!E || !T)) || (mem != RGF_MEM_HOST && mem != RGF_MEM_DEVICE)) {
        set_error("rgf_transmission: invalid arguments");
        return RGF_E_INVALID;
    }
    if (!p->blocks_set || !p->lead_set[0] || !p->lead_set[1]) {
        set_error("rgf_transmission: device blocks and both leads must be set first");
        return RGF_E_STATE;
    }
    if (n_E == 0) return RGF_OK;
    std::lock_guard<std::mutex> lk(p->exec_mu);
    return rgf::run_transmission(p, E, n_E, T, err, flags, mem);
}

rgf_status rgf_submit(rgf_plan_t p, const double* E, int n_E, rgf_ticket_t* ticket) {
    RGF_TRY(check_plan(p));
    if (!ticket || n_E < 0 || (n_E > 0 && !E)) {
        set_error("rgf_submit: invalid arguments");
        return RGF_E_INVALID;
    }
    if (!p->blocks_set || !p->lead_set[0] || !p->lead_set[1]) {
        set_error("rgf_submit: device blocks and both leads must be set first");
        return RGF_E_STATE;
    }
    auto job = std::make_shared<rgf_job>();
    job->id = g_next_ticket.fetch_add(1);
    job->plan = p;
    job->E.assign(E, E + n_E);
    job->T.assign(n_E, 0.0);
    job->err.assign(n_E, 0.0);
    job->flags.assign(n_E, 0);
    {
        std::lock_guard<std::mutex> lk(g_jobs_mu);
        g_jobs[job->id] = job;
    }
    {
        std::lock_guard<std::mutex> lk(p->mu);
        if (!p->worker_started) {
            p->worker = std::thread(worker_loop, p);
            p->worker_started = true;
        }
        p->queue.push_back(job.get());
    }
    p->cv.notify_all();
    *ticket = job->id;
    return RGF_OK;
}

rgf_status rgf_poll(rgf_ticket_t ticket, double* T, double* err, int* flags, int timeout_us) {
    std::shared_ptr<rgf_job> job;
    std::unique_lock<std::mutex> lk(g_jobs_mu);
    auto it = g_jobs.find(ticket);
    if (it == g_jobs.end()) {
        set_error("rgf_poll: unknown ticket %llu", (unsigned long long)ticket);
        return RGF_E_INVALID;
    }
    job = it->second;
    if (!job->done) {
        if (timeout_us == 0) return RGF_E_NOT_READY;
        if (timeout_us < 0) {
            g_jobs_cv.wait(lk, [&] { return job->done; });
        } else if (!g_jobs_cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return job->done; })) {
            set_error("rgf_poll: ticket %llu not done after %d us", (unsigned long long)ticket, timeout_us);
            return RGF_E_TIMEOUT;
        }
    }
    if (job->status != RGF_OK) {
        set_error("%s", job->message.c_str());
        g_jobs.erase(ticket);
        return job->status;
    }
    if (!job->E.empty()) {
        if (!T) {
            set_error("rgf_poll: null T");
            return RGF_E_INVALID;
        }
        std::memcpy(T, job->T.data(), sizeof(double) * job->T.size());
        if (err) std::memcpy(err, job->err.data(), sizeof(double) * job->err.size());
        if (flags) std::memcpy(flags, job->flags.data(), sizeof(int) * job->flags.size());
    }
    g_jobs.erase(ticket);
    return RGF_OK;
}

}  // extern "C"

namespace {
void worker_loop(rgf_plan_s* p) {
    for (;;) {
        rgf_job* job = nullptr;
        {
            std::unique_lock<std::mutex> lk(p->mu);
            p->cv.wait(lk, [&] { return p->stop || !p->queue.empty(); });
            if (p->stop && p->queue.empty()) return;
            job = p->queue.front();
            p->queue.pop_front();
        }
        rgf_status s = RGF_OK;
        if (!job->E.empty()) {
            std::lock_guard<std::mutex> ex(p->exec_mu);
            s = rgf::run_transmission(p, job->E.data(), (int)job->E.size(), job->T.data(), job->err.data(),
                                      job->flags.data(), RGF_MEM_HOST);
        }
        {
            std::lock_guard<std::mutex> lk2(g_jobs_mu);
            job->status = s;
            if (s != RGF_OK) job->message = rgf::get_error();
            job->done = true;
        }
        g_jobs_cv.notify_all();
    }
}
}  // namespace
