// Run-time counters of the library: kernel launches, and CUDA-event timing
// of the slice-product GEMM launches (the dominant kernel of the mixed path).
#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/rgf_kernels.h"
#include "common.cuh"
#include "metrics.h"

namespace rgf {

namespace {
std::atomic<unsigned long long> g_launches{0};
std::mutex g_mu;
std::atomic<bool> g_timing{false};
struct Rec {
    cudaEvent_t a, b;
    double flops;
};
std::vector<Rec> g_recs;
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
std::mutex g_debug_mu;
std::vector<unsigned (*)()>& debug_units() {
    static std::vector<unsigned (*)()> v;
    return v;
}
}  // namespace

void debug_register(unsigned (*collect)()) {
    std::lock_guard<std::mutex> lk(g_debug_mu);
    debug_units().push_back(collect);
}

bool gemm_timing_enabled() { return g_timing.load(std::memory_order_relaxed); }

void gemm_timing_before(cudaStream_t st, cudaEvent_t* a) {
    cudaEventCreate(a);
    cudaEventRecord(*a, st);
}

void gemm_timing_after(cudaStream_t st, cudaEvent_t a, double flops) {
    cudaEvent_t b;
    cudaEventCreate(&b);
    cudaEventRecord(b, st);
    std::lock_guard<std::mutex> lk(g_mu);
    g_recs.push_back({a, b, flops});
}

}  // namespace rgf

extern "C" {

unsigned long long rgf_launch_count(void) { return rgf::g_launches.load(); }

int rgf_debug_build(void) {
#ifdef RGF_DEBUG
    return 1;
#else
    return 0;
#endif
}

unsigned rgf_debug_flags(void) {
    std::lock_guard<std::mutex> lk(rgf::g_debug_mu);
    unsigned w = 0;
    for (auto f : rgf::debug_units()) w |= f();
    return w;
}

rgf_status rgf_gemm_timing(int enable, double* total_ms, long long* launches, double* flops) {
    std::lock_guard<std::mutex> lk(rgf::g_mu);
    if (total_ms || launches || flops) {
        double ms = 0.0, fl = 0.0;
        for (auto& r : rgf::g_recs) {
            if (cudaEventSynchronize(r.b) != cudaSuccess) {
                rgf::set_error("rgf_gemm_timing: event wait failed");
                return RGF_E_CUDA;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, r.a, r.b);
            ms += t;
            fl += r.flops;
        }
        if (total_ms) *total_ms = ms;
        if (launches) *launches = (long long)rgf::g_recs.size();
        if (flops) *flops = fl;
    }
    for (auto& r : rgf::g_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    rgf::g_recs.clear();
    rgf::g_timing.store(enable != 0);
    return RGF_OK;
}

}  // extern "C"
