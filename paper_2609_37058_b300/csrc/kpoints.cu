// Transverse Bloch sums X(k) = sum_R exp(2 pi i k.R) X(R) (rgf_kpoints.h).
// HBM-bound: reads n_R blocks and writes one per output element.  The
// phases are computed on the host in FP64 and passed by value.
#include <cmath>
#include <vector>

#include "../../include/rgf_kpoints.h"
#include "common.cuh"

namespace rgf {
namespace {

constexpr int kMaxR = 64;

struct Phases {
    double2 p[kMaxR];
};

__global__ void k_bloch_sum(int n_R, long n, const double2* __restrict__ XR, double2* __restrict__ Xk, Phases ph) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int r = 0; r < n_R; ++r) cfma(acc, ph.p[r], XR[(long)r * n + i]);
        Xk[i] = acc;
    }
}

__global__ void k_kmesh_mean(int n_k, int n_E, const double* __restrict__ Tk, const double* __restrict__ w,
                             double* __restrict__ T) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_E) return;
    double s = 0.0;
    for (int k = 0; k < n_k; ++k) s = fma(w[k], Tk[(long)k * n_E + e], s);
    T[e] = s;
}

}  // namespace
}  // namespace rgf

extern "C" rgf_status rgf_bloch_sum(int n_R, const int* R, const double* kfrac, int n_blocks, int b,
                                    const double* X_R, double* X_k, void* cuda_stream) {
    if (n_R < 1 || n_R > rgf::kMaxR || n_blocks < 1 || b < 1 || !R || !kfrac || !X_R || !X_k) {
        rgf::set_error("rgf_bloch_sum: invalid arguments (1 <= n_R <= %d, n_blocks, b >= 1, non-null pointers)",
                       rgf::kMaxR);
        return RGF_E_INVALID;
    }
    rgf::Phases ph{};
    const double two_pi = 6.283185307179586476925286766559;
    for (int r = 0; r < n_R; ++r) {
        // Reduce k.R to [0, 1) before the trigonometric call so that large
        // lattice vectors keep the phase accurate.
        double t = kfrac[0] * R[2 * r] + kfrac[1] * R[2 * r + 1];
        t -= std::floor(t);
        ph.p[r] = make_double2(std::cos(two_pi * t), std::sin(two_pi * t));
    }
    const long n = (long)n_blocks * b * b;
    const int threads = 256;
    long blocks = (n + threads - 1) / threads;
    if (blocks > 148L * 16) blocks = 148L * 16;
    rgf::k_bloch_sum<<<(int)blocks, threads, 0, (cudaStream_t)cuda_stream>>>(
        n_R, n, (const double2*)X_R, (double2*)X_k, ph);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

extern "C" rgf_status rgf_kmesh_mean(int n_k, int n_E, const double* T_k, const double* w, double* T,
                                     void* cuda_stream) {
    if (n_k < 1 || n_E < 1 || !T_k || !w || !T) {
        rgf::set_error("rgf_kmesh_mean: invalid arguments");
        return RGF_E_INVALID;
    }
    rgf::k_kmesh_mean<<<(n_E + 127) / 128, 128, 0, (cudaStream_t)cuda_stream>>>(n_k, n_E, T_k, w, T);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}
