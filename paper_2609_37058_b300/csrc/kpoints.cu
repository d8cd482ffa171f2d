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

extern "C" rgf_status rgf_kmesh_transmission(rgf_server_t server, const rgf_kdevice* dev, int n_k, const double* kfrac,
                                             const double* w, const double* E, int n_E, double eta, int group,
                                             double* T, double* T_k, void* cuda_stream) {
    if (!server || !dev || !kfrac || !w || !E || !T || n_k < 1 || n_E < 1 || !(eta > 0.0) || group < 1 ||
        group > 64 || dev->n_R < 1 || dev->n_R > rgf::kMaxR || !dev->R || dev->n_layers < 1 || dev->b < 1 ||
        dev->b > 512 || !dev->H_diag || !dev->S_diag || !dev->lead[0] || !dev->lead[1] ||
        (dev->n_layers > 1 && (!dev->H_lower || !dev->S_lower))) {
        rgf::set_error("rgf_kmesh_transmission: invalid arguments");
        return RGF_E_INVALID;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int N = dev->n_layers, b = dev->b, nR = dev->n_R;
    const size_t bb = (size_t)b * b;
    const size_t per_k = bb * (2 * (size_t)N + 2 * (size_t)(N - 1) + 12);  // complex128 entries of one device
    const int G = group < n_k ? group : n_k;
    // One allocation: G devices of Bloch-summed blocks, the energies, T(E, k).
    double* buf = nullptr;
    const size_t bytes = (size_t)G * per_k * 16 + (size_t)n_E * 8 + (size_t)n_k * 8 + (size_t)n_k * n_E * 8;
    RGF_CUDA_TRY(cudaMalloc(&buf, bytes));
    struct Free {
        double* p;
        ~Free() { cudaFree(p); }
    } guard{buf};
    double* dE = buf + (size_t)G * per_k * 2;
    double* dw = dE + n_E;
    double* Tk = T_k ? T_k : dw + n_k;
    RGF_CUDA_TRY(cudaMemcpyAsync(dE, E, sizeof(double) * n_E, cudaMemcpyHostToDevice, st));
    RGF_CUDA_TRY(cudaMemcpyAsync(dw, w, sizeof(double) * n_k, cudaMemcpyHostToDevice, st));
    std::vector<rgf_ticket_t> tickets(G);
    for (int k0 = 0; k0 < n_k; k0 += G) {
        const int nk = (n_k - k0) < G ? (n_k - k0) : G;
        std::vector<rgf_request> reqs(nk);
        for (int j = 0; j < nk; ++j) {
            const double* kf = kfrac + 2 * (size_t)(k0 + j);
            double* base = buf + (size_t)j * per_k * 2;
            double* Hd = base;
            double* Sd = Hd + bb * N * 2;
            double* Hl = Sd + bb * N * 2;
            double* Sl = Hl + bb * (N - 1) * 2;
            double* L[2] = {Sl + bb * (N - 1) * 2, Sl + bb * (N - 1) * 2 + bb * 6 * 2};
            RGF_TRY(rgf_bloch_sum(nR, dev->R, kf, N, b, dev->H_diag, Hd, st));
            RGF_TRY(rgf_bloch_sum(nR, dev->R, kf, N, b, dev->S_diag, Sd, st));
            if (N > 1) {
                RGF_TRY(rgf_bloch_sum(nR, dev->R, kf, N - 1, b, dev->H_lower, Hl, st));
                RGF_TRY(rgf_bloch_sum(nR, dev->R, kf, N - 1, b, dev->S_lower, Sl, st));
            }
            for (int s = 0; s < 2; ++s) RGF_TRY(rgf_bloch_sum(nR, dev->R, kf, 6, b, dev->lead[s], L[s], st));
            rgf_request& r = reqs[j];
            r = rgf_request{};
            r.n_layers = N;
            r.b = b;
            r.eta = eta;
            r.H_diag = Hd;
            r.S_diag = Sd;
            r.H_lower = N > 1 ? Hl : nullptr;
            r.S_lower = N > 1 ? Sl : nullptr;
            for (int s = 0; s < 2; ++s)
                for (int q = 0; q < 6; ++q) r.lead[s][q] = L[s] + bb * q * 2;
            r.E = dE;
            r.n_E = n_E;
            r.mem = RGF_MEM_DEVICE;
        }
        // The server reads the blocks on its own streams once it admits them.
        RGF_CUDA_TRY(cudaStreamSynchronize(st));
        rgf_status first_err = RGF_OK;
        int submitted = 0;
        for (; submitted < nk; ++submitted) {
            first_err = rgf_server_submit(server, &reqs[submitted], &tickets[submitted]);
            if (first_err != RGF_OK) break;
        }
        for (int j = 0; j < submitted; ++j) {
            // Every ticket is collected (so the server lets go of the blocks)
            // before the buffers are reused or freed.
            const rgf_status s =
                rgf_server_poll(server, tickets[j], Tk + (size_t)(k0 + j) * n_E, nullptr, nullptr, nullptr, -1);
            if (s != RGF_OK && first_err == RGF_OK) first_err = s;
        }
        if (first_err != RGF_OK) return first_err;
    }
    RGF_TRY(rgf_kmesh_mean(n_k, n_E, Tk, dw, T, cuda_stream));
    RGF_CUDA_TRY(cudaStreamSynchronize(st));
    return RGF_OK;
}
