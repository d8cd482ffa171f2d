// Layer-resolved density of states of a mixed-precision plan
// (rgf_observables.h): forward sweep keeping every left-connected g_i, then
// the backward recursion for the diagonal and first off-diagonal blocks of
// G, each followed by its contribution to -(1/pi) Im Tr[(G S)_ii].
#include <mutex>

#include "../../include/rgf_observables.h"
#include "df.cuh"
#include "mixed_ops.h"
#include "plan.h"

namespace rgf {
namespace {

// out[e * N + layer] += coef * Im sum_jk A_e[j][k] B'[k][j] with
// B' = B (mode 0: Im Tr(A B)) or B' = B^dagger (mode 1: Im Tr(A B^dagger)).
__global__ void k_trace_im_acc(int b, const float4* __restrict__ A, const float4* __restrict__ B, int mode,
                               double coef, double* __restrict__ out, int N, int layer) {
    __shared__ double sh[32];
    const long nn = (long)b * b, off = (long)blockIdx.x * nn;
    double im = 0.0;
    for (long i = threadIdx.x; i < nn; i += blockDim.x) {
        const int j = (int)(i / b), k = (int)(i % b);
        const float4 a4 = A[off + i];
        const double ar = df_to_double(re_of(a4)), ai = df_to_double(im_of(a4));
        const float4 b4 = mode == 0 ? B[(long)k * b + j] : B[i];
        const double br = df_to_double(re_of(b4));
        const double bi = mode == 0 ? df_to_double(im_of(b4)) : -df_to_double(im_of(b4));
        im += ar * bi + ai * br;
    }
    for (int o = 16; o > 0; o >>= 1) im += __shfl_xor_sync(0xffffffffu, im, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = im;
    __syncthreads();
    if (w == 0) {
        im = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) im += __shfl_xor_sync(0xffffffffu, im, o);
        if (l == 0) out[(long)blockIdx.x * N + layer] += coef * im;
    }
}

rgf_status trace_im_acc(int batch, int b, const float4* A, const float4* B, int mode, double coef, double* out,
                        int N, int layer, cudaStream_t st) {
    k_trace_im_acc<<<batch, 256, 0, st>>>(b, A, B, mode, coef, out, N, layer);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

constexpr double kInvPi = 0.31830988618379067154;

// One wave of W energies already in p->d_E; D (W x N, device) receives the
// layer DOS.  g_store holds N x W df matrices.
rgf_status ldos_wave(rgf_plan_s* p, int W, float4* g_store, double* D) {
    auto* pm = (PlanMixed*)p->mixed;
    MixedState* m = &pm->ms;
    cudaStream_t st = p->stream;
    const int b = p->b, N = p->N;
    const long nn = (long)b * b;
    const double eta = p->opt.eta;
    const double* E = p->d_E;
    Ctx c{m, st, nn, b, p->opt.ns_steps, p->d_err, p->d_flags, &p->n_reseeds};
    auto U = [&](int unit) { return m->pool + (long)unit * W * nn; };
    auto g = [&](int i) { return g_store + (long)i * W * nn; };
    RGF_TRY(mixed_leads(p, W, c));
    float4 *sigL = U(0), *sigR = U(0) + (long)W * nn;
    float4 *Ut = U(4), *Lt = U(5), *X = U(6), *Z = U(7), *Y = U(8), *Gup = U(9), *M = U(12), *P = U(13),
           *Rs = U(14);
    float4* Gn[2] = {U(10), U(11)};

    // Forward sweep, keeping g_i.
    FormSrcDf a0{{pm->S_diag, nullptr}, {pm->H_diag, nullptr}, {0, 0}};
    RGF_TRY(form_dfc(W, 1, b, E, eta, a0, M, sigL, nullptr, st));
    if (N == 1) RGF_TRY(axpy_dfc(W, b, -1.0f, sigR, M, st));
    RGF_TRY(inv_mixed(c, W, W, M, g(0), Rs, nullptr, p->d_flags));
    for (int i = 1; i < N; ++i) {
        const float4* Sl = pm->S_lower + (long)(i - 1) * nn;
        const float4* Hl = pm->H_lower + (long)(i - 1) * nn;
        FormSrcDf up{{Sl, nullptr}, {Hl, nullptr}, {1, 0}};
        FormSrcDf lo{{Sl, nullptr}, {Hl, nullptr}, {0, 0}};
        FormSrcDf ai{{pm->S_diag + (long)i * nn, nullptr}, {pm->H_diag + (long)i * nn, nullptr}, {0, 0}};
        RGF_TRY(form_dfc(W, 1, b, E, eta, up, Ut, nullptr, nullptr, st));
        RGF_TRY(form_dfc(W, 1, b, E, eta, lo, Lt, nullptr, nullptr, st));
        RGF_TRY(form_dfc(W, 1, b, E, eta, ai, M, (i == N - 1) ? sigR : nullptr, nullptr, st));
        RGF_TRY(sliceA(c, W, 0, g(i - 1), nullptr));
        RGF_TRY(sliceB(c, W, 0, Ut, nullptr));
        RGF_TRY(mm(c, W, 0, 0, -1.0f, nullptr, 0, P, nullptr));  // P = -g tau'
        RGF_TRY(sliceA(c, W, 0, Lt, nullptr));
        RGF_TRY(sliceB(c, W, 0, P, nullptr));
        RGF_TRY(mm(c, W, 0, 0, 1.0f, M, 0, M, nullptr));  // M += tau P
        RGF_TRY(inv_mixed(c, W, W, M, g(i), Rs, nullptr, p->d_flags));
    }

    // Backward recursion: G_{N-1,N-1} = g_{N-1}; for i = N-2 .. 0
    //   X = g_i tau'_{i+1}, Z = tau_{i+1} g_i, Y = G_{i+1,i+1} Z,
    //   G_ii = g_i + X Y, G_{i,i+1} = -X G_{i+1,i+1}, G_{i+1,i} = -Y.
    RGF_CUDA_TRY(cudaMemsetAsync(D, 0, sizeof(double) * W * N, st));
    RGF_TRY(copy_dfc(W, b, Gn[(N - 1) & 1], g(N - 1), nullptr, st));
    RGF_TRY(trace_im_acc(W, b, Gn[(N - 1) & 1], pm->S_diag + (long)(N - 1) * nn, 0, -kInvPi, D, N, N - 1, st));
    for (int i = N - 2; i >= 0; --i) {
        float4* Gnext = Gn[(i + 1) & 1];
        float4* Gii = Gn[i & 1];
        const float4* Sl = pm->S_lower + (long)i * nn;  // S_{i+1,i}
        const float4* Hl = pm->H_lower + (long)i * nn;
        FormSrcDf up{{Sl, nullptr}, {Hl, nullptr}, {1, 0}};
        FormSrcDf lo{{Sl, nullptr}, {Hl, nullptr}, {0, 0}};
        RGF_TRY(form_dfc(W, 1, b, E, eta, up, Ut, nullptr, nullptr, st));  // tau'_{i+1} = M_{i,i+1}
        RGF_TRY(form_dfc(W, 1, b, E, eta, lo, Lt, nullptr, nullptr, st));  // tau_{i+1} = M_{i+1,i}
        RGF_TRY(sliceA(c, W, 0, g(i), nullptr));
        RGF_TRY(sliceB(c, W, 0, Ut, nullptr));
        RGF_TRY(mm(c, W, 0, 0, 1.0f, nullptr, 0, X, nullptr));
        RGF_TRY(sliceA(c, W, 1, Lt, nullptr));
        RGF_TRY(sliceB(c, W, 1, g(i), nullptr));
        RGF_TRY(mm(c, W, 1, 1, 1.0f, nullptr, 0, Z, nullptr));
        RGF_TRY(sliceA(c, W, 1, Gnext, nullptr));
        RGF_TRY(sliceB(c, W, 1, Z, nullptr));
        RGF_TRY(mm(c, W, 1, 1, 1.0f, nullptr, 0, Y, nullptr));
        RGF_TRY(sliceA(c, W, 0, X, nullptr));
        RGF_TRY(sliceB(c, W, 0, Y, nullptr));
        RGF_TRY(mm(c, W, 0, 0, 1.0f, g(i), 0, Gii, nullptr));  // G_ii = g_i + X Y
        RGF_TRY(sliceB(c, W, 1, Gnext, nullptr));
        RGF_TRY(mm(c, W, 0, 1, -1.0f, nullptr, 0, Gup, nullptr));  // G_{i,i+1} = -X G_{i+1,i+1}
        RGF_TRY(trace_im_acc(W, b, Gii, pm->S_diag + (long)i * nn, 0, -kInvPi, D, N, i, st));
        RGF_TRY(trace_im_acc(W, b, Gup, Sl, 0, -kInvPi, D, N, i, st));  // Tr(G_{i,i+1} S_{i+1,i})
        // Tr(G_{i+1,i} S_{i,i+1}) = -Tr(Y S_{i+1,i}^dagger)
        RGF_TRY(trace_im_acc(W, b, Y, Sl, 1, kInvPi, D, N, i + 1, st));
    }
    int h_status = 0;
    RGF_CUDA_TRY(cudaMemcpyAsync(&h_status, m->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    RGF_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_status != 0) {
        set_error("tensor-core GEMM pipeline timed out (status 0x%x)", h_status);
        return RGF_E_CUDA;
    }
    return RGF_OK;
}

}  // namespace
}  // namespace rgf

extern "C" rgf_status rgf_ldos(rgf_plan_t p, const double* E, int n_E, double* D, int mem) {
    if (!p || n_E < 0 || (n_E > 0 && (!E || !D)) || (mem != RGF_MEM_HOST && mem != RGF_MEM_DEVICE)) {
        rgf::set_error("rgf_ldos: invalid arguments");
        return RGF_E_INVALID;
    }
    if (p->opt.precision != RGF_MIXED) {
        rgf::set_error("rgf_ldos: needs a plan created with RGF_MIXED");
        return RGF_E_STATE;
    }
    if (!p->blocks_set || !p->lead_set[0] || !p->lead_set[1]) {
        rgf::set_error("rgf_ldos: device blocks and both leads must be set first");
        return RGF_E_STATE;
    }
    if (n_E == 0) return RGF_OK;
    std::lock_guard<std::mutex> lk(p->exec_mu);
    const int N = p->N, b = p->b;
    const size_t per_energy = (size_t)N * b * b * sizeof(float4) + (size_t)N * sizeof(double);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        rgf::set_error("rgf_ldos: cudaMemGetInfo failed");
        return RGF_E_CUDA;
    }
    int W = p->W;
    const size_t budget = (size_t)(0.6 * (double)free_b);
    if ((size_t)W * per_energy > budget) W = (int)(budget / per_energy);
    if (W < 1) {
        rgf::set_error("rgf_ldos: one energy needs %zu bytes for the stored layer inverses", per_energy);
        return RGF_E_OOM;
    }
    float4* g_store = nullptr;
    double* Dd = nullptr;
    if (cudaMalloc((void**)&g_store, (size_t)W * N * b * b * sizeof(float4)) != cudaSuccess ||
        cudaMalloc((void**)&Dd, (size_t)W * N * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(g_store);
        rgf::set_error("rgf_ldos: allocation failed");
        return RGF_E_OOM;
    }
    const cudaMemcpyKind kin = mem == RGF_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind kout = mem == RGF_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    rgf_status s = RGF_OK;
    for (int w0 = 0; w0 < n_E && s == RGF_OK; w0 += W) {
        const int Wc = (n_E - w0) < W ? (n_E - w0) : W;
        if (cudaMemcpyAsync(p->d_E, E + w0, sizeof(double) * Wc, kin, p->stream) != cudaSuccess) {
            s = RGF_E_CUDA;
            break;
        }
        s = rgf::ldos_wave(p, Wc, g_store, Dd);
        if (s == RGF_OK &&
            cudaMemcpyAsync(D + (size_t)w0 * N, Dd, sizeof(double) * Wc * N, kout, p->stream) != cudaSuccess)
            s = RGF_E_CUDA;
    }
    if (cudaStreamSynchronize(p->stream) != cudaSuccess && s == RGF_OK) s = RGF_E_CUDA;
    if (s == RGF_E_CUDA && rgf::get_error()[0] == '\0') rgf::set_error("rgf_ldos: CUDA error");
    cudaFree(g_store);
    cudaFree(Dd);
    return s;
}
