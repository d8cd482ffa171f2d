// Landauer current from T(E) (rgf_observables.h): one CTA per bias, the
// trapezoidal sum over energy intervals reduced with warp shuffles.
#include "../../include/rgf_observables.h"
#include "common.cuh"

namespace rgf {
namespace {

constexpr double kG0 = 7.748091729863649e-5;  // 2 e^2 / h in siemens

// Fermi function 1 / (1 + exp(x / kT)) written with tanh (no overflow); the
// step function with value 1/2 at x = 0 when kT = 0.
__device__ __forceinline__ double fermi(double x, double kT) {
    if (kT > 0.0) return 0.5 * (1.0 - tanh(0.5 * x / kT));
    return x < 0.0 ? 1.0 : (x > 0.0 ? 0.0 : 0.5);
}

__global__ void k_current(int n_E, const double* __restrict__ E, const double* __restrict__ T,
                          const double* __restrict__ V, double E_F, double kT, double* __restrict__ I) {
    __shared__ double sh[32];
    const double v = V[blockIdx.x];
    const double muL = E_F + 0.5 * v, muR = E_F - 0.5 * v;
    double s = 0.0;
    for (int i = threadIdx.x; i < n_E - 1; i += blockDim.x) {
        const double e0 = E[i], e1 = E[i + 1];
        const double g0 = T[i] * (fermi(e0 - muL, kT) - fermi(e0 - muR, kT));
        const double g1 = T[i + 1] * (fermi(e1 - muL, kT) - fermi(e1 - muR, kT));
        s += 0.5 * (e1 - e0) * (g0 + g1);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = s;
    __syncthreads();
    if (w == 0) {
        s = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (l == 0) I[blockIdx.x] = kG0 * s;
    }
}

}  // namespace
}  // namespace rgf

extern "C" rgf_status rgf_current(int n_E, const double* E, const double* T, int n_V, const double* V, double E_F,
                                  double kT, double* I, void* cuda_stream) {
    if (n_E < 2 || n_V < 1 || !(kT >= 0.0) || !E || !T || !V || !I) {
        rgf::set_error("rgf_current: invalid arguments");
        return RGF_E_INVALID;
    }
    rgf::k_current<<<n_V, 256, 0, (cudaStream_t)cuda_stream>>>(n_E, E, T, V, E_F, kT, I);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}
