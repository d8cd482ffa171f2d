// FP32 seed inverse of the mixed path with its trailing updates on the
// tensor cores: blocked Gauss-Jordan with partial pivoting (panel and row
// interchanges on the CUDA cores, gj_tmpl.cuh), each update C += Pbar T a
// tcgen05 product of BF16 splits accumulated in FP32 (gj_update_tc,
// tc_gemm.cu).
#include <algorithm>
#include <cstdlib>

#include "gj_tmpl.cuh"

namespace rgf {

size_t inv_c32_workspace_bytes(int batch, int b) {
    // Pbar splits (b rows) and T splits (2b rows) per entry, then pivots.
    const size_t tc = (size_t)batch * ((size_t)kGjSplits * 3 * b * kGjKp * sizeof(__nv_bfloat16) +
                                       (size_t)b * sizeof(int)) +
                      256;
    return std::max(tc, inv_workspace_bytes_t<float2>(batch, b));
}

// Tensor-core update unless RGF_GJ_TC=0 in the environment (read once).
static bool gj_tc_enabled() {
    static const bool on = [] {
        const char* e = getenv("RGF_GJ_TC");
        return !(e && e[0] == '0');
    }();
    return on;
}

rgf_status inv_c32(int batch, int b, float2* A, long sA, void* ws, int* flags, const int* active, int* status,
                   cudaStream_t st, int nb_override) {
    return inv_t<float2>(batch, b, A, sA, ws, flags, active, st, nb_override, gj_tc_enabled() ? status : nullptr);
}

rgf_status inv_c32_to(int batch, int b, float2* A, long sA, void* ws, int* flags, const int* active, int* status,
                      cudaStream_t st, int nb_override, float4* out_df, double2* out_c128) {
    if ((out_df != nullptr) == (out_c128 != nullptr)) {
        set_error("inv_c32_to: exactly one output is required");
        return RGF_E_INVALID;
    }
    return inv_t<float2>(batch, b, A, sA, ws, flags, active, st, nb_override, gj_tc_enabled() ? status : nullptr,
                         out_df, out_c128);
}

}  // namespace rgf
