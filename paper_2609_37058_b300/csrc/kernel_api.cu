// Kernel-level C entry points (include/rgf_kernels.h): each copies host
// inputs to temporary device memory, runs one building block and copies the
// result back.
#include <vector>

#include "../../include/rgf_kernels.h"
#include "df.cuh"
#include "gj_tmpl.cuh"
#include "mixed.h"

namespace {

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { cudaFree(p); }
};

rgf_status dalloc(DevBuf& b, size_t bytes) {
    if (cudaMalloc(&b.p, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        rgf::set_error("cudaMalloc(%zu) failed", bytes);
        return RGF_E_OOM;
    }
    return RGF_OK;
}

__global__ void k_dfc_to_f64(long n, const float4* X, double2* Y) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float4 v = X[i];
        Y[i] = make_double2(rgf::df_to_double(make_float2(v.x, v.y)), rgf::df_to_double(make_float2(v.z, v.w)));
    }
}

bool dims_ok(int batch, int m, int n, int k) {
    return batch >= 0 && batch <= 65535 && m >= 1 && n >= 1 && k >= 1 && m <= 4096 && n <= 4096 && k <= 4096;
}

}  // namespace

extern "C" {

rgf_status rgf_kernel_zgemm_f64(int batch, int m, int n, int k, const double* A, const double* B, double* C) {
    if (!dims_ok(batch, m, n, k) || !A || !B || !C) {
        rgf::set_error("rgf_kernel_zgemm_f64: invalid arguments");
        return RGF_E_INVALID;
    }
    if (batch == 0) return RGF_OK;
    const size_t sa = (size_t)m * k, sb = (size_t)k * n, sc = (size_t)m * n;
    DevBuf dA, dB, dC;
    RGF_TRY(dalloc(dA, batch * sa * 16));
    RGF_TRY(dalloc(dB, batch * sb * 16));
    RGF_TRY(dalloc(dC, batch * sc * 16));
    RGF_CUDA_TRY(cudaMemcpy(dA.p, A, batch * sa * 16, cudaMemcpyHostToDevice));
    RGF_CUDA_TRY(cudaMemcpy(dB.p, B, batch * sb * 16, cudaMemcpyHostToDevice));
    rgf::ZGemm g{};
    g.batch = batch;
    g.m = m;
    g.n = n;
    g.k = k;
    g.alpha = make_double2(1, 0);
    g.beta = make_double2(0, 0);
    g.A = (const double2*)dA.p;
    g.lda = k;
    g.sA = (long)sa;
    g.B = (const double2*)dB.p;
    g.ldb = n;
    g.sB = (long)sb;
    g.C = (double2*)dC.p;
    g.ldc = n;
    g.sC = (long)sc;
    RGF_TRY(rgf::zgemm_f64(g, 0));
    RGF_CUDA_TRY(cudaMemcpy(C, dC.p, batch * sc * 16, cudaMemcpyDeviceToHost));
    return RGF_OK;
}

rgf_status rgf_kernel_inverse_f64(int batch, int b, double* A, int* flags) {
    if (batch < 0 || batch > 65535 || b < 1 || b > 512 || !A) {
        rgf::set_error("rgf_kernel_inverse_f64: invalid arguments");
        return RGF_E_INVALID;
    }
    if (batch == 0) return RGF_OK;
    const size_t nn = (size_t)b * b;
    DevBuf dA, ws, df;
    RGF_TRY(dalloc(dA, batch * nn * 16));
    RGF_TRY(dalloc(ws, rgf::inv_f64_workspace_bytes(batch, b)));
    RGF_TRY(dalloc(df, batch * sizeof(int)));
    RGF_CUDA_TRY(cudaMemcpy(dA.p, A, batch * nn * 16, cudaMemcpyHostToDevice));
    RGF_CUDA_TRY(cudaMemset(df.p, 0, batch * sizeof(int)));
    RGF_TRY(rgf::inv_f64(batch, b, (double2*)dA.p, (long)nn, ws.p, (int*)df.p, nullptr, 0));
    RGF_CUDA_TRY(cudaMemcpy(A, dA.p, batch * nn * 16, cudaMemcpyDeviceToHost));
    if (flags) RGF_CUDA_TRY(cudaMemcpy(flags, df.p, batch * sizeof(int), cudaMemcpyDeviceToHost));
    return RGF_OK;
}

rgf_status rgf_kernel_inverse_c64(int batch, int b, float* A, int* flags) {
    if (batch < 0 || batch > 65535 || b < 1 || b > 512 || !A) {
        rgf::set_error("rgf_kernel_inverse_c64: invalid arguments");
        return RGF_E_INVALID;
    }
    if (batch == 0) return RGF_OK;
    const size_t nn = (size_t)b * b;
    DevBuf dA, ws, df, dst;
    RGF_TRY(dalloc(dA, batch * nn * 8));
    RGF_TRY(dalloc(ws, rgf::inv_c32_workspace_bytes(batch, b)));
    RGF_TRY(dalloc(df, batch * sizeof(int)));
    RGF_TRY(dalloc(dst, sizeof(int)));
    RGF_CUDA_TRY(cudaMemcpy(dA.p, A, batch * nn * 8, cudaMemcpyHostToDevice));
    RGF_CUDA_TRY(cudaMemset(df.p, 0, batch * sizeof(int)));
    RGF_CUDA_TRY(cudaMemset(dst.p, 0, sizeof(int)));
    RGF_TRY(rgf::inv_c32(batch, b, (float2*)dA.p, (long)nn, ws.p, (int*)df.p, nullptr, (int*)dst.p, 0));
    int status = 0;
    RGF_CUDA_TRY(cudaMemcpy(&status, dst.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (status != 0) {
        rgf::set_error("rgf_kernel_inverse_c64: tensor-core pipeline timed out (status 0x%x)", status);
        return RGF_E_CUDA;
    }
    RGF_CUDA_TRY(cudaMemcpy(A, dA.p, batch * nn * 8, cudaMemcpyDeviceToHost));
    if (flags) RGF_CUDA_TRY(cudaMemcpy(flags, df.p, batch * sizeof(int), cudaMemcpyDeviceToHost));
    return RGF_OK;
}

static rgf_status zgemm_mixed_impl(int batch, int m, int n, int k, const double* A, const double* B, double* C,
                                   int core, unsigned long long test_wait_ns, int* status_out, int nsl = 0);
static rgf_status zgemm_hp_impl(int batch, int m, int n, int k, const double* A, const double* B, double* C,
                                int nsl);

rgf_status rgf_kernel_zgemm_mixed(int batch, int m, int n, int k, const double* A, const double* B, double* C,
                                  int core) {
    return zgemm_mixed_impl(batch, m, n, k, A, B, C, core, 0, nullptr);
}

rgf_status rgf_kernel_zgemm_slices(int batch, int m, int n, int k, const double* A, const double* B, double* C,
                                   int fp64_operands, int nsl) {
    if (fp64_operands) {
        if (nsl != 5 && nsl != 7) {
            rgf::set_error("rgf_kernel_zgemm_slices: FP64 operands take 5 or 7 slices, not %d", nsl);
            return RGF_E_INVALID;
        }
        return zgemm_hp_impl(batch, m, n, k, A, B, C, nsl == 7 ? 0 : nsl);
    }
    if (nsl != 4 && nsl != 5 && nsl != 6) {
        rgf::set_error("rgf_kernel_zgemm_slices: double-float operands take 4, 5 or 6 slices, not %d", nsl);
        return RGF_E_INVALID;
    }
    return zgemm_mixed_impl(batch, m, n, k, A, B, C, 0, 0, nullptr, nsl == 6 ? 0 : nsl);
}

rgf_status rgf_kernel_tc_timeout_probe(int wait_us, int* status_bits) {
    if (wait_us < 1 || wait_us > 1000000 || !status_bits) {
        rgf::set_error("rgf_kernel_tc_timeout_probe: wait_us in [1, 1e6] and a status pointer required");
        return RGF_E_INVALID;
    }
    const int b = 64, batch = 2;
    std::vector<double> A(2 * (size_t)batch * b * b, 0.5), B(2 * (size_t)batch * b * b, 0.25), C(2 * (size_t)batch * b * b);
    return zgemm_mixed_impl(batch, b, b, b, A.data(), B.data(), C.data(), 0, 1000ull * wait_us, status_bits);
}

static rgf_status zgemm_mixed_impl(int batch, int m, int n, int k, const double* A, const double* B, double* C,
                                   int core, unsigned long long test_wait_ns, int* status_out, int nsl) {
    if (!dims_ok(batch, m, n, k) || !A || !B || !C || (core != 0 && core != 1)) {
        rgf::set_error("rgf_kernel_zgemm_mixed: invalid arguments");
        return RGF_E_INVALID;
    }
    if (batch == 0) return RGF_OK;
    const size_t sa = (size_t)m * k, sb = (size_t)k * n, sc = (size_t)m * n;
    const int Kp = rgf::slice_pitch(k);
    DevBuf dA, dB, fA, fB, fC, dC, SA, SB, status;
    RGF_TRY(dalloc(dA, batch * sa * 16));
    RGF_TRY(dalloc(dB, batch * sb * 16));
    RGF_TRY(dalloc(fA, batch * sa * 16));
    RGF_TRY(dalloc(fB, batch * sb * 16));
    RGF_TRY(dalloc(fC, batch * sc * 16));
    RGF_TRY(dalloc(dC, batch * sc * 16));
    const size_t sab = (size_t)batch * rgf::kSlices * m * Kp * 2, sbb = (size_t)batch * rgf::kSlices * 2 * n * Kp * 2;
    RGF_TRY(dalloc(SA, sab));
    RGF_TRY(dalloc(SB, sbb));
    RGF_TRY(dalloc(status, sizeof(int)));
    RGF_CUDA_TRY(cudaMemset(SA.p, 0, sab));
    RGF_CUDA_TRY(cudaMemset(SB.p, 0, sbb));
    RGF_CUDA_TRY(cudaMemset(status.p, 0, sizeof(int)));
    RGF_CUDA_TRY(cudaMemcpy(dA.p, A, batch * sa * 16, cudaMemcpyHostToDevice));
    RGF_CUDA_TRY(cudaMemcpy(dB.p, B, batch * sb * 16, cudaMemcpyHostToDevice));
    RGF_TRY(rgf::to_dfc((long)(batch * sa), (const double2*)dA.p, (float4*)fA.p, 0));
    RGF_TRY(rgf::to_dfc((long)(batch * sb), (const double2*)dB.p, (float4*)fB.p, 0));
    RGF_TRY(rgf::slice_rows(batch, m, k, (const float4*)fA.p, (long)sa, (__nv_bfloat16*)SA.p, Kp, nullptr, 0));
    RGF_TRY(rgf::slice_cols(batch, k, n, (const float4*)fB.p, (long)sb, (__nv_bfloat16*)SB.p, Kp,
                            nullptr, 0));
    rgf::OzGemm g{};
    g.batch = batch;
    g.m = m;
    g.n = n;
    g.k = k;
    g.As = (const __nv_bfloat16*)SA.p;
    g.Bs = (const __nv_bfloat16*)SB.p;
    g.Kp = Kp;
    g.alpha = 1.0f;
    g.C = (float4*)fC.p;
    g.sC = (long)sc;
    g.status = (int*)status.p;
    g.test_wait_ns = test_wait_ns;
    g.nsl = nsl;
    RGF_TRY(rgf::oz_gemm(g, core, 0));
    k_dfc_to_f64<<<1024, 256>>>((long)(batch * sc), (const float4*)fC.p, (double2*)dC.p);
    RGF_LAUNCH_CHECK();
    int h_status = 0;
    RGF_CUDA_TRY(cudaMemcpy(&h_status, status.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (status_out) *status_out = h_status;
    if (h_status) {
        rgf::set_error("tensor-core pipeline timeout (status 0x%x)", h_status);
        return RGF_E_CUDA;
    }
    RGF_CUDA_TRY(cudaMemcpy(C, dC.p, batch * sc * 16, cudaMemcpyDeviceToHost));
    return RGF_OK;
}

rgf_status rgf_kernel_zgemm_hp(int batch, int m, int n, int k, const double* A, const double* B, double* C) {
    return zgemm_hp_impl(batch, m, n, k, A, B, C, 0);
}

static rgf_status zgemm_hp_impl(int batch, int m, int n, int k, const double* A, const double* B, double* C,
                                int nsl) {
    if (!dims_ok(batch, m, n, k) || !A || !B || !C) {
        rgf::set_error("rgf_kernel_zgemm_hp: invalid arguments");
        return RGF_E_INVALID;
    }
    if (batch == 0) return RGF_OK;
    const size_t sa = (size_t)m * k, sb = (size_t)k * n, sc = (size_t)m * n;
    const int Kp = rgf::slice_pitch(k);
    DevBuf dA, dB, dC, SA, SB, status;
    RGF_TRY(dalloc(dA, batch * sa * 16));
    RGF_TRY(dalloc(dB, batch * sb * 16));
    RGF_TRY(dalloc(dC, batch * sc * 16));
    const size_t sab = (size_t)batch * rgf::kSlicesHP * m * Kp * 2, sbb = (size_t)batch * rgf::kSlicesHP * 2 * n * Kp * 2;
    RGF_TRY(dalloc(SA, sab));
    RGF_TRY(dalloc(SB, sbb));
    RGF_TRY(dalloc(status, sizeof(int)));
    RGF_CUDA_TRY(cudaMemset(SA.p, 0, sab));
    RGF_CUDA_TRY(cudaMemset(SB.p, 0, sbb));
    RGF_CUDA_TRY(cudaMemset(status.p, 0, sizeof(int)));
    RGF_CUDA_TRY(cudaMemcpy(dA.p, A, batch * sa * 16, cudaMemcpyHostToDevice));
    RGF_CUDA_TRY(cudaMemcpy(dB.p, B, batch * sb * 16, cudaMemcpyHostToDevice));
    RGF_TRY(rgf::slice_rows_f64(batch, m, k, (const double2*)dA.p, (long)sa, (__nv_bfloat16*)SA.p, Kp, nullptr, 0));
    RGF_TRY(rgf::slice_cols_f64(batch, k, n, (const double2*)dB.p, (long)sb, (__nv_bfloat16*)SB.p, Kp,
                                nullptr, 0));
    rgf::OzGemmHP g{};
    g.batch = batch;
    g.m = m;
    g.n = n;
    g.k = k;
    g.As = (const __nv_bfloat16*)SA.p;
    g.Bs = (const __nv_bfloat16*)SB.p;
    g.Kp = Kp;
    g.alpha = 1.0f;
    g.C = (double2*)dC.p;
    g.sC = (long)sc;
    g.status = (int*)status.p;
    g.nsl = nsl;
    RGF_TRY(rgf::oz_gemm_hp(g, 0));
    int h_status = 0;
    RGF_CUDA_TRY(cudaMemcpy(&h_status, status.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (h_status) {
        rgf::set_error("tensor-core pipeline timeout (status 0x%x)", h_status);
        return RGF_E_CUDA;
    }
    RGF_CUDA_TRY(cudaMemcpy(C, dC.p, batch * sc * 16, cudaMemcpyDeviceToHost));
    return RGF_OK;
}

}  // extern "C"
