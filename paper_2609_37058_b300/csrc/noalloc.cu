// Allocation-free variant of the FP64 batched inverse (see rgf_kernels.h).
//
// The Gauss-Jordan workspace (panel copies, row blocks, pivots) lives in one
// file-scope device array instead of memory from cudaMalloc.  Host code must
// not use the array's name as a pointer: on the host it is only a stand-in
// symbol.  Its device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and cached.
#include <mutex>

#include "../../include/rgf_kernels.h"
#include "gj_tmpl.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;  // 16 MiB on every GPU that loads the library
static __device__ __align__(256) unsigned char g_inverse_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

rgf_status scratch_for_current_device(void** out) {
    int dev = -1;
    RGF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        rgf::set_error("rgf_inverse_f64_noalloc: device ordinal %d out of range", dev);
        return RGF_E_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_inverse_scratch);
        if (e != cudaSuccess || !p) {
            rgf::set_error("rgf_inverse_f64_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return RGF_E_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return RGF_OK;
}

}  // namespace

extern "C" {

size_t rgf_inverse_f64_noalloc_limit(void) { return kNoAllocScratchBytes; }

rgf_status rgf_inverse_f64_noalloc(int batch, int b, double* A, int* flags, void* cuda_stream) {
    if (batch < 0 || batch > 65535 || b < 1 || b > 512 || (batch > 0 && !A)) {
        rgf::set_error("rgf_inverse_f64_noalloc: invalid arguments (batch %d, b %d)", batch, b);
        return RGF_E_INVALID;
    }
    const size_t need = rgf::inv_workspace_bytes_t<double2>(batch, b);
    if (need > kNoAllocScratchBytes) {
        rgf::set_error("rgf_inverse_f64_noalloc: batch %d of %d x %d matrices needs %zu bytes of scratch, more than "
                       "the fixed %zu",
                       batch, b, b, need, kNoAllocScratchBytes);
        return RGF_E_INVALID;
    }
    // The inverse's own shared-memory limit, checked here so that a call it
    // would reject fails before the flags are cleared.
    const int nb = rgf::gj_nb(b);
    const size_t smem = ((size_t)b * (nb + 1) + b) * sizeof(double2);
    if (smem > 200 * 1024) {
        rgf::set_error("rgf_inverse_f64_noalloc: b = %d needs %zu bytes of shared memory", b, smem);
        return RGF_E_INVALID;
    }
    if (batch == 0) return RGF_OK;
    void* scratch = nullptr;
    RGF_TRY(scratch_for_current_device(&scratch));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (flags) RGF_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * batch, st));
    return rgf::inv_t<double2>(batch, b, reinterpret_cast<double2*>(A), (long)b * b, scratch, flags, nullptr, st);
}

}  // extern "C"
