// Shared device helpers of the RGF library: complex arithmetic on
// double2/float2, error plumbing, launch geometry.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/rgf.h"
#include "nvtx3/nvToolsExt.h"

namespace rgf {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
const char* get_error();

#define RGF_CUDA_TRY(expr)                                                          \
    do {                                                                            \
        cudaError_t _e = (expr);                                                    \
        if (_e != cudaSuccess) {                                                    \
            ::rgf::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr,             \
                             cudaGetErrorString(_e));                              \
            return RGF_E_CUDA;                                                      \
        }                                                                           \
    } while (0)

#define RGF_TRY(expr)                          \
    do {                                       \
        rgf_status _s = (expr);                \
        if (_s != RGF_OK) return _s;           \
    } while (0)

void count_launch();

#define RGF_LAUNCH_CHECK()                                                          \
    do {                                                                            \
        ::rgf::count_launch();                                                      \
        cudaError_t _e = cudaGetLastError();                                        \
        if (_e != cudaSuccess) {                                                    \
            ::rgf::set_error("%s:%d kernel launch: %s", __FILE__, __LINE__,         \
                             cudaGetErrorString(_e));                              \
            return RGF_E_CUDA;                                                      \
        }                                                                           \
    } while (0)

// ---------------------------------------------------------------- complex
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) {
    return make_double2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) {
    return make_double2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
// acc += a * b
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ double2 cinv(double2 d) {
    double s = 1.0 / (d.x * d.x + d.y * d.y);
    return make_double2(d.x * s, -d.y * s);
}

__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
    return make_float2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float2 cinv(float2 d) {
    float s = 1.0f / (d.x * d.x + d.y * d.y);
    return make_float2(d.x * s, -d.y * s);
}

inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// Named NVTX range for the lifetime of the object (profilers group the
// launches of a phase under it; without a profiler attached it costs a
// function-pointer check).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------- debug checks
// The build with -DRGF_DEBUG checks on the device the indices that come from
// data (pivot rows of the Gauss-Jordan inverses, entries of the server's
// slot table).  A failed check ORs its bit into this translation unit's
// device word and the kernel goes on with a safe index or skips the access:
// no trap, no early exit before a barrier.  rgf_debug_flags() collects and
// clears the words of every unit.  In the normal build RGF_DCHECK is true.
enum : unsigned { RGF_DBG_PIVOT = 1u, RGF_DBG_SLOT = 2u, RGF_DBG_POINTER = 4u };
void debug_register(unsigned (*collect)());
#ifdef RGF_DEBUG
static __device__ unsigned int g_debug_word;
__device__ __forceinline__ bool debug_fail(unsigned bit) {
    atomicOr(&g_debug_word, bit);
    return false;
}
namespace {
unsigned debug_collect_unit() {
    unsigned h = 0, z = 0;
    if (cudaMemcpyFromSymbol(&h, g_debug_word, sizeof(h)) != cudaSuccess) return 0x80000000u;
    cudaMemcpyToSymbol(g_debug_word, &z, sizeof(z));
    return h;
}
const int g_debug_unit_registered = (debug_register(&debug_collect_unit), 0);
}  // namespace
#define RGF_DCHECK(cond, bit) ((cond) || ::rgf::debug_fail(bit))
#else
#define RGF_DCHECK(cond, bit) true
#endif

}  // namespace rgf
