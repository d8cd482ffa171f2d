// FP64 kernels of the RGF library: block formation z S - H, batched complex
// GEMM, batched blocked Gauss-Jordan inverse, decimation updates and the
// Caroli trace.  All matrices are b x b complex128 (double2), row-major,
// one matrix per batch entry unless a stride says otherwise.
#include <cstdarg>
#include <cstdio>

#include "kernels.h"
#include "gj_tmpl.cuh"

namespace rgf {

// ------------------------------------------------------------------ errors
static thread_local char g_err[1024] = "";
void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
const char* get_error() { return g_err; }

static inline int grid_for(long n, int threads, int cap = 1024) {
    long g = (n + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// ------------------------------------------------------------------ form
__global__ void k_form_f64(int W, int b, const double* __restrict__ E, double eta, FormSrc src,
                           double2* __restrict__ out, const double2* __restrict__ sub,
                           double sub_coef, const int* __restrict__ active) {
    const int be = blockIdx.y;
    if (active && !active[be]) return;
    const int s = be / W, e = be % W;
    const double2 z = make_double2(E[e], eta);
    const double2* S = src.S[s];
    const double2* H = src.H[s];
    const int tr = src.trans[s];
    const long nn = (long)b * b;
    double2* o = out + (long)be * nn;
    const double2* sb = sub ? sub + (long)be * nn : nullptr;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < nn;
         idx += (long)gridDim.x * blockDim.x) {
        const int r = (int)(idx / b), c = (int)(idx % b);
        const long src_idx = tr ? (long)c * b + r : idx;
        double2 sv = S ? S[src_idx] : make_double2(0.0, 0.0);
        double2 hv = H[src_idx];
        if (tr) {
            sv = cconj(sv);
            hv = cconj(hv);
        }
        double2 v = csub(cmul(z, sv), hv);
        if (sb) {
            v.x -= sub_coef * sb[idx].x;
            v.y -= sub_coef * sb[idx].y;
        }
        o[idx] = v;
    }
}

rgf_status form_f64(int W, int nsrc, int b, const double* E, double eta, const FormSrc& src,
                    double2* out, const double2* sub, double sub_coef, const int* active,
                    cudaStream_t st) {
    if (W <= 0) return RGF_OK;
    dim3 grid(grid_for((long)b * b, 256, 64), W * nsrc);
    k_form_f64<<<grid, 256, 0, st>>>(W, b, E, eta, src, out, sub, sub_coef, active);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

// ------------------------------------------------------------------ GEMM / inverse
rgf_status zgemm_f64(const ZGemm& g, cudaStream_t st) { return zgemm_t<double2>(g, st); }

size_t inv_f64_workspace_bytes(int batch, int b) { return inv_workspace_bytes_t<double2>(batch, b); }

rgf_status inv_f64(int batch, int b, double2* A, long sA, void* ws, int* flags, const int* active,
                   cudaStream_t st) {
    return inv_t<double2>(batch, b, A, sA, ws, flags, active, st);
}

// ------------------------------------------------------------------ elementwise
__global__ void k_identity_f64(int b, double2* A) {
    const long nn = (long)b * b;
    double2* Ab = A + (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x)
        Ab[i] = make_double2((i / b) == (i % b) ? 1.0 : 0.0, 0.0);
}

rgf_status set_identity_f64(int batch, int b, double2* A, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_identity_f64<<<dim3(grid_for((long)b * b, 256, 64), batch), 256, 0, st>>>(b, A);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_dec_update_f64(int b, double2* eps_s, double2* eps, const double2* agb,
                                 const double2* bga, const int* active) {
    if (active && !active[blockIdx.y]) return;
    const long nn = (long)b * b, off = (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const double2 x = agb[off + i], y = bga[off + i];
        eps_s[off + i] = csub(eps_s[off + i], x);
        eps[off + i] = csub(csub(eps[off + i], x), y);
    }
}

rgf_status dec_update_f64(int batch, int b, double2* eps_s, double2* eps, const double2* agb,
                          const double2* bga, const int* active, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_dec_update_f64<<<dim3(grid_for((long)b * b, 256, 64), batch), 256, 0, st>>>(b, eps_s, eps, agb, bga,
                                                                              active);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_gamma_f64(int b, const double2* sigma, double2* gamma) {
    const long nn = (long)b * b, off = (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / b), c = (int)(i % b);
        const double2 s = sigma[off + i];
        const double2 st = sigma[off + (long)c * b + r];
        // i (s - conj(st)) = i ((s.x - st.x) + i (s.y + st.y))
        gamma[off + i] = make_double2(-(s.y + st.y), s.x - st.x);
    }
}

rgf_status gamma_f64(int batch, int b, const double2* sigma, double2* gamma, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_gamma_f64<<<dim3(grid_for((long)b * b, 256, 64), batch), 256, 0, st>>>(b, sigma, gamma);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__device__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;  // valid on thread 0
}

__global__ void k_dec_check_f64(int b, const double2* alpha, const double2* beta, const double* anorm,
                                double tol, int it, int* active, int* iters, int* remaining) {
    const int bi = blockIdx.x;
    if (!active[bi]) return;
    __shared__ double sh[32];
    const long nn = (long)b * b, off = (long)bi * nn;
    double sa = 0.0, sb = 0.0;
    for (long i = threadIdx.x; i < nn; i += blockDim.x) {
        sa += cabs2(alpha[off + i]);
        sb += cabs2(beta[off + i]);
    }
    const double ta = block_sum(sa, sh);
    const double tb = block_sum(sb, sh);
    if (threadIdx.x == 0) {
        iters[bi] = it;
        const double lim = tol * anorm[bi];
        if (sqrt(ta) <= lim && sqrt(tb) <= lim) {
            active[bi] = 0;
        } else {
            atomicAdd(remaining, 1);
        }
    }
}

rgf_status dec_check_f64(int batch, int b, const double2* alpha, const double2* beta,
                         const double* anorm, double tol, int it, int* active, int* iters,
                         int* remaining, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_dec_check_f64<<<batch, 256, 0, st>>>(b, alpha, beta, anorm, tol, it, active, iters, remaining);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_fro_norm_f64(int b, const double2* A, double* out) {
    __shared__ double sh[32];
    const long nn = (long)b * b, off = (long)blockIdx.x * nn;
    double s = 0.0;
    for (long i = threadIdx.x; i < nn; i += blockDim.x) s += cabs2(A[off + i]);
    const double t = block_sum(s, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = sqrt(t);
}

rgf_status fro_norm_f64(int batch, int b, const double2* A, double* out, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_fro_norm_f64<<<batch, 256, 0, st>>>(b, A, out);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

// Tr[Gamma_L G Gamma_R G^dag] = sum_jk X_jk conj(Y_jk) with X = Gamma_L G and
// Y = G Gamma_R (Gamma_R Hermitian); one CTA per energy, warp-shuffle sums.
__global__ void k_trace_xy_f64(int b, const double2* X, const double2* Y, double* T, double* Ti) {
    __shared__ double sh[32];
    const long nn = (long)b * b, off = (long)blockIdx.x * nn;
    double re = 0.0, im = 0.0;
    for (long i = threadIdx.x; i < nn; i += blockDim.x) {
        const double2 x = X[off + i], y = Y[off + i];
        re += x.x * y.x + x.y * y.y;
        im += x.y * y.x - x.x * y.y;
    }
    const double tr = block_sum(re, sh);
    const double ti = block_sum(im, sh);
    if (threadIdx.x == 0) {
        T[blockIdx.x] = tr;
        if (Ti) Ti[blockIdx.x] = ti;
    }
}

rgf_status trace_xy_f64(int batch, int b, const double2* X, const double2* Y, double* T, double* Timag,
                        cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_trace_xy_f64<<<batch, 256, 0, st>>>(b, X, Y, T, Timag);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_copy_f64(int b, double2* dst, const double2* src, const int* active) {
    if (active && !active[blockIdx.y]) return;
    const long nn = (long)b * b, off = (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x)
        dst[off + i] = src[off + i];
}

rgf_status copy_f64(int batch, int b, double2* dst, const double2* src, const int* active,
                    cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_copy_f64<<<dim3(grid_for((long)b * b, 256, 64), batch), 256, 0, st>>>(b, dst, src, active);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_axpy_f64(int b, double alpha, const double2* X, double2* Y) {
    const long nn = (long)b * b, off = (long)blockIdx.y * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const double2 x = X[off + i];
        double2 y = Y[off + i];
        y.x += alpha * x.x;
        y.y += alpha * x.y;
        Y[off + i] = y;
    }
}

rgf_status axpy_f64(int batch, int b, double alpha, const double2* X, double2* Y, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_axpy_f64<<<dim3(grid_for((long)b * b, 256, 64), batch), 256, 0, st>>>(b, alpha, X, Y);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_merge_dec_flags(int W, const int* dec_flags, const int* dec_active, int* flags) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= W) return;
    int f = flags[e] | dec_flags[e] | dec_flags[W + e];
    if (dec_active[e]) f |= RGF_FLAG_NOCONV_L;
    if (dec_active[W + e]) f |= RGF_FLAG_NOCONV_R;
    flags[e] = f;
}

rgf_status merge_dec_flags(int W, const int* dec_flags, const int* dec_active, int* flags,
                           cudaStream_t st) {
    if (W <= 0) return RGF_OK;
    k_merge_dec_flags<<<ceil_div(W, 128), 128, 0, st>>>(W, dec_flags, dec_active, flags);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

// ------------------------------------------------------------- Newton refinement
__global__ void k_newton_mask(int n, const int* mask, const int* dec_active, int* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ((mask ? mask[i] : 1) && !dec_active[i]) ? 1 : 0;
}

rgf_status newton_mask(int n, const int* mask, const int* dec_active, int* out, cudaStream_t st) {
    if (n <= 0) return RGF_OK;
    k_newton_mask<<<ceil_div(n, 128), 128, 0, st>>>(n, mask, dec_active, out);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_stein_check_f64(int b, const double2* A, const double2* B, double tol, double growth,
                                  int first, double* p0, int* status, int* active, int* remaining) {
    const int bi = blockIdx.x;
    if (!active[bi]) return;
    __shared__ double sh[32];
    const long nn = (long)b * b, off = (long)bi * nn;
    double sa = 0.0, sb = 0.0;
    for (long i = threadIdx.x; i < nn; i += blockDim.x) {
        sa += cabs2(A[off + i]);
        sb += cabs2(B[off + i]);
    }
    const double ta = block_sum(sa, sh);
    const double tb = block_sum(sb, sh);
    if (threadIdx.x == 0) {
        const double p = sqrt(ta) * sqrt(tb);
        if (first) p0[bi] = p;
        if (p <= tol) {
            status[bi] = 1;
            active[bi] = 0;
        } else if (!isfinite(p) || p > growth * p0[bi]) {
            status[bi] = 2;
            active[bi] = 0;
        } else {
            atomicAdd(remaining, 1);
        }
    }
}

rgf_status stein_check_f64(int batch, int b, const double2* A, const double2* B, double tol, double growth,
                           int first, double* p0, int* status, int* active, int* remaining, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_stein_check_f64<<<batch, 256, 0, st>>>(b, A, B, tol, growth, first, p0, status, active, remaining);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_newton_finish_f64(int b, const double2* X, double2* g, const int* mask, const int* status,
                                    double again, int* next, int* flags, int* remaining) {
    const int bi = blockIdx.x;
    if (!mask[bi]) {
        if (threadIdx.x == 0) next[bi] = 0;
        return;
    }
    __shared__ double sh[32];
    const long nn = (long)b * b, off = (long)bi * nn;
    const bool ok = status[bi] == 1;
    double sx = 0.0, sg = 0.0;
    for (long i = threadIdx.x; i < nn; i += blockDim.x) {
        double2 v = g[off + i];
        if (ok) {
            const double2 x = X[off + i];
            v.x += x.x;
            v.y += x.y;
            g[off + i] = v;
            sx += cabs2(x);
        }
        sg += cabs2(v);
    }
    const double tx = block_sum(sx, sh);
    const double tg = block_sum(sg, sh);
    if (threadIdx.x == 0) {
        const int more = ok && sqrt(tx) > again * sqrt(tg);
        next[bi] = more;
        if (more) atomicAdd(remaining, 1);
        if (!ok) atomicOr(&flags[bi], RGF_FLAG_LEAD_NEWTON);
    }
}

rgf_status newton_finish_f64(int batch, int b, const double2* X, double2* g, const int* mask, const int* status,
                             double again, int* next, int* flags, int* remaining, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_newton_finish_f64<<<batch, 256, 0, st>>>(b, X, g, mask, status, again, next, flags, remaining);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_sub_f64(int b, const double2* A, const double2* B, double2* C, const int* active) {
    const int bi = blockIdx.y;
    if (active && !active[bi]) return;
    const long nn = (long)b * b, off = (long)bi * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x)
        C[off + i] = csub(A[off + i], B[off + i]);
}

rgf_status sub_f64(int batch, int b, const double2* A, const double2* B, double2* C, const int* active,
                   cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    dim3 g(ceil_div((long)b * b, 256) < 16 ? ceil_div((long)b * b, 256) : 16, batch);
    k_sub_f64<<<g, 256, 0, st>>>(b, A, B, C, active);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_axpy_masked_f64(int b, double alpha, const double2* X, double2* Y, const int* active) {
    const int bi = blockIdx.y;
    if (active && !active[bi]) return;
    const long nn = (long)b * b, off = (long)bi * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const double2 x = X[off + i];
        double2 y = Y[off + i];
        y.x = fma(alpha, x.x, y.x);
        y.y = fma(alpha, x.y, y.y);
        Y[off + i] = y;
    }
}

rgf_status axpy_masked_f64(int batch, int b, double alpha, const double2* X, double2* Y, const int* active,
                           cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    dim3 g(ceil_div((long)b * b, 256) < 16 ? ceil_div((long)b * b, 256) : 16, batch);
    k_axpy_masked_f64<<<g, 256, 0, st>>>(b, alpha, X, Y, active);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

__global__ void k_add_identity_f64(int b, double s, double2* A, const int* active) {
    const int bi = blockIdx.x;
    if (active && !active[bi]) return;
    for (int r = threadIdx.x; r < b; r += blockDim.x) A[(long)bi * b * b + (long)r * b + r].x += s;
}

rgf_status add_identity_f64(int batch, int b, double s, double2* A, const int* active, cudaStream_t st) {
    if (batch <= 0) return RGF_OK;
    k_add_identity_f64<<<batch, 128, 0, st>>>(b, s, A, active);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

}  // namespace rgf
