// Table-driven kernels of the multi-device engine (see engine.h).
#include "df.cuh"
#include "engine.h"

namespace rgf {

namespace {

inline int chunks(long n, int threads, int cap) {
    long g = (n + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

__device__ __forceinline__ float4 df_zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

__global__ void k_pad_to_dfc(int b, int bc, const double2* __restrict__ src, float4* __restrict__ dst,
                             double diag_fill) {
    const long nb = (long)bc * bc;
    const double2* s = src + (long)blockIdx.y * b * b;
    float4* d = dst + (long)blockIdx.y * nb;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / bc), c = (int)(i % bc);
        float4 v;
        if (r < b && c < b) {
            const double2 x = s[(long)r * b + c];
            v = cdf(df_from_double(x.x), df_from_double(x.y));
        } else if (r == c) {
            v = cdf(df_from_double(diag_fill), make_float2(0.f, 0.f));
        } else {
            v = df_zero();
        }
        d[i] = v;
    }
}

__global__ void k_pad_f64(int b, int bc, const double2* __restrict__ src, double2* __restrict__ dst,
                          double diag_fill) {
    const long nb = (long)bc * bc;
    const double2* s = src + (long)blockIdx.y * b * b;
    double2* d = dst + (long)blockIdx.y * nb;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / bc), c = (int)(i % bc);
        double2 v = make_double2(0.0, 0.0);
        if (r < b && c < b)
            v = s[(long)r * b + c];
        else if (r == c)
            v.x = diag_fill;
        d[i] = v;
    }
}

__global__ void k_refill(int S, int bc, const SlotTab* __restrict__ tab, const int* __restrict__ refill,
                         const float4* __restrict__ ready, float4* __restrict__ store, const double* dec_err,
                         const int* dec_flags, double* slot_err, int* slot_flags) {
    const int s = blockIdx.y;
    if (!refill[s]) return;
    const int r = tab[s].ready, D = tab[s].ready_D;
    if (!RGF_DCHECK(r >= 0 && r < D, RGF_DBG_SLOT)) return;
    const long nn = (long)bc * bc;
    for (int k = 0; k < 4; ++k) {
        const float4* src = ready + ((long)k * D + r) * nn;
        float4* dst = store + ((long)k * S + s) * nn;
        for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x)
            dst[i] = src[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        slot_err[s] = dec_err[r];
        slot_flags[s] = dec_flags[r];
    }
}

// (zr + i zi)(S') - H' in df, S' = S or S^dagger.
__device__ __forceinline__ float4 zs_minus_h(float2 zr, float2 zi, float4 sv, float4 hv) {
    const float2 sr = re_of(sv), sim = im_of(sv);
    const float2 re = df_sub(df_sub(df_mul(zr, sr), df_mul(zi, sim)), re_of(hv));
    const float2 im = df_sub(df_add(df_mul(zr, sim), df_mul(zi, sr)), im_of(hv));
    return cdf(re, im);
}

__device__ __forceinline__ float4 dagger_elem(const float4* A, int bc, int r, int c) {
    float4 v = A[(long)c * bc + r];
    v.z = -v.z;
    v.w = -v.w;
    return v;
}

__global__ void k_form_step(int S, int bc, const SlotTab* __restrict__ tab, SlotMasks mk,
                            const float4* __restrict__ sigL, const float4* __restrict__ sigR, float4* __restrict__ M,
                            float4* __restrict__ Ut, float4* __restrict__ Lt) {
    const int s = blockIdx.y;
    if (!mk.act[s]) return;
    const SlotTab t = tab[s];
    const int nf = mk.nf ? mk.nf[s] : 0, fi = mk.first[s], la = mk.last[s];
    if (!RGF_DCHECK(t.Sii && t.Hii && (!nf || (t.Sl && t.Hl)), RGF_DBG_POINTER)) return;
    const float2 zr = df_from_double(t.E), zi = df_from_double(t.eta);
    const long nn = (long)bc * bc, off = (long)s * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / bc), c = (int)(i % bc);
        float4 m = zs_minus_h(zr, zi, t.Sii[i], t.Hii[i]);
        if (fi) m = cdf_sub(m, sigL[off + i]);
        if (la) m = cdf_sub(m, sigR[off + i]);
        M[off + i] = m;
        if (nf) {
            Lt[off + i] = zs_minus_h(zr, zi, t.Sl[i], t.Hl[i]);
            Ut[off + i] = zs_minus_h(zr, zi, dagger_elem(t.Sl, bc, r, c), dagger_elem(t.Hl, bc, r, c));
        }
    }
}

__global__ void k_identity_masked(int bc, float4* A, const int* mask) {
    const int s = blockIdx.y;
    if (!mask[s]) return;
    const long nn = (long)bc * bc;
    float4* a = A + (long)s * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / bc), c = (int)(i % bc);
        a[i] = make_float4(r == c ? 1.f : 0.f, 0.f, 0.f, 0.f);
    }
}

__device__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void k_trace_masked(int bc, const float4* X, const float4* Y, const int* mask, double* T) {
    __shared__ double sh[32];
    const int s = blockIdx.x;
    if (!mask[s]) return;
    const long nn = (long)bc * bc, off = (long)s * nn;
    double re = 0.0;
    for (long i = threadIdx.x; i < nn; i += blockDim.x) {
        const float4 x4 = X[off + i], y4 = Y[off + i];
        const double xr = df_to_double(re_of(x4)), xi = df_to_double(im_of(x4));
        const double yr = df_to_double(re_of(y4)), yi = df_to_double(im_of(y4));
        re += xr * yr + xi * yi;
    }
    const double tr = block_sum(re, sh);
    if (threadIdx.x == 0) T[s] = tr;
}

__global__ void k_finish(int S, const SlotTab* __restrict__ tab, const int* last, const double* slot_T,
                         const double* slot_err, const int* slot_flags) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S || !last[s]) return;
    const SlotTab t = tab[s];
    if (!RGF_DCHECK(t.outT && t.outErr && t.outFlags, RGF_DBG_POINTER)) return;
    *t.outT = slot_T[s];
    *t.outErr = slot_err[s];
    *t.outFlags = slot_flags[s];
}

// Entry be = side * D + j; lead block k of side s at lead + (6 s + k) nn.
__global__ void k_form_dec(int D, int bc, const DecTab* __restrict__ tab, double2* eps_s, double2* eps,
                           double2* alpha, double2* beta) {
    const int be = blockIdx.y;
    const int side = be / D, j = be % D;
    const DecTab t = tab[j];
    const long nn = (long)bc * bc;
    const double2* L = t.lead + (long)6 * side * nn;
    const double2 z = make_double2(t.E, t.eta);
    const long off = (long)be * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / bc), c = (int)(i % bc);
        const long ti = (long)c * bc + r;
        const double2 a = csub(cmul(z, L[nn + i]), L[i]);
        eps_s[off + i] = a;
        eps[off + i] = a;
        // M_{j,j+1} of a lead cell pair is the conjugate transpose of the lower block.
        const double2 lo = csub(cmul(z, L[3 * nn + i]), L[2 * nn + i]);
        const double2 up = csub(cmul(z, cconj(L[3 * nn + ti])), cconj(L[2 * nn + ti]));
        // Left lead: outward coupling M_{j,j-1} (lower); right lead: M_{j,j+1} (upper).
        alpha[off + i] = side == 0 ? lo : up;
        beta[off + i] = side == 0 ? up : lo;
    }
}

__global__ void k_form_coupling(int D, int bc, const DecTab* __restrict__ tab, double2* x1, double2* x2) {
    const int be = blockIdx.y;
    const int side = be / D, j = be % D;
    const DecTab t = tab[j];
    const long nn = (long)bc * bc;
    const double2* L = t.lead + (long)6 * side * nn;
    const double2 z = make_double2(t.E, t.eta);
    const long off = (long)be * nn;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / bc), c = (int)(i % bc);
        const long ti = (long)c * bc + r;
        const double2 lo = csub(cmul(z, L[5 * nn + i]), L[4 * nn + i]);
        const double2 up = csub(cmul(z, cconj(L[5 * nn + ti])), cconj(L[4 * nn + ti]));
        x1[off + i] = side == 0 ? lo : up;
        x2[off + i] = side == 0 ? up : lo;
    }
}

}  // namespace

rgf_status pad_to_dfc(int nblk, int b, int bc, const double2* src, float4* dst, double diag_fill, cudaStream_t st) {
    if (nblk <= 0) return RGF_OK;
    k_pad_to_dfc<<<dim3(chunks((long)bc * bc, 256, 64), nblk), 256, 0, st>>>(b, bc, src, dst, diag_fill);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

rgf_status pad_f64(int nblk, int b, int bc, const double2* src, double2* dst, double diag_fill, cudaStream_t st) {
    if (nblk <= 0) return RGF_OK;
    k_pad_f64<<<dim3(chunks((long)bc * bc, 256, 64), nblk), 256, 0, st>>>(b, bc, src, dst, diag_fill);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

rgf_status engine_refill(int S, int bc, const SlotTab* tab, const int* refill, const float4* ready,
                         float4* store, const double* dec_err, const int* dec_flags, double* slot_err,
                         int* slot_flags, cudaStream_t st) {
    k_refill<<<dim3(chunks((long)bc * bc, 256, 32), S), 256, 0, st>>>(S, bc, tab, refill, ready, store, dec_err,
                                                                      dec_flags, slot_err, slot_flags);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

rgf_status engine_form_step(int S, int bc, const SlotTab* tab, SlotMasks mk, const float4* sigL, const float4* sigR,
                            float4* M, float4* Ut, float4* Lt, cudaStream_t st) {
    k_form_step<<<dim3(chunks((long)bc * bc, 256, 64), S), 256, 0, st>>>(S, bc, tab, mk, sigL, sigR, M, Ut, Lt);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

rgf_status set_identity_masked_dfc(int S, int bc, float4* A, const int* mask, cudaStream_t st) {
    k_identity_masked<<<dim3(chunks((long)bc * bc, 256, 64), S), 256, 0, st>>>(bc, A, mask);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

rgf_status trace_masked_dfc(int S, int bc, const float4* X, const float4* Y, const int* mask, double* T,
                            cudaStream_t st) {
    k_trace_masked<<<S, 256, 0, st>>>(bc, X, Y, mask, T);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

rgf_status engine_finish(int S, const SlotTab* tab, const int* last, const double* slot_T, const double* slot_err,
                         const int* slot_flags, cudaStream_t st) {
    k_finish<<<ceil_div(S, 128), 128, 0, st>>>(S, tab, last, slot_T, slot_err, slot_flags);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

rgf_status engine_form_dec(int D, int bc, const DecTab* tab, double2* eps_s, double2* eps, double2* alpha,
                           double2* beta, cudaStream_t st) {
    k_form_dec<<<dim3(chunks((long)bc * bc, 256, 64), 2 * D), 256, 0, st>>>(D, bc, tab, eps_s, eps, alpha, beta);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

rgf_status engine_form_coupling(int D, int bc, const DecTab* tab, double2* x1, double2* x2, cudaStream_t st) {
    k_form_coupling<<<dim3(chunks((long)bc * bc, 256, 64), 2 * D), 256, 0, st>>>(D, bc, tab, x1, x2);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

}  // namespace rgf
