// Non-orthogonal kernel polynomial method for the Fermi level (rgf_kpm.h).
//
// B300 layout of the work: FP64 is the precision (the recursion runs over
// hundreds of moments and the moments are compared with an FP64 oracle),
// and the FP64 pipe is narrow on this part (about two FP64 FMAs per clock
// and SM), so every SM must be busy with FP64 FMAs.  The random vectors are
// independent: one CTA owns one vector and runs the whole Chebyshev
// recursion for it, one layer after the other, with no communication
// between CTAs.  Per layer and step it streams six b x b blocks (H_ii,
// H_{i,i-1}, H_{i,i+1}, F_i in the forward pass; D_i^-1, F_{i+1}^dag in the
// backward pass) from L2/HBM; the CTAs of one launch walk the layers in
// step, so a block read by one CTA is mostly served from L2 to the others.
// A warp reduces each output row: lanes read consecutive entries of the
// row (coalesced), multiply by the vector held in shared memory and
// combine with shuffles.
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/rgf_kpm.h"
#include "common.cuh"
#include "kernels.h"

namespace rgf {
namespace {

constexpr int kKpmThreads = 256;
constexpr int kKpmWarps = kKpmThreads / 32;

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// The conjugate transposes of n b x b blocks.
__global__ void k_ctrans(long n_blocks, int b, const double2* __restrict__ X, double2* __restrict__ Y) {
    const long nn = (long)b * b;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n_blocks * nn; e += (long)gridDim.x * blockDim.x) {
        const long blk = e / nn, rc = e % nn;
        const int r = (int)(rc / b), c = (int)(rc % b);
        Y[blk * nn + (long)c * b + r] = cconj(X[e]);
    }
}

struct KpmArgs {
    int N, b, n_rand, n_mom;
    double alpha, beta;
    const double2* Hd;    // N blocks H_ii
    const double2* Hl;    // N-1 blocks H_{i,i-1} (index i-1)
    const double2* Hu;    // N-1 blocks H_{i-1,i} (index i-1)
    const double2* F;     // N-1 blocks F_i = S_{i,i-1} D_{i-1}^-1 (index i-1)
    const double2* G;     // N-1 blocks F_i^dag (index i-1)
    const double2* Dinv;  // N blocks D_i^-1
    const double2* R;     // n_rand random vectors, vector-major
    double2* work;        // n_rand x 3 vectors of N b
    double* mu_part;      // [n_mom][n_rand]
};

// One block row of y = sum_t X_t u_t over up to four (block, vector) terms
// with signs, for the b rows of a layer: warp w takes rows w, w + 8, ...
template <int NT>
__device__ __forceinline__ void block_rows(int b, const double2* const (&X)[NT], const double2* const (&u)[NT],
                                           const double (&sgn)[NT], double2* y_smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < b; r += kKpmWarps) {
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            if (!X[t]) continue;
            const double2* row = X[t] + (long)r * b;
            double2 s = make_double2(0.0, 0.0);
            for (int k = lane; k < b; k += 32) cfma(s, row[k], u[t][k]);
            acc.x = fma(sgn[t], s.x, acc.x);
            acc.y = fma(sgn[t], s.y, acc.y);
        }
        acc = warp_sum(acc);
        if (lane == 0) y_smem[r] = acc;
    }
}

// The whole Chebyshev recursion of one random vector per CTA.  With POWER
// the same passes run a power iteration instead: v <- S^-1 H v / |S^-1 H v|
// (alpha = 1, beta = 0), mu_part[n] receiving |S^-1 H v_{n-1}| for the
// normalized v_{n-1} (one CTA).
// Shared memory: vectors vm (v_{i-1}), v0 (v_i), vp (v_{i+1}), wprev (w_{i-1}
// or x_{i+1}), y (the layer's result), 5 b entries.
template <bool POWER>
__global__ void __launch_bounds__(kKpmThreads) k_kpm_chebyshev(KpmArgs a) {
    extern __shared__ double2 sm[];
    const int b = a.b, N = a.N;
    const long Nb = (long)N * b;
    double2* vm = sm;
    double2* v0 = sm + b;
    double2* vp = sm + 2 * b;
    double2* wprev = sm + 3 * b;
    double2* y = sm + 4 * b;
    __shared__ double red[kKpmWarps];
    const double2* r = a.R + (long)blockIdx.x * Nb;
    double2* P = a.work + (long)blockIdx.x * 3 * Nb;  // the older vector (v_{n-2}), overwritten by v_n
    double2* Q = P + Nb;                               // the latest vector (v_{n-1})
    double2* W = Q + Nb;                               // forward-substitution results w
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;

    auto block_reduce = [&](double v) -> double {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp] = v;
        __syncthreads();
        double s = 0.0;
        if (tid == 0)
            for (int w = 0; w < kKpmWarps; ++w) s += red[w];
        __syncthreads();
        return s;
    };

    // v_0 = r: Q <- r, mu_0 (POWER: Q <- r / |r|).
    double d0 = 0.0;
    for (long e = tid; e < Nb; e += kKpmThreads) {
        const double2 x = r[e];
        Q[e] = x;
        d0 += x.x * x.x + x.y * x.y;
    }
    d0 = block_reduce(d0);
    __shared__ double bcast;
    if (tid == 0) {
        a.mu_part[blockIdx.x] = POWER ? sqrt(d0) : d0;
        bcast = d0;
    }
    __syncthreads();
    if (POWER) {
        const double sc = 1.0 / sqrt(bcast);
        for (long e = tid; e < Nb; e += kKpmThreads) Q[e] = make_double2(Q[e].x * sc, Q[e].y * sc);
        __syncthreads();
    }

    const double ia = 1.0 / a.alpha;
    for (int n = 1; n < a.n_mom; ++n) {
        // Forward pass: t_i = H_ii v_i + H_{i,i-1} v_{i-1} + H_{i,i+1} v_{i+1},
        // w_i = t_i - F_i w_{i-1}.
        for (int k = tid; k < b; k += kKpmThreads) {
            vm[k] = make_double2(0.0, 0.0);
            v0[k] = Q[k];
            vp[k] = N > 1 ? Q[b + k] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        for (int i = 0; i < N; ++i) {
            const long bb = (long)b * b;
            const double2* X[4] = {a.Hd + i * bb, i > 0 ? a.Hl + (i - 1) * bb : nullptr,
                                   i < N - 1 ? a.Hu + i * bb : nullptr, i > 0 ? a.F + (i - 1) * bb : nullptr};
            const double2* u[4] = {v0, vm, vp, wprev};
            const double s[4] = {1.0, 1.0, 1.0, -1.0};
            block_rows<4>(b, X, u, s, y);
            __syncthreads();
            // w_i to memory and into wprev; shift the v window.
            for (int k = tid; k < b; k += kKpmThreads) {
                W[(long)i * b + k] = y[k];
                wprev[k] = y[k];
                vm[k] = v0[k];
                v0[k] = vp[k];
                vp[k] = (i + 2 < N) ? Q[(long)(i + 2) * b + k] : make_double2(0.0, 0.0);
            }
            __syncthreads();
        }
        // Backward pass: x_i = D_i^-1 w_i - F_{i+1}^dag x_{i+1}; then
        // v_n = 2 (x - beta v_{n-1}) / alpha - v_{n-2} (v_1 = (x - beta v_0) / alpha)
        // into P, and the moment sum r^dag v_n.
        double dot = 0.0;
        for (int i = N - 1; i >= 0; --i) {
            const long bb = (long)b * b;
            for (int k = tid; k < b; k += kKpmThreads) v0[k] = W[(long)i * b + k];
            __syncthreads();
            const double2* X[2] = {a.Dinv + i * bb, i < N - 1 ? a.G + i * bb : nullptr};
            const double2* u[2] = {v0, wprev};
            const double s[2] = {1.0, -1.0};
            block_rows<2>(b, X, u, s, y);
            __syncthreads();
            for (int k = tid; k < b; k += kKpmThreads) {
                const long e = (long)i * b + k;
                const double2 x = y[k];
                wprev[k] = x;  // x_i for the next (lower) layer
                if (POWER) {
                    P[e] = x;
                    dot += x.x * x.x + x.y * x.y;
                    continue;
                }
                const double2 q = Q[e];
                double2 vn = make_double2((x.x - a.beta * q.x) * ia, (x.y - a.beta * q.y) * ia);
                if (n > 1) {
                    const double2 p = P[e];
                    vn = make_double2(2.0 * vn.x - p.x, 2.0 * vn.y - p.y);
                }
                P[e] = vn;
                const double2 rr = r[e];
                dot += rr.x * vn.x + rr.y * vn.y;  // Re(conj(r) v_n)
            }
            __syncthreads();
        }
        dot = block_reduce(dot);
        if (tid == 0) {
            a.mu_part[(long)n * a.n_rand + blockIdx.x] = POWER ? sqrt(dot) : dot;
            bcast = dot;
        }
        __syncthreads();
        if (POWER) {
            const double sc = 1.0 / sqrt(bcast);
            for (long e = tid; e < Nb; e += kKpmThreads) P[e] = make_double2(P[e].x * sc, P[e].y * sc);
            __syncthreads();
        }
        double2* t = P;
        P = Q;
        Q = t;
        __syncthreads();
    }
}

// mu[n] = (1/R) sum_c mu_part[n][c], in a fixed order (deterministic).
__global__ void k_kpm_reduce(int n_mom, int n_rand, const double* __restrict__ part, double* __restrict__ mu) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_mom) return;
    double s = 0.0;
    for (int c = 0; c < n_rand; ++c) s += part[(long)n * n_rand + c];
    mu[n] = s / n_rand;
}

// Bisection for E_F: each iteration evaluates spin * N(x_mid) with the
// Jackson-damped closed form, threads sharing the moment sum.
__global__ void k_kpm_fermi(int n_mom, const double* __restrict__ mu, double alpha, double beta, double n_el,
                            double spin, double* E_F) {
    __shared__ double part[256];
    __shared__ double lohi[2];
    const int tid = threadIdx.x;
    const double M = (double)n_mom;
    const double q = M_PI / (M + 1.0);
    const double cotq = cos(q) / sin(q);
    if (tid == 0) {
        lohi[0] = -1.0;
        lohi[1] = 1.0;
    }
    __syncthreads();
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lohi[0] + lohi[1]);
        const double theta = acos(fmin(fmax(mid, -1.0), 1.0));
        double s = 0.0;
        for (int n = 1 + tid; n < n_mom; n += blockDim.x) {
            const double g = ((M - n + 1.0) * cos(q * n) + sin(q * n) * cotq) / (M + 1.0);
            s += g * mu[n] * sin(n * theta) / n;
        }
        part[tid] = s;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (tid < o) part[tid] += part[tid + o];
            __syncthreads();
        }
        if (tid == 0) {
            // g_0 = 1
            const double states = mu[0] * (M_PI - theta) / M_PI - (2.0 / M_PI) * part[0];
            if (spin * states < n_el)
                lohi[0] = mid;
            else
                lohi[1] = mid;
        }
        __syncthreads();
    }
    if (tid == 0) *E_F = beta + alpha * 0.5 * (lohi[0] + lohi[1]);
}

}  // namespace
}  // namespace rgf

struct rgf_kpm_s {
    int N = 0, b = 0, device = 0;
    cudaStream_t st = nullptr;
    double2* buf = nullptr;  // Hd, Hl, Hu, Sd, Sl, Su, F, G, Dinv
    double2 *Hd, *Hl, *Hu, *Sd, *Sl, *Su, *F, *G, *Dinv;
};

extern "C" {

rgf_status rgf_kpm_create(rgf_kpm_t* out, int N, int b, const double* H_diag, const double* S_diag,
                          const double* H_lower, const double* S_lower, int mem, void* cuda_stream) {
    if (!out || N < 1 || b < 1 || b > 512 || !H_diag || !S_diag || (N > 1 && (!H_lower || !S_lower)) ||
        (mem != RGF_MEM_HOST && mem != RGF_MEM_DEVICE)) {
        rgf::set_error("rgf_kpm_create: invalid arguments");
        return RGF_E_INVALID;
    }
    *out = nullptr;
    auto* k = new rgf_kpm_s();
    struct Guard {
        rgf_kpm_s*& k;
        bool keep = false;
        ~Guard() {
            if (!keep) {
                cudaFree(k->buf);
                delete k;
            }
        }
    } guard{k};
    k->N = N;
    k->b = b;
    k->st = (cudaStream_t)cuda_stream;
    RGF_CUDA_TRY(cudaGetDevice(&k->device));
    const long bb = (long)b * b;
    const long L = N > 1 ? N - 1 : 1;
    const size_t n_el = (size_t)bb * (3 * (size_t)N + 6 * (size_t)L);
    RGF_CUDA_TRY(cudaMalloc(&k->buf, n_el * sizeof(double2)));
    double2* p = k->buf;
    k->Hd = p; p += bb * N;
    k->Sd = p; p += bb * N;
    k->Dinv = p; p += bb * N;
    k->Hl = p; p += bb * L;
    k->Hu = p; p += bb * L;
    k->Sl = p; p += bb * L;
    k->Su = p; p += bb * L;
    k->F = p; p += bb * L;
    k->G = p;
    const cudaMemcpyKind kind = mem == RGF_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaStream_t st = k->st;
    RGF_CUDA_TRY(cudaMemcpyAsync(k->Hd, H_diag, sizeof(double2) * bb * N, kind, st));
    RGF_CUDA_TRY(cudaMemcpyAsync(k->Sd, S_diag, sizeof(double2) * bb * N, kind, st));
    if (N > 1) {
        RGF_CUDA_TRY(cudaMemcpyAsync(k->Hl, H_lower, sizeof(double2) * bb * (N - 1), kind, st));
        RGF_CUDA_TRY(cudaMemcpyAsync(k->Sl, S_lower, sizeof(double2) * bb * (N - 1), kind, st));
        const int g = (int)std::min<long>((bb * (N - 1) + 255) / 256, 148L * 16);
        rgf::k_ctrans<<<g, 256, 0, st>>>(N - 1, b, (const double2*)k->Hl, k->Hu);
        RGF_LAUNCH_CHECK();
        rgf::k_ctrans<<<g, 256, 0, st>>>(N - 1, b, (const double2*)k->Sl, k->Su);
        RGF_LAUNCH_CHECK();
    }
    // Block LDL of S: D_0 = S_00; F_i = S_{i,i-1} D_{i-1}^-1; D_i = S_ii - F_i S_{i-1,i}.
    // Dinv holds D_i, inverted in place once F_{i+1} no longer needs it... the
    // recursion needs D_{i-1}^-1 only, so each D_i is inverted as soon as formed.
    void* ws = nullptr;
    RGF_CUDA_TRY(cudaMalloc(&ws, rgf::inv_f64_workspace_bytes(1, b) + sizeof(int)));
    struct WsFree {
        void* p;
        ~WsFree() { cudaFree(p); }
    } wsf{ws};
    int* d_flag = (int*)((char*)ws + rgf::inv_f64_workspace_bytes(1, b));
    RGF_CUDA_TRY(cudaMemsetAsync(d_flag, 0, sizeof(int), st));
    RGF_CUDA_TRY(cudaMemcpyAsync(k->Dinv, k->Sd, sizeof(double2) * bb, cudaMemcpyDeviceToDevice, st));
    RGF_TRY(rgf::inv_f64(1, b, k->Dinv, bb, ws, d_flag, nullptr, st));
    for (int i = 1; i < N; ++i) {
        rgf::ZGemm g{};
        g.batch = 1;
        g.m = g.n = g.k = b;
        g.alpha = make_double2(1.0, 0.0);
        g.beta = make_double2(0.0, 0.0);
        g.A = k->Sl + (i - 1) * bb;
        g.lda = b;
        g.B = k->Dinv + (i - 1) * bb;
        g.ldb = b;
        g.C = k->F + (i - 1) * bb;
        g.ldc = b;
        g.skip0 = g.skip1 = 0;
        RGF_TRY(rgf::zgemm_f64(g, st));  // F_i
        g.alpha = make_double2(-1.0, 0.0);
        g.beta = make_double2(1.0, 0.0);
        g.A = k->F + (i - 1) * bb;
        g.B = k->Su + (i - 1) * bb;
        g.Cin = k->Sd + i * bb;
        g.ldcin = b;
        g.C = k->Dinv + i * bb;
        RGF_TRY(rgf::zgemm_f64(g, st));  // D_i
        RGF_TRY(rgf::inv_f64(1, b, k->Dinv + i * bb, bb, ws, d_flag, nullptr, st));
    }
    if (N > 1) {
        const int g = (int)std::min<long>((bb * (N - 1) + 255) / 256, 148L * 16);
        rgf::k_ctrans<<<g, 256, 0, st>>>(N - 1, b, (const double2*)k->F, k->G);
        RGF_LAUNCH_CHECK();
    }
    int h_flag = 0;
    RGF_CUDA_TRY(cudaMemcpyAsync(&h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    RGF_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_flag) {
        rgf::set_error("rgf_kpm_create: the overlap's block factorization met an exactly zero pivot");
        return RGF_E_INVALID;
    }
    guard.keep = true;
    *out = k;
    return RGF_OK;
}

rgf_status rgf_kpm_scale(rgf_kpm_t k, const double* x0, int iters, double margin, double* alpha, double* beta) {
    if (!k || !x0 || iters < 1 || iters > 100000 || !(margin >= 0.0) || !alpha || !beta) {
        rgf::set_error("rgf_kpm_scale: invalid arguments");
        return RGF_E_INVALID;
    }
    const long Nb = (long)k->N * k->b;
    double2* work = nullptr;
    RGF_CUDA_TRY(cudaMalloc(&work, sizeof(double2) * 3 * Nb + sizeof(double) * (iters + 1)));
    struct Free {
        void* p;
        ~Free() { cudaFree(p); }
    } f{work};
    double* rho = (double*)(work + 3 * Nb);
    rgf::KpmArgs a{k->N, k->b, 1, iters + 1, 1.0, 0.0, k->Hd, k->Hl, k->Hu, k->F, k->G, k->Dinv,
                   (const double2*)x0, work, rho};
    rgf::k_kpm_chebyshev<true><<<1, rgf::kKpmThreads, sizeof(double2) * 5 * k->b, k->st>>>(a);
    RGF_LAUNCH_CHECK();
    double h = 0.0;
    RGF_CUDA_TRY(cudaMemcpyAsync(&h, rho + iters, sizeof(double), cudaMemcpyDeviceToHost, k->st));
    RGF_CUDA_TRY(cudaStreamSynchronize(k->st));
    if (!(h > 0.0) || !std::isfinite(h)) {
        rgf::set_error("rgf_kpm_scale: power iteration gave %g", h);
        return RGF_E_INVALID;
    }
    *alpha = (1.0 + margin) * h;
    *beta = 0.0;
    return RGF_OK;
}

rgf_status rgf_kpm_moments(rgf_kpm_t k, double alpha, double beta, int n_rand, const double* R, int n_mom,
                           double* mu) {
    if (!k || !(alpha > 0.0) || n_rand < 1 || !R || n_mom < 2 || n_mom > (1 << 20) || !mu) {
        rgf::set_error("rgf_kpm_moments: invalid arguments");
        return RGF_E_INVALID;
    }
    const long Nb = (long)k->N * k->b;
    double2* work = nullptr;
    double* part = nullptr;
    RGF_CUDA_TRY(cudaMalloc(&work, sizeof(double2) * 3 * Nb * n_rand));
    struct Free {
        void* p;
        ~Free() { cudaFree(p); }
    } f1{work};
    RGF_CUDA_TRY(cudaMalloc(&part, sizeof(double) * (size_t)n_mom * n_rand));
    Free f2{part};
    rgf::KpmArgs a{k->N, k->b, n_rand, n_mom, alpha, beta, k->Hd, k->Hl, k->Hu, k->F, k->G, k->Dinv,
                   (const double2*)R, work, part};
    const size_t smem = sizeof(double2) * 5 * k->b;
    rgf::k_kpm_chebyshev<false><<<n_rand, rgf::kKpmThreads, smem, k->st>>>(a);
    RGF_LAUNCH_CHECK();
    rgf::k_kpm_reduce<<<(n_mom + 127) / 128, 128, 0, k->st>>>(n_mom, n_rand, part, mu);
    RGF_LAUNCH_CHECK();
    // |T_n(x)| <= 1 on [-1, 1]: moments far above mu_0 mean that alpha, beta
    // do not map the spectrum into [-1, 1] (the recursion then grows
    // exponentially).
    std::vector<double> h(n_mom);
    RGF_CUDA_TRY(cudaMemcpyAsync(h.data(), mu, sizeof(double) * n_mom, cudaMemcpyDeviceToHost, k->st));
    RGF_CUDA_TRY(cudaStreamSynchronize(k->st));
    for (int n = 1; n < n_mom; ++n)
        if (!std::isfinite(h[n]) || std::fabs(h[n]) > 10.0 * std::fabs(h[0])) {
            rgf::set_error("rgf_kpm_moments: moment %d is %g against mu_0 = %g: the spectrum is not inside "
                           "[beta - alpha, beta + alpha]",
                           n, h[n], h[0]);
            return RGF_E_INVALID;
        }
    return RGF_OK;
}

rgf_status rgf_kpm_fermi(int n_mom, const double* mu, double alpha, double beta, double n_electrons, double spin,
                         double* E_F, void* cuda_stream) {
    if (n_mom < 1 || !mu || !E_F || !(alpha > 0.0) || !(spin > 0.0)) {
        rgf::set_error("rgf_kpm_fermi: invalid arguments");
        return RGF_E_INVALID;
    }
    rgf::k_kpm_fermi<<<1, 256, 0, (cudaStream_t)cuda_stream>>>(n_mom, mu, alpha, beta, n_electrons, spin, E_F);
    RGF_LAUNCH_CHECK();
    return RGF_OK;
}

rgf_status rgf_kpm_destroy(rgf_kpm_t k) {
    if (!k) return RGF_OK;
    cudaStreamSynchronize(k->st);
    cudaFree(k->buf);
    delete k;
    return RGF_OK;
}

}  // extern "C"
