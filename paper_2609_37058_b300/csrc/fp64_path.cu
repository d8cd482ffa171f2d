// The plain FP64 RGF path: Sancho-Rubio decimation of both leads, lead
// self-energies and broadenings, the left-to-right block sweep and the
// Caroli trace, every step in IEEE binary64 on the CUDA cores.  Energies
// of one wave are the batch dimension of every kernel.
#include <utility>

#include "kernels.h"
#include "plan.h"

namespace rgf {

namespace {
constexpr int kPoolMats = 22;  // in units of W matrices

struct Pool {
    double2* base;
    long nn;
    int W;
    double2* at(int unit) const { return base + (long)unit * W * nn; }
};

inline ZGemm gemm_sq(int batch, int b, double2 alpha, const double2* A, const double2* B,
                     double2* C, const int* active) {
    ZGemm g{};
    g.batch = batch;
    g.m = g.n = g.k = b;
    g.alpha = alpha;
    g.beta = make_double2(0.0, 0.0);
    g.A = A;
    g.lda = b;
    g.sA = (long)b * b;
    g.B = B;
    g.ldb = b;
    g.sB = (long)b * b;
    g.C = C;
    g.ldc = b;
    g.sC = (long)b * b;
    g.active = active;
    g.skip0 = g.skip1 = 0;
    return g;
}
}  // namespace

// Sancho-Rubio decimation of both leads in FP64 for batch entries s*W + e
// (s = 0 left, 1 right) whose mask entry is nonzero (mask may be null: all).
// pool must hold kDecMats*2W matrices, inv_ws inv_f64_workspace_bytes(2W, b).
// On return *g_out points at the 2W surface Green's functions inside pool
// (entries outside the mask untouched), p->d_dec_flags gathers SINGULAR bits
// and dec_active[i] != 0 marks entries that hit dec_max_iter.
rgf_status fp64_decimate(rgf_plan_s* p, int W, const int* mask, double2* pool_base, void* inv_ws,
                         int* dec_active, double2** g_out) {
    cudaStream_t st = p->stream;
    const int b = p->b;
    const long nn = (long)b * b;
    const double eta = p->opt.eta;
    const double2 one = make_double2(1.0, 0.0), mone = make_double2(-1.0, 0.0);
    Pool pool{pool_base, nn, W};
    const double* E = p->d_E;
    double2 *eps_s = pool.at(0), *eps = pool.at(2), *alpha = pool.at(4), *beta = pool.at(6);
    double2 *g = pool.at(8), *ga = pool.at(10), *gb = pool.at(12);
    double2 *t1 = pool.at(14), *t2 = pool.at(16), *t3 = pool.at(18), *t4 = pool.at(20);
    const int W2 = 2 * W;
    double2** L = p->lead[0];
    double2** R = p->lead[1];
    {
        FormSrc a{{L[1], R[1]}, {L[0], R[0]}, {0, 0}};
        RGF_TRY(form_f64(W, 2, b, E, eta, a, eps, nullptr, 0.0, mask, st));
        RGF_TRY(copy_f64(W2, b, eps_s, eps, mask, st));
        // Outward coupling: left lead M_{j,j-1} (lower), right lead M_{j,j+1} (upper).
        FormSrc al{{L[3], R[3]}, {L[2], R[2]}, {0, 1}};
        FormSrc be{{L[3], R[3]}, {L[2], R[2]}, {1, 0}};
        RGF_TRY(form_f64(W, 2, b, E, eta, al, alpha, nullptr, 0.0, mask, st));
        RGF_TRY(form_f64(W, 2, b, E, eta, be, beta, nullptr, 0.0, mask, st));
        RGF_TRY(fro_norm_f64(W2, b, eps, p->d_anorm, st));
    }
    int* act = dec_active;
    if (mask) {
        RGF_CUDA_TRY(cudaMemcpyAsync(act, mask, sizeof(int) * W2, cudaMemcpyDeviceToDevice, st));
    } else {
        std::vector<int> ones(W2, 1);
        RGF_CUDA_TRY(cudaMemcpyAsync(act, ones.data(), sizeof(int) * W2, cudaMemcpyHostToDevice, st));
    }
    RGF_CUDA_TRY(cudaMemsetAsync(p->d_iters, 0, sizeof(int) * W2, st));
    for (int it = 1; it <= p->opt.dec_max_iter; ++it) {
        RGF_TRY(copy_f64(W2, b, g, eps, act, st));
        RGF_TRY(inv_f64(W2, b, g, nn, inv_ws, p->d_dec_flags, act, st));
        RGF_TRY(zgemm_f64(gemm_sq(W2, b, one, g, alpha, ga, act), st));
        RGF_TRY(zgemm_f64(gemm_sq(W2, b, one, g, beta, gb, act), st));
        RGF_TRY(zgemm_f64(gemm_sq(W2, b, one, alpha, gb, t1, act), st));   // alpha g beta
        RGF_TRY(zgemm_f64(gemm_sq(W2, b, one, beta, ga, t2, act), st));    // beta g alpha
        RGF_TRY(zgemm_f64(gemm_sq(W2, b, mone, alpha, ga, t3, act), st));  // -alpha g alpha
        RGF_TRY(zgemm_f64(gemm_sq(W2, b, mone, beta, gb, t4, act), st));   // -beta g beta
        RGF_TRY(dec_update_f64(W2, b, eps_s, eps, t1, t2, act, st));
        std::swap(alpha, t3);
        std::swap(beta, t4);
        RGF_CUDA_TRY(cudaMemsetAsync(p->d_remaining, 0, sizeof(int), st));
        RGF_TRY(dec_check_f64(W2, b, alpha, beta, p->d_anorm, p->opt.dec_tol, it, act, p->d_iters,
                              p->d_remaining, st));
        RGF_CUDA_TRY(cudaMemcpyAsync(p->h_remaining, p->d_remaining, sizeof(int), cudaMemcpyDeviceToHost, st));
        RGF_CUDA_TRY(cudaStreamSynchronize(st));
        if (*p->h_remaining == 0) break;
    }
    // g_s = eps_s^-1
    RGF_TRY(copy_f64(W2, b, g, eps_s, mask, st));
    RGF_TRY(inv_f64(W2, b, g, nn, inv_ws, nullptr, mask, st));

    // Newton steps on the fixed-point equation g = (a - alpha g beta)^-1 for
    // the converged entries: the decimation's recursion loses digits at some
    // energies (relative errors up to ~1e-5 in FP64 with residuals up to
    // ~1e-2); Newton takes g to the FP64 rounding level.  With
    // r = (a - alpha g beta) g - I the correction X solves the Stein equation
    // X = -g r + (g alpha) X (beta g), summed by doubling until
    // |A|_F |B|_F <= dec_tol^2.  A doubling that grows instead (above 1e4
    // times its first value: a g outside Newton's basin, near band edges at
    // small eta) drops the step: g keeps its decimation value and the energy
    // is flagged RGF_FLAG_LEAD_NEWTON.  Another step (up to three) follows for
    // the entries whose correction exceeded 1e-10 |g|_F: what a correction c
    // leaves is of order K c^2 (K up to ~1e6 near band edges), below the FP64
    // bar's need for c <= 1e-10.  a, alpha and beta are formed again (the
    // decimation overwrote them).
    {
        double2 *a0 = pool.at(0), *al0 = pool.at(2), *be0 = pool.at(4), *Wm = pool.at(6), *r = pool.at(10);
        double2 *A = pool.at(12), *B = pool.at(14), *X = pool.at(16), *u1 = pool.at(18), *u2 = pool.at(20);
        int* nm = p->d_nmask;
        int* nx = p->d_nnext;
        int* sm = p->d_smask;
        RGF_TRY(newton_mask(W2, mask, act, nm, st));
        FormSrc a{{L[1], R[1]}, {L[0], R[0]}, {0, 0}};
        FormSrc al{{L[3], R[3]}, {L[2], R[2]}, {0, 1}};
        FormSrc be{{L[3], R[3]}, {L[2], R[2]}, {1, 0}};
        RGF_TRY(form_f64(W, 2, b, E, eta, a, a0, nullptr, 0.0, nm, st));
        RGF_TRY(form_f64(W, 2, b, E, eta, al, al0, nullptr, 0.0, nm, st));
        RGF_TRY(form_f64(W, 2, b, E, eta, be, be0, nullptr, 0.0, nm, st));
        const double stol = p->opt.dec_tol * p->opt.dec_tol;
        for (int step = 0; step < 3; ++step) {
            RGF_TRY(zgemm_f64(gemm_sq(W2, b, one, al0, g, u1, nm), st));   // alpha g
            RGF_TRY(zgemm_f64(gemm_sq(W2, b, one, u1, be0, u2, nm), st));  // alpha g beta
            RGF_TRY(sub_f64(W2, b, a0, u2, Wm, nm, st));
            RGF_TRY(zgemm_f64(gemm_sq(W2, b, one, Wm, g, r, nm), st));
            RGF_TRY(add_identity_f64(W2, b, -1.0, r, nm, st));              // r
            RGF_TRY(zgemm_f64(gemm_sq(W2, b, mone, g, r, X, nm), st));      // X = -g r
            RGF_TRY(zgemm_f64(gemm_sq(W2, b, one, g, al0, A, nm), st));
            RGF_TRY(zgemm_f64(gemm_sq(W2, b, one, be0, g, B, nm), st));
            RGF_CUDA_TRY(cudaMemcpyAsync(sm, nm, sizeof(int) * W2, cudaMemcpyDeviceToDevice, st));
            RGF_CUDA_TRY(cudaMemsetAsync(p->d_status, 0, sizeof(int) * W2, st));
            for (int k = 0; k < p->opt.dec_max_iter; ++k) {
                RGF_TRY(zgemm_f64(gemm_sq(W2, b, one, A, X, u1, sm), st));  // A X
                ZGemm acc = gemm_sq(W2, b, one, u1, B, X, sm);             // X + A X B
                acc.beta = one;
                acc.Cin = X;
                acc.ldcin = b;
                acc.sCin = nn;
                RGF_TRY(zgemm_f64(acc, st));
                RGF_TRY(zgemm_f64(gemm_sq(W2, b, one, A, A, u2, sm), st));
                std::swap(A, u2);
                RGF_TRY(zgemm_f64(gemm_sq(W2, b, one, B, B, u2, sm), st));
                std::swap(B, u2);
                RGF_CUDA_TRY(cudaMemsetAsync(p->d_remaining, 0, sizeof(int), st));
                RGF_TRY(stein_check_f64(W2, b, A, B, stol, 1e4, k == 0, p->d_p0, p->d_status, sm, p->d_remaining,
                                        st));
                RGF_CUDA_TRY(cudaMemcpyAsync(p->h_remaining, p->d_remaining, sizeof(int), cudaMemcpyDeviceToHost, st));
                RGF_CUDA_TRY(cudaStreamSynchronize(st));
                if (*p->h_remaining == 0) break;
            }
            RGF_CUDA_TRY(cudaMemsetAsync(p->d_remaining, 0, sizeof(int), st));
            RGF_TRY(newton_finish_f64(W2, b, X, g, nm, p->d_status, 1e-10, nx, p->d_dec_flags, p->d_remaining, st));
            RGF_CUDA_TRY(cudaMemcpyAsync(p->h_remaining, p->d_remaining, sizeof(int), cudaMemcpyDeviceToHost, st));
            RGF_CUDA_TRY(cudaStreamSynchronize(st));
            if (*p->h_remaining == 0) break;
            std::swap(nm, nx);
        }
    }
    *g_out = g;
    return RGF_OK;
}

size_t fp64_workspace_bytes(int W, int b) {
    const size_t nn = (size_t)b * b;
    return (size_t)kPoolMats * W * nn * sizeof(double2) + inv_f64_workspace_bytes(2 * W, b) + 1024;
}

rgf_status fp64_wave(rgf_plan_s* p, int W) {
    NvtxRange wave_range("rgf fp64 wave");
    cudaStream_t st = p->stream;
    const int b = p->b, N = p->N;
    const long nn = (long)b * b;
    const double eta = p->opt.eta;
    const double2 one = make_double2(1.0, 0.0), mone = make_double2(-1.0, 0.0);
    Pool pool{(double2*)p->ws, nn, W};
    void* inv_ws = (void*)((char*)p->ws + (size_t)kPoolMats * W * nn * sizeof(double2));
    const double* E = p->d_E;

    RGF_CUDA_TRY(cudaMemsetAsync(p->d_flags, 0, sizeof(int) * W, st));
    RGF_CUDA_TRY(cudaMemsetAsync(p->d_dec_flags, 0, sizeof(int) * 2 * W, st));
    RGF_CUDA_TRY(cudaMemsetAsync(p->d_err, 0, sizeof(double) * W, st));

    // ---------------------------------------------------------- decimation
    double2* g = nullptr;
    RGF_TRY(fp64_decimate(p, W, nullptr, pool.at(0), inv_ws, p->d_active, &g));
    RGF_TRY(merge_dec_flags(W, p->d_dec_flags, p->d_active, p->d_flags, st));
    const int W2 = 2 * W;
    double2 *t1 = pool.at(14), *t2 = pool.at(16), *t3 = pool.at(18);
    double2** L = p->lead[0];
    double2** R = p->lead[1];

    // ---------------------------------------------------------- self-energies
    // Sigma_L = Lc_L g_L Uc_L, Sigma_R = Uc_R g_R Lc_R with Lc = z Sc - Hc
    // (lower) and Uc its upper partner; Gamma = i (Sigma - Sigma^dagger).
    double2* sigma = pool.at(0);  // [L: W][R: W]
    double2* gamma = pool.at(2);
    {
        FormSrc x1{{L[5], R[5]}, {L[4], R[4]}, {0, 1}};
        FormSrc x2{{L[5], R[5]}, {L[4], R[4]}, {1, 0}};
        RGF_TRY(form_f64(W, 2, b, E, eta, x1, t1, nullptr, 0.0, nullptr, st));
        RGF_TRY(form_f64(W, 2, b, E, eta, x2, t2, nullptr, 0.0, nullptr, st));
        RGF_TRY(zgemm_f64(gemm_sq(W2, b, one, t1, g, t3, nullptr), st));
        RGF_TRY(zgemm_f64(gemm_sq(W2, b, one, t3, t2, sigma, nullptr), st));
        RGF_TRY(gamma_f64(W2, b, sigma, gamma, st));
    }
    double2* sigL = sigma;
    double2* sigR = sigma + (long)W * nn;
    double2* gamL = gamma;
    double2* gamR = gamma + (long)W * nn;

    // ---------------------------------------------------------- sweep
    double2 *gi = pool.at(4), *P = pool.at(5), *M = pool.at(6), *Lt = pool.at(7), *Ut = pool.at(8);
    double2 *Q = pool.at(9), *Qn = pool.at(10), *G = pool.at(11), *X = pool.at(12), *Y = pool.at(13);
    if (N == 1) {
        FormSrc a0{{p->S_diag, nullptr}, {p->H_diag, nullptr}, {0, 0}};
        RGF_TRY(form_f64(W, 1, b, E, eta, a0, gi, sigL, 1.0, nullptr, st));
        RGF_TRY(axpy_f64(W, b, -1.0, sigR, gi, st));
        RGF_TRY(inv_f64(W, b, gi, nn, inv_ws, p->d_flags, nullptr, st));
        std::swap(G, gi);
    } else {
        FormSrc a0{{p->S_diag, nullptr}, {p->H_diag, nullptr}, {0, 0}};
        RGF_TRY(form_f64(W, 1, b, E, eta, a0, gi, sigL, 1.0, nullptr, st));
        RGF_TRY(inv_f64(W, b, gi, nn, inv_ws, p->d_flags, nullptr, st));
        for (int i = 1; i < N; ++i) {
            const double2* Sl = p->S_lower + (long)(i - 1) * nn;
            const double2* Hl = p->H_lower + (long)(i - 1) * nn;
            FormSrc up{{Sl, nullptr}, {Hl, nullptr}, {1, 0}};
            FormSrc lo{{Sl, nullptr}, {Hl, nullptr}, {0, 0}};
            FormSrc ai{{p->S_diag + (long)i * nn, nullptr}, {p->H_diag + (long)i * nn, nullptr}, {0, 0}};
            RGF_TRY(form_f64(W, 1, b, E, eta, up, Ut, nullptr, 0.0, nullptr, st));
            RGF_TRY(form_f64(W, 1, b, E, eta, lo, Lt, nullptr, 0.0, nullptr, st));
            RGF_TRY(form_f64(W, 1, b, E, eta, ai, M, (i == N - 1) ? sigR : nullptr, 1.0, nullptr, st));
            RGF_TRY(zgemm_f64(gemm_sq(W, b, mone, gi, Ut, P, nullptr), st));  // P = -g tau'
            ZGemm gm = gemm_sq(W, b, one, Lt, P, M, nullptr);                 // M += tau P
            gm.beta = one;
            gm.Cin = M;
            gm.ldcin = b;
            gm.sCin = nn;
            RGF_TRY(zgemm_f64(gm, st));
            RGF_TRY(inv_f64(W, b, M, nn, inv_ws, p->d_flags, nullptr, st));
            std::swap(gi, M);
            if (i == 1) {
                std::swap(Q, P);
            } else {
                RGF_TRY(zgemm_f64(gemm_sq(W, b, one, Q, P, Qn, nullptr), st));
                std::swap(Q, Qn);
            }
        }
        RGF_TRY(zgemm_f64(gemm_sq(W, b, one, Q, gi, G, nullptr), st));
    }

    // ---------------------------------------------------------- Caroli trace
    RGF_TRY(zgemm_f64(gemm_sq(W, b, one, gamL, G, X, nullptr), st));
    RGF_TRY(zgemm_f64(gemm_sq(W, b, one, G, gamR, Y, nullptr), st));
    RGF_TRY(trace_xy_f64(W, b, X, Y, p->d_T, p->d_Ti, st));
    return RGF_OK;
}

}  // namespace rgf
