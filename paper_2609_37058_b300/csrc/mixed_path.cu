// Mixed-precision RGF path.  Every complex GEMM is an exact BF16 slice
// product on the tensor cores with a double-float (about 48-bit) result;
// every inverse is an FP32 Gauss-Jordan seed refined by Newton-Schulz steps
// X <- X + X (I - M X) whose residual and correction are again slice
// products.  Matrices between kernels are double-float complex (float4).
// The final Caroli trace is reduced in FP64.
#include <algorithm>
#include <cstdlib>
#include <utility>
#include <vector>

#include "gj_tmpl.cuh"
#include "mixed_ops.h"
#include "plan.h"

namespace rgf {

namespace {

size_t sa_bytes(int cnt, int b, int Kp, int nsl = kSlices) {
    return (size_t)cnt * nsl * b * Kp * sizeof(__nv_bfloat16);
}
size_t sb_bytes(int cnt, int b, int Kp, int nsl = kSlices) {
    return (size_t)cnt * nsl * 2 * b * Kp * sizeof(__nv_bfloat16);
}
}  // namespace

// Slice A by rows into sa[ia], B by columns into sb[ib] (the first `planes` slices).
rgf_status sliceA(const Ctx& c, int cnt, int ia, const float4* A, const int* act, int planes) {
    return slice_rows(cnt, c.b, c.b, A, c.nn, c.m->sa[ia], c.m->Kp, act, c.st, planes);
}
rgf_status sliceB(const Ctx& c, int cnt, int ib, const float4* B, const int* act, int planes) {
    return slice_cols(cnt, c.b, c.b, B, c.nn, c.m->sb[ib], c.m->Kp, act, c.st, planes);
}

// Slices that mm4 reads: four on the tcgen05 core, all six on the reference core.
static int mm4_planes(const Ctx& c) { return c.m->core == 1 ? kSlices : 4; }
// C = alpha * A B (+ D) (+ I) from already sliced operands.
rgf_status mm(const Ctx& c, int cnt, int ia, int ib, float alpha, const float4* D, int addI, float4* C,
              const int* act, float2* C2, float* rsq, double2* rtr) {
    OzGemm g{};
    g.batch = cnt;
    g.m = g.n = g.k = c.b;
    g.As = c.m->sa[ia];
    g.Bs = c.m->sb[ib];
    g.Kp = c.m->Kp;
    g.alpha = alpha;
    g.D = D;
    g.sD = c.nn;
    g.add_identity = addI;
    g.C = C;
    g.sC = c.nn;
    g.C2 = C2;
    g.rsq = rsq;
    g.rtr = rtr;
    g.active = act;
    g.status = c.m->status;
    g.bn = c.m->bn;
    return oz_gemm(g, c.m->core, c.st);
}

// C = A B + D with four of the six slices of each operand (corrections).
rgf_status mm4(const Ctx& c, int cnt, int ia, int ib, const float4* D, float4* C, const int* act) {
    OzGemm g{};
    g.batch = cnt;
    g.m = g.n = g.k = c.b;
    g.As = c.m->sa[ia];
    g.Bs = c.m->sb[ib];
    g.Kp = c.m->Kp;
    g.alpha = 1.0f;
    g.D = D;
    g.sD = c.nn;
    g.C = C;
    g.sC = c.nn;
    g.active = act;
    g.status = c.m->status;
    g.bn = c.m->bn;
    g.nsl = mm4_planes(c) == kSlices ? 0 : mm4_planes(c);
    return oz_gemm(g, c.m->core, c.st);
}

// Seven-slice (FP64-class) counterparts for FP64 matrices.
rgf_status hsliceA(const Ctx& c, int cnt, int ia, const double2* A, const int* act) {
    return slice_rows_f64(cnt, c.b, c.b, A, c.nn, c.m->hsa[ia], c.m->Kp, act, c.st);
}
rgf_status hsliceB(const Ctx& c, int cnt, int ib, const double2* B, const int* act) {
    return slice_cols_f64(cnt, c.b, c.b, B, c.nn, c.m->hsb[ib], c.m->Kp, act, c.st);
}
rgf_status hmm(const Ctx& c, int cnt, int ia, int ib, float alpha, const double2* D, int addI, double2* C,
               const int* act, int nsl) {
    OzGemmHP g{};
    g.nsl = nsl;
    g.batch = cnt;
    g.m = g.n = g.k = c.b;
    g.As = c.m->hsa[ia];
    g.Bs = c.m->hsb[ib];
    g.Kp = c.m->Kp;
    g.alpha = alpha;
    g.D = D;
    g.sD = c.nn;
    g.add_identity = addI;
    g.C = C;
    g.sC = c.nn;
    g.active = act;
    g.status = c.m->status;
    return oz_gemm_hp(g, c.st);
}

// X = M^-1 for cnt FP64 matrices: FP32 Gauss-Jordan seed, then Newton-Schulz
// steps with seven-slice products (FP64-class), FP64 Gauss-Jordan reseed of
// seeds that do not contract.  Uses hsa[1] for M, hsa[0]/hsb[0] for the steps.
rgf_status inv_hp(const Ctx& c, int cnt, int W, const double2* M, double2* X, double2* R, const int* act,
                  int* gj_flags, const double2* X_prev) {
    MixedState* m = c.m;
    RGF_TRY(c128_to_c64(cnt, c.b, M, m->c64, act, c.st));
    RGF_TRY(inv_c32_to(cnt, c.b, m->c64, c.nn, m->inv_ws, nullptr, act, m->status, c.st, 0, nullptr, X));
    if (c.ns_steps == 0) return RGF_OK;
    // Seeds up to kHpBad are refined rather than replaced: allow the steps
    // they need (entries stop as soon as they converge).
    const int steps = c.ns_steps > kHpSteps ? c.ns_steps : kHpSteps;
    int* cur = m->nsact[0];
    int* nxt = m->nsact[1];
    RGF_TRY(mask_init(cnt, act, cur, c.st));
    RGF_TRY(hsliceA(c, cnt, 1, M, act));
    for (int s = 0; s < steps; ++s) {
        RGF_TRY(hsliceB(c, cnt, 0, X, cur));
        RGF_TRY(hmm(c, cnt, 1, 0, -1.0f, nullptr, 1, R, cur));  // R = I - M X
        if (s == 0) RGF_CUDA_TRY(cudaMemsetAsync(m->bad_count, 0, sizeof(int), c.st));
        RGF_CUDA_TRY(cudaMemsetAsync(m->more_count, 0, sizeof(int), c.st));
        RGF_TRY(ns_check_f64(cnt, W, c.b, R, c.err, c.flags, s, steps, cur, nxt, m->bad, m->bad_count, c.st,
                             m->more_count));
        RGF_CUDA_TRY(cudaMemcpyAsync(m->h_more, m->more_count, sizeof(int), cudaMemcpyDeviceToHost, c.st));
        if (s > 0) RGF_CUDA_TRY(cudaStreamSynchronize(c.st));
        if (s == 0) {
            RGF_CUDA_TRY(cudaMemcpyAsync(m->h_bad, m->bad_count, sizeof(int), cudaMemcpyDeviceToHost, c.st));
            RGF_CUDA_TRY(cudaStreamSynchronize(c.st));
            int n_bad = *m->h_bad;
            int* need64 = m->bad;
            if (n_bad > 0 && X_prev) {
                // The nearby matrix's inverse as the seed of these entries.
                RGF_TRY(copy_f64(cnt, c.b, X, X_prev, m->bad, c.st));
                RGF_TRY(hsliceB(c, cnt, 0, X, m->bad));
                RGF_TRY(hmm(c, cnt, 1, 0, -1.0f, nullptr, 1, R, m->bad));
                RGF_CUDA_TRY(cudaMemsetAsync(m->bad_count, 0, sizeof(int), c.st));
                RGF_TRY(recheck_f64(cnt, c.b, R, m->bad, m->bad2, m->bad_count, nxt, c.st));
                RGF_CUDA_TRY(cudaMemcpyAsync(m->h_bad, m->bad_count, sizeof(int), cudaMemcpyDeviceToHost, c.st));
                RGF_CUDA_TRY(cudaStreamSynchronize(c.st));
                n_bad = *m->h_bad;
                need64 = m->bad2;
            }
            if (n_bad > 0) {
                if (c.n_reseeds) *c.n_reseeds += n_bad;
                RGF_TRY(copy_f64(cnt, c.b, m->c128, M, need64, c.st));
                RGF_TRY(inv_t<double2>(cnt, c.b, m->c128, c.nn, m->inv64_ws, gj_flags, need64, c.st));
                RGF_TRY(copy_f64(cnt, c.b, X, m->c128, need64, c.st));
                RGF_TRY(hsliceB(c, cnt, 0, X, need64));
                RGF_TRY(hmm(c, cnt, 1, 0, -1.0f, nullptr, 1, R, need64));
            }
        }
        RGF_TRY(hsliceA(c, cnt, 0, X, cur));
        RGF_TRY(hsliceB(c, cnt, 0, R, cur));
        // X += X R: a correction (the next residual is formed from all seven
        // slices and removes its error; the last one is below 3e-7 relative),
        // so five slices of each operand suffice.
        RGF_TRY(hmm(c, cnt, 0, 0, 1.0f, X, 0, X, cur, 5));
        std::swap(cur, nxt);
        // A zero count: every entry is done (reseeded entries always continue).
        if (*m->h_more == 0) break;
    }
    return RGF_OK;
}

// Sancho-Rubio decimation of the 2W lead entries formed in units 0, 2, 4, 6
// of the decimation pool, with FP64 storage and seven-slice products, then
// one Newton step on the fixed-point equation for the converged entries
// (see hp_newton_step).
// The doubling's remainder after round k is A^(2^k) X B^(2^k), at most
// |A^(2^k)|_F |B^(2^k)|_F |X|_F: stopping at a product of 1e-4 leaves X
// accurate to 1e-4 relative.  X is a correction (a second step, taken while
// |X|_F > 1e-8 |g|_F, solves again from the corrected g), so g keeps at most
// 1e-12 relative from the truncation.
constexpr double kSteinTol = 1e-4;

rgf_status hp_newton_step(const Ctx& c, int W, double stol, int max_iter, const double2* a0, const double2* al0,
                          const double2* be0, double2* g);

rgf_status hp_decimate_run(const Ctx& c, int W, double tol, int max_iter, double2** g_out) {
    MixedState* m = c.m;
    cudaStream_t st = c.st;
    const int b = c.b, W2 = 2 * W;
    auto U = [&](int unit) { return dec_unit(m, W, unit); };
    double2 *eps_s = U(0), *eps = U(2), *alpha = U(4), *beta = U(6), *g = U(8), *ga = U(10), *gb = U(12);
    double2 *t1 = U(14), *t2 = U(16), *t3 = U(18), *t4 = U(20), *R = U(22), *g_prev = U(24);
    // The lead's own a, alpha, beta for the Newton step (the decimation overwrites them).
    RGF_TRY(copy_f64(W2, b, U(26), eps_s, nullptr, st));
    RGF_TRY(copy_f64(W2, b, U(28), alpha, nullptr, st));
    RGF_TRY(copy_f64(W2, b, U(30), beta, nullptr, st));
    RGF_TRY(fro_norm_f64(W2, b, eps, m->dec_anorm, st));
    std::vector<int> ones(W2, 1);
    RGF_CUDA_TRY(cudaMemcpyAsync(m->dec_active, ones.data(), sizeof(int) * W2, cudaMemcpyHostToDevice, st));
    RGF_CUDA_TRY(cudaMemsetAsync(m->dec_iters, 0, sizeof(int) * W2, st));
    RGF_CUDA_TRY(cudaMemsetAsync(m->dec_flags, 0, sizeof(int) * W2, st));
    int* act = m->dec_active;
    for (int it = 1; it <= max_iter; ++it) {
        // From the second iteration on, entries whose FP32 seed does not
        // contract start from the previous iteration's inverse (eps changes by
        // alpha g beta + beta g alpha, which shrinks as the decimation
        // converges) before resorting to an FP64 Gauss-Jordan inverse.
        RGF_TRY(inv_hp(c, W2, W, eps, g, R, act, m->dec_flags, it > 1 ? g_prev : nullptr));
        RGF_TRY(copy_f64(W2, b, g_prev, g, act, st));
        RGF_TRY(hsliceA(c, W2, 0, g, act));
        RGF_TRY(hsliceB(c, W2, 0, alpha, act));
        RGF_TRY(hmm(c, W2, 0, 0, 1.0f, nullptr, 0, ga, act));  // g alpha
        RGF_TRY(hsliceB(c, W2, 1, beta, act));
        RGF_TRY(hmm(c, W2, 0, 1, 1.0f, nullptr, 0, gb, act));  // g beta
        RGF_TRY(hsliceB(c, W2, 0, gb, act));
        RGF_TRY(hsliceB(c, W2, 1, ga, act));
        RGF_TRY(hsliceA(c, W2, 0, alpha, act));
        RGF_TRY(hmm(c, W2, 0, 0, 1.0f, nullptr, 0, t1, act));   // alpha g beta
        RGF_TRY(hmm(c, W2, 0, 1, -1.0f, nullptr, 0, t3, act));  // -alpha g alpha
        RGF_TRY(hsliceA(c, W2, 0, beta, act));
        RGF_TRY(hmm(c, W2, 0, 1, 1.0f, nullptr, 0, t2, act));   // beta g alpha
        RGF_TRY(hmm(c, W2, 0, 0, -1.0f, nullptr, 0, t4, act));  // -beta g beta
        RGF_TRY(dec_update_f64(W2, b, eps_s, eps, t1, t2, act, st));
        std::swap(alpha, t3);
        std::swap(beta, t4);
        RGF_CUDA_TRY(cudaMemsetAsync(m->dec_remaining, 0, sizeof(int), st));
        RGF_TRY(dec_check_f64(W2, b, alpha, beta, m->dec_anorm, tol, it, act, m->dec_iters, m->dec_remaining, st));
        RGF_CUDA_TRY(cudaMemcpyAsync(m->h_remaining, m->dec_remaining, sizeof(int), cudaMemcpyDeviceToHost, st));
        RGF_CUDA_TRY(cudaStreamSynchronize(st));
        if (*m->h_remaining == 0) break;
    }
    RGF_TRY(merge_dec_flags(W, m->dec_flags, m->dec_active, c.flags, st));
    RGF_TRY(inv_hp(c, W2, W, eps_s, g, R, nullptr, m->dec_flags));
    RGF_TRY(merge_dec_flags(W, m->dec_flags, m->dec_active, c.flags, st));
    RGF_TRY(hp_newton_step(c, W, kSteinTol, max_iter, U(26), U(28), U(30), g));
    RGF_TRY(merge_dec_flags(W, m->dec_flags, m->dec_active, c.flags, st));
    *g_out = g;
    return RGF_OK;
}

// Newton steps on g = (a - alpha g beta)^-1 for the entries whose
// decimation converged: Sancho-Rubio's recursion loses digits at some
// energies (FP64-class results off by up to ~1e-5 relative, with fixed-point
// residuals up to ~1e-2).  r = (a - alpha g beta) g - I from seven-slice
// products (FP64-class, it is a small difference); the correction X solves
// X = -g r + (g alpha) X (beta g), summed by doubling (X += A X B, A = A A,
// B = B B) until |A|_F |B|_F <= stol, with five-slice products (X is a
// correction); g += X.  A doubling that grows instead (above 1e4 times its
// first value) drops the step: g keeps its decimation value and the entry is
// flagged RGF_FLAG_LEAD_NEWTON.  A second step follows for the entries whose
// correction exceeded 1e-8 |g|_F (what a correction c leaves is of order
// K c^2 with K up to ~1e6, far below the mixed path's 1e-6 bar in T; the FP64
// path, held to 1e-9, takes up to three steps at 1e-10).  Uses
// decimation-pool units 0..7, 10..17.
rgf_status hp_newton_step(const Ctx& c, int W, double stol, int max_iter, const double2* a0, const double2* al0,
                          const double2* be0, double2* g) {
    MixedState* m = c.m;
    cudaStream_t st = c.st;
    const int b = c.b, W2 = 2 * W;
    auto U = [&](int unit) { return dec_unit(m, W, unit); };
    double2 *Wm = U(0), *negr = U(2), *A = U(4), *B = U(6), *X = U(10), *u1 = U(12), *u2 = U(14), *u3 = U(16);
    int* nm = m->dec_newton;
    int* nx = m->dec_next;
    int* sm = m->dec_smask;
    RGF_TRY(newton_mask(W2, nullptr, m->dec_active, nm, st));
    for (int step = 0; step < 2; ++step) {
        RGF_TRY(hsliceA(c, W2, 0, al0, nm));
        RGF_TRY(hsliceB(c, W2, 0, g, nm));
        RGF_TRY(hmm(c, W2, 0, 0, 1.0f, nullptr, 0, u1, nm));           // alpha g
        RGF_TRY(hsliceA(c, W2, 0, u1, nm));
        RGF_TRY(hsliceB(c, W2, 1, be0, nm));
        RGF_TRY(hmm(c, W2, 0, 1, 1.0f, nullptr, 0, u2, nm));           // alpha g beta
        RGF_TRY(sub_f64(W2, b, a0, u2, Wm, nm, st));                     // a - alpha g beta
        RGF_TRY(hsliceA(c, W2, 0, Wm, nm));
        RGF_TRY(hmm(c, W2, 0, 0, -1.0f, nullptr, 1, negr, nm));        // I - (a - alpha g beta) g = -r
        RGF_TRY(hsliceA(c, W2, 0, g, nm));
        RGF_TRY(hsliceB(c, W2, 0, negr, nm));
        RGF_TRY(hmm(c, W2, 0, 0, 1.0f, nullptr, 0, X, nm, 5));         // X = -g r
        RGF_TRY(hsliceB(c, W2, 1, al0, nm));
        RGF_TRY(hmm(c, W2, 0, 1, 1.0f, nullptr, 0, A, nm, 5));         // A = g alpha
        RGF_TRY(hsliceA(c, W2, 0, be0, nm));
        RGF_TRY(hsliceB(c, W2, 0, g, nm));
        RGF_TRY(hmm(c, W2, 0, 0, 1.0f, nullptr, 0, B, nm, 5));         // B = beta g
        RGF_CUDA_TRY(cudaMemcpyAsync(sm, nm, sizeof(int) * W2, cudaMemcpyDeviceToDevice, st));
        RGF_CUDA_TRY(cudaMemsetAsync(m->dec_status, 0, sizeof(int) * W2, st));
        for (int k = 0; k < max_iter; ++k) {
            RGF_TRY(hsliceA(c, W2, 0, A, sm));
            RGF_TRY(hsliceB(c, W2, 0, X, sm));
            RGF_TRY(hmm(c, W2, 0, 0, 1.0f, nullptr, 0, u1, sm, 5));    // A X
            RGF_TRY(hsliceA(c, W2, 1, u1, sm));
            RGF_TRY(hsliceB(c, W2, 1, B, sm));
            RGF_TRY(hmm(c, W2, 1, 1, 1.0f, X, 0, X, sm, 5));           // X + A X B
            RGF_TRY(hsliceB(c, W2, 0, A, sm));
            RGF_TRY(hmm(c, W2, 0, 0, 1.0f, nullptr, 0, u2, sm, 5));    // A A
            RGF_TRY(hsliceA(c, W2, 1, B, sm));
            RGF_TRY(hmm(c, W2, 1, 1, 1.0f, nullptr, 0, u3, sm, 5));    // B B
            std::swap(A, u2);
            std::swap(B, u3);
            RGF_CUDA_TRY(cudaMemsetAsync(m->dec_remaining, 0, sizeof(int), st));
            RGF_TRY(stein_check_f64(W2, b, A, B, stol, 1e4, k == 0, m->dec_p0, m->dec_status, sm, m->dec_remaining,
                                    st));
            RGF_CUDA_TRY(cudaMemcpyAsync(m->h_remaining, m->dec_remaining, sizeof(int), cudaMemcpyDeviceToHost, st));
            RGF_CUDA_TRY(cudaStreamSynchronize(st));
            if (*m->h_remaining == 0) break;
        }
        RGF_CUDA_TRY(cudaMemsetAsync(m->dec_remaining, 0, sizeof(int), st));
        RGF_TRY(newton_finish_f64(W2, b, X, g, nm, m->dec_status, 1e-8, nx, m->dec_flags, m->dec_remaining, st));
        RGF_CUDA_TRY(cudaMemcpyAsync(m->h_remaining, m->dec_remaining, sizeof(int), cudaMemcpyDeviceToHost, st));
        RGF_CUDA_TRY(cudaStreamSynchronize(st));
        if (*m->h_remaining == 0) break;
        std::swap(nm, nx);
    }
    return RGF_OK;
}

// X = M^-1 for cnt matrices (batch entries i, energy i mod W): an FP32
// Gauss-Jordan seed, then up to ns_steps Newton-Schulz steps X += X (I - M X)
// in place, each entry stopping once its residual predicts convergence.
// A seed whose residual is >= 0.5 gets a Sherman-Morrison-scaled first
// correction (see ns_check); entries still at >= 0.5 after it are reseeded
// with the FP64 Gauss-Jordan inverse.
// Uses sa[1] for M, sa[0]/sb[0] for the steps and R as df scratch.
rgf_status inv_mixed(const Ctx& c, int cnt, int W, const float4* M, float4* X, float4* R, const int* act,
                     int* gj_flags, bool m64_ready) {
    return inv_mixed_steps(c, cnt, W, M, X, R, act, gj_flags, 0, c.ns_steps, m64_ready);
}

rgf_status inv_mixed_steps(const Ctx& c, int cnt, int W, const float4* M, float4* X, float4* R, const int* act,
                           int* gj_flags, int s_begin, int s_end, bool m64_ready) {
    MixedState* m = c.m;
    const int steps = c.ns_steps;
    if (s_end > steps) s_end = steps;
    if (s_begin == 0) {
        if (!m64_ready) RGF_TRY(dfc_hi_to_c64(cnt, c.b, M, m->c64, act, c.st));
        // An FP32 seed with a zero pivot is not reported: its residual is not
        // finite, so it is reseeded in FP64 below, which reports its own pivots.
        RGF_TRY(inv_c32_to(cnt, c.b, m->c64, c.nn, m->inv_ws, nullptr, act, m->status, c.st, m->gj_nb, X, nullptr));
        if (steps == 0) return RGF_OK;
        RGF_TRY(mask_init(cnt, act, m->nsact[0], c.st));
        RGF_TRY(sliceA(c, cnt, 1, M, act));
    }
    // Step s works on the mask nsact[s % 2] and writes nsact[(s + 1) % 2].
    int* cur = m->nsact[s_begin & 1];
    int* nxt = m->nsact[(s_begin + 1) & 1];
    // The tcgen05 residual GEMM also returns |R|_F and tr R per block, so
    // that the check does not read R again (the legacy core does not).
    float* rsq = m->core == 0 ? m->r_sumsq : nullptr;
    for (int s = s_begin; s < s_end; ++s) {
        RGF_TRY(sliceB(c, cnt, 0, X, cur));
        double2* rtr = (rsq && s == 0) ? m->r_trace : nullptr;
        RGF_TRY(mm(c, cnt, 1, 0, -1.0f, nullptr, 1, R, cur, nullptr, rsq, rtr));  // R = I - M X
        if (s == 1) RGF_CUDA_TRY(cudaMemsetAsync(m->bad_count, 0, sizeof(int), c.st));
        // From step 1 on the entries that need a further step are counted.
        // Outside graph capture the count is read back (step 1 synchronises
        // anyway) so that steps nobody needs are not launched; in a graph the
        // caller reads it after the step-1 graph.
        const bool count_more = s >= 1;
        if (count_more) RGF_CUDA_TRY(cudaMemsetAsync(m->more_count, 0, sizeof(int), c.st));
        RGF_TRY(ns_check(cnt, W, c.b, R, c.err, c.flags, s, steps, cur, nxt, m->bad, m->bad_count, m->theta, c.st,
                         count_more ? m->more_count : nullptr, rsq, rtr));
        if (count_more && !c.graph && s >= 2) {
            RGF_CUDA_TRY(cudaMemcpyAsync(m->h_more, m->more_count, sizeof(int), cudaMemcpyDeviceToHost, c.st));
            RGF_CUDA_TRY(cudaStreamSynchronize(c.st));
        }
        if (s == 0) RGF_TRY(scale_theta(cnt, c.b, R, m->theta, cur, c.st));
        if (s == 1 && c.graph) {
            RGF_TRY(accumulate_count(m->reseed_acc, m->bad_count, c.st));
            RGF_TRY(dfc_to_c128(cnt, c.b, M, m->c128, m->bad, c.st));
            RGF_TRY(inv_t<double2>(cnt, c.b, m->c128, c.nn, m->inv64_ws, gj_flags, m->bad, c.st));
            RGF_TRY(c128_to_dfc(cnt, c.b, m->c128, X, m->bad, c.st));
            RGF_TRY(sliceB(c, cnt, 0, X, m->bad));
            RGF_TRY(mm(c, cnt, 1, 0, -1.0f, nullptr, 1, R, m->bad));
        } else if (s == 1) {
            RGF_CUDA_TRY(cudaMemcpyAsync(m->h_bad, m->bad_count, sizeof(int), cudaMemcpyDeviceToHost, c.st));
            RGF_CUDA_TRY(cudaMemcpyAsync(m->h_more, m->more_count, sizeof(int), cudaMemcpyDeviceToHost, c.st));
            RGF_CUDA_TRY(cudaStreamSynchronize(c.st));
            if (*m->h_bad > 0) {
                if (c.n_reseeds) *c.n_reseeds += *m->h_bad;
                RGF_TRY(dfc_to_c128(cnt, c.b, M, m->c128, m->bad, c.st));
                RGF_TRY(inv_t<double2>(cnt, c.b, m->c128, c.nn, m->inv64_ws, gj_flags, m->bad, c.st));
                RGF_TRY(c128_to_dfc(cnt, c.b, m->c128, X, m->bad, c.st));
                RGF_TRY(sliceB(c, cnt, 0, X, m->bad));
                RGF_TRY(mm(c, cnt, 1, 0, -1.0f, nullptr, 1, R, m->bad));
            }
        }
        // Operands of the correction are sliced only as far as mm4 reads them.
        RGF_TRY(sliceA(c, cnt, 0, X, cur, mm4_planes(c)));
        RGF_TRY(sliceB(c, cnt, 0, R, cur, mm4_planes(c)));
        RGF_TRY(mm4(c, cnt, 0, 0, X, X, cur));  // X += X R (a correction: four slices suffice)
        std::swap(cur, nxt);
        // Entries reseeded in FP64 at step 1 always continue (their check saw
        // the old seed), so a zero count means every entry is done.
        if (count_more && !c.graph && *m->h_more == 0) break;
    }
    return RGF_OK;
}

size_t mixed_workspace_bytes(int W, int b, int slice_entries, int inv_entries) {
    const int Kp = slice_pitch(b);
    const size_t nn = (size_t)b * b;
    size_t s = (size_t)kPoolUnits * W * nn * sizeof(float4);
    s += 2 * sa_bytes(slice_entries, b, Kp) + 2 * sb_bytes(slice_entries, b, Kp);
    s += (size_t)inv_entries * nn * sizeof(float2) + inv_c32_workspace_bytes(inv_entries, b);
    s += (size_t)inv_entries * nn * sizeof(double2) + inv_workspace_bytes_t<double2>(inv_entries, b);
    s += (size_t)inv_entries * 4 * sizeof(int) +
         (size_t)inv_entries * sizeof(double2) + 8192;
    s += (size_t)inv_entries * rstat_slots(b) * (sizeof(float) + sizeof(double2)) + 512;
    return s;
}

size_t mixed_workspace_bytes(int W, int b) { return mixed_workspace_bytes(W, b, 2 * W, 2 * W); }

size_t mixed_dec_bytes(int Wd, int b) {
    const int Kp = slice_pitch(b);
    return (size_t)kDecUnits * Wd * b * b * sizeof(double2) + 2 * sa_bytes(2 * Wd, b, Kp, kSlicesHP) +
           2 * sb_bytes(2 * Wd, b, Kp, kSlicesHP) + (size_t)2 * Wd * (7 * sizeof(int) + 2 * sizeof(double)) + 4096;
}

rgf_status mixed_state_init(MixedState* m, int b, int W, void* ws, cudaStream_t st, int Wd, int slice_entries) {
    if (Wd <= 0 || Wd > W) Wd = W;
    if (slice_entries <= 0) slice_entries = 2 * W;
    const int inv_entries = std::max(W, 2 * Wd);
    m->b = b;
    m->W = W;
    m->Wd = Wd;
    m->slice_entries = slice_entries;
    m->inv_entries = inv_entries;
    m->Kp = slice_pitch(b);
    const size_t nn = (size_t)b * b;
    const char* env = getenv("RGF_OZ_CORE");
    m->core = (env && env[0] == '1') ? 1 : 0;
    auto alloc = [&](void** ptr, size_t bytes) -> rgf_status {
        if (cudaMalloc(ptr, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            set_error("mixed workspace: cudaMalloc(%zu) failed", bytes);
            return RGF_E_OOM;
        }
        return RGF_OK;
    };
    if (!ws) {
        RGF_TRY(alloc(&m->own, mixed_workspace_bytes(W, b, slice_entries, inv_entries)));
        ws = m->own;
    }
    // Carve the workspace.
    char* w = (char*)ws;
    m->pool = (float4*)w;
    w += (size_t)kPoolUnits * W * nn * sizeof(float4);
    for (int i = 0; i < 2; ++i) {
        m->sa[i] = (__nv_bfloat16*)w;
        w += sa_bytes(slice_entries, b, m->Kp);
    }
    for (int i = 0; i < 2; ++i) {
        m->sb[i] = (__nv_bfloat16*)w;
        w += sb_bytes(slice_entries, b, m->Kp);
    }
    m->c64 = (float2*)w;
    w += (size_t)inv_entries * nn * sizeof(float2);
    w = (char*)(((uintptr_t)w + 255) & ~(uintptr_t)255);  // the seed's BF16 splits are read by TMA
    m->inv_ws = (void*)w;
    w += inv_c32_workspace_bytes(inv_entries, b);
    w = (char*)(((uintptr_t)w + 255) & ~(uintptr_t)255);
    m->c128 = (double2*)w;
    w += (size_t)inv_entries * nn * sizeof(double2);
    m->inv64_ws = (void*)w;
    w += inv_workspace_bytes_t<double2>(inv_entries, b);
    w = (char*)(((uintptr_t)w + 255) & ~(uintptr_t)255);
    m->nsact[0] = (int*)w;
    w += (size_t)inv_entries * sizeof(int);
    m->nsact[1] = (int*)w;
    w += (size_t)inv_entries * sizeof(int);
    m->bad = (int*)w;
    w += (size_t)inv_entries * sizeof(int);
    m->bad2 = (int*)w;
    w += (size_t)inv_entries * sizeof(int);
    w = (char*)(((uintptr_t)w + 15) & ~(uintptr_t)15);
    m->theta = (double2*)w;
    w += (size_t)inv_entries * sizeof(double2);
    w = (char*)(((uintptr_t)w + 255) & ~(uintptr_t)255);
    m->r_sumsq = (float*)w;
    w += (size_t)inv_entries * rstat_slots(b) * sizeof(float);
    w = (char*)(((uintptr_t)w + 255) & ~(uintptr_t)255);
    m->r_trace = (double2*)w;
    w += (size_t)inv_entries * rstat_slots(b) * sizeof(double2);
    // Zero the slice buffers once: the K padding is never written again.
    RGF_CUDA_TRY(cudaMemsetAsync(m->sa[0], 0,
                                 2 * sa_bytes(slice_entries, b, m->Kp) + 2 * sb_bytes(slice_entries, b, m->Kp), st));
    RGF_TRY(alloc((void**)&m->status, 8 * sizeof(int)));
    m->bad_count = m->status + 1;
    m->reseed_acc = (long long*)(m->status + 2);
    m->more_count = m->status + 4;
    {
        char* d = nullptr;
        RGF_TRY(alloc((void**)&d, mixed_dec_bytes(Wd, b)));
        m->dec_own = d;
        m->dec_pool = (double2*)d;
        d += (size_t)kDecUnits * Wd * nn * sizeof(double2);
        for (int i = 0; i < 2; ++i) {
            m->hsa[i] = (__nv_bfloat16*)d;
            d += sa_bytes(2 * Wd, b, m->Kp, kSlicesHP);
        }
        for (int i = 0; i < 2; ++i) {
            m->hsb[i] = (__nv_bfloat16*)d;
            d += sb_bytes(2 * Wd, b, m->Kp, kSlicesHP);
        }
        m->dec_anorm = (double*)d;
        d += (size_t)2 * Wd * sizeof(double);
        m->dec_active = (int*)d;
        d += (size_t)2 * Wd * sizeof(int);
        m->dec_iters = (int*)d;
        d += (size_t)2 * Wd * sizeof(int);
        m->dec_flags = (int*)d;
        d += (size_t)2 * Wd * sizeof(int);
        m->dec_remaining = (int*)d;
        d += 16;
        m->dec_newton = (int*)d;
        d += (size_t)2 * Wd * sizeof(int);
        m->dec_smask = (int*)d;
        d += (size_t)2 * Wd * sizeof(int);
        m->dec_next = (int*)d;
        d += (size_t)2 * Wd * sizeof(int);
        m->dec_status = (int*)d;
        d += (size_t)2 * Wd * sizeof(int);
        d = (char*)(((uintptr_t)d + 15) & ~(uintptr_t)15);
        m->dec_p0 = (double*)d;
        // The K padding of the slice buffers is never written: zero it once.
        RGF_CUDA_TRY(cudaMemsetAsync(m->hsa[0], 0,
                                     2 * sa_bytes(2 * Wd, b, m->Kp, kSlicesHP) + 2 * sb_bytes(2 * Wd, b, m->Kp, kSlicesHP),
                                     st));
    }
    if (cudaMallocHost((void**)&m->h_bad, 4 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        set_error("mixed workspace: cudaMallocHost failed");
        return RGF_E_OOM;
    }
    m->h_remaining = m->h_bad + 1;
    m->h_more = m->h_bad + 2;
    RGF_CUDA_TRY(cudaMemsetAsync(m->status, 0, 8 * sizeof(int), st));
    RGF_CUDA_TRY(cudaStreamSynchronize(st));
    return RGF_OK;
}

void mixed_state_free(MixedState* m) {
    cudaFree(m->status);
    cudaFree(m->dec_own);
    cudaFree(m->own);
    if (m->h_bad) cudaFreeHost(m->h_bad);
    m->status = nullptr;
    m->dec_own = m->own = nullptr;
    m->h_bad = nullptr;
}

rgf_status mixed_init(rgf_plan_s* p) {
    auto* pm = new PlanMixed();
    p->mixed = pm;
    const int b = p->b, N = p->N;
    const size_t nn = (size_t)b * b;
    auto alloc = [&](void** ptr, size_t bytes) -> rgf_status {
        if (cudaMalloc(ptr, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            set_error("mixed_init: cudaMalloc(%zu) failed", bytes);
            return RGF_E_OOM;
        }
        return RGF_OK;
    };
    RGF_TRY(alloc((void**)&pm->H_diag, nn * N * sizeof(float4)));
    RGF_TRY(alloc((void**)&pm->S_diag, nn * N * sizeof(float4)));
    if (N > 1) {
        RGF_TRY(alloc((void**)&pm->H_lower, nn * (N - 1) * sizeof(float4)));
        RGF_TRY(alloc((void**)&pm->S_lower, nn * (N - 1) * sizeof(float4)));
    }
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < 6; ++k) RGF_TRY(alloc((void**)&pm->lead[s][k], nn * sizeof(float4)));
    return mixed_state_init(&pm->ms, b, p->W, p->ws, p->stream);
}

void mixed_free(rgf_plan_s* p) {
    auto* pm = (PlanMixed*)p->mixed;
    if (!pm) return;
    cudaFree(pm->H_diag);
    cudaFree(pm->S_diag);
    cudaFree(pm->H_lower);
    cudaFree(pm->S_lower);
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < 6; ++k) cudaFree(pm->lead[s][k]);
    mixed_state_free(&pm->ms);
    delete pm;
    p->mixed = nullptr;
}

rgf_status mixed_on_blocks(rgf_plan_s* p) {
    auto* m = (PlanMixed*)p->mixed;
    const long nn = (long)p->b * p->b;
    RGF_TRY(to_dfc(nn * p->N, p->H_diag, m->H_diag, p->stream));
    RGF_TRY(to_dfc(nn * p->N, p->S_diag, m->S_diag, p->stream));
    if (p->N > 1) {
        RGF_TRY(to_dfc(nn * (p->N - 1), p->H_lower, m->H_lower, p->stream));
        RGF_TRY(to_dfc(nn * (p->N - 1), p->S_lower, m->S_lower, p->stream));
    }
    RGF_CUDA_TRY(cudaStreamSynchronize(p->stream));
    return RGF_OK;
}

rgf_status mixed_on_lead(rgf_plan_s* p, int side) {
    auto* m = (PlanMixed*)p->mixed;
    const long nn = (long)p->b * p->b;
    for (int k = 0; k < 6; ++k) RGF_TRY(to_dfc(nn, p->lead[side][k], m->lead[side][k], p->stream));
    RGF_CUDA_TRY(cudaStreamSynchronize(p->stream));
    return RGF_OK;
}

// Decimation of both leads, self-energies and broadening matrices for the
// W energies in p->d_E: Sigma_L, Sigma_R in pool unit 0 (2W entries),
// Gamma_L, Gamma_R in unit 2.  Clears and fills p->d_flags / p->d_err.
rgf_status mixed_leads(rgf_plan_s* p, int W, const Ctx& c) {
    auto* pm = (PlanMixed*)p->mixed;
    MixedState* m = &pm->ms;
    cudaStream_t st = p->stream;
    const int b = p->b;
    const long nn = (long)b * b;
    const double eta = p->opt.eta;
    const double* E = p->d_E;
    auto U = [&](int unit) { return m->pool + (long)unit * W * nn; };
    const int W2 = 2 * W;

    RGF_CUDA_TRY(cudaMemsetAsync(p->d_flags, 0, sizeof(int) * W, st));
    RGF_CUDA_TRY(cudaMemsetAsync(p->d_err, 0, sizeof(double) * W, st));
    RGF_CUDA_TRY(cudaMemsetAsync(m->status, 0, sizeof(int), st));

    // ---------------------------------------------------------- decimation
    // Lead decimation runs with FP64 storage and seven-slice products: the
    // Sancho-Rubio recursion inverts matrices with condition numbers up to
    // ~1e7 at some energies and needs FP64-class arithmetic there.
    float4 *g = U(8), *t1 = U(14), *t2 = U(16), *t3 = U(18);
    float4** L = pm->lead[0];
    float4** Rl = pm->lead[1];
    {
        double2** L64 = p->lead[0];
        double2** R64 = p->lead[1];
        auto D = [&](int unit) { return dec_unit(m, W, unit); };
        FormSrc a{{L64[1], R64[1]}, {L64[0], R64[0]}, {0, 0}};
        RGF_TRY(form_f64(W, 2, b, E, eta, a, D(2), nullptr, 0.0, nullptr, st));
        RGF_TRY(copy_f64(W2, b, D(0), D(2), nullptr, st));
        // Outward coupling: left lead M_{j,j-1} (lower), right lead M_{j,j+1} (upper).
        FormSrc al{{L64[3], R64[3]}, {L64[2], R64[2]}, {0, 1}};
        FormSrc be{{L64[3], R64[3]}, {L64[2], R64[2]}, {1, 0}};
        RGF_TRY(form_f64(W, 2, b, E, eta, al, D(4), nullptr, 0.0, nullptr, st));
        RGF_TRY(form_f64(W, 2, b, E, eta, be, D(6), nullptr, 0.0, nullptr, st));
        double2* g64 = nullptr;
        RGF_TRY(hp_decimate_run(c, W, p->opt.dec_tol, p->opt.dec_max_iter, &g64));
        RGF_TRY(c128_to_dfc(W2, b, g64, g, nullptr, st));
    }

    // ---------------------------------------------------------- self-energies
    float4* sigma = U(0);
    float4* gamma = U(2);
    FormSrcDf x1{{L[5], Rl[5]}, {L[4], Rl[4]}, {0, 1}};
    FormSrcDf x2{{L[5], Rl[5]}, {L[4], Rl[4]}, {1, 0}};
    RGF_TRY(form_dfc(W, 2, b, E, eta, x1, t1, nullptr, nullptr, st));
    RGF_TRY(form_dfc(W, 2, b, E, eta, x2, t2, nullptr, nullptr, st));
    RGF_TRY(sliceA(c, W2, 0, t1, nullptr));
    RGF_TRY(sliceB(c, W2, 0, g, nullptr));
    RGF_TRY(mm(c, W2, 0, 0, 1.0f, nullptr, 0, t3, nullptr));
    RGF_TRY(sliceA(c, W2, 0, t3, nullptr));
    RGF_TRY(sliceB(c, W2, 0, t2, nullptr));
    RGF_TRY(mm(c, W2, 0, 0, 1.0f, nullptr, 0, sigma, nullptr));
    RGF_TRY(gamma_dfc(W2, b, sigma, gamma, st));
    return RGF_OK;
}

rgf_status mixed_wave(rgf_plan_s* p, int W) {
    auto* pm = (PlanMixed*)p->mixed;
    MixedState* m = &pm->ms;
    cudaStream_t st = p->stream;
    const int b = p->b, N = p->N;
    const long nn = (long)b * b;
    const double eta = p->opt.eta;
    const double* E = p->d_E;
    Ctx c{m, st, nn, b, p->opt.ns_steps, p->d_err, p->d_flags, &p->n_reseeds};
    auto U = [&](int unit) { return m->pool + (long)unit * W * nn; };
    cudaEvent_t ev[3];
    for (auto& e : ev) RGF_CUDA_TRY(cudaEventCreate(&e));
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard() {
            for (int i = 0; i < 3; ++i) cudaEventDestroy(e[i]);
        }
    } guard{ev};
    NvtxRange wave_range("rgf mixed wave");
    RGF_CUDA_TRY(cudaEventRecord(ev[0], st));
    {
        NvtxRange r("rgf lead decimation + self-energies");
        RGF_TRY(mixed_leads(p, W, c));
    }
    NvtxRange sweep_range("rgf sweep + trace");
    RGF_CUDA_TRY(cudaEventRecord(ev[1], st));
    float4* sigma = U(0);
    float4* gamma = U(2);
    float4* sigL = sigma;
    float4* sigR = sigma + (long)W * nn;
    float4* gamL = gamma;
    float4* gamR = gamma + (long)W * nn;

    // ---------------------------------------------------------- sweep
    float4 *gi = U(4), *P = U(5), *M = U(6), *Q = U(9), *Qn = U(10);
    // The tcgen05 GEMM that forms M also writes the seed inverse's complex64
    // input (the legacy mma.sync core does not).
    float2* m64 = m->core == 0 ? m->c64 : nullptr;
    float4 *G = U(11), *Xt = U(12), *Yt = U(13), *Rs = U(14);
    if (N == 1) {
        FormSrcDf a0{{pm->S_diag, nullptr}, {pm->H_diag, nullptr}, {0, 0}};
        RGF_TRY(form_dfc(W, 1, b, E, eta, a0, M, sigL, nullptr, st));
        RGF_TRY(axpy_dfc(W, b, -1.0f, sigR, M, st));
        RGF_TRY(inv_mixed(c, W, W, M, gi, Rs, nullptr, p->d_flags));
        G = gi;
    } else {
        FormSrcDf a0{{pm->S_diag, nullptr}, {pm->H_diag, nullptr}, {0, 0}};
        RGF_TRY(form_dfc(W, 1, b, E, eta, a0, M, sigL, nullptr, st));
        RGF_TRY(inv_mixed(c, W, W, M, gi, Rs, nullptr, p->d_flags));
        for (int i = 1; i < N; ++i) {
            const float4* Sl = pm->S_lower + (long)(i - 1) * nn;
            const float4* Hl = pm->H_lower + (long)(i - 1) * nn;
            FormSrcDf ai{{pm->S_diag + (long)i * nn, nullptr}, {pm->H_diag + (long)i * nn, nullptr}, {0, 0}};
            RGF_TRY(form_dfc(W, 1, b, E, eta, ai, M, (i == N - 1) ? sigR : nullptr, nullptr, st));
            // tau' and tau go straight to their slices (never stored as matrices).
            RGF_TRY(sliceA(c, W, 0, gi, nullptr));
            RGF_TRY(form_slice_cols_dag(W, b, E, eta, Sl, Hl, m->sb[0], m->Kp, st));
            RGF_TRY(mm(c, W, 0, 0, -1.0f, nullptr, 0, P, nullptr));  // P = -g tau'
            RGF_TRY(form_slice_rows(W, b, E, eta, Sl, Hl, m->sa[0], m->Kp, st));
            RGF_TRY(sliceB(c, W, 0, P, nullptr));
            RGF_TRY(mm(c, W, 0, 0, 1.0f, M, 0, M, nullptr, m64));  // M += tau P (and its complex64 copy)
            if (i == 1) {
                std::swap(Q, P);
            } else {
                RGF_TRY(sliceA(c, W, 1, Q, nullptr));
                RGF_TRY(mm(c, W, 1, 0, 1.0f, nullptr, 0, Qn, nullptr));  // Q P
                std::swap(Q, Qn);
            }
            RGF_TRY(inv_mixed(c, W, W, M, gi, Rs, nullptr, p->d_flags, m64 != nullptr));
        }
        RGF_TRY(sliceA(c, W, 0, Q, nullptr));
        RGF_TRY(sliceB(c, W, 0, gi, nullptr));
        RGF_TRY(mm(c, W, 0, 0, 1.0f, nullptr, 0, G, nullptr));
    }

    // ---------------------------------------------------------- Caroli trace
    RGF_TRY(sliceA(c, W, 0, gamL, nullptr));
    RGF_TRY(sliceB(c, W, 0, G, nullptr));
    RGF_TRY(mm(c, W, 0, 0, 1.0f, nullptr, 0, Xt, nullptr));
    RGF_TRY(sliceA(c, W, 0, G, nullptr));
    RGF_TRY(sliceB(c, W, 0, gamR, nullptr));
    RGF_TRY(mm(c, W, 0, 0, 1.0f, nullptr, 0, Yt, nullptr));
    RGF_TRY(trace_dfc(W, b, Xt, Yt, p->d_T, p->d_Ti, st));
    RGF_CUDA_TRY(cudaEventRecord(ev[2], st));

    int h_status = 0;
    RGF_CUDA_TRY(cudaMemcpyAsync(&h_status, m->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    RGF_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_status != 0) {
        set_error("tensor-core GEMM pipeline timed out (status 0x%x)", h_status);
        return RGF_E_CUDA;
    }
    float t_lead = 0.f, t_sweep = 0.f;
    RGF_CUDA_TRY(cudaEventElapsedTime(&t_lead, ev[0], ev[1]));
    RGF_CUDA_TRY(cudaEventElapsedTime(&t_sweep, ev[1], ev[2]));
    p->lead_ms += t_lead;
    p->sweep_ms += t_sweep;
    return RGF_OK;
}

}  // namespace rgf
