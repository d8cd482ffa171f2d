/* Extended-precision CPU oracle for the RGF transmission T(E).
 * TEST INFRASTRUCTURE ONLY: only tests/, the golden-value script beside them,
 * __graft_entry__.smoke() and the CPU-baseline leg of bench.py may load it.
 * The CUDA library never calls it and shares no code with it.
 *
 * It evaluates exactly the textbook steps of the FP64 oracle (oracle/rgf_oracle.py),
 * but every complex number is a pair of x87 80-bit `long double` values (64-bit
 * significand, unit roundoff 2^-64, i.e. 2048 times finer than binary64).  Its job
 * is to settle the energies where the FP64 problem is itself worse conditioned
 * than the FP64 parity bar: there, the difference between the FP64 oracle and this
 * one measures the FP64 oracle's own rounding error.
 *
 * What it computes (the paper's Results, the paragraph on the cost of each part:
 * transmission from a block-tridiagonal nonorthogonal Hamiltonian, cost linear in
 * the number of principal layers per energy point; Results: the generalized
 * problem H c = eps S c; Methods, transport paragraph: electrode self-energies
 * with the device Hamiltonian).  The paper prints no RGF equation, so the steps
 * are the textbook ones:
 *   z = E + i eta multiplies S everywhere; M = z S - H;
 *   lead surface Green's function: the retarded fixed point of
 *   g = (a - alpha g beta)^-1, reached by Sancho-Rubio decimation of (a, alpha,
 *   beta) and then, when the decimation converged, Newton steps on the
 *   fixed-point equation (the decimation's recursion loses digits at some
 *   energies: its result can leave a residual far above the rounding level,
 *   which the Newton steps remove);
 *   Sigma_L = M_{0,-1} g_L M_{-1,0},  Sigma_R = M_{N-1,N} g_R M_{N,N-1};
 *   Gamma = i (Sigma - Sigma^dag);
 *   left-to-right sweep g_0 = (A_0 - Sigma_L)^-1, Q_0 = I,
 *     P_i = -g_{i-1} tau'_i, M_i = A_i + tau_i P_i (- Sigma_R at the last layer),
 *     g_i = M_i^-1, Q_i = Q_{i-1} P_i, G_{0,N-1} = Q_{N-1} g_{N-1};
 *   T = Re Tr[Gamma_L G Gamma_R G^dag]  (the imaginary part is returned too).
 * Inverses are Gauss-Jordan elimination with partial pivoting on [M | I].
 *
 * Newton step for the fixed point: with r = (a - alpha g beta) g - I, the
 * correction X solves the linearized (Stein) equation X = -g r + (g alpha) X
 * (beta g), summed by doubling: X <- X + A X B, A <- A A, B <- B B, from
 * X = -g r, A = g alpha, B = beta g, until |A|_F |B|_F <= tol; g <- g + X.
 *
 * Pins (tests/test_oracle_ext.py): mpmath dense inversion at 40 digits on tiny
 * random devices, with the surface Green's function checked by its fixed-point
 * residual at 40 digits; the uniform-chain closed form evaluated in mpmath; the
 * FP64 oracle on well-conditioned energies.
 *
 * Layout of the inputs: complex128 as interleaved (re, im) doubles, row-major b x b
 * blocks, layer-major; H_lower[i-1] = H_{i,i-1}.  A lead is six blocks in the order
 * H00, S00, H10, S10, Hc, Sc (H10 = H_{j+1,j} in the device's orientation; Hc is
 * H_{0,-1} for the left lead and H_{N,N-1} for the right lead).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef long double real;
typedef struct { real re, im; } cplx;

static inline cplx cmul(cplx a, cplx b) {
    cplx r = { a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re };
    return r;
}

/* z X - Y for complex128 inputs X, Y (conj-transposed when dag != 0). */
static void form(cplx *out, const double *X, const double *Y, cplx z, int b, int dag) {
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) {
            size_t s = dag ? ((size_t)c * b + r) : ((size_t)r * b + c);
            real xr = X[2 * s], xi = X[2 * s + 1], yr = Y[2 * s], yi = Y[2 * s + 1];
            if (dag) { xi = -xi; yi = -yi; }
            cplx x = { xr, xi };
            cplx zx = cmul(z, x);
            out[(size_t)r * b + c].re = zx.re - yr;
            out[(size_t)r * b + c].im = zx.im - yi;
        }
}

/* C = A B (C distinct from A and B).  Each entry is one dot product over k with
 * its sum kept in registers (B is read through a transposed copy in bt). */
static void gemm_t(cplx *C, const cplx *A, const cplx *B, int b, cplx *bt) {
    for (int k = 0; k < b; ++k)
        for (int j = 0; j < b; ++j) bt[(size_t)j * b + k] = B[(size_t)k * b + j];
    for (int i = 0; i < b; ++i) {
        const cplx *Ai = A + (size_t)i * b;
        for (int j = 0; j < b; ++j) {
            const cplx *Bj = bt + (size_t)j * b;
            real sr = 0.0L, si = 0.0L;
            for (int k = 0; k < b; ++k) {
                sr += Ai[k].re * Bj[k].re - Ai[k].im * Bj[k].im;
                si += Ai[k].re * Bj[k].im + Ai[k].im * Bj[k].re;
            }
            C[(size_t)i * b + j].re = sr;
            C[(size_t)i * b + j].im = si;
        }
    }
}

/* C = A B with a per-thread transposed-copy buffer (OpenMP threads each own one). */
static __thread cplx *tls_bt = NULL;
static __thread size_t tls_bt_n = 0;

static void gemm(cplx *C, const cplx *A, const cplx *B, int b) {
    size_t n = (size_t)b * b;
    if (tls_bt_n < n) {
        free(tls_bt);
        tls_bt = (cplx *)malloc(n * sizeof(cplx));
        tls_bt_n = n;
    }
    gemm_t(C, A, B, b, tls_bt);
}

/* Ainv = A^-1 by Gauss-Jordan with partial pivoting on the augmented [A | I].
 * work holds b x 2b entries.  Returns 0, or 1 on an exactly zero pivot. */
static int inverse(cplx *Ainv, const cplx *A, int b, cplx *work) {
    int w = 2 * b;
    for (int r = 0; r < b; ++r) {
        for (int c = 0; c < b; ++c) work[(size_t)r * w + c] = A[(size_t)r * b + c];
        for (int c = 0; c < b; ++c) {
            work[(size_t)r * w + b + c].re = (r == c) ? 1.0L : 0.0L;
            work[(size_t)r * w + b + c].im = 0.0L;
        }
    }
    for (int k = 0; k < b; ++k) {
        int p = k;
        real best = -1.0L;
        for (int r = k; r < b; ++r) {
            cplx v = work[(size_t)r * w + k];
            real m = v.re * v.re + v.im * v.im;
            if (m > best) { best = m; p = r; }
        }
        if (best == 0.0L) return 1;
        if (p != k)
            for (int c = 0; c < w; ++c) {
                cplx t = work[(size_t)k * w + c];
                work[(size_t)k * w + c] = work[(size_t)p * w + c];
                work[(size_t)p * w + c] = t;
            }
        cplx piv = work[(size_t)k * w + k];
        real den = piv.re * piv.re + piv.im * piv.im;
        cplx inv = { piv.re / den, -piv.im / den };
        for (int c = 0; c < w; ++c) work[(size_t)k * w + c] = cmul(work[(size_t)k * w + c], inv);
        for (int r = 0; r < b; ++r) {
            if (r == k) continue;
            cplx f = work[(size_t)r * w + k];
            if (f.re == 0.0L && f.im == 0.0L) continue;
            for (int c = 0; c < w; ++c) {
                cplx t = cmul(f, work[(size_t)k * w + c]);
                work[(size_t)r * w + c].re -= t.re;
                work[(size_t)r * w + c].im -= t.im;
            }
        }
    }
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) Ainv[(size_t)r * b + c] = work[(size_t)r * w + b + c];
    return 0;
}

static real fro(const cplx *A, int b) {
    real s = 0.0L;
    for (size_t i = 0; i < (size_t)b * b; ++i) s += A[i].re * A[i].re + A[i].im * A[i].im;
    return sqrtl(s);
}

/* Surface Green's function of a semi-infinite chain by Sancho-Rubio decimation:
 * g = eps^-1; eps_s -= alpha g beta; eps -= alpha g beta + beta g alpha;
 * alpha = -alpha g alpha; beta = -beta g beta; until
 * max(||alpha||_F, ||beta||_F) <= tol ||a||_F.  alpha, beta are overwritten.
 * Returns the iteration count (negated when it did not converge). */
static int sancho_rubio(cplx *gs, const cplx *a, cplx *alpha, cplx *beta, int b, real tol,
                        int max_iter, cplx *work) {
    size_t bb = (size_t)b * b;
    cplx *eps_s = work, *eps = work + bb, *g = work + 2 * bb, *ga = work + 3 * bb,
         *gb = work + 4 * bb, *agb = work + 5 * bb, *bga = work + 6 * bb, *gj = work + 7 * bb;
    memcpy(eps_s, a, sizeof(cplx) * bb);
    memcpy(eps, a, sizeof(cplx) * bb);
    real na = fro(a, b);
    int it;
    for (it = 1; it <= max_iter; ++it) {
        inverse(g, eps, b, gj);
        gemm(gb, g, beta, b);
        gemm(ga, g, alpha, b);
        gemm(agb, alpha, gb, b);
        gemm(bga, beta, ga, b);
        for (size_t e = 0; e < bb; ++e) {
            eps_s[e].re -= agb[e].re; eps_s[e].im -= agb[e].im;
            eps[e].re -= agb[e].re + bga[e].re; eps[e].im -= agb[e].im + bga[e].im;
        }
        gemm(g, alpha, ga, b);              /* alpha g alpha */
        for (size_t e = 0; e < bb; ++e) { alpha[e].re = -g[e].re; alpha[e].im = -g[e].im; }
        gemm(g, beta, gb, b);               /* beta g beta */
        for (size_t e = 0; e < bb; ++e) { beta[e].re = -g[e].re; beta[e].im = -g[e].im; }
        real na_ = fro(alpha, b), nb_ = fro(beta, b);
        if ((na_ > nb_ ? na_ : nb_) <= tol * na) break;
    }
    inverse(gs, eps_s, b, gj);
    return it <= max_iter ? it : -max_iter;
}

/* Newton steps on g = (a - alpha g beta)^-1 (see the header); alpha, beta are
 * the lead's original couplings (not the decimated ones).  work: 9 bb.  A step
 * whose doubling grows (|A|_F |B|_F above 1e4 times its first value, not
 * finite, or not below tol after 200 doublings) is dropped and the function
 * returns 0 with g as it was; another step follows while the last correction
 * exceeded 1e-14 |g|_F (what a correction c leaves is of order K c^2, K up to
 * ~1e6).  Returns 1 when the refinement held. */
static int newton_refine(cplx *g, const cplx *a, const cplx *alpha, const cplx *beta, int b, real tol,
                         int steps, cplx *work) {
    size_t bb = (size_t)b * b;
    cplx *W = work, *r = work + bb, *A = work + 2 * bb, *B = work + 3 * bb, *X = work + 4 * bb,
         *t1 = work + 5 * bb, *t2 = work + 6 * bb;
    for (int s = 0; s < steps; ++s) {
        gemm(t1, alpha, g, b);   /* alpha g */
        gemm(t2, t1, beta, b);   /* alpha g beta */
        for (size_t e = 0; e < bb; ++e) { W[e].re = a[e].re - t2[e].re; W[e].im = a[e].im - t2[e].im; }
        gemm(r, W, g, b);        /* (a - alpha g beta) g */
        for (int q = 0; q < b; ++q) r[(size_t)q * b + q].re -= 1.0L;
        gemm(X, g, r, b);
        for (size_t e = 0; e < bb; ++e) { X[e].re = -X[e].re; X[e].im = -X[e].im; }
        gemm(A, g, alpha, b);
        gemm(B, beta, g, b);
        real p0 = -1.0L;
        int converged = 0;
        for (int k = 0; k < 200; ++k) {
            gemm(t1, A, X, b);
            gemm(t2, t1, B, b);
            for (size_t e = 0; e < bb; ++e) { X[e].re += t2[e].re; X[e].im += t2[e].im; }
            gemm(t1, A, A, b);
            memcpy(A, t1, sizeof(cplx) * bb);
            gemm(t1, B, B, b);
            memcpy(B, t1, sizeof(cplx) * bb);
            real p = fro(A, b) * fro(B, b);
            if (p0 < 0.0L) p0 = p;
            if (p <= tol) { converged = 1; break; }
            if (!(p == p) || p > 1e4L * p0 || isinf(p)) break;
        }
        if (!converged) return 0;
        for (size_t e = 0; e < bb; ++e) { g[e].re += X[e].re; g[e].im += X[e].im; }
        if (fro(X, b) <= 1e-14L * fro(g, b)) break;
    }
    return 1;
}

/* Per-lead blocks of M = z S - H: on-site a, outward alpha, inward beta, and the
 * device-lead couplings c_lower (row right of column) and c_upper. */
static void lead_blocks(const double *const *lead, cplx z, int b, int right, cplx *a, cplx *alpha,
                        cplx *beta, cplx *c_lower, cplx *c_upper) {
    form(a, lead[1], lead[0], z, b, 0);
    /* lower = M_{j+1,j}, upper = M_{j,j+1} */
    if (right) {
        form(alpha, lead[3], lead[2], z, b, 1);
        form(beta, lead[3], lead[2], z, b, 0);
    } else {
        form(alpha, lead[3], lead[2], z, b, 0);
        form(beta, lead[3], lead[2], z, b, 1);
    }
    form(c_lower, lead[5], lead[4], z, b, 0);
    form(c_upper, lead[5], lead[4], z, b, 1);
}

/* One energy.  Returns T's real part in *T, imaginary part in *Ti, decimation
 * iteration counts in it[0..1] (negative: not converged). */
static void one_energy(int N, int b, const double *Hd, const double *Sd, const double *Hl,
                       const double *Sl, const double *const *leadL, const double *const *leadR,
                       double E, double eta, real tol, int max_iter, int newton_steps, double *T,
                       double *Ti, int *it) {
    size_t bb = (size_t)b * b;
    cplx z = { (real)E, (real)eta };
    cplx *buf = (cplx *)calloc(bb * 28, sizeof(cplx));
    cplx *a = buf, *al = buf + bb, *be = buf + 2 * bb, *cl = buf + 3 * bb, *cu = buf + 4 * bb;
    cplx *gL = buf + 5 * bb, *gR = buf + 6 * bb, *sL = buf + 7 * bb, *sR = buf + 8 * bb;
    cplx *t1 = buf + 9 * bb, *g = buf + 10 * bb, *Q = buf + 11 * bb, *P = buf + 12 * bb;
    cplx *M = buf + 13 * bb, *t2 = buf + 14 * bb, *work = buf + 15 * bb; /* 9 bb */
    cplx *gj = buf + 24 * bb;                                            /* 2 bb (b x 2b) */
    cplx *al0 = buf + 26 * bb, *be0 = buf + 27 * bb;                     /* original couplings */

    /* Left lead: Sigma_L = M_{0,-1} g_L M_{-1,0} = c_lower g_L c_upper. */
    lead_blocks(leadL, z, b, 0, a, al, be, cl, cu);
    memcpy(al0, al, sizeof(cplx) * bb);
    memcpy(be0, be, sizeof(cplx) * bb);
    it[0] = sancho_rubio(gL, a, al, be, b, tol, max_iter, work);
    if (newton_steps > 0 && it[0] > 0) newton_refine(gL, a, al0, be0, b, tol * tol, newton_steps, work);
    gemm(t1, cl, gL, b);
    gemm(sL, t1, cu, b);
    /* Right lead: Sigma_R = M_{N-1,N} g_R M_{N,N-1} = c_upper g_R c_lower. */
    lead_blocks(leadR, z, b, 1, a, al, be, cl, cu);
    memcpy(al0, al, sizeof(cplx) * bb);
    memcpy(be0, be, sizeof(cplx) * bb);
    it[1] = sancho_rubio(gR, a, al, be, b, tol, max_iter, work);
    if (newton_steps > 0 && it[1] > 0) newton_refine(gR, a, al0, be0, b, tol * tol, newton_steps, work);
    gemm(t1, cu, gR, b);
    gemm(sR, t1, cl, b);

    /* Sweep. */
    form(M, Sd, Hd, z, b, 0);
    for (size_t e = 0; e < bb; ++e) { M[e].re -= sL[e].re; M[e].im -= sL[e].im; }
    if (N == 1)
        for (size_t e = 0; e < bb; ++e) { M[e].re -= sR[e].re; M[e].im -= sR[e].im; }
    inverse(g, M, b, gj);
    memset(Q, 0, sizeof(cplx) * bb);
    for (int r = 0; r < b; ++r) Q[(size_t)r * b + r].re = 1.0L;
    for (int i = 1; i < N; ++i) {
        form(t1, Sl + 2 * bb * (i - 1), Hl + 2 * bb * (i - 1), z, b, 1); /* tau'_i */
        gemm(P, g, t1, b);
        for (size_t e = 0; e < bb; ++e) { P[e].re = -P[e].re; P[e].im = -P[e].im; }
        form(t1, Sl + 2 * bb * (i - 1), Hl + 2 * bb * (i - 1), z, b, 0); /* tau_i */
        gemm(t2, t1, P, b);
        form(M, Sd + 2 * bb * i, Hd + 2 * bb * i, z, b, 0);              /* A_i */
        for (size_t e = 0; e < bb; ++e) { M[e].re += t2[e].re; M[e].im += t2[e].im; }
        if (i == N - 1)
            for (size_t e = 0; e < bb; ++e) { M[e].re -= sR[e].re; M[e].im -= sR[e].im; }
        inverse(g, M, b, gj);
        gemm(t2, Q, P, b);
        memcpy(Q, t2, sizeof(cplx) * bb);
    }
    cplx *G = P;
    gemm(G, Q, g, b);

    /* Gamma = i (Sigma - Sigma^dag): entry (r,c) = i (s_rc - conj(s_cr)). */
    cplx *gamL = t1, *gamR = t2;
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) {
            cplx x = sL[(size_t)r * b + c], y = sL[(size_t)c * b + r];
            cplx d = { x.re - y.re, x.im + y.im };
            gamL[(size_t)r * b + c].re = -d.im; gamL[(size_t)r * b + c].im = d.re;
            x = sR[(size_t)r * b + c]; y = sR[(size_t)c * b + r];
            cplx d2 = { x.re - y.re, x.im + y.im };
            gamR[(size_t)r * b + c].re = -d2.im; gamR[(size_t)r * b + c].im = d2.re;
        }
    /* Tr[Gamma_L G Gamma_R G^dag] = sum_jk (Gamma_L G Gamma_R)_jk conj(G_jk). */
    gemm(M, gamL, G, b);
    gemm(Q, M, gamR, b);
    real tr = 0.0L, ti = 0.0L;
    for (size_t e = 0; e < bb; ++e) {
        tr += Q[e].re * G[e].re + Q[e].im * G[e].im;
        ti += Q[e].im * G[e].re - Q[e].re * G[e].im;
    }
    *T = (double)tr;
    *Ti = (double)ti;
    free(buf);
}

/* T(E) for n_E energies.  leads_L and leads_R point to six complex128 blocks each
 * (H00, S00, H10, S10, Hc, Sc).  Energies run in parallel when OpenMP is on (each
 * energy is independent).  T_imag and iters (2 per energy) may be NULL. */
void rgf_ext_transmission(int N, int b, const double *H_diag, const double *S_diag,
                          const double *H_lower, const double *S_lower,
                          const double *const *lead_L, const double *const *lead_R,
                          const double *E, int n_E, double eta, double tol, int max_iter,
                          int newton_steps, double *T, double *T_imag, int *iters) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < n_E; ++k) {
        double ti;
        int it[2];
        one_energy(N, b, H_diag, S_diag, H_lower, S_lower, lead_L, lead_R, E[k], eta,
                   (real)tol, max_iter, newton_steps, &T[k], &ti, it);
        if (T_imag) T_imag[k] = ti;
        if (iters) { iters[2 * k] = it[0]; iters[2 * k + 1] = it[1]; }
    }
}

/* Surface Green's function of one lead alone (for the fixed-point pin): side 0 =
 * left, 1 = right.  g_out is complex128 b x b; the result is rounded from 80 bits,
 * and g_out_lo receives the rounding remainder (g80 - (double)g80) so that callers
 * can see the value to about 2^-64 of its magnitude. */
int rgf_ext_surface_gf(int b, const double *const *lead, int side, double E, double eta,
                       double tol, int max_iter, int newton_steps, double *g_out, double *g_out_lo) {
    size_t bb = (size_t)b * b;
    cplx z = { (real)E, (real)eta };
    cplx *buf = (cplx *)calloc(bb * 18, sizeof(cplx));
    cplx *a = buf, *al = buf + bb, *be = buf + 2 * bb, *cl = buf + 3 * bb, *cu = buf + 4 * bb;
    cplx *gs = buf + 5 * bb, *work = buf + 6 * bb, *al0 = buf + 16 * bb, *be0 = buf + 17 * bb;
    lead_blocks(lead, z, b, side, a, al, be, cl, cu);
    memcpy(al0, al, sizeof(cplx) * bb);
    memcpy(be0, be, sizeof(cplx) * bb);
    int it = sancho_rubio(gs, a, al, be, b, (real)tol, max_iter, work);
    if (newton_steps > 0 && it > 0) newton_refine(gs, a, al0, be0, b, (real)tol * (real)tol, newton_steps, work);
    for (size_t e = 0; e < bb; ++e) {
        double hr = (double)gs[e].re, hi = (double)gs[e].im;
        g_out[2 * e] = hr; g_out[2 * e + 1] = hi;
        if (g_out_lo) {
            g_out_lo[2 * e] = (double)(gs[e].re - (real)hr);
            g_out_lo[2 * e + 1] = (double)(gs[e].im - (real)hi);
        }
    }
    free(buf);
    return it;
}
