"""FP64 CPU oracle for the RGF transmission path.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or run this module.  The CUDA library never calls it
and shares no code with it.

What it computes (the paper's Results section, RGF paragraph: transmission
from a block-tridiagonal nonorthogonal Hamiltonian, cost linear in the number
of principal layers per energy point; Methods: DFT electrode self-energies
combined with the device Hamiltonian; Results: the generalized problem
H c = eps S c in a nonorthogonal basis).  The paper prints no RGF equation,
so the formulas are the textbook ones, in this notation:

* z = E + i*eta multiplies S everywhere (device, couplings, leads).
* M = z S - H is block tridiagonal with on-site blocks A_i = z S_ii - H_ii,
  lower blocks tau_i = z S_{i,i-1} - H_{i,i-1} and upper blocks
  tau'_i = z S_{i-1,i} - H_{i-1,i} = z S_{i,i-1}^dag - H_{i,i-1}^dag.
* Lead surface Green's functions g_s solve g_s = (a - alpha g_s beta)^-1,
  with a the lead on-site block of M, alpha the coupling from the surface
  cell to the next cell away from the device, beta the coupling back (the
  retarded fixed point).  Sancho-Rubio decimation approaches it; at some
  energies its recursion loses digits (the FP64 result can leave a fixed-
  point residual of 1e-4 and a relative error of 1e-5), so Newton steps on
  the fixed-point equation follow it: with r = (a - alpha g beta) g - I the
  correction X solves the linearized (Stein) equation
  X = -g r + (g alpha) X (beta g), summed by doubling (see newton_refine for
  the rules that drop a step whose doubling grows instead of converging).
* Sigma_L = tau_c^L g_L tau'_c^L sits on block (0,0); Sigma_R =
  tau'_c^R g_R tau_c^R sits on block (N-1,N-1); Gamma = i (Sigma - Sigma^dag).
* G = (M - Sigma_L (+) Sigma_R)^-1, and T(E) = Re Tr[Gamma_L G_{0,N-1}
  Gamma_R G_{0,N-1}^dag].

Pins (all in ``tests/test_oracle_pins.py``): the closed-form uniform chain
(surface GF, self-energy, Gamma and T at finite eta), brute-force dense
inversion against the block recursion on tiny random devices, the
surface-GF fixed-point residual, Hermiticity and positivity of Gamma,
left-right sweep equality, the H -> H + cS energy shift, block-unitary
gauge invariance, zero coupling, and 0 <= T <= channel count.  Every
function below is covered by at least one of them.
"""
from __future__ import annotations

import numpy as np

_inv = np.linalg.inv


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def lead_blocks(lead, z, side):
    """On-site block a, outward coupling alpha, inward coupling beta of M = zS - H
    for one lead, and the device-lead couplings (into device, out of device).

    side 'R': the lead extends to the right; outward = upper block M_{j,j+1}.
    side 'L': the lead extends to the left; outward = lower block M_{j,j-1}.
    """
    a = z * lead.S00 - lead.H00
    lower = z * lead.S10 - lead.H10            # M_{j+1,j}
    upper = z * _dag(lead.S10) - _dag(lead.H10)  # M_{j,j+1}
    c_lower = z * lead.Sc - lead.Hc
    c_upper = z * _dag(lead.Sc) - _dag(lead.Hc)
    if side == "R":
        return a, upper, lower, c_lower, c_upper
    if side == "L":
        return a, lower, upper, c_lower, c_upper
    raise ValueError(side)


def sancho_rubio(a, alpha, beta, tol=1e-14, max_iter=100):
    """Surface Green's function of a semi-infinite chain by decimation.

    Each iteration eliminates every other cell of the current chain: with
    g = eps^-1, the surface block loses alpha g beta, bulk blocks lose
    alpha g beta + beta g alpha, and the couplings become -alpha g alpha and
    -beta g beta (the Schur complement of the three-cell chain).  Stops when
    max(||alpha||_F, ||beta||_F) <= tol * ||a||_F.  Returns (g_s, iterations,
    converged).
    """
    eps_s = a.copy()
    eps = a.copy()
    na = np.linalg.norm(a)
    for it in range(1, max_iter + 1):
        g = _inv(eps)
        g_beta = g @ beta
        g_alpha = g @ alpha
        agb = alpha @ g_beta
        bga = beta @ g_alpha
        eps_s = eps_s - agb
        eps = eps - agb - bga
        alpha = -(alpha @ g_alpha)
        beta = -(beta @ g_beta)
        if max(np.linalg.norm(alpha), np.linalg.norm(beta)) <= tol * na:
            return _inv(eps_s), it, True
    return _inv(eps_s), max_iter, False


def newton_refine(a, alpha, beta, g, max_steps=3, tol=1e-28, max_doublings=100, growth=1e4,
                  again=1e-12):
    """Newton steps on g = (a - alpha g beta)^-1.  Returns (g, ok).

    One step: r = (a - alpha g beta) g - I; the correction X solves the
    linearized (Stein) equation X = -g r + A X B with A = g alpha, B = beta g,
    summed by doubling (X <- X + A X B, A <- A A, B <- B B) until
    p = |A|_F |B|_F <= tol; then g <- g + X.  The doubling converges when the
    spectral radii of A and B multiply to less than one, as they do at the
    retarded fixed point; a g far enough from it can break that (near band
    edges at small eta), and the sums then grow: when p exceeds growth times
    its first value, turns non-finite or has not reached tol after
    max_doublings, the step is dropped, g is kept and ok is False.  Another
    step follows while the last correction exceeded again |g|_F: Newton
    converges quadratically, so what a correction of size c leaves is of
    order K c^2 (K up to ~1e6 near band edges at eta = 1e-6), below the FP64
    level for c <= 1e-12."""
    n = a.shape[0]
    eye = np.eye(n, dtype=np.complex128)
    for _ in range(max_steps):
        r = (a - alpha @ g @ beta) @ g - eye
        A = g @ alpha
        B = beta @ g
        X = -(g @ r)
        p0 = None
        converged = False
        for _ in range(max_doublings):
            X = X + A @ X @ B
            A = A @ A
            B = B @ B
            p = np.linalg.norm(A) * np.linalg.norm(B)
            if p0 is None:
                p0 = p
            if p <= tol:
                converged = True
                break
            if not np.isfinite(p) or p > growth * p0:
                break
        if not converged:
            return g, False
        g = g + X
        if np.linalg.norm(X) <= again * np.linalg.norm(g):
            break
    return g, True


def self_energies(dev, z, tol=1e-14, max_iter=100, newton_steps=3):
    """Sigma_L, Sigma_R, Gamma_L, Gamma_R, the decimation iteration counts and
    whether each lead's Newton refinement held (refined = (left, right))."""
    aL, alL, beL, cLlow, cLup = lead_blocks(dev.lead_L, z, "L")
    aR, alR, beR, cRlow, cRup = lead_blocks(dev.lead_R, z, "R")
    gL, itL, okL = sancho_rubio(aL, alL, beL, tol, max_iter)
    gR, itR, okR = sancho_rubio(aR, alR, beR, tol, max_iter)
    # Newton steps follow a converged decimation only (a truncated one is
    # reported as such, and its result stays as it is).
    refL = refR = False
    if newton_steps > 0 and okL:
        gL, refL = newton_refine(aL, alL, beL, gL, newton_steps)
    if newton_steps > 0 and okR:
        gR, refR = newton_refine(aR, alR, beR, gR, newton_steps)
    # Left: Sigma_L = M_{0,-1} g_L M_{-1,0}; M_{0,-1} is the lower block Lc.
    sig_L = cLlow @ gL @ cLup
    # Right: Sigma_R = M_{N-1,N} g_R M_{N,N-1}; M_{N-1,N} is the upper block.
    sig_R = cRup @ gR @ cRlow
    gam_L = 1j * (sig_L - _dag(sig_L))
    gam_R = 1j * (sig_R - _dag(sig_R))
    return dict(sigma_L=sig_L, sigma_R=sig_R, gamma_L=gam_L, gamma_R=gam_R,
                g_L=gL, g_R=gR, iters=(itL, itR), converged=(okL and okR), refined=(refL, refR))


def _A(dev, z, i):
    return z * dev.S_diag[i] - dev.H_diag[i]


def _tau(dev, z, i):
    """Lower block M_{i,i-1}, i >= 1."""
    return z * dev.S_lower[i - 1] - dev.H_lower[i - 1]


def _tau_up(dev, z, i):
    """Upper block M_{i-1,i}, i >= 1."""
    return z * _dag(dev.S_lower[i - 1]) - _dag(dev.H_lower[i - 1])


def rgf_G1N(dev, z, sigma_L, sigma_R):
    """G_{0,N-1} by the left-to-right recursive sweep.

    g_0 = (A_0 - Sigma_L)^-1, Q_0 = I; for i = 1..N-1:
    P_i = -g_{i-1} tau'_i, M_i = A_i + tau_i P_i (- Sigma_R at i = N-1),
    g_i = M_i^-1, Q_i = Q_{i-1} P_i; finally G_{0,N-1} = Q_{N-1} g_{N-1}.
    (The minus in P keeps the sign of the exact block of the inverse.)
    """
    N = dev.n_layers
    b = dev.b
    if N == 1:
        return _inv(_A(dev, z, 0) - sigma_L - sigma_R)
    g = _inv(_A(dev, z, 0) - sigma_L)
    Q = np.eye(b, dtype=np.complex128)
    for i in range(1, N):
        P = -(g @ _tau_up(dev, z, i))
        M = _A(dev, z, i) + _tau(dev, z, i) @ P
        if i == N - 1:
            M = M - sigma_R
        g = _inv(M)
        Q = Q @ P
    return Q @ g


def rgf_G1N_right_sweep(dev, z, sigma_L, sigma_R):
    """G_{0,N-1} by the mirror sweep from the right lead towards the left.

    gr_{N-1} = (A_{N-1} - Sigma_R)^-1; for i = N-2..0:
    R_i = -gr_{i+1} tau_{i+1}, M_i = A_i + tau'_{i+1} R_i (- Sigma_L at i = 0),
    gr_i = M_i^-1, and G_{0,N-1} = gr_0 tau'_1 ... with the right-connected
    chain: G_{0,N-1} = gr_0 (-tau'_1 gr_1) (-tau'_2 gr_2) ... .
    """
    N = dev.n_layers
    if N == 1:
        return _inv(_A(dev, z, 0) - sigma_L - sigma_R)
    grs = [None] * N
    grs[N - 1] = _inv(_A(dev, z, N - 1) - sigma_R)
    for i in range(N - 2, -1, -1):
        R = -(grs[i + 1] @ _tau(dev, z, i + 1))
        M = _A(dev, z, i) + _tau_up(dev, z, i + 1) @ R
        if i == 0:
            M = M - sigma_L
        grs[i] = _inv(M)
    G = grs[0]
    for i in range(1, N):
        G = G @ (-(_tau_up(dev, z, i) @ grs[i]))
    return G


def assemble_dense(dev, z, sigma_L, sigma_R):
    """The full (N b) x (N b) matrix z S - H - Sigma_L (+) Sigma_R."""
    N, b = dev.n_layers, dev.b
    M = np.zeros((N * b, N * b), dtype=np.complex128)
    for i in range(N):
        M[i * b:(i + 1) * b, i * b:(i + 1) * b] = _A(dev, z, i)
    for i in range(1, N):
        M[i * b:(i + 1) * b, (i - 1) * b:i * b] = _tau(dev, z, i)
        M[(i - 1) * b:i * b, i * b:(i + 1) * b] = _tau_up(dev, z, i)
    M[:b, :b] -= sigma_L
    M[(N - 1) * b:, (N - 1) * b:] -= sigma_R
    return M


def dense_G1N(dev, z, sigma_L, sigma_R):
    """Block (0, N-1) of the full inverse, by a dense solve against the last
    block column of the identity."""
    N, b = dev.n_layers, dev.b
    M = assemble_dense(dev, z, sigma_L, sigma_R)
    rhs = np.zeros((N * b, b), dtype=np.complex128)
    rhs[(N - 1) * b:, :] = np.eye(b)
    X = np.linalg.solve(M, rhs)
    return X[:b, :]


def caroli(gamma_L, G1N, gamma_R):
    """Tr[Gamma_L G Gamma_R G^dag] as a complex number (its imaginary part is
    a diagnostic that should vanish)."""
    return np.trace(gamma_L @ G1N @ gamma_R @ _dag(G1N))


def transmission(dev, energies, eta, method="rgf", tol=1e-14, max_iter=100,
                 return_info=False, newton_steps=3):
    """T(E) for each energy.  method: 'rgf' (left sweep), 'rgf_right'
    (mirror sweep) or 'dense' (full inversion)."""
    energies = np.asarray(energies, dtype=np.float64)
    T = np.empty(energies.shape[0])
    info = []
    for k, E in enumerate(energies):
        z = complex(E, eta)
        se = self_energies(dev, z, tol, max_iter, newton_steps)
        if method == "rgf":
            G = rgf_G1N(dev, z, se["sigma_L"], se["sigma_R"])
        elif method == "rgf_right":
            G = rgf_G1N_right_sweep(dev, z, se["sigma_L"], se["sigma_R"])
        elif method == "dense":
            G = dense_G1N(dev, z, se["sigma_L"], se["sigma_R"])
        else:
            raise ValueError(method)
        t = caroli(se["gamma_L"], G, se["gamma_R"])
        T[k] = t.real
        if return_info:
            info.append(dict(trace_imag=t.imag, iters=se["iters"], converged=se["converged"],
                             refined=se["refined"]))
    return (T, info) if return_info else T


def transmission_one(dev, E, eta, **kw):
    return float(transmission(dev, [E], eta, **kw)[0])
