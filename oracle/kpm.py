"""Plain CPU oracle of the non-orthogonal kernel polynomial method (KPM) for
the Fermi level.  TEST INFRASTRUCTURE ONLY: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the CUDA library never calls it and shares no code with it.

What it computes (the paper's Results: the generalized problem
H c = eps S c in a nonorthogonal basis; the rescaled operator
A~ = S^-1 (H - b S) / a expanded in Chebyshev polynomials, its action on a
vector evaluated by solving linear systems with S instead of forming S^-1;
the Chebyshev moments reconstruct the density of states, which fixes the
Fermi level through the electron count; the cost paragraph: O(N_mom N_rand N)
with N_mom moments and N_rand stochastic random vectors).  In the notation
below the paper's scale and shift (a, b) are called ``alpha`` and ``beta``
(``b`` is the block size elsewhere in this project).

The paper gives no formulas beyond that; these readings are the textbook
KPM (Weisse, Wellein, Alvermann, Fehske, Rev. Mod. Phys. 78, 275 (2006)):

* moments mu_n = (1/R) sum_r Re(r^dag T_n(A~) r), with T_0 r = r,
  T_1 r = A~ r, T_{n+1} r = 2 A~ T_n r - T_{n-1} r; random vectors r with
  E[r r^dag] = I are inputs (unit-modulus random phases in the tests);
  the trace of T_n(A~) is real (the eigenvalues of S^-1 H are), so the
  real part is taken;
* Jackson kernel g_n = ((M - n + 1) cos(pi n / (M + 1))
  + sin(pi n / (M + 1)) cot(pi / (M + 1))) / (M + 1), M = N_mom;
* number of states below x = (E - beta) / alpha, with theta = arccos x:
  N(x) = g_0 mu_0 (pi - theta) / pi - (2 / pi) sum_{n>=1} g_n mu_n sin(n theta) / n
  (the integral of the kernel-damped Chebyshev density of states);
* electron count spin * N(x); the Fermi level is the E where it equals the
  target count, found by bisection on x in [-1, 1];
* the scale (a silent point of the paper): alpha from a power iteration on
  S^-1 H from a given start vector (the largest |eps| from below) with a
  safety margin, beta = 0.  For diagonally dominant overlaps a Gershgorin
  bound also serves (used by the pins).

Pins (tests/test_oracle_kpm.py): with the full unit-vector basis as random
vectors the moments equal sum_i T_n(lambda_i) over the generalized
eigenvalues of scipy.linalg.eigh(H, S); the integrated density of states
counts those eigenvalues inside spectral gaps; the Fermi level falls in the
gap that the exact count selects; N(1) = mu_0.
"""
from __future__ import annotations

import numpy as np


def dense_blocks(dev):
    """Dense H and S of the device region (block tridiagonal, upper blocks
    the conjugate transposes of the stored lower blocks)."""
    N, b = dev.n_layers, dev.b
    H = np.zeros((N * b, N * b), dtype=np.complex128)
    S = np.zeros_like(H)
    for i in range(N):
        H[i * b:(i + 1) * b, i * b:(i + 1) * b] = dev.H_diag[i]
        S[i * b:(i + 1) * b, i * b:(i + 1) * b] = dev.S_diag[i]
    for i in range(1, N):
        H[i * b:(i + 1) * b, (i - 1) * b:i * b] = dev.H_lower[i - 1]
        S[i * b:(i + 1) * b, (i - 1) * b:i * b] = dev.S_lower[i - 1]
        H[(i - 1) * b:i * b, i * b:(i + 1) * b] = dev.H_lower[i - 1].conj().T
        S[(i - 1) * b:i * b, i * b:(i + 1) * b] = dev.S_lower[i - 1].conj().T
    return H, S


def moments(H, S, alpha, beta, R, n_mom):
    """mu_n, n < n_mom, for the random vectors in the columns of R (dense
    H, S).  A~ v = S^-1 (H v - beta S v) / alpha by a linear solve with S."""
    apply = lambda V: np.linalg.solve(S, H @ V - beta * (S @ V)) / alpha
    nR = R.shape[1]
    mu = np.empty(n_mom)
    v_prev = R.astype(np.complex128)
    mu[0] = np.real(np.sum(np.conj(R) * v_prev)) / nR
    if n_mom == 1:
        return mu
    v = apply(v_prev)
    mu[1] = np.real(np.sum(np.conj(R) * v)) / nR
    for n in range(2, n_mom):
        v_next = 2.0 * apply(v) - v_prev
        mu[n] = np.real(np.sum(np.conj(R) * v_next)) / nR
        v_prev, v = v, v_next
    return mu


def jackson(n_mom):
    M = n_mom
    n = np.arange(M)
    q = np.pi / (M + 1)
    return ((M - n + 1) * np.cos(q * n) + np.sin(q * n) / np.tan(q)) / (M + 1)


def states_below(mu, x):
    """N(x): kernel-damped integrated density of states below x in [-1, 1]."""
    g = jackson(len(mu))
    theta = np.arccos(np.clip(x, -1.0, 1.0))
    n = np.arange(1, len(mu))
    s = g[0] * mu[0] * (np.pi - theta) / np.pi
    return s - (2.0 / np.pi) * np.sum(g[1:] * mu[1:] * np.sin(n * theta) / n)


def fermi_level(mu, alpha, beta, n_electrons, spin=2.0, iters=200):
    """E_F with spin * N((E_F - beta) / alpha) = n_electrons, by bisection."""
    lo, hi = -1.0, 1.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if spin * states_below(mu, mid) < n_electrons:
            lo = mid
        else:
            hi = mid
    return beta + alpha * 0.5 * (lo + hi)


def gershgorin_scale(H, S, margin=0.01):
    """(alpha, beta) that map every generalized eigenvalue into [-1, 1]:
    |eps| <= rho_H / g_S, rho_H the largest absolute row sum of H and g_S the
    smallest Gershgorin lower bound of S (S must be diagonally dominant
    enough that g_S > 0); beta = 0."""
    rho = np.max(np.sum(np.abs(H), axis=1))
    d = np.real(np.diag(S))
    off = np.sum(np.abs(S), axis=1) - np.abs(np.diag(S))
    g = np.min(d - off)
    if g <= 0:
        raise ValueError("overlap not diagonally dominant: no Gershgorin bound")
    return (1.0 + margin) * rho / g, 0.0


def power_scale(H, S, x0, iters=100, margin=0.05):
    """(alpha, beta): x <- S^-1 H x / |S^-1 H x| from x0, iters steps; the
    last |S^-1 H x| for unit x estimates max |eps|; alpha = (1 + margin) of
    it, beta = 0."""
    x = np.asarray(x0, dtype=np.complex128).reshape(-1)
    x = x / np.linalg.norm(x)
    rho = 0.0
    for _ in range(iters):
        y = np.linalg.solve(S, H @ x)
        rho = np.linalg.norm(y)
        x = y / rho
    return (1.0 + margin) * rho, 0.0
