"""Polynomial filter application, Fig. ChebFD (Sec. 3.1 step 5) - oracle side.

The block X (N x n_b) is replaced by p[H] X = sum_n gc[n] T_n(alpha H + beta) X
through the three-term recurrence of Sec. 2.1, in exactly the step order of
Fig. ChebFD: two start steps, then N_p - 2 steps that each apply
A = alpha H + beta once and add gc[n] w to the accumulated block.  A u is
evaluated as alpha (H u) + beta u, with H u a CSR product (ascending columns).

The Chebyshev moments of Sec. 4, mu_n[k] = <x_k, T_n(A) x_k>, are computed
here literally from their definition (the original x_k kept aside), for
n = 0 .. 2 N_p - 1.
"""
import numpy as np


def apply_A(H, alpha, beta, v):
    """(alpha H + beta 1) v."""
    return alpha * (H @ v) + beta * v


def filter_block(H, alpha, beta, gc, X):
    """Return p[H] X following Fig. ChebFD; H is a scipy CSR matrix."""
    Np = len(gc) - 1
    if Np < 2:
        raise ValueError("Fig. ChebFD needs N_p >= 2")
    x = np.array(X, copy=True)
    u = apply_A(H, alpha, beta, x)                 # u = A x
    w = 2.0 * apply_A(H, alpha, beta, u) - x       # w = 2 A u - x
    x = gc[0] * x + gc[1] * u + gc[2] * w          # x = g0c0 x + g1c1 u + g2c2 w
    for n in range(3, Np + 1):
        u, w = w, u                                # swap(w, u)
        w = 2.0 * apply_A(H, alpha, beta, u) - w   # w = 2 A u - w
        x = x + gc[n] * w                          # x = x + gn cn w
    return x


def chebyshev_vectors(H, alpha, beta, X, nmax):
    """T_0(A) X .. T_nmax(A) X by the recurrence T_{n+1} = 2 A T_n - T_{n-1}."""
    out = [np.array(X, copy=True)]
    if nmax >= 1:
        out.append(apply_A(H, alpha, beta, out[0]))
    for _ in range(2, nmax + 1):
        out.append(2.0 * apply_A(H, alpha, beta, out[-1]) - out[-2])
    return out


def moments(H, alpha, beta, X, count):
    """mu_n[k] = Re <x_k, T_n(A) x_k>, n = 0..count-1 (Sec. 4): array count x n_b."""
    T = chebyshev_vectors(H, alpha, beta, X, count - 1)
    return np.array([np.real(np.sum(np.conj(X) * Tn, axis=0)) for Tn in T])
