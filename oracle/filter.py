"""Polynomial filter application (Sec. 2.1, Sec. 3.1 step 5) - oracle side.

The block X (N x n_b) is replaced by p[H] X = sum_{n=0}^{N_p} gc[n] T_n(A) X with
A = alpha H + beta, the Chebyshev polynomials of A applied to X by their
three-term recurrence T_0 = 1, T_1(A) = A, T_{n+1}(A) = 2 A T_n(A) - T_{n-1}(A).
Each T_n(A) X costs one product with A and is added to the sum as soon as it
exists (ascending n, the order the filter of Fig. ChebFD uses), so only the
two latest vectors are kept.  A v is evaluated as alpha (H v) + beta v, with
H v a CSR product (ascending columns).

The Chebyshev moments of Sec. 4, mu_n[k] = <x_k, T_n(A) x_k>, are computed
here literally from their definition (the original x_k kept aside), for
n = 0 .. 2 N_p - 1.
"""
import numpy as np


def apply_A(H, alpha, beta, v):
    """(alpha H + beta 1) v."""
    return alpha * (H @ v) + beta * v


def filter_block(H, alpha, beta, gc, X):
    """Return sum_n gc[n] T_n(A) X (Sec. 2.1); H is a scipy CSR matrix, N_p >= 2."""
    Np = len(gc) - 1
    if Np < 2:
        raise ValueError("the filter needs N_p >= 2")
    t_prev = np.array(X, copy=True)                 # T_0(A) X
    t_cur = apply_A(H, alpha, beta, t_prev)         # T_1(A) X
    y = gc[0] * t_prev + gc[1] * t_cur
    for n in range(2, Np + 1):
        t_prev, t_cur = t_cur, 2.0 * apply_A(H, alpha, beta, t_cur) - t_prev   # T_n(A) X
        y = y + gc[n] * t_cur
    return y


def chebyshev_vectors(H, alpha, beta, X, nmax):
    """T_0(A) X .. T_nmax(A) X by the recurrence T_{n+1} = 2 A T_n - T_{n-1}."""
    out = [np.array(X, copy=True)]
    if nmax >= 1:
        out.append(apply_A(H, alpha, beta, out[0]))
    for _ in range(2, nmax + 1):
        out.append(2.0 * apply_A(H, alpha, beta, out[-1]) - out[-2])
    return out


def moments(H, alpha, beta, X, count):
    """mu_n[k] = Re <x_k, T_n(A) x_k>, n = 0..count-1 (Sec. 4): array count x n_b.
    T_n(A) X from the recurrence, keeping only the two latest blocks."""
    X = np.asarray(X)
    out = np.zeros((count, X.shape[1]))
    t_prev, t_cur = None, np.array(X, copy=True)
    for n in range(count):
        out[n] = np.real(np.sum(np.conj(X) * t_cur, axis=0))
        if n + 1 == count:
            break
        if n == 0:
            t_prev, t_cur = t_cur, apply_A(H, alpha, beta, X)
        else:
            t_prev, t_cur = t_cur, 2.0 * apply_A(H, alpha, beta, t_cur) - t_prev
    return out
