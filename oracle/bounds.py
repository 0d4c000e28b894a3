"""Spectral interval [a, b] from a short Lanczos run (Sec. 3.1 step 1, 20-30
steps preferred over Gershgorin) - oracle side.

The paper does not state the start vector or a safety margin.  Reading taken:
m Lanczos steps in FP64 with full reorthogonalisation from a start vector of
SplitMix64 stream 4 (entries 2u-1, real and imaginary parts at word indices
2i, 2i+1); Ritz values theta_i with residual bounds rho_i = |beta_m s_{m,i}|;
a = theta_min - rho_min, b = theta_max + rho_max; then widened by 1% of b - a on
each side and clamped to the Gershgorin interval.  ||H|| := max(|a|, |b|)
(Sec. 3.1 step 8).
"""
import numpy as np

from . import rng

STREAM_LANCZOS = 4


def start_vector(seed, D, complex_values):
    if complex_values:
        u = rng.uniform(seed, STREAM_LANCZOS, np.arange(2 * D, dtype=np.uint64))
        v = (2.0 * u[0::2] - 1.0) + 1j * (2.0 * u[1::2] - 1.0)
    else:
        u = rng.uniform(seed, STREAM_LANCZOS, np.arange(D, dtype=np.uint64))
        v = 2.0 * u - 1.0
    return v


def gershgorin(H):
    Hc = H.tocsr()
    d = Hc.diagonal()
    radius = np.asarray(abs(Hc).sum(axis=1)).ravel() - np.abs(d)
    return float(np.min(np.real(d) - radius)), float(np.max(np.real(d) + radius))


def lanczos_bounds(H, steps=30, seed=0, margin=0.01):
    D = H.shape[0]
    cplx = np.iscomplexobj(H.data)
    v = start_vector(seed, D, cplx)
    v = v / np.linalg.norm(v)
    V = [v]
    alphas, betas = [], []
    m = min(steps, D)
    for j in range(m):
        w = H @ V[j]
        a_j = np.real(np.vdot(V[j], w))
        w = w - a_j * V[j]
        if j > 0:
            w = w - betas[j - 1] * V[j - 1]
        Vm = np.array(V).T
        w = w - Vm @ (Vm.conj().T @ w)                  # full reorthogonalisation
        b_j = np.linalg.norm(w)
        alphas.append(a_j)
        betas.append(b_j)
        if b_j == 0.0 or j == m - 1:
            break
        V.append(w / b_j)
    k = len(alphas)
    T = np.diag(alphas) + np.diag(betas[:k - 1], 1) + np.diag(betas[:k - 1], -1)
    theta, S = np.linalg.eigh(T)
    rho = np.abs(betas[k - 1] * S[k - 1, :])
    a = theta[0] - rho[0]
    b = theta[-1] + rho[-1]
    width = b - a
    a -= margin * width
    b += margin * width
    g_lo, g_hi = gershgorin(H)
    return max(a, g_lo), min(b, g_hi)


def norm_from_bounds(a, b):
    return max(abs(a), abs(b))
