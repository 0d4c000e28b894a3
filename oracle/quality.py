"""Filter quality analysis of Sec. 2.3 and the effort model of Sec. 2.4.

sigma(N_p) = max_{x in [a,b] \\ I_S} |p(x)| / min_{x in I_T} |p(x)|   (Sec. 2.3)
eta(N_p)   = -N_p / log10 sigma                                   (Sec. 2.3)
N_iter     ~ log10 eps / log10 sigma                              (Sec. 2.3)

p is evaluated on a uniform theta grid (x = cos theta) with 32 points per
period 2 pi / N_p through a DCT-III of the coefficients, plus exact sums at the
interval end points; the optimal N_p is an integer search (coarse scan, then
every integer near the coarse minimum).
"""
import numpy as np
import scipy.fft

from . import coeffs


def _poly_on_grid(gc, M):
    """p(cos theta_j) at theta_j = pi (j + 1/2) / M, j = 0..M-1 (DCT-III)."""
    x = np.zeros(M)
    x[0] = gc[0]
    x[1:len(gc)] = 0.5 * gc[1:]
    return scipy.fft.dct(x, type=3)


def damping_sigma(Np, delta, delta_p, c=0.0, a=-1.0, b=1.0, kind="lanczos", mu=2.0,
                  per_period=64, inset=0.0):
    """sigma for I_T = [c-delta, c+delta], I_S = [c-delta-delta', c+delta+delta'];
    p sampled at ``per_period`` points per theta period 2 pi / N_p.  The window
    of p is I_T narrowed by ``inset`` of its half-width (0: I_T itself)."""
    lo, hi = c - delta, c + delta
    w = (1.0 - inset) * delta
    gc = coeffs.filter_coeffs(a, b, c - w, c + w, Np, kind, mu)
    alpha, beta = coeffs.scaling(a, b)
    M = max(per_period * Np // 2, 4096)
    pg = _poly_on_grid(gc, M)
    xg = np.cos(np.pi * (np.arange(M) + 0.5) / M)
    x_lo, x_hi = alpha * lo + beta, alpha * hi + beta
    s_lo, s_hi = alpha * (lo - delta_p) + beta, alpha * (hi + delta_p) + beta
    ends = coeffs.eval_poly(gc, np.array([x_lo, x_hi, s_lo, s_hi, -1.0, 1.0]))
    inside = np.abs(pg[(xg >= x_lo) & (xg <= x_hi)])
    pmin = min(inside.min() if inside.size else np.inf, abs(ends[0]), abs(ends[1]))
    outside = np.abs(pg[(xg < s_lo) | (xg > s_hi)])
    pmax = max(outside.max() if outside.size else 0.0, abs(ends[2]), abs(ends[3]),
               abs(ends[4]), abs(ends[5]))
    return pmax / pmin


def eta(Np, delta, delta_p, **kw):
    s = damping_sigma(Np, delta, delta_p, **kw)
    if not s < 1.0:
        return np.inf
    return -Np / np.log10(s)


def optimal_Np(delta, delta_p, n_lo=None, n_hi=None, ratio=1.003, keep=6, **kw):
    """(N_p^opt, eta^opt): integer minimiser of eta (Sec. 2.3, Fig. polyeff1).

    eta(N_p) has narrow cusps (the maximiser of |p| outside I_S jumps between
    side lobes), so the coarse scan is a fine geometric grid at 16 points per
    period, and every integer around its ``keep`` best local minima is then
    evaluated at 64 points per period."""
    S_w = (kw.get("b", 1.0) - kw.get("a", -1.0)) / 2.0
    guess = 6.0 * S_w / delta_p
    n_lo = n_lo or max(4, int(0.1 * guess))
    n_hi = n_hi or int(3.0 * guess) + 8
    count = int(np.log(n_hi / n_lo) / np.log(ratio)) + 2
    grid = np.unique(np.round(np.geomspace(n_lo, n_hi, count)).astype(int))
    vals = np.array([eta(int(n), delta, delta_p, per_period=16, **kw) for n in grid])
    interior = [k for k in range(len(grid))
                if vals[k] <= vals[max(k - 1, 0)] and vals[k] <= vals[min(k + 1, len(grid) - 1)]]
    interior.sort(key=lambda k: vals[k])
    best_n, best_e = None, np.inf
    for k in interior[:keep]:
        lo = grid[max(k - 2, 0)]
        hi = grid[min(k + 2, len(grid) - 1)]
        for n in range(int(lo), int(hi) + 1):
            e = eta(n, delta, delta_p, **kw)
            if e < best_e:
                best_n, best_e = n, e
    return best_n, float(best_e)


def n_iter_estimate(eps, sigma):
    """N_iter ~ log10 eps / log10 sigma (Sec. 2.3)."""
    return np.log10(eps) / np.log10(sigma)


def effort_flat(eta0, S_w, delta, N_T, N_S):
    """eta N_S for a flat DOS, Eq. etanflat."""
    return eta0 * S_w / delta * N_T / (1.0 - N_T / N_S)


def effort_linear(eta0, S_w, delta, N_T, N_S):
    """eta N_S for a linear DOS, Eq. etanlinear (minimal at N_S = 4 N_T)."""
    r = np.sqrt(N_S / N_T)
    return eta0 * S_w / delta * N_T * r / (1.0 - 1.0 / r)


def margin_flat(N_S, N_T):
    """delta'/delta = N_S/N_T - 1 for a flat DOS (Sec. 2.4)."""
    return N_S / N_T - 1.0


def margin_linear(N_S, N_T):
    """delta'/delta = sqrt(N_S/N_T) - 1 for a linear DOS (Sec. 2.4)."""
    return np.sqrt(N_S / N_T) - 1.0
