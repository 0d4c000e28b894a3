"""Kernel polynomial method with stochastic trace (Sec. 3.1 step 1-2; method of
Weisse, Wellein, Alvermann, Fehske, Rev. Mod. Phys. 78 (2006), cited as WWAF06).

Normalised moments  mu_n = Tr T_n(A) / D ~ (1/(R D)) sum_r <r, T_n(A) r>
with R probe vectors r whose entries are independent with E[r r^H] = 1:
real entries s = +-1 (bit 0 of the SplitMix64 word), complex entries
(s0 + i s1)/sqrt(2) (bits 0 and 1), stream 2, word index i*R + r.

The eigenvalue count inside [lam_lo, lam_hi] (Eq. DOS:target) is the integral
of the damped expansion rho(x) = (g_0 mu_0 + 2 sum g_n mu_n T_n(x)) /
(pi sqrt(1-x^2)) over the scaled window, which equals D sum_n g_n mu_n c_n with
the window coefficients c_n of Sec. 2.1.  The Jackson factors for M moments
are those of Tab. Kernel with N_p = M + 1 (the form of WWAF06).
"""
import numpy as np

from . import coeffs, filter as filt, rng


def probe_vectors(seed, D, R, complex_values):
    idx = (np.arange(D, dtype=np.uint64)[:, None] * np.uint64(R)
           + np.arange(R, dtype=np.uint64)[None, :])
    w = rng.words(seed, rng.STREAM_KPM, idx)
    s0 = 1.0 - 2.0 * (w & np.uint64(1)).astype(np.float64)
    if not complex_values:
        return s0
    s1 = 1.0 - 2.0 * ((w >> np.uint64(1)) & np.uint64(1)).astype(np.float64)
    return (s0 + 1j * s1) * (1.0 / np.sqrt(2.0))


def moments(H, alpha, beta, M, R, seed, complex_values):
    """mu_0..mu_{M-1}, the stochastic trace estimate of Tr T_n(A)/D; the
    recurrence T_{n+1} = 2 A T_n - T_{n-1} is run once, keeping two vectors."""
    D = H.shape[0]
    r = probe_vectors(seed, D, R, complex_values)
    per = np.zeros((M, R))
    t_prev, t_cur = None, r
    for n in range(M):
        per[n] = np.real(np.sum(np.conj(r) * t_cur, axis=0))
        if n == 0:
            t_prev, t_cur = t_cur, filt.apply_A(H, alpha, beta, r)
        else:
            t_prev, t_cur = t_cur, 2.0 * filt.apply_A(H, alpha, beta, t_cur) - t_prev
    return per.sum(axis=1) / (R * D)


def jackson_kpm(M):
    return coeffs.kernel_gn("jackson", M + 1)[:M]


def count_in_window(mu, D, a, b, lam_lo, lam_hi, g=None):
    """Estimated N_T of Eq. DOS:target: D sum_n g_n mu_n c_n."""
    M = len(mu)
    g = jackson_kpm(M) if g is None else g
    c = coeffs.window_cn(a, b, lam_lo, lam_hi, M - 1)
    return D * float(np.sum(g * mu * c))


def dos(mu, D, a, b, lam, g=None):
    """rho(lambda) in states per unit lambda (for plots and checks)."""
    M = len(mu)
    g = jackson_kpm(M) if g is None else g
    alpha, beta = coeffs.scaling(a, b)
    x = np.clip(alpha * np.asarray(lam) + beta, -1 + 1e-15, 1 - 1e-15)
    th = np.arccos(x)
    n = np.arange(M)
    w = np.where(n == 0, 1.0, 2.0) * g * mu
    series = np.cos(np.multiply.outer(th, n)) @ w
    return D * alpha * series / (np.pi * np.sqrt(1.0 - x * x))
