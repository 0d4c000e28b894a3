"""Filter polynomial construction, Sec. 2.1 (Eq. W1, Eq. W2, Tab. Kernel).

Reading of the printed closed form for c_n (Sec. 2.1): with
theta(l) = arccos(alpha l + beta) and theta_lo = theta(lambda_lo) >
theta_hi = theta(lambda_hi), the integral of the rectangular window W against
T_n with weight (1-x^2)^(-1/2) gives

    c_0 = (theta_lo - theta_hi) / pi
    c_n = 2 / (pi n) (sin(n theta_lo) - sin(n theta_hi))      (n >= 1)

which is the printed expression with the overall sign reversed; the printed
sign would make p(x) ~ -1 inside the window, contradicting p ~ 1 there
(Sec. 2.2).  The sign does not change span{p[H] x_k}.  Arguments of arccos
are clamped to [-1, 1].
"""
import numpy as np

KERNELS = ("none", "fejer", "jackson", "lanczos")


def scaling(a, b):
    """alpha = 2/(b-a), beta = (a+b)/(a-b) of Eq. W1, mapping [a,b] onto [-1,1]."""
    if not b > a:
        raise ValueError("need b > a")
    return 2.0 / (b - a), (a + b) / (a - b)


def window_cn(a, b, lam_lo, lam_hi, Np):
    """Chebyshev coefficients c_0..c_Np of the rectangular window (Sec. 2.1)."""
    alpha, beta = scaling(a, b)
    th_lo = np.arccos(np.clip(alpha * lam_lo + beta, -1.0, 1.0))
    th_hi = np.arccos(np.clip(alpha * lam_hi + beta, -1.0, 1.0))
    n = np.arange(Np + 1, dtype=np.float64)
    c = np.empty(Np + 1)
    c[0] = (th_lo - th_hi) / np.pi
    c[1:] = 2.0 / (np.pi * n[1:]) * (np.sin(n[1:] * th_lo) - np.sin(n[1:] * th_hi))
    return c


def kernel_gn(kind, Np, mu=2.0):
    """Damping factors g_0..g_Np of Tab. Kernel ('none' = all ones, Sec. 2.3)."""
    n = np.arange(Np + 1, dtype=np.float64)
    if kind == "none":
        return np.ones(Np + 1)
    if kind == "fejer":
        return (Np - n + 1.0) / (Np + 1.0)
    if kind == "jackson":
        q = np.pi / Np
        return ((Np - n) * np.cos(q * n) + np.sin(q * n) / np.tan(q)) / Np
    if kind == "lanczos":
        g = np.ones(Np + 1)
        arg = np.pi * n[1:] / (Np + 1.0)
        g[1:] = (np.sin(arg) / arg) ** mu
        return g
    raise ValueError(kind)


def filter_coeffs(a, b, lam_lo, lam_hi, Np, kind="lanczos", mu=2.0):
    """gc[n] = g_n c_n, n = 0..Np: the coefficients of p(x) in Eq. W2."""
    return kernel_gn(kind, Np, mu) * window_cn(a, b, lam_lo, lam_hi, Np)


def eval_poly(gc, x):
    """p(x) = sum_n gc[n] T_n(x) for x in [-1, 1], T_n(cos t) = cos(n t) (Sec. 2.1)."""
    th = np.arccos(np.clip(np.asarray(x, dtype=np.float64), -1.0, 1.0))
    n = np.arange(len(gc), dtype=np.float64)
    return np.cos(np.multiply.outer(th, n)) @ gc
