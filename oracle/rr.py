"""Rayleigh-Ritz projection and residuals (Sec. 3.1 step 7) - oracle side.

For an orthonormal basis Y: G = Y^H (H Y), symmetrised (G + G^H)/2, eigenpairs
(theta_k, s_k) in ascending order; Ritz vectors V = Y S; residual norms
r_k = ||H v_k - theta_k v_k|| formed as ||(H Y) s_k - theta_k Y s_k||, which
needs no further product with H.

Harmonic Ritz extraction (the alternative named in Sec. 3.1 step 7 and
Sec. 6, after Morgan 1991 and Paige, Parlett, van der Vorst 1995), with a
target tau (the window centre): with Z = (H - tau) Y, the pairs (mu_k, s_k) of
the Hermitian-definite problem (Y^H Z) s = mu (Z^H Z) s give the harmonic Ritz
values tau + 1/mu_k (equivalently: the Ritz values of (H - tau)^-1 on the
subspace Z spans, inverted and shifted back).  Reading: the eigenvalue
estimate of a harmonic vector v_k = Y s_k / ||Y s_k|| is its Rayleigh quotient
rho_k = v_k^H H v_k, its residual ||H v_k - rho_k v_k||; pairs are ordered by
ascending rho.  When Z^H Z is not positive definite (a basis vector is an
exact eigenvector at tau) the ordinary Ritz pairs are returned instead.
"""
import numpy as np
import scipy.linalg


def rayleigh_ritz(H, Y):
    HY = H @ Y
    G = Y.conj().T @ HY
    G = 0.5 * (G + G.conj().T)
    theta, S = np.linalg.eigh(G)
    V = Y @ S
    HV = HY @ S
    res = np.linalg.norm(HV - V * theta[None, :], axis=0)
    return theta, V, res


def residual_norms(H, V, theta):
    """||H v_k - theta_k v_k|| for given pairs (one product with H)."""
    return np.linalg.norm(H @ V - V * np.asarray(theta)[None, :], axis=0)


def harmonic_ritz(H, Y, tau):
    """(rho, V, res, theta_h) for an orthonormal basis Y and target tau: Rayleigh
    quotients, unit harmonic Ritz vectors, residual norms, harmonic Ritz values
    tau + 1/mu; ascending rho."""
    HY = H @ Y
    Z = HY - tau * Y
    G = Y.conj().T @ Z
    G = 0.5 * (G + G.conj().T)
    K = Z.conj().T @ Z
    K = 0.5 * (K + K.conj().T)
    try:
        mu, S = scipy.linalg.eigh(G, K)
    except np.linalg.LinAlgError:
        theta, V, res = rayleigh_ritz(H, Y)
        return theta, V, res, theta.copy()
    S = S / np.linalg.norm(Y @ S, axis=0)[None, :]
    V = Y @ S
    HV = HY @ S
    rho = np.real(np.sum(V.conj() * HV, axis=0))
    order = np.argsort(rho, kind="stable")
    rho, V, HV, mu = rho[order], V[:, order], HV[:, order], mu[order]
    res = np.linalg.norm(HV - V * rho[None, :], axis=0)
    with np.errstate(divide="ignore"):
        theta_h = tau + 1.0 / mu
    return rho, V, res, theta_h

