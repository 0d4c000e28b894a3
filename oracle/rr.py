"""Rayleigh-Ritz projection and residuals (Sec. 3.1 step 7) - oracle side.

For an orthonormal basis Y: G = Y^H (H Y), symmetrised (G + G^H)/2, eigenpairs
(theta_k, s_k) in ascending order; Ritz vectors V = Y S; residual norms
r_k = ||H v_k - theta_k v_k|| formed as ||(H Y) s_k - theta_k Y s_k||, which
needs no further product with H.
"""
import numpy as np


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
