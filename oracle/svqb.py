"""Rank-revealing SVQB orthonormalisation (Sec. 3.1 step 6; method of
Stathopoulos and Wu, SIAM J. Sci. Comput. 23 (2002)) - oracle side.

The paper names SVQB and asks for refilling the search space with new random
vectors when orthogonalisation reduces its size, but gives no steps.  Reading:
  1. S = Y^H Y (FP64; the paper's Kahan-summed dot products are an accuracy
     device for long vectors, the oracle forms the plain FP64 product);
  2. D = diag(S)^(-1/2) (a zero column gets d = 0);
  3. D S D = U Theta U^H (dense Hermitian eigensolver);
  4. directions with Theta_i < n_s 2^-52 max Theta are dropped;
  5. Y <- Y D U Theta^(-1/2) over the kept directions; dropped directions are
     replaced by fresh random vectors (SplitMix64 stream 3, the q-th refill
     column of the run takes word indices q*N + i, x2 for complex parts);
  6. repeat (at most 3 passes) while refilled or while max|Y^H Y - I| > 1e-12.
"""
import numpy as np

from . import rng


def refill_vectors(seed, D, first, count, complex_values):
    cols = []
    for q in range(first, first + count):
        if complex_values:
            idx = np.uint64(2 * q * D) + np.arange(2 * D, dtype=np.uint64)
            u = rng.uniform(seed, rng.STREAM_REFILL, idx)
            cols.append((2 * u[0::2] - 1) + 1j * (2 * u[1::2] - 1))
        else:
            idx = np.uint64(q * D) + np.arange(D, dtype=np.uint64)
            cols.append(2 * rng.uniform(seed, rng.STREAM_REFILL, idx) - 1)
    return np.array(cols).T


def svqb(Y, seed=0, refill_counter=0, max_pass=3, tol=1e-12):
    """Return (Q, rank of the first pass, updated refill counter)."""
    Y = np.array(Y, copy=True)
    D, ns = Y.shape
    cplx = np.iscomplexobj(Y)
    first_rank = None
    for _ in range(max_pass):
        S = Y.conj().T @ Y
        diag = np.real(np.diag(S))
        d = np.where(diag > 0, 1.0 / np.sqrt(np.where(diag > 0, diag, 1.0)), 0.0)
        DSD = d[:, None] * S * d[None, :]
        DSD = 0.5 * (DSD + DSD.conj().T)
        theta, U = np.linalg.eigh(DSD)
        keep = theta >= ns * 2.0 ** -52 * theta.max()
        r = int(keep.sum())
        if first_rank is None:
            first_rank = r
        Y = Y @ (d[:, None] * U[:, keep] / np.sqrt(theta[keep])[None, :])
        if r < ns:
            Y = np.concatenate([Y, refill_vectors(seed, D, refill_counter, ns - r, cplx)], axis=1)
            refill_counter += ns - r
            continue
        err = np.abs(Y.conj().T @ Y - np.eye(ns)).max()
        if err <= tol:
            break
    return Y, first_rank, refill_counter
