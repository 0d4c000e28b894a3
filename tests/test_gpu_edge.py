"""Degenerate and edge inputs of the CUDA path against the oracle and dense
diagonalisation: the minimum degree N_p = 2 (only the two start steps run),
matrices smaller than one SELL chunk (1, 3, 5 and 17 rows against C = 1..32
and sorting windows sigma up to 16), single-column complex blocks, a search
space as large as the matrix, and a window at the lower edge of the
spectrum (an exterior window)."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import paper_1510_04895_gb300 as pkg
from oracle import coeffs, filter as ofilt

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _random_hermitian(n, cplx, seed, density=0.5):
    rs = np.random.default_rng(seed)
    A = rs.uniform(-1, 1, (n, n)) * (rs.uniform(0, 1, (n, n)) < density)
    if cplx:
        A = A + 1j * rs.uniform(-1, 1, (n, n)) * (rs.uniform(0, 1, (n, n)) < density)
    A = A + A.conj().T + np.diag(rs.uniform(-1, 1, n))
    return sp.csr_matrix(A)


@pytest.mark.parametrize("n,C,sigma", [(1, 1, 1), (3, 4, 8), (5, 32, 1), (17, 8, 16)])
@pytest.mark.parametrize("cplx,nb", [(True, 1), (True, 3), (False, 2), (False, 6)])
@pytest.mark.parametrize("Np", [2, 3])
def test_filter_tiny_matrices_minimum_degree(n, C, sigma, cplx, nb, Np):
    Hs = _random_hermitian(n, cplx, seed=n * 10 + nb)
    Hs.sort_indices()
    H = pkg.chebfd_matrix_create_csr(Hs.indptr.astype(np.int64), Hs.indices.astype(np.int32),
                                     Hs.data, sell_C=C, sell_sigma=sigma)
    bound = float(np.abs(Hs.toarray()).sum(axis=1).max()) + 0.1     # Gershgorin
    alpha, beta = coeffs.scaling(-bound, bound)
    gc = coeffs.filter_coeffs(-bound, bound, -0.2, 0.3, Np, "lanczos")
    rs = np.random.default_rng(3)
    X0 = rs.uniform(-1, 1, (n, nb)) + (1j * rs.uniform(-1, 1, (n, nb)) if cplx else 0)
    X = torch.from_numpy(X0).to(DEV)
    pkg.chebfd_filter_block(H, alpha, beta, gc, X)
    ref = ofilt.filter_block(Hs, alpha, beta, gc, X0)
    got = X.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())


def test_solve_search_space_as_large_as_the_matrix():
    """n_s = N = 48 (diagonal H): the filtered block spans the whole space, so
    Rayleigh-Ritz is exact; every eigenvalue of the window is found."""
    lam = np.linspace(-1.0, 1.0, 48)
    Hs = sp.diags(lam).tocsr()
    Hs.sort_indices()
    H = pkg.chebfd_matrix_create_csr(Hs.indptr.astype(np.int64), Hs.indices.astype(np.int32),
                                     Hs.data)
    r = pkg.chebfd_solve(H, -0.3, 0.3, 48, 20, eps=1e-10, kernel="lanczos", a=-1.01, b=1.01)
    exact = lam[np.abs(lam) <= 0.3]
    assert r["converged"] and r["nev"] == len(exact)
    assert np.abs(np.sort(r["lam"]) - exact).max() <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed_df"])
def test_solve_window_at_the_lower_edge_of_the_spectrum(precision):
    """An exterior window [-1.05, -0.9] on a flat-spectrum diagonal (D = 400):
    the lowest 20 eigenvalues, found to 1e-9 ||H|| by both precisions."""
    D = 400
    lam = -1.0 + 2.0 * np.arange(D) / (D - 1)
    Hs = sp.diags(lam).tocsr()
    Hs.sort_indices()
    H = pkg.chebfd_matrix_create_csr(Hs.indptr.astype(np.int64), Hs.indices.astype(np.int32),
                                     Hs.data, also_single=True)
    r = pkg.chebfd_solve(H, -1.05, -0.9, 64, 120, eps=1e-9, kernel="lanczos", a=-1.01, b=1.01,
                         precision=precision, max_iter=40)
    exact = lam[(lam >= -1.05) & (lam <= -0.9)]
    assert len(exact) == 20
    assert r["converged"] and r["nev"] == len(exact)
    assert np.abs(np.sort(r["lam"]) - exact).max() <= 1e-9 * 1.01
