"""The double-float filter (hi + lo floats, error-free FP32 transformations)
against the FP64 oracle: the filtered FP64 block within 1e-11 relative
Frobenius norm, the same bar as the FP64 kernels."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import paper_1510_04895_gb300 as pkg
from oracle import bounds as obounds, coeffs, filter as ofilt, lattice
from paper_1510_04895_gb300 import workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _lattice(kind, Lx, Ly, Lz, W, seed, **kw):
    H = pkg.chebfd_matrix_create_lattice(kind, Lx, Ly, Lz, t=1.0, m=1.0, W=W, seed=seed,
                                         also_single=True, **kw)
    if kind == "topi":
        csr = lattice.topi_csr(Lx, Ly, Lz, t=1.0, m=1.0, W=W, seed=seed)
    else:
        csr = lattice.graphene_csr(Lx, Ly, t=1.0, W=W, seed=seed)
    return H, lattice.to_scipy(*csr)


def _df_case(H, Ho, nb, Np, kernel, window, xseed=0):
    a, b = obounds.lanczos_bounds(Ho, 30, seed=0)
    alpha, beta = coeffs.scaling(a, b)
    gc = coeffs.filter_coeffs(a, b, window[0], window[1], Np, kernel)
    X0 = workloads.random_block(xseed, H.n, nb, H.is_complex)
    X = torch.from_numpy(X0).to(DEV)
    pkg.chebfd_filter_block_df(H, alpha, beta, gc, X)
    torch.cuda.synchronize()
    return X.cpu().numpy(), ofilt.filter_block(Ho, alpha, beta, gc, X0)


def test_df_filter_smallest_insulator():
    """8x8x8x4, n_b = 64 (two 32-column panels), N_p = 200, Jackson."""
    H, Ho = _lattice("topi", 8, 8, 8, 0.5, 0)
    got, ref = _df_case(H, Ho, 64, 200, "jackson", (-0.1, 0.1))
    assert rel(got, ref) <= 1e-11, rel(got, ref)


@pytest.mark.parametrize("nb,C,sigma", [(4, 1, 1), (36, 4, 1), (2, 8, 16), (18, 2, 1)])
def test_df_filter_ragged_panels_and_orders(nb, C, sigma):
    H, Ho = _lattice("topi", 3, 5, 7, 1.2, 5, sell_C=C, sell_sigma=sigma)
    got, ref = _df_case(H, Ho, nb, 37, "lanczos", (-0.3, 0.4))
    assert rel(got, ref) <= 1e-11, rel(got, ref)


@pytest.mark.parametrize("nb", [64, 80, 2])
def test_df_filter_graphene_real(nb):
    H, Ho = _lattice("graphene", 20, 17, 1, 1.0, 2)
    got, ref = _df_case(H, Ho, nb, 150, "lanczos", (-0.2, 0.2))
    assert rel(got, ref) <= 1e-11, rel(got, ref)


def test_df_filter_variable_row_lengths():
    """A random Hermitian matrix with rows of 1..20 entries (generic SELL path)."""
    rs = np.random.default_rng(11)
    n = 700
    A = sp.random(n, n, density=0.012, random_state=rs, format="csr")
    A = A + 1j * sp.random(n, n, density=0.012, random_state=rs, format="csr")
    Hs = (A + A.conj().T + sp.diags(rs.uniform(-1, 1, n))).tocsr()
    Hs.sort_indices()
    H = pkg.chebfd_matrix_create_csr(Hs.indptr.astype(np.int64), Hs.indices.astype(np.int32),
                                     Hs.data.astype(np.complex128), sell_C=4, sell_sigma=32,
                                     also_single=True)
    got, ref = _df_case(H, Hs, 24, 80, "lanczos", (-0.2, 0.3))
    assert rel(got, ref) <= 1e-11, rel(got, ref)


def test_df_filter_diagonal_closed_form():
    """T_n(cos t) = cos(n t) on a diagonal matrix: entry-wise closed form."""
    D = 4096
    lam = lattice.linear_dos_eigs(D)
    rp, c, v = lattice.diagonal_csr(lam)
    H = pkg.chebfd_matrix_create_csr(rp, c, v, also_single=True)
    gc = coeffs.filter_coeffs(-1.0, 1.0, -0.05, 0.05, 300, "lanczos")
    X0 = workloads.random_block(3, D, 8, False)
    X = torch.from_numpy(X0).to(DEV)
    pkg.chebfd_filter_block_df(H, 1.0, 0.0, gc, X)
    p = np.cos(np.outer(np.arccos(lam), np.arange(301))) @ gc
    assert np.abs(X.cpu().numpy() - p[:, None] * X0).max() <= 1e-12 * np.abs(gc).sum()


def test_df_filter_full_size_insulator():
    """64x64x32x4 (N = 524288), n_b = 32, N_p = 6: within 1e-11 of the oracle."""
    w = workloads.TOPI_MEDIUM
    H, Ho = _lattice("topi", w["Lx"], w["Ly"], w["Lz"], w["W"], w["seed"])
    got, ref = _df_case(H, Ho, 32, 6, "lanczos", (-0.1, 0.1))
    assert rel(got, ref) <= 1e-11, rel(got, ref)


def test_df_filter_needs_the_single_copy():
    H = pkg.chebfd_matrix_create_lattice("topi", 3, 3, 3, W=0.5, seed=0)
    X = torch.zeros((H.n, 8), dtype=torch.complex128, device=DEV)
    with pytest.raises(pkg.ChebFDError):
        pkg.chebfd_filter_block_df(H, 0.2, 0.0, np.ones(5), X)


@pytest.mark.parametrize("blocked", [True, False])
def test_df_filter_slab_blocked_and_sell(blocked):
    """Eq. Ham slab: the blocked double-float step (site blocks, padded at
    the open surfaces) and the SELL one both within 1e-11 of the oracle."""
    H = pkg.chebfd_matrix_create_lattice("topi_slab", 5, 6, 4, t=1.0, m=2.0, W=2.0, seed=2,
                                         also_single=True)
    assert H.blocked_width == 7
    H.set_blocked(blocked)
    Ho = lattice.to_scipy(*lattice.topi_slab_csr(5, 6, 4, t=1.0, m=2.0, W=2.0, seed=2))
    got, ref = _df_case(H, Ho, 40, 90, "lanczos", (-0.06, 0.06))
    assert rel(got, ref) <= 1e-11, rel(got, ref)


@pytest.mark.parametrize("kind,L,t,nb", [("topi", (6, 5, 4), 1.0, 40), ("topi", (2, 3, 2), 0.7, 3),
                                         ("topi_slab", (5, 6, 4), 1.1, 32),
                                         ("topi_slab", (4, 4, 1), 1.0, 17)])
def test_df_filter_matrix_free(kind, L, t, nb):
    """The double-float step with H's entries rebuilt in registers (hopping
    t/2 split into hi + lo, onsite + beta/alpha summed in FP64 and split):
    within 1e-11 of the oracle and of the stored-matrix double-float filter,
    on both lattices, a ragged second panel and edges 1-2 (coinciding
    neighbours); t = 0.7, 1.1 have no exact float."""
    m = 2.0 if kind == "topi_slab" else 1.0
    H = pkg.chebfd_matrix_create_lattice(kind, *L, t=t, m=m, W=1.3, seed=4, also_single=True)
    gen = lattice.topi_slab_csr if kind == "topi_slab" else lattice.topi_csr
    Ho = lattice.to_scipy(*gen(*L, t=t, m=m, W=1.3, seed=4))
    H.set_matrix_free(True)
    got, ref = _df_case(H, Ho, nb, 60, "lanczos", (-0.08, 0.08))
    assert rel(got, ref) <= 1e-11, rel(got, ref)
    H.set_matrix_free(False)
    stored, _ = _df_case(H, Ho, nb, 60, "lanczos", (-0.08, 0.08))
    assert rel(got, stored) <= 1e-11, rel(got, stored)
