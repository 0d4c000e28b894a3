"""The blocked-ELL copy and its complex64 Chebyshev step (4 rows of a lattice
site computed together) against the FP64 oracle and against the SELL kernel."""
import numpy as np
import pytest
import torch

import paper_1510_04895_gb300 as pkg
from oracle import coeffs, filter as ofilt, lattice
from paper_1510_04895_gb300 import workloads

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_blocked_copy_only_for_its_shape():
    topi = dict(t=1.0, m=1.0, W=0.5, seed=1)
    assert pkg.chebfd_matrix_create_lattice("topi", 4, 3, 5, also_single=True,
                                            **topi).blocked_width == 7
    # no single-precision copy, a sigma-sorted row order, or a real matrix: none
    assert pkg.chebfd_matrix_create_lattice("topi", 4, 3, 5, **topi).blocked_width == 0
    assert pkg.chebfd_matrix_create_lattice("topi", 4, 3, 5, sell_sigma=8, also_single=True,
                                            **topi).blocked_width == 0
    assert pkg.chebfd_matrix_create_lattice("graphene", 8, 8, W=1.0, seed=1,
                                            also_single=True).blocked_width == 0
    # a complex CSR whose 4-row blocks touch too many column blocks: none
    rs = np.random.default_rng(3)
    n = 400
    lens = np.full(n, 12)
    rowptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    col = np.concatenate([np.sort(rs.choice(n, 12, replace=False)) for _ in range(n)]).astype(np.int32)
    val = rs.standard_normal(rowptr[-1]) + 1j * rs.standard_normal(rowptr[-1])
    H = pkg.chebfd_matrix_create_csr(rowptr, col, val, also_single=True)
    assert H.blocked_width == 0
    with pytest.raises(pkg.ChebFDError):
        H.set_blocked(True)


def _step_case(Lx, Ly, Lz, W, seed, nb, ld=None):
    H = pkg.chebfd_matrix_create_lattice("topi", Lx, Ly, Lz, t=1.0, m=1.0, W=W, seed=seed,
                                         also_single=True)
    assert H.blocked_width == 7
    Ho = lattice.to_scipy(*lattice.topi_csr(Lx, Ly, Lz, t=1.0, m=1.0, W=W, seed=seed))
    ld = ld or nb
    mk = lambda s: torch.from_numpy(workloads.random_block(s, H.n, ld, True)).to(
        DEV).to(torch.complex64)
    U, W0, Y0 = mk(1), mk(2), mk(3)
    alpha, beta, c = 0.23, -0.041, 0.37
    ref_u = U[:, :nb].cpu().numpy().astype(np.complex128)
    ref_w = 2.0 * ofilt.apply_A(Ho, alpha, beta, ref_u) - W0[:, :nb].cpu().numpy()
    ref_y = Y0[:, :nb].cpu().numpy() + c * ref_w
    out = {}
    for blocked in (True, False):
        H.set_blocked(blocked)
        Wt, Yt = W0.clone(), Y0.clone()
        pkg.chebfd_chebyshev_step(H, alpha, beta, c, U[:, :nb], Wt[:, :nb], Yt[:, :nb])
        torch.cuda.synchronize()
        out[blocked] = (Wt.cpu().numpy(), Yt.cpu().numpy())
        # columns beyond nb are untouched
        assert torch.equal(Wt[:, nb:], W0[:, nb:]) and torch.equal(Yt[:, nb:], Y0[:, nb:])
    return out, ref_w, ref_y, nb


@pytest.mark.parametrize("Lx,Ly,Lz,nb", [(6, 5, 4, 64), (5, 3, 7, 32), (4, 4, 4, 16), (3, 5, 3, 8),
                                         (6, 2, 3, 2), (2, 2, 3, 64), (1, 3, 2, 16)])
def test_blocked_step_matches_oracle_and_sell(Lx, Ly, Lz, nb):
    """One fused step w = 2(aH+b)u - w, y += c w: the blocked kernel (group
    widths 32, 16 and 8 lanes; lattices with edges 1 and 2, where neighbour
    sites coincide and blocks are merged or padded) within FP32 rounding of
    the FP64 oracle on the same complex64 inputs, and of the SELL kernel."""
    out, ref_w, ref_y, nb = _step_case(Lx, Ly, Lz, 1.3, 5, nb)
    tol = 30 * 2.0 ** -24
    for blocked in (True, False):
        w, y = out[blocked]
        assert rel(w[:, :nb], ref_w) <= tol, (blocked, rel(w[:, :nb], ref_w))
        assert rel(y[:, :nb], ref_y) <= tol
    assert rel(out[True][0], out[False][0]) <= 2 * tol


def test_blocked_step_strided_panel():
    """A panel of 32 columns inside rows of 48 (ld = 48): only the panel changes."""
    out, ref_w, ref_y, nb = _step_case(4, 6, 5, 0.9, 2, 32, ld=48)
    w, y = out[True]
    assert rel(w[:, :nb], ref_w) <= 30 * 2.0 ** -24


def test_blocked_filter_full_size_insulator():
    """64x64x32x4 (N = 524288), n_b = 64, complex64 filter through the blocked
    kernel, N_p = 6: within the FP32 bound of the FP64 oracle, and equal to the
    SELL kernel's filter to FP32 rounding."""
    w = workloads.TOPI_MEDIUM
    H = pkg.chebfd_matrix_create_lattice("topi", w["Lx"], w["Ly"], w["Lz"], t=w["t"], m=w["m"],
                                         W=w["W"], seed=w["seed"], also_single=True)
    Ho = lattice.to_scipy(*lattice.topi_csr(w["Lx"], w["Ly"], w["Lz"], t=w["t"], m=w["m"],
                                            W=w["W"], seed=w["seed"]))
    a, b = -4.2, 4.2
    alpha, beta = coeffs.scaling(a, b)
    gc = coeffs.filter_coeffs(a, b, -0.1, 0.1, 6, "lanczos")
    X0 = torch.from_numpy(workloads.random_block(0, H.n, 64, True)).to(DEV).to(torch.complex64)
    got = {}
    for blocked in (True, False):
        H.set_blocked(blocked)
        X = X0.clone()
        pkg.chebfd_filter_block(H, alpha, beta, gc, X)
        got[blocked] = X.cpu().numpy()
    ref = ofilt.filter_block(Ho, alpha, beta, gc, X0.cpu().numpy().astype(np.complex128))
    bound = 6 * 30 * 2.0 ** -24 * np.linalg.norm(X0.cpu().numpy()) / np.linalg.norm(ref)
    assert rel(got[True], ref) <= bound
    assert rel(got[True], got[False]) <= bound


@pytest.mark.parametrize("single", [True, False])
def test_slab_filter_matches_oracle(single):
    """Eq. Ham slab (open in z: 11-entry surface rows, so the blocked copy has
    padded block columns and the SELL path its generic variable-width loop):
    the filter within 1e-11 (FP64) or the FP32 bound (complex64) of the oracle."""
    Lx, Ly, Lz = 6, 5, 4
    H = pkg.chebfd_matrix_create_lattice("topi_slab", Lx, Ly, Lz, t=1.0, m=2.0, W=2.0, seed=3,
                                         also_single=True)
    assert H.blocked_width == 7
    Ho = lattice.to_scipy(*lattice.topi_slab_csr(Lx, Ly, Lz, t=1.0, m=2.0, W=2.0, seed=3))
    a, b = -5.5, 5.5
    alpha, beta = coeffs.scaling(a, b)
    gc = coeffs.filter_coeffs(a, b, -0.06, 0.06, 120, "lanczos")
    X0 = workloads.random_block(4, H.n, 64, True)
    X = torch.from_numpy(X0).to(DEV)
    if single:
        X = X.to(torch.complex64)
    Xin = X.cpu().numpy().astype(np.complex128)
    pkg.chebfd_filter_block(H, alpha, beta, gc, X)
    ref = ofilt.filter_block(Ho, alpha, beta, gc, Xin)
    err = rel(X.cpu().numpy(), ref)
    tol = 120 * 30 * 2.0 ** -24 * np.linalg.norm(Xin) / np.linalg.norm(ref) if single else 1e-11
    assert err <= tol, (err, tol)


@pytest.mark.parametrize("kind,L,nb", [("topi", (6, 5, 4), 64), ("topi", (5, 3, 7), 32),
                                       ("topi", (2, 2, 3), 16), ("topi", (1, 3, 2), 8),
                                       ("topi_slab", (6, 5, 4), 64), ("topi_slab", (3, 4, 2), 2),
                                       ("topi_slab", (4, 4, 1), 16)])
def test_matrix_free_step_matches_oracle(kind, L, nb):
    """The matrix-free step (entries rebuilt in registers from the lattice
    description; coinciding neighbours on edges 1 and 2; open slab surfaces)
    within FP32 rounding of the FP64 oracle step and of the stored-matrix step."""
    m = 2.0 if kind == "topi_slab" else 1.0
    H = pkg.chebfd_matrix_create_lattice(kind, *L, t=1.0, m=m, W=1.3, seed=5, also_single=True)
    gen = lattice.topi_slab_csr if kind == "topi_slab" else lattice.topi_csr
    Ho = lattice.to_scipy(*gen(*L, t=1.0, m=m, W=1.3, seed=5))
    mk = lambda s: torch.from_numpy(workloads.random_block(s, H.n, nb, True)).to(
        DEV).to(torch.complex64)
    U, W0, Y0 = mk(1), mk(2), mk(3)
    alpha, beta, c = 0.21, 0.037, -0.43
    ref_w = 2.0 * ofilt.apply_A(Ho, alpha, beta, U.cpu().numpy().astype(np.complex128)) \
        - W0.cpu().numpy()
    ref_y = Y0.cpu().numpy() + c * ref_w
    got = {}
    for free in (True, False):
        H.set_matrix_free(free)
        Wt, Yt = W0.clone(), Y0.clone()
        pkg.chebfd_chebyshev_step(H, alpha, beta, c, U, Wt, Yt)
        got[free] = (Wt.cpu().numpy(), Yt.cpu().numpy())
    tol = 30 * 2.0 ** -24
    assert rel(got[True][0], ref_w) <= tol and rel(got[True][1], ref_y) <= tol
    assert rel(got[True][0], got[False][0]) <= 2 * tol


def test_matrix_free_only_for_insulator_lattices():
    g = pkg.chebfd_matrix_create_lattice("graphene", 8, 8, W=1.0, seed=1, also_single=True)
    with pytest.raises(pkg.ChebFDError):
        g.set_matrix_free(True)
    t = pkg.chebfd_matrix_create_lattice("topi", 4, 4, 4, W=1.0, seed=1)   # no single copy
    with pytest.raises(pkg.ChebFDError):
        t.set_matrix_free(True)


@pytest.mark.parametrize("kind,L", [("topi", (200, 160, 2)), ("topi_slab", (208, 152, 2))])
def test_tiled_site_order_visits_every_site(kind, L):
    """Lattices whose two x-y planes of 64-column rows exceed L2 are visited
    in tiles of the x-y plane (200 = 8 x 25, 160 = 8 x 20, 208 = 13 x 16,
    152 = 8 x 19): the blocked and the matrix-free steps still reproduce the
    oracle step on every row."""
    m = 2.0 if kind == "topi_slab" else 1.0
    H = pkg.chebfd_matrix_create_lattice(kind, *L, t=1.0, m=m, W=0.8, seed=2, also_single=True)
    gen = lattice.topi_slab_csr if kind == "topi_slab" else lattice.topi_csr
    Ho = lattice.to_scipy(*gen(*L, t=1.0, m=m, W=0.8, seed=2))
    nb = 64
    mk = lambda s: torch.from_numpy(workloads.random_block(s, H.n, nb, True)).to(
        DEV).to(torch.complex64)
    U, W0, Y0 = mk(1), mk(2), mk(3)
    alpha, beta, c = 0.2, -0.01, 0.5
    ref_w = 2.0 * ofilt.apply_A(Ho, alpha, beta, U.cpu().numpy().astype(np.complex128)) \
        - W0.cpu().numpy()
    for free in (False, True):
        H.set_matrix_free(free)
        Wt, Yt = W0.clone(), Y0.clone()
        pkg.chebfd_chebyshev_step(H, alpha, beta, c, U, Wt, Yt)
        w = Wt.cpu().numpy()
        # every row updated correctly (a skipped or doubled site shows up row-wise)
        row_err = np.linalg.norm(w - ref_w, axis=1) / np.linalg.norm(ref_w, axis=1)
        assert row_err.max() <= 1e-5, (free, row_err.max())


@pytest.mark.parametrize("kind,L,Np", [("topi", (16, 8, 12), 9), ("topi", (8, 16, 20), 12),
                                       ("topi", (8, 8, 3), 7), ("topi_slab", (24, 8, 8), 10)])
def test_two_step_matrix_free_filter(kind, L, Np):
    """Two Chebyshev steps per pass (matrix-free insulator, 16-column panels,
    8 x 8 x-y tiles with a one-site halo, z-segments of Z planes): the filter
    of a 16-column block equals, bit for bit, the same block filtered with
    single matrix-free steps (the same per-site arithmetic); odd and even
    N_p (a single step left over), periodic and open z, and it agrees with the
    FP64 oracle within the complex64 bound."""
    Lx, Ly, Lz = L
    kw = dict(t=1.0, m=(1.0 if kind == "topi" else 2.0), W=1.2, seed=7, also_single=True)
    H = pkg.chebfd_matrix_create_lattice(kind, Lx, Ly, Lz, **kw)
    H.set_matrix_free(True, pairs=True)
    gen = lattice.topi_csr if kind == "topi" else lattice.topi_slab_csr
    Ho = lattice.to_scipy(*gen(Lx, Ly, Lz, t=kw["t"], m=kw["m"], W=kw["W"], seed=kw["seed"]))
    a, b = -5.6, 5.6
    alpha, beta = coeffs.scaling(a, b)
    gc = coeffs.filter_coeffs(a, b, -0.3, 0.1, Np, "lanczos")
    X0 = workloads.random_block(Lx + Np, H.n, 16, True).astype(np.complex64)
    X = torch.from_numpy(X0).to(DEV)
    pkg.chebfd_filter_block(H, alpha, beta, gc, X)
    H.set_matrix_free(True)      # single steps for the reference
    Xs = torch.from_numpy(X0).to(DEV)
    pkg.chebfd_filter_block(H, alpha, beta, gc, Xs)
    got = X.cpu().numpy()
    assert np.array_equal(got, Xs.cpu().numpy())
    ref = ofilt.filter_block(Ho, alpha, beta, gc, X0.astype(np.complex128))
    bound = Np * 30 * 2.0 ** -24 * np.linalg.norm(X0) / np.linalg.norm(ref)
    assert rel(got, ref) <= bound
