"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Matrix construction and the SELL permutation are compared bit for bit; the
FP64 filtered block within 1e-11 relative Frobenius norm; single-precision
results within bounds derived from FP32 rounding (unit roundoff 6e-8 times the
growth of the recurrence)."""
import numpy as np
import pytest
import torch

import paper_1510_04895_gb300 as pkg
from oracle import bounds as obounds, coeffs, filter as ofilt, kpm as okpm, lattice, sell as osell
from oracle import solve as osolve
from paper_1510_04895_gb300 import workloads

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TDT = {(True, False): torch.complex128, (True, True): torch.complex64,
       (False, False): torch.float64, (False, True): torch.float32}


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def oracle_csr(kind, Lx, Ly, Lz=1, t=1.0, m=1.0, W=0.0, seed=0):
    if kind == "topi":
        return lattice.topi_csr(Lx, Ly, Lz, t=t, m=m, W=W, seed=seed)
    if kind == "topi_slab":
        return lattice.topi_slab_csr(Lx, Ly, Lz, t=t, m=m, W=W, seed=seed)
    return lattice.graphene_csr(Lx, Ly, t=t, W=W, seed=seed)


def assert_sell_equal(got, ref):
    for key in ("chunk_ptr", "chunk_len", "col", "perm"):
        assert np.array_equal(got[key], ref[key]), key
    # bitwise equality of the values (signed zeros included)
    g = got["val"].view(np.uint64)
    r = np.ascontiguousarray(ref["val"]).view(np.uint64)
    assert np.array_equal(g, r)


# ------------------------------------------------------------------ matrices


@pytest.mark.parametrize("spec", [
    ("topi", 8, 8, 8, 0.5, 0, 1, 1), ("topi", 3, 4, 5, 2.0, 7, 4, 1), ("topi", 2, 2, 3, 0.7, 3, 2, 1),
    ("topi", 2, 1, 3, 1.1, 9, 8, 16), ("graphene", 16, 12, 1, 1.0, 2, 1, 1),
    ("graphene", 2, 5, 1, 1.0, 4, 32, 64), ("graphene", 1, 3, 1, 0.3, 1, 4, 4),
    ("topi_slab", 6, 5, 4, 2.0, 3, 1, 1), ("topi_slab", 2, 3, 1, 2.0, 5, 4, 8),
    ("topi_slab", 3, 2, 7, 0.7, 1, 8, 32),
])
def test_lattice_generator_and_sell_bit_exact(spec):
    kind, Lx, Ly, Lz, W, seed, C, sigma = spec
    m = 2.0 if kind == "topi_slab" else 1.0
    H = pkg.chebfd_matrix_create_lattice(kind, Lx, Ly, Lz, t=1.0, m=m, W=W, seed=seed,
                                         sell_C=C, sell_sigma=sigma)
    ref = osell.sell_from_csr(*oracle_csr(kind, Lx, Ly, Lz, 1.0, m, W, seed), C, sigma)
    assert_sell_equal(H.export_sell(), ref)


@pytest.mark.parametrize("C,sigma", [(1, 1), (4, 1), (8, 32), (32, 1000), (2, 3)])
def test_csr_upload_and_sell_bit_exact(C, sigma):
    rs = np.random.default_rng(C + 10 * sigma)
    n = 1000
    lens = rs.integers(1, 12, n)
    rowptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    col = np.concatenate([np.sort(rs.choice(n, l, replace=False)) for l in lens]).astype(np.int32)
    val = rs.standard_normal(rowptr[-1]) + 1j * rs.standard_normal(rowptr[-1])
    H = pkg.chebfd_matrix_create_csr(rowptr, col, val, sell_C=C, sell_sigma=sigma)
    assert_sell_equal(H.export_sell(), osell.sell_from_csr(rowptr, col, val, C, sigma))


def test_full_size_insulator_matrix_sampled():
    """64x64x32x4 insulator (N = 524288): the device SELL equals the oracle CSR."""
    w = workloads.TOPI_MEDIUM
    H = pkg.chebfd_matrix_create_lattice("topi", w["Lx"], w["Ly"], w["Lz"], t=w["t"], m=w["m"],
                                         W=w["W"], seed=w["seed"])
    got = H.export_sell()
    rp, c, v = lattice.topi_csr(w["Lx"], w["Ly"], w["Lz"], t=w["t"], m=w["m"], W=w["W"], seed=w["seed"])
    assert np.array_equal(got["chunk_ptr"], rp) and np.array_equal(got["col"], c)
    assert np.array_equal(got["val"].view(np.uint64), v.view(np.uint64))
    assert np.array_equal(got["perm"], np.arange(len(rp) - 1))


# ------------------------------------------------------------------ kernels


def _gpu_block(X, single):
    t = torch.from_numpy(np.ascontiguousarray(X)).to(DEV)
    if single:
        t = t.to(torch.complex64 if t.is_complex() else torch.float32)
    return t


@pytest.mark.parametrize("kind,single,nb", [("topi", False, 64), ("topi", True, 64), ("topi", False, 16),
                                             ("topi", True, 2), ("graphene", False, 128),
                                             ("graphene", True, 4), ("topi", False, 80)])
def test_spmv_matches_oracle(kind, single, nb):
    args = ("topi", 5, 4, 6, 1.0, 1.0, 1.5, 3) if kind == "topi" else ("graphene", 24, 20, 1, 1.0, 0.0, 1.0, 4)
    H = pkg.chebfd_matrix_create_lattice(*args[:4], t=args[4], m=args[5], W=args[6], seed=args[7],
                                         also_single=True)
    Ho = lattice.to_scipy(*oracle_csr(*args))
    X0 = workloads.random_block(1, H.n, nb, H.is_complex)
    X = _gpu_block(X0, single)
    Y = torch.empty_like(X)
    pkg.chebfd_spmv(H, 0.37, -0.21, X, Y)
    ref = ofilt.apply_A(Ho, 0.37, -0.21, X.cpu().numpy().astype(X0.dtype))
    tol = 2e-6 if single else 1e-14
    assert rel(Y.cpu().numpy(), ref) < tol


def _filter_case(kind, Lx, Ly, Lz, W, seed, nb, Np, kernel, window, single, C=1, sigma=1,
                 moments=False, xseed=0):
    H = pkg.chebfd_matrix_create_lattice(kind, Lx, Ly, Lz, t=1.0, m=1.0, W=W, seed=seed,
                                         sell_C=C, sell_sigma=sigma, also_single=True)
    Ho = lattice.to_scipy(*oracle_csr(kind, Lx, Ly, Lz, 1.0, 1.0, W, seed))
    a, b = obounds.lanczos_bounds(Ho, 30, seed=0)
    alpha, beta = coeffs.scaling(a, b)
    gc = coeffs.filter_coeffs(a, b, window[0], window[1], Np, kernel)
    X0 = workloads.random_block(xseed, H.n, nb, H.is_complex)
    X = _gpu_block(X0, single)
    Xin = X.cpu().numpy().astype(X0.dtype)
    mom = None
    if moments:
        mom = torch.zeros((2 * Np, nb), dtype=torch.float64, device=DEV)
    pkg.chebfd_filter_block(H, alpha, beta, gc, X, moments=mom)
    torch.cuda.synchronize()
    ref = ofilt.filter_block(Ho, alpha, beta, gc, Xin)
    out = dict(got=X.cpu().numpy(), ref=ref, gc=gc, Xin=Xin, H=Ho, alpha=alpha, beta=beta)
    if moments:
        out["mom"] = mom.cpu().numpy()
        out["mom_ref"] = ofilt.moments(Ho, alpha, beta, Xin, 2 * Np)
    return out


def test_filter_smallest_insulator_fp64_parity():
    """8x8x8x4 insulator, n_b = 64, N_p = 200, Jackson: rel. Frobenius <= 1e-11."""
    w = workloads.TOPI_SMALL
    r = _filter_case("topi", 8, 8, 8, 0.5, 0, 64, 200, "jackson", w["window"], False)
    assert rel(r["got"], r["ref"]) <= 1e-11


def test_filter_smallest_insulator_complex64_error():
    """complex64 recurrence with FP32 accumulation: error vs the FP64 oracle."""
    r = _filter_case("topi", 8, 8, 8, 0.5, 0, 64, 200, "jackson", (-0.1, 0.1), True)
    err = rel(r["got"], r["ref"])
    # N_p steps, each with relative rounding ~ 13 * 2^-24 growth bounded by ||X||/||Y||
    bound = 200 * 13 * 2.0 ** -24 * np.linalg.norm(r["Xin"]) / np.linalg.norm(r["ref"])
    assert err <= bound, (err, bound)


@pytest.mark.parametrize("nb,single,C,sigma", [(16, False, 1, 1), (2, True, 4, 8), (80, False, 2, 1),
                                                (48, True, 8, 1), (1, False, 32, 1)])
def test_filter_ragged_widths_and_chunks(nb, single, C, sigma):
    r = _filter_case("topi", 3, 5, 7, 1.2, 5, nb, 37, "lanczos", (-0.3, 0.4), single, C=C, sigma=sigma)
    tol = 1e-11 if not single else 37 * 13 * 2.0 ** -24 * np.linalg.norm(r["Xin"]) / np.linalg.norm(r["ref"])
    assert rel(r["got"], r["ref"]) <= tol


@pytest.mark.parametrize("single", [False, True])
def test_filter_graphene_real(single):
    r = _filter_case("graphene", 20, 17, 1, 1.0, 2, 64, 150, "lanczos", (-0.2, 0.2), single)
    tol = 1e-11 if not single else 150 * 4 * 2.0 ** -24 * np.linalg.norm(r["Xin"]) / np.linalg.norm(r["ref"])
    assert rel(r["got"], r["ref"]) <= tol


def test_filter_moments_match_definition():
    r = _filter_case("topi", 4, 4, 5, 0.8, 1, 16, 60, "fejer", (-0.5, 0.5), False, moments=True)
    assert rel(r["got"], r["ref"]) <= 1e-11
    assert np.abs(r["mom"] - r["mom_ref"]).max() <= 1e-10 * np.abs(r["mom_ref"][0]).max()


def test_filter_on_diagonal_matrix_closed_form():
    """T_n(cos t) = cos(n t): for diagonal H the filtered entries are
    sum_n gc_n cos(n arccos(alpha l_i + beta)) times the input."""
    D = 4096
    lam = lattice.linear_dos_eigs(D)
    rp, c, v = lattice.diagonal_csr(lam)
    H = pkg.chebfd_matrix_create_csr(rp, c, v)
    gc = coeffs.filter_coeffs(-1.0, 1.0, -0.05, 0.05, 300, "lanczos")
    X0 = workloads.random_block(3, D, 8, False)
    X = torch.from_numpy(X0).to(DEV)
    pkg.chebfd_filter_block(H, 1.0, 0.0, gc, X)
    p = np.cos(np.outer(np.arccos(lam), np.arange(301))) @ gc
    assert np.abs(X.cpu().numpy() - p[:, None] * X0).max() <= 1e-13 * np.abs(gc).sum()


def test_filter_divergence_is_reported():
    """With [a,b] not containing spec(H), |T_n| grows and the moment check
    returns ENUMERIC (a host-side status, no device fault)."""
    H = pkg.chebfd_matrix_create_lattice("topi", 4, 4, 4, W=0.5, seed=0)
    a, b = -1.0, 1.0                      # spectrum reaches +-4
    alpha, beta = coeffs.scaling(a, b)
    gc = coeffs.filter_coeffs(a, b, -0.1, 0.1, 50, "jackson")
    X = torch.from_numpy(workloads.random_block(0, H.n, 16, True)).to(DEV)
    mom = torch.zeros((100, 16), dtype=torch.float64, device=DEV)
    with pytest.raises(pkg.ChebFDError) as e:
        pkg.chebfd_filter_block(H, alpha, beta, gc, X, moments=mom)
    assert e.value.status == 4


def test_filter_full_size_insulator_launch_config():
    """64x64x32x4 (N = 524288), n_b = 64, the benchmark's kernel configuration,
    N_p = 6 (oracle time): FP64 within 1e-11, complex64 within its FP32 bound."""
    w = workloads.TOPI_MEDIUM
    for single in (False, True):
        r = _filter_case("topi", w["Lx"], w["Ly"], w["Lz"], w["W"], w["seed"], 64, 6, "lanczos",
                         (-0.1, 0.1), single)
        e = rel(r["got"], r["ref"])
        tol = 1e-11 if not single else 6 * 13 * 2.0 ** -24 * np.linalg.norm(r["Xin"]) / np.linalg.norm(r["ref"])
        assert e <= tol, (single, e, tol)


# ------------------------------------------------------------------ helpers


def test_random_block_matches_oracle_search_vectors():
    X = torch.zeros((777, 24), dtype=torch.complex128, device=DEV)
    pkg.chebfd_random_block(X, col0=0, ns_total=24, seed=9)
    ref = osolve.search_vectors(9, 777, 24, True)
    assert np.array_equal(X.cpu().numpy(), ref)
    Xr = torch.zeros((301, 10), dtype=torch.float64, device=DEV)
    pkg.chebfd_random_block(Xr, col0=0, ns_total=10, seed=4)
    assert np.array_equal(Xr.cpu().numpy(), osolve.search_vectors(4, 301, 10, False))


@pytest.mark.parametrize("kind", ["topi", "graphene"])
def test_scale_bounds_enclose_spectrum(kind):
    args = ("topi", 5, 4, 4, 1.0, 1.0, 1.5, 2) if kind == "topi" else ("graphene", 12, 10, 1, 1.0, 0.0, 1.0, 2)
    H = pkg.chebfd_matrix_create_lattice(*args[:4], t=args[4], m=args[5], W=args[6], seed=args[7])
    Ho = lattice.to_scipy(*oracle_csr(*args))
    e = np.linalg.eigvalsh(Ho.toarray())
    a, b, al, be = pkg.chebfd_scale_bounds(H, 30, seed=1)
    assert a <= e[0] and b >= e[-1] and (b - a) <= 1.06 * (e[-1] - e[0])
    ao, bo = obounds.lanczos_bounds(Ho, 30, seed=1)
    assert abs(a - ao) <= 1e-6 * (bo - ao) and abs(b - bo) <= 1e-6 * (bo - ao)
    assert al == pytest.approx(2 / (b - a)) and be == pytest.approx((a + b) / (a - b))


def test_kpm_moments_match_oracle():
    H = pkg.chebfd_matrix_create_lattice("topi", 4, 4, 4, W=1.0, seed=4)
    Ho = lattice.to_scipy(*lattice.topi_csr(4, 4, 4, W=1.0, seed=4))
    a, b = -4.8, 4.8
    alpha, beta = coeffs.scaling(a, b)
    mu = pkg.chebfd_kpm_moments(H, alpha, beta, 64, 8, seed=3)
    ref = okpm.moments(Ho, alpha, beta, 64, 8, seed=3, complex_values=True)
    assert np.abs(mu - ref).max() <= 1e-12


@pytest.mark.parametrize("dtype,nb", [(torch.complex64, 200), (torch.complex128, 72),
                                      (torch.float32, 136), (torch.float64, 8)])
def test_host_block_filter_equals_device_filter(dtype, nb):
    """chebfd_filter_block_host streams a host block through the device panel
    by panel (ring of three device panels, copies on two streams overlapping
    the filter): bit-identical to chebfd_filter_block on a device copy, with
    more panels than ring slots, a ragged last panel and a padded host row
    stride; a page-locked and a pageable host block."""
    cplx = dtype.is_complex
    H = (pkg.chebfd_matrix_create_lattice("topi", 6, 5, 7, t=1.0, m=1.0, W=1.0, seed=3,
                                          also_single=True) if cplx else
         pkg.chebfd_matrix_create_lattice("graphene", 20, 17, 1, t=1.0, W=1.0, seed=2,
                                          also_single=True))
    gc = pkg.chebfd_window_coeffs(-4.5, 4.5, -0.2, 0.3, 40, "lanczos", 2.0)
    ld = nb + (8 if dtype in (torch.complex64, torch.float32) else 2)  # 16-byte rows, padded
    X0 = workloads.random_block(9, H.n, ld, cplx)
    Xd = torch.from_numpy(X0).to(dtype).to(DEV)
    pkg.chebfd_filter_block(H, 0.21, 0.0, gc, Xd[:, :nb])
    ref = Xd.cpu()
    for pinned in (True, False):
        Xh = torch.from_numpy(X0).to(dtype)
        if pinned:
            Xh = Xh.pin_memory()
        pkg.chebfd_filter_block_host(H, 0.21, 0.0, gc, Xh[:, :nb])
        torch.cuda.synchronize()
        assert torch.equal(Xh[:, :nb], ref[:, :nb])
        assert torch.equal(Xh[:, nb:], torch.from_numpy(X0).to(dtype)[:, nb:])  # padding untouched


def test_host_block_filter_rejects_bad_blocks():
    H = pkg.chebfd_matrix_create_lattice("topi", 3, 3, 3, W=0.5, seed=0, also_single=True)
    gc = np.ones(5)
    Xh = torch.zeros((H.n, 6), dtype=torch.complex64)       # 48-byte rows: fine
    with pytest.raises(pkg.ChebFDError):
        pkg.chebfd_filter_block_host(H, 0.2, 0.0, gc, Xh[:, :3])   # 24 bytes per row
    with pytest.raises(pkg.ChebFDError):
        pkg.chebfd_filter_block_host(H, 0.2, 0.0, gc[:2], Xh)     # N_p < 2
    with pytest.raises(pkg.ChebFDError):
        pkg.chebfd_filter_block_host(H, 0.2, 0.0, gc, torch.zeros((H.n, 8)))  # real vs complex
