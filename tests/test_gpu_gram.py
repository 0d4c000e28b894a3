"""The tall Gram product of the orthonormalisation and Rayleigh-Ritz steps
(Sec. 3.1 steps 6-7), A^H B for N x m blocks, by the three methods of
chebfd_gram: cuBLAS FP64, the double-float kernel and the split onto the bf16
tensor cores.  The reference is the plain definition: on small cases every
entry is the exactly rounded dot product (error-free products by Dekker's
split, summed by math.fsum); on large ones numpy's FP64 product, whose own
error is bounded by the same relative scale."""
import math

import numpy as np
import pytest
import torch

import paper_1510_04895_gb300 as pkg
from paper_1510_04895_gb300 import workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _two_prod(a, b):
    p = a * b
    c = 134217729.0
    ah = a * c
    ah = ah - (ah - a)
    al = a - ah
    bh = b * c
    bh = bh - (bh - b)
    bl = b - bh
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def exact_gram(A, B):
    """A^H B with every entry the correctly rounded sum of exact products."""
    Ar, Ai = np.real(A), np.imag(A) if np.iscomplexobj(A) else np.zeros_like(A)
    Br, Bi = np.real(B), np.imag(B) if np.iscomplexobj(B) else np.zeros_like(B)
    m = A.shape[1]
    G = np.zeros((m, m), np.complex128 if np.iscomplexobj(A) else np.float64)

    def dot(x, y):
        p, e = _two_prod(x, y)
        return np.concatenate([p, e])

    for p_ in range(m):
        for q in range(m):
            re = math.fsum(np.concatenate([dot(Ar[:, p_], Br[:, q]), dot(Ai[:, p_], Bi[:, q])]))
            if np.iscomplexobj(A):
                im = math.fsum(np.concatenate([dot(Ar[:, p_], Bi[:, q]), -dot(Ai[:, p_], Br[:, q])]))
                G[p_, q] = re + 1j * im
            else:
                G[p_, q] = re
    return G


def scale_of(A, B):
    """|A|^H |B| (entrywise moduli): the scale of a dot product's rounding error."""
    return np.abs(A).T @ np.abs(B)


@pytest.mark.parametrize("cplx", [True, False])
@pytest.mark.parametrize("n,m", [(1, 1), (63, 5), (64, 7), (513, 3), (1000, 12), (4097, 9)])
def test_gram_small_against_exact_definition(cplx, n, m):
    """Ragged N around the 64-row K-blocks and the 512-row exact chunks,
    m from 1 to 12 (partial 128 x 64 tiles), A != B and A == B."""
    A0 = workloads.random_block(n + m, n, m, cplx)
    B0 = workloads.random_block(n + 2 * m, n, m, cplx)
    A = torch.from_numpy(A0).to(DEV)
    B = torch.from_numpy(B0).to(DEV)
    for X0, Y0, X, Y in ((A0, B0, A, B), (A0, A0, A, A)):
        ref = exact_gram(X0, Y0)
        sc = scale_of(X0, Y0)
        for method in ("tensor", "double_float", "fp64"):
            G = pkg.chebfd_gram(X, None if Y is X else Y, method=method).cpu().numpy()
            err = (np.abs(G - ref) / sc).max()
            tol = {"tensor": 2.0 ** -52, "double_float": 2.0 ** -44, "fp64": 2.0 ** -52 * n}[method]
            assert err <= tol, (method, err, tol)


def test_gram_wide_column_scales_and_zero_columns():
    """Columns scaled by 2^-300 .. 2^300 (each column's own power-of-two scale),
    an all-zero column and subnormal entries: every entry to FP64 accuracy
    relative to its own scale."""
    n, m = 2000, 8
    rs = np.random.default_rng(4)
    A0 = rs.uniform(-1, 1, (n, m)) * np.ldexp(1.0, np.arange(m) * 85 - 300)[None, :]
    B0 = rs.uniform(-1, 1, (n, m)) * np.ldexp(1.0, 290 - np.arange(m) * 83)[None, :]
    A0[:, 3] = 0.0
    B0[:7, 5] = 1e-310                      # subnormals among normal entries
    ref = exact_gram(A0, B0)
    sc = scale_of(A0, B0)
    G = pkg.chebfd_gram(torch.from_numpy(A0).to(DEV), torch.from_numpy(B0).to(DEV),
                        method="tensor").cpu().numpy()
    assert np.all(G[3, :] == 0.0)
    ok = sc > 0
    assert (np.abs(G - ref)[ok] / sc[ok]).max() <= 2.0 ** -50


@pytest.mark.parametrize("cplx", [True, False])
def test_gram_large_methods_agree(cplx):
    """70001 x 128 (several row splits per tile, 137 chunks) and an
    orthonormalised 131072 x 96 block (11 chunks per CTA): the tensor-core
    Gram agrees with numpy's FP64 product and with cuBLAS within 1e-13 of
    |A|^H |B|, and with cuBLAS within 2e-15 on the orthonormal block (whose
    distance from the identity, ~3e-14 with some LAPACKs, belongs to the QR
    factor, not to the product)."""
    n, m = 70001, 128 if cplx else 200
    A0 = workloads.random_block(31, n, m, cplx)
    B0 = workloads.random_block(32, n, m, cplx)
    A, B = torch.from_numpy(A0).to(DEV), torch.from_numpy(B0).to(DEV)
    ref = A0.conj().T @ B0
    sc = scale_of(A0, B0)
    for method in ("tensor", "fp64"):
        G = pkg.chebfd_gram(A, B, method=method).cpu().numpy()
        assert (np.abs(G - ref) / sc).max() <= 1e-13, method
    Q0 = np.linalg.qr(workloads.random_block(33, 131072, 96, cplx))[0]
    Q = torch.from_numpy(np.ascontiguousarray(Q0)).to(DEV)
    G = pkg.chebfd_gram(Q, method="tensor").cpu().numpy()
    Gb = pkg.chebfd_gram(Q, method="fp64").cpu().numpy()
    assert np.abs(G - Gb).max() <= 2e-15
    assert np.abs(G - Q0.conj().T @ Q0).max() <= 2e-15 + 96 * 2.0 ** -53


def exact_product(Y, M):
    """Y @ M with every entry the correctly rounded sum of exact products."""
    cplx = np.iscomplexobj(Y)
    out = np.zeros((Y.shape[0], M.shape[1]), np.complex128 if cplx else np.float64)
    Yr, Yi = np.real(Y), np.imag(Y) if cplx else np.zeros_like(Y)
    Mr, Mi = np.real(M), np.imag(M) if cplx else np.zeros_like(M)

    def dot(x, y):
        p, e = _two_prod(x, y)
        return np.concatenate([p, e])

    for p_ in range(Y.shape[0]):
        for i in range(M.shape[1]):
            re = math.fsum(np.concatenate([dot(Yr[p_], Mr[:, i]), -dot(Yi[p_], Mi[:, i])]))
            if cplx:
                im = math.fsum(np.concatenate([dot(Yr[p_], Mi[:, i]), dot(Yi[p_], Mr[:, i])]))
                out[p_, i] = re + 1j * im
            else:
                out[p_, i] = re
    return out


@pytest.mark.parametrize("cplx", [True, False])
@pytest.mark.parametrize("n,k,r", [(1, 1, 1), (127, 5, 7), (130, 48, 48), (64, 300, 9),
                                   (257, 33, 70)])
def test_block_update_small_against_exact_definition(cplx, n, k, r):
    """T = Y M (the block update of steps 6-7) on ragged shapes: partial
    128-row and 64-column tiles, k = 300 complex (K = 600 real: two 512-row
    exact chunks), every entry within 2^-52 of |Y| |M| of the exactly rounded
    product (tensor), cuBLAS and the double-float kernel within their bounds."""
    Y0 = workloads.random_block(n + k, n, k, cplx)
    M0 = workloads.random_block(n + k + r, k, r, cplx)
    ref = exact_product(Y0, M0)
    sc = np.abs(Y0) @ np.abs(M0)
    Y, M = torch.from_numpy(Y0).to(DEV), torch.from_numpy(M0).to(DEV)
    for method, tol in (("tensor", 2.0 ** -52), ("double_float", 2.0 ** -44),
                        ("fp64", 2.0 ** -52 * k)):
        T = pkg.chebfd_block_update(Y, M, method=method).cpu().numpy()
        err = (np.abs(T - ref) / sc).max()
        assert err <= tol, (method, err, tol)


@pytest.mark.parametrize("cplx", [True, False])
def test_block_update_large_methods_agree(cplx):
    """524288 x 192 times 192 x 192 (the benchmark's n_s), with rows of very
    different scales (2^-200 .. 2^200): tensor and cuBLAS agree within 1e-14
    of |Y| |M| row by row."""
    n, k = 524288, 192
    Y0 = workloads.random_block(41, n, k, cplx)
    Y0 *= np.ldexp(1.0, (np.arange(n) % 401) - 200)[:, None]
    M0 = workloads.random_block(42, k, k, cplx)
    Y, M = torch.from_numpy(Y0).to(DEV), torch.from_numpy(M0).to(DEV)
    Tt = pkg.chebfd_block_update(Y, M, method="tensor").cpu().numpy()
    Tf = pkg.chebfd_block_update(Y, M, method="fp64").cpu().numpy()
    sc = np.abs(Y0) @ np.abs(M0)
    assert (np.abs(Tt - Tf) / sc).max() <= 1e-14


def test_gram_and_block_update_in_row_chunks():
    """Blocks long enough that the tensor-core path works in row chunks (2 GiB
    of digit slices at a time: 65536 rows of 2048 real columns): a real
    150001 x 2048 Gram (three chunks, the last ragged, their K-splits added in
    place) and a complex 150001 x 1024 block times 1024 x 40 agree with cuBLAS
    within 1e-13 of |A|^T |A| and |Y| |M|."""
    n = 150001
    g = torch.Generator(device=DEV).manual_seed(5)
    A = torch.randn(n, 2048, dtype=torch.float64, device=DEV, generator=g)
    A[:, 7] *= 2.0 ** 40                      # a column on another scale
    Gt = pkg.chebfd_gram(A, method="tensor")
    Gf = pkg.chebfd_gram(A, method="fp64")
    sc = A.abs().T @ A.abs()
    assert float(((Gt - Gf).abs() / sc).max()) <= 1e-13
    assert torch.equal(Gt, Gt.T)               # mirrored: exactly symmetric
    del A, Gt, Gf, sc
    torch.cuda.empty_cache()
    Y = torch.randn(n, 1024, dtype=torch.complex128, device=DEV, generator=g)
    M = torch.randn(1024, 40, dtype=torch.complex128, device=DEV, generator=g)
    Tt = pkg.chebfd_block_update(Y, M, method="tensor")
    Tf = pkg.chebfd_block_update(Y, M, method="fp64")
    sc = Y.abs() @ M.abs()
    assert float(((Tt - Tf).abs() / sc).max()) <= 1e-13
