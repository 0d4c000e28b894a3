"""Parity at the benchmark workloads' full sizes, in the launch configuration
bench.py times, on outputs the oracle computes one by one (the oracle cannot
hold the 16e6-row matrix's filter) or on whole results where it can."""
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


def test_large_insulator_step_sampled_rows():
    """200x200x100x4 insulator (N = 16e6), n_b = 64, complex64 blocked step:
    w = 2(aH+b)u - w and y += c w at 256 random rows (4 orbitals of 64 sites,
    including the first and last site) against the oracle rows of those sites,
    in FP64 on the same complex64 inputs."""
    w = workloads.TOPI_LARGE
    H = pkg.chebfd_matrix_create_lattice("topi", w["Lx"], w["Ly"], w["Lz"], t=w["t"], m=w["m"],
                                         W=w["W"], seed=w["seed"], also_single=True)
    assert H.n == 16_000_000 and H.blocked_width == 7
    nb = 64
    U = torch.empty((H.n, nb), dtype=torch.complex64, device=DEV)
    W0 = torch.empty_like(U)
    Y0 = torch.empty_like(U)
    pkg.chebfd_random_block(U, ns_total=nb, seed=1)
    pkg.chebfd_random_block(W0, ns_total=nb, seed=2)
    pkg.chebfd_random_block(Y0, ns_total=nb, seed=3)
    rs = np.random.default_rng(5)
    sites = np.unique(np.concatenate([[0, H.n // 4 - 1], rs.integers(0, H.n // 4, 62)]))
    rows = (4 * sites[:, None] + np.arange(4)).ravel()
    rp, c, v = lattice.topi_csr(w["Lx"], w["Ly"], w["Lz"], t=w["t"], m=w["m"], W=w["W"],
                                seed=w["seed"], sites=sites)
    need = np.unique(c)
    u_need = U[torch.from_numpy(need).to(DEV)].cpu().numpy().astype(np.complex128)
    w_in = W0[torch.from_numpy(rows).to(DEV)].cpu().numpy().astype(np.complex128)
    y_in = Y0[torch.from_numpy(rows).to(DEV)].cpu().numpy().astype(np.complex128)
    alpha, beta, cc = 0.24, 0.0013, 0.37
    pkg.chebfd_chebyshev_step(H, alpha, beta, cc, U, W0, Y0)
    torch.cuda.synchronize()
    w_got = W0[torch.from_numpy(rows).to(DEV)].cpu().numpy()
    y_got = Y0[torch.from_numpy(rows).to(DEV)].cpu().numpy()
    pos = {col: k for k, col in enumerate(need)}
    hu = np.zeros((len(rows), nb), np.complex128)
    for i in range(len(rows)):
        for p in range(rp[i], rp[i + 1]):
            hu[i] += v[p] * u_need[pos[c[p]]]
    u_rows = u_need[[pos[r] for r in rows]]
    w_ref = 2.0 * (alpha * hu + beta * u_rows) - w_in
    y_ref = y_in + cc * w_ref
    tol = 30 * 2.0 ** -24
    assert rel(w_got, w_ref) <= tol and rel(y_got, y_ref) <= tol


@pytest.mark.parametrize("single", [True, False])
def test_graphene_full_size_filter(single):
    """1024x1024 graphene (N = 2097152), n_b = 128 (the benchmark's panel), N_p = 4:
    FP64 within 1e-11 of the oracle, FP32 within its rounding bound."""
    w = workloads.GRAPHENE
    H = pkg.chebfd_matrix_create_lattice("graphene", w["Lx"], w["Ly"], t=w["t"], W=w["W"],
                                         seed=w["seed"], also_single=True)
    Ho = lattice.to_scipy(*lattice.graphene_csr(w["Lx"], w["Ly"], t=w["t"], W=w["W"],
                                                seed=w["seed"]))
    a, b = -3.25, 3.25
    alpha, beta = coeffs.scaling(a, b)
    gc = coeffs.filter_coeffs(a, b, -0.02, 0.02, 4, "lanczos")
    X0 = workloads.random_block(6, H.n, 128, False)
    X = torch.from_numpy(X0).to(DEV)
    if single:
        X = X.to(torch.float32)
    Xin = X.cpu().numpy().astype(np.float64)
    pkg.chebfd_filter_block(H, alpha, beta, gc, X)
    ref = ofilt.filter_block(Ho, alpha, beta, gc, Xin)
    err = rel(X.cpu().numpy(), ref)
    tol = 4 * 8 * 2.0 ** -24 * np.linalg.norm(Xin) / np.linalg.norm(ref) if single else 1e-11
    assert err <= tol, (err, tol)


def test_full_ensemble_sampled_members():
    """The 512-member ensemble (N_total = 7.67e6) with the autotuned layout,
    N_p = 12: members 0, 255 and 511 equal their own filters bitwise and the
    oracle within the FP32 bound."""
    e = workloads.ENSEMBLE
    members = workloads.ensemble_members(e["count"], e["first_seed"])
    mats = [pkg.chebfd_matrix_create_lattice("topi", L, L, L, t=e["t"], m=e["m"], W=W, seed=s,
                                             also_single=True) for L, W, s in members]
    n = sum(4 * L ** 3 for L, _, _ in members)
    X = torch.empty((n, e["ns"]), dtype=torch.complex64, device=DEV)
    E, _ = pkg.chebfd_ensemble_autotune(mats, X)
    Np = 12
    al, be, gcs = [], [], []
    for L, W, s in members:
        bound = 1.01 * (abs(e["m"]) + 3 * e["t"] + W / 2)
        x, y = coeffs.scaling(-bound, bound)
        al.append(x)
        be.append(y)
        gcs.append(pkg.chebfd_window_coeffs(-bound, bound, e["window"][0], e["window"][1], Np,
                                            "lanczos", 2.0))
    E.set_coeffs(np.array(al), np.array(be), np.array(gcs))
    X0 = workloads.random_block(9, n, e["ns"], True).astype(np.complex64)
    Xe = torch.from_numpy(X0).to(DEV)
    E.filter(Xe)
    torch.cuda.synchronize()
    got = Xe.cpu().numpy()
    for i in (0, 255, 511):
        L, W, s = members[i]
        r0, r1 = E.offsets[i], E.offsets[i + 1]
        Xi = torch.from_numpy(np.ascontiguousarray(X0[r0:r1])).to(DEV)
        pkg.chebfd_filter_block(mats[i], al[i], be[i], gcs[i], Xi)
        torch.cuda.synchronize()
        assert np.array_equal(got[r0:r1], Xi.cpu().numpy()), i
        Ho = lattice.to_scipy(*lattice.topi_csr(L, L, L, t=e["t"], m=e["m"], W=W, seed=s))
        xin = X0[r0:r1].astype(np.complex128)
        ref = ofilt.filter_block(Ho, al[i], be[i], gcs[i], xin)
        tol = Np * 30 * 2.0 ** -24 * np.linalg.norm(xin) / np.linalg.norm(ref)
        assert rel(got[r0:r1], ref) <= tol, i


def test_medium_insulator_host_block_filter_full_size():
    """The benchmark's end-to-end path at its full size: the 64x64x32x4
    insulator (N = 524288), the 256-column complex64 search block in
    page-locked host memory (1.07 GB), N_p = 8, streamed through the device by
    chebfd_filter_block_host (four 64-column panels through a ring of three):
    bit-identical to chebfd_filter_block on a device copy, and within
    complex64 rounding of the oracle on 64 sampled rows."""
    w = workloads.TOPI_MEDIUM
    H = pkg.chebfd_matrix_create_lattice("topi", w["Lx"], w["Ly"], w["Lz"], t=w["t"], m=w["m"],
                                         W=w["W"], seed=w["seed"], also_single=True)
    a, b = -4.2, 4.2
    alpha, beta = coeffs.scaling(a, b)
    gc = pkg.chebfd_window_coeffs(a, b, -0.14, 0.14, 8, "lanczos", 2.0)
    Xd = torch.empty((H.n, 256), dtype=torch.complex64, device=DEV)
    pkg.chebfd_random_block(Xd, ns_total=256, seed=3)
    X0 = Xd.cpu()
    Xh = X0.clone().pin_memory()
    pkg.chebfd_filter_block(H, alpha, beta, gc, Xd)
    pkg.chebfd_filter_block_host(H, alpha, beta, gc, Xh)
    torch.cuda.synchronize()
    assert torch.equal(Xh, Xd.cpu())
    # sampled rows against the oracle's filter (FP64 on the same inputs)
    rs = np.random.default_rng(8)
    sites = np.unique(np.concatenate([[0, H.n // 4 - 1], rs.integers(0, H.n // 4, 14)]))
    rows = (4 * sites[:, None] + np.arange(4)[None, :]).reshape(-1)
    Ho = lattice.to_scipy(*lattice.topi_csr(w["Lx"], w["Ly"], w["Lz"], t=w["t"], m=w["m"],
                                            W=w["W"], seed=w["seed"]))
    ref = ofilt.filter_block(Ho, alpha, beta, coeffs.filter_coeffs(a, b, -0.14, 0.14, 8,
                                                                    "lanczos", 2.0),
                             X0.numpy()[:, :8].astype(np.complex128))
    got = Xh.numpy()[rows, :8].astype(np.complex128)
    assert np.abs(got - ref[rows]).max() <= 1e-4 * np.abs(ref).max()
