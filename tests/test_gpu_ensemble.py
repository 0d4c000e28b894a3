"""Batched ensembles: many independent insulator Hamiltonians of uneven size
filtered by one fused launch per Chebyshev step (replayed from a CUDA graph)
must give, member by member, what the single-matrix filter gives (bitwise:
same arithmetic per row or per site) and what the oracle gives (FP64 1e-11)."""
import numpy as np
import pytest
import torch

import paper_1510_04895_gb300 as pkg
from oracle import coeffs, filter as ofilt, lattice
from paper_1510_04895_gb300 import workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

MEMBERS = [(3, 0.4, 100), (4, 1.7, 101), (5, 0.9, 102), (3, 2.0, 103), (6, 0.2, 104)]


def _members(single=True):
    mats, ranges = [], []
    for L, W, seed in MEMBERS:
        mats.append(pkg.chebfd_matrix_create_lattice("topi", L, L, L, t=1.0, m=1.0, W=W, seed=seed,
                                                     also_single=single))
        bound = 1.0 + 3.0 + W / 2 + 0.05          # |m| + 3t + W/2 encloses the spectrum
        ranges.append((-bound, bound))
    return mats, ranges


def _coeffs(ranges, Np, window=(-0.3, 0.3)):
    al, be, gc = [], [], []
    for a, b in ranges:
        x, y = coeffs.scaling(a, b)
        al.append(x)
        be.append(y)
        gc.append(pkg.chebfd_window_coeffs(a, b, window[0], window[1], Np, "lanczos", 2.0))
    return np.array(al), np.array(be), np.array(gc)


@pytest.mark.parametrize("dt,nb,C", [(torch.complex64, 48, 1), (torch.complex64, 48, 4),
                                      (torch.complex128, 32, 2), (torch.complex64, 16, 1)])
def test_ensemble_filter_matches_single_filters_and_oracle(dt, nb, C):
    mats, ranges = _members()
    E = pkg.chebfd_ensemble_create(mats, sell_C=C)
    assert E.count == len(MEMBERS) and E.n == sum(4 * L ** 3 for L, _, _ in MEMBERS)
    Np = 60
    al, be, gc = _coeffs(ranges, Np)
    E.set_coeffs(al, be, gc)
    X0 = workloads.random_block(7, E.n, nb, True)
    Xe = torch.from_numpy(X0).to(DEV).to(dt)
    Xin = Xe.cpu().numpy().astype(np.complex128)
    E.filter(Xe, use_graph=True)
    torch.cuda.synchronize()
    got = Xe.cpu().numpy()
    for i, (L, W, seed) in enumerate(MEMBERS):
        r0, r1 = E.offsets[i], E.offsets[i + 1]
        Xi = torch.from_numpy(np.ascontiguousarray(X0[r0:r1])).to(DEV).to(dt)
        # members and ensemble both run the blocked complex64 step (the
        # members' blocked copies are concatenated into the ensemble's)
        assert mats[i].blocked_width == 7
        pkg.chebfd_filter_block(mats[i], al[i], be[i], gc[i], Xi)
        torch.cuda.synchronize()
        assert np.array_equal(got[r0:r1], Xi.cpu().numpy()), "member %d differs from single" % i
        Ho = lattice.to_scipy(*lattice.topi_csr(L, L, L, t=1.0, m=1.0, W=W, seed=seed))
        ref = ofilt.filter_block(Ho, al[i], be[i], gc[i], Xin[r0:r1])
        err = np.linalg.norm(got[r0:r1] - ref) / np.linalg.norm(ref)
        tol = 1e-11 if dt == torch.complex128 else \
            Np * 13 * 2.0 ** -24 * np.linalg.norm(Xin[r0:r1]) / np.linalg.norm(ref)
        assert err <= tol, (i, err, tol)


def test_ensemble_graph_replay_and_coefficient_update():
    mats, ranges = _members()
    E = pkg.chebfd_ensemble_create(mats, sell_C=1)
    al, be, gc = _coeffs(ranges, 40)
    E.set_coeffs(al, be, gc)
    X0 = torch.from_numpy(workloads.random_block(3, E.n, 32, True)).to(DEV).to(torch.complex64)
    A, B, Cx = X0.clone(), X0.clone(), X0.clone()
    E.filter(A, use_graph=False)
    E.filter(B, use_graph=True)     # capture + launch
    E.filter(Cx, use_graph=True)    # replay
    torch.cuda.synchronize()
    assert torch.equal(A, B) and torch.equal(A, Cx)
    # new coefficients of the same degree are picked up by the cached graph
    al2, be2, gc2 = _coeffs(ranges, 40, window=(-0.6, 0.1))
    E.set_coeffs(al2, be2, gc2)
    D, F = X0.clone(), X0.clone()
    E.filter(D, use_graph=True)
    E.filter(F, use_graph=False)
    torch.cuda.synchronize()
    assert torch.equal(D, F) and not torch.equal(D, A)


def test_ensemble_autotune_returns_a_working_layout():
    mats, ranges = _members()
    n = sum(4 * L ** 3 for L, _, _ in MEMBERS)
    X = torch.zeros((n, 48), dtype=torch.complex64, device=DEV)
    E, ms = pkg.chebfd_ensemble_autotune(mats, X)
    assert ms > 0 and E.sell_C in (1, 2, 4) and E.panel in (16, 32, 48) and E.tile in (1, 4, 16)
    al, be, gc = _coeffs(ranges, 30)
    E.set_coeffs(al, be, gc)
    X0 = workloads.random_block(5, n, 48, True)
    Xe = torch.from_numpy(X0).to(DEV).to(torch.complex64)
    E.filter(Xe)
    ref = pkg.chebfd_ensemble_create(mats, sell_C=1)
    ref.set_coeffs(al, be, gc)
    Xr = torch.from_numpy(X0).to(DEV).to(torch.complex64)
    ref.filter(Xr)
    torch.cuda.synchronize()
    assert torch.equal(Xe, Xr)


def test_ensemble_rejects_mismatched_members():
    a = pkg.chebfd_matrix_create_lattice("topi", 3, 3, 3, W=0.5, seed=1)
    g = pkg.chebfd_matrix_create_lattice("graphene", 4, 4, W=0.5, seed=1)
    with pytest.raises(pkg.ChebFDError):
        pkg.chebfd_ensemble_create([a, g])
    s = pkg.chebfd_matrix_create_lattice("topi", 3, 3, 3, W=0.5, seed=1, sell_C=4)
    with pytest.raises(pkg.ChebFDError):
        pkg.chebfd_ensemble_create([a, s])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_solve_matches_dense_per_member(precision):
    """chebfd_solve_batched on a 5-member ensemble: every member's window
    eigenvalues equal the dense eigensolver's within 1e-10 ||H||, residuals
    <= 1e-9 ||H||."""
    members = [(4, 0.4, 100), (5, 1.7, 101), (4, 0.9, 102), (6, 2.0, 103), (5, 0.2, 104)]
    mats, a, b = [], [], []
    for L, W, seed in members:
        mats.append(pkg.chebfd_matrix_create_lattice("topi", L, L, L, t=1.0, m=1.0, W=W,
                                                     seed=seed, also_single=True))
        bound = 1.01 * (1.0 + 3.0 + W / 2)
        a.append(-bound)
        b.append(bound)
    E = pkg.chebfd_ensemble_create(mats, sell_C=1)
    res, its = pkg.chebfd_solve_batched(E, mats, a, b, -0.3, 0.3, 32, 160, eps=1e-9,
                                        precision=precision, max_iter=40, vectors=True)
    assert its >= 1
    for i, (L, W, seed) in enumerate(members):
        e = np.linalg.eigvalsh(lattice.to_scipy(*lattice.topi_csr(L, L, L, t=1.0, m=1.0, W=W,
                                                                  seed=seed)).toarray())
        exact = np.sort(e[np.abs(e) <= 0.3])
        r = res[i]
        normH = max(abs(a[i]), abs(b[i]))
        assert r["converged"] and r["nev"] == len(exact), (i, r["nev"], len(exact))
        if not len(exact):
            continue                      # a window inside this member's gap
        assert np.abs(np.sort(r["lam"]) - exact).max() <= 1e-10 * normH
        assert r["res"].max() <= 1e-9 * normH
        V = r["V"].cpu().numpy()
        assert np.abs(V.conj().T @ V - np.eye(r["nev"])).max() <= 1e-12
