"""Parity of the dense FP64 steps and of the whole ChebFD iteration (through the
C ABI) with the CPU oracle and with dense diagonalisation."""
import numpy as np
import pytest
import torch

import paper_1510_04895_gb300 as pkg
from oracle import bounds as obounds, lattice, rr as orr, solve as osolve, svqb as osvqb
from paper_1510_04895_gb300 import workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def span_distance(A, B):
    """max-norm of B minus its projection onto span(A) (A, B orthonormal): zero
    exactly when span(B) lies in span(A); linear in a perturbation of either."""
    return float(np.abs(B - A @ (A.conj().T @ B)).max())


@pytest.mark.parametrize("cplx", [True, False])
def test_orthonormalize_full_rank_matches_oracle(cplx):
    Y0 = workloads.random_block(7, 3001 if cplx else 3000, 48, cplx)
    Y0[:, 5] *= 1e-5
    Y = torch.from_numpy(Y0).to(DEV)
    rank, cnt = pkg.chebfd_orthonormalize(Y, seed=3)
    Q = Y.cpu().numpy()
    Qo, rank_o, cnt_o = osvqb.svqb(Y0, seed=3)
    assert rank == rank_o == 48 and cnt == cnt_o == 0
    assert np.abs(Q.conj().T @ Q - np.eye(48)).max() <= 1e-12
    assert span_distance(Q, Qo) <= 1e-10


def test_orthonormalize_rank_deficient_refills_like_oracle():
    Y0 = workloads.random_block(8, 2000, 12, True)
    Z = np.concatenate([Y0, Y0 @ workloads.random_block(9, 12, 8, True)], axis=1)  # rank 12 of 20
    Y = torch.from_numpy(np.ascontiguousarray(Z)).to(DEV)
    rank, cnt = pkg.chebfd_orthonormalize(Y, seed=5, refill_counter=3)
    Qo, rank_o, cnt_o = osvqb.svqb(Z, seed=5, refill_counter=3)
    assert rank == rank_o == 12 and cnt == cnt_o == 11
    Q = Y.cpu().numpy()
    assert np.abs(Q.conj().T @ Q - np.eye(20)).max() <= 1e-12
    assert span_distance(Q, Qo) <= 1e-9


@pytest.mark.parametrize("kind", ["topi", "graphene"])
def test_rayleigh_ritz_matches_oracle(kind):
    if kind == "topi":
        H = pkg.chebfd_matrix_create_lattice("topi", 4, 5, 6, W=1.1, seed=4)
        Ho = lattice.to_scipy(*lattice.topi_csr(4, 5, 6, W=1.1, seed=4))
    else:
        H = pkg.chebfd_matrix_create_lattice("graphene", 30, 20, W=1.0, seed=4)
        Ho = lattice.to_scipy(*lattice.graphene_csr(30, 20, W=1.0, seed=4))
    Y0, _, _ = osvqb.svqb(workloads.random_block(1, H.n, 32, H.is_complex))
    Y = torch.from_numpy(np.ascontiguousarray(Y0)).to(DEV)
    theta, res = pkg.chebfd_rayleigh_ritz(H, Y)
    th_o, V_o, res_o = orr.rayleigh_ritz(Ho, Y0)
    normH = abs(Ho).sum(axis=1).max()
    assert np.abs(theta - th_o).max() <= 1e-12 * normH
    assert np.abs(res - res_o).max() <= 1e-11 * normH
    V = Y.cpu().numpy()
    assert np.allclose(orr.residual_norms(Ho, V, theta), res, atol=1e-11 * normH)
    r2 = pkg.chebfd_residuals(H, Y, theta)
    assert np.allclose(r2, res, atol=1e-11 * normH)


def test_rayleigh_ritz_exact_invariant_subspace():
    H = pkg.chebfd_matrix_create_lattice("topi", 3, 3, 3, W=0.8, seed=9)
    Ho = lattice.to_scipy(*lattice.topi_csr(3, 3, 3, W=0.8, seed=9))
    lam, Vd = np.linalg.eigh(Ho.toarray())
    Y = torch.from_numpy(np.ascontiguousarray(Vd[:, 40:52])).to(DEV)
    theta, res = pkg.chebfd_rayleigh_ritz(H, Y)
    assert np.abs(theta - lam[40:52]).max() <= 1e-12
    assert res.max() <= 1e-12


@pytest.mark.parametrize("kind", ["topi", "graphene"])
def test_harmonic_ritz_matches_oracle(kind):
    """Harmonic Ritz extraction (Sec. 6) on a random orthonormal block: the
    Rayleigh quotients of the oracle's harmonic vectors, unit vectors whose
    residuals recomputed on the CPU equal the returned ones."""
    if kind == "topi":
        H = pkg.chebfd_matrix_create_lattice("topi", 4, 5, 6, W=1.1, seed=4)
        Ho = lattice.to_scipy(*lattice.topi_csr(4, 5, 6, W=1.1, seed=4))
        tau = 0.1
    else:
        H = pkg.chebfd_matrix_create_lattice("graphene", 30, 20, W=1.0, seed=4)
        Ho = lattice.to_scipy(*lattice.graphene_csr(30, 20, W=1.0, seed=4))
        tau = -0.05
    Y0, _, _ = osvqb.svqb(workloads.random_block(1, H.n, 32, H.is_complex))
    Y = torch.from_numpy(np.ascontiguousarray(Y0)).to(DEV)
    theta, res = pkg.chebfd_harmonic_ritz(H, Y, tau)
    rho_o, V_o, res_o, _ = orr.harmonic_ritz(Ho, Y0, tau)
    normH = abs(Ho).sum(axis=1).max()
    assert np.all(np.diff(theta) >= 0)
    assert np.abs(theta - rho_o).max() <= 1e-10 * normH
    assert np.abs(res - res_o).max() <= 1e-10 * normH
    V = Y.cpu().numpy()
    assert np.abs(np.linalg.norm(V, axis=0) - 1.0).max() <= 1e-12
    assert np.allclose(orr.residual_norms(Ho, V, theta), res, atol=1e-11 * normH)


def test_harmonic_ritz_exact_subspace_and_singular_fallback():
    """On eigenvectors the harmonic pairs are exact; with tau equal to one of
    their eigenvalues (Z^H Z singular) the ordinary Ritz pairs come back."""
    H = pkg.chebfd_matrix_create_lattice("topi", 3, 3, 3, W=0.8, seed=9)
    Ho = lattice.to_scipy(*lattice.topi_csr(3, 3, 3, W=0.8, seed=9))
    lam, Vd = np.linalg.eigh(Ho.toarray())
    Y = torch.from_numpy(np.ascontiguousarray(Vd[:, 40:52])).to(DEV)
    theta, res = pkg.chebfd_harmonic_ritz(H, Y, 0.5 * (lam[40] + lam[51]) + 1e-3)
    assert np.abs(theta - lam[40:52]).max() <= 1e-11
    assert res.max() <= 1e-11
    n = 64
    d = np.arange(n) / 8.0 - 3.0                       # exact binary eigenvalues
    D = pkg.chebfd_matrix_create_csr(np.arange(n + 1), np.arange(n), d)
    E = np.zeros((n, 8))
    E[np.arange(8) * 5, np.arange(8)] = 1.0            # unit vectors of eigenvalues d[5 k]
    Ye = torch.from_numpy(E).to(DEV)
    theta, res = pkg.chebfd_harmonic_ritz(D, Ye, d[15])
    assert np.array_equal(theta, np.sort(d[np.arange(8) * 5]))
    assert res.max() == 0.0


def test_convert_block_round_trip():
    X0 = workloads.random_block(2, 1000, 16, True)
    X = torch.from_numpy(X0).to(DEV)
    Y = torch.empty((1000, 16), dtype=torch.complex64, device=DEV)
    pkg.chebfd_convert_block(X, Y)
    assert np.array_equal(Y.cpu().numpy(), X0.astype(np.complex64))
    Z = torch.empty_like(X)
    pkg.chebfd_convert_block(Y, Z)
    assert np.array_equal(Z.cpu().numpy(), X0.astype(np.complex64).astype(np.complex128))


def _dense_window(Ho, lo, hi):
    e = np.linalg.eigvalsh(Ho.toarray())
    return e[(e >= lo) & (e <= hi)], e


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_df"])
def test_solve_smallest_insulator_against_dense(precision):
    """8x8x8x4 insulator (N = 2048), W = 0.5, window [-0.1, 0.1], n_s = 64,
    N_p = 200, Jackson: all window eigenvalues within 1e-10 ||H|| of the dense
    eigensolver, residuals <= 1e-9 ||H||, chiral +- pairing."""
    w = workloads.TOPI_SMALL
    H = pkg.chebfd_matrix_create_lattice("topi", 8, 8, 8, t=1.0, m=1.0, W=0.5, seed=0,
                                         also_single=True)
    Ho = lattice.to_scipy(*lattice.topi_csr(8, 8, 8, t=1.0, m=1.0, W=0.5, seed=0))
    r = pkg.chebfd_solve(H, -0.1, 0.1, 64, 200, eps=1e-9, kernel="jackson", precision=precision)
    ew, e = _dense_window(Ho, -0.1, 0.1)
    normH = max(abs(r["a"]), abs(r["b"]))
    assert r["converged"] and r["nev"] == len(ew) > 0
    assert np.abs(np.sort(r["lam"]) - ew).max() <= 1e-10 * normH
    assert r["res"].max() <= 1e-9 * normH
    V = r["V"].cpu().numpy()
    assert np.abs(V.conj().T @ V - np.eye(r["nev"])).max() <= 1e-12
    assert np.abs(orr.residual_norms(Ho, V, r["lam"])).max() <= 1e-9 * normH
    th = np.sort(r["lam"])
    assert np.abs(th + th[::-1]).max() <= 1e-10 * normH
    if precision != "fp64":
        assert 1 <= r["fp64_iterations"] < r["iterations"]
    # the oracle run on the same workload finds the same eigenvalues
    ro = osolve.chebfd(Ho, r["a"], r["b"], -0.1, 0.1, 64, 200, 1e-9, kind="jackson", seed=0)
    assert np.abs(np.sort(ro["theta"]) - th).max() <= 1e-10 * normH


@pytest.mark.parametrize("precision", ["mixed", "mixed_df"])
def test_solve_graphene_real_against_dense(precision):
    H = pkg.chebfd_matrix_create_lattice("graphene", 40, 36, W=1.0, seed=2, also_single=True)
    Ho = lattice.to_scipy(*lattice.graphene_csr(40, 36, W=1.0, seed=2))
    r = pkg.chebfd_solve(H, -0.05, 0.05, 48, 400, eps=1e-9, kernel="lanczos", precision=precision)
    ew, _ = _dense_window(Ho, -0.05, 0.05)
    normH = max(abs(r["a"]), abs(r["b"]))
    assert r["converged"] and r["nev"] == len(ew) > 0
    assert np.abs(np.sort(r["lam"]) - ew).max() <= 1e-10 * normH
    assert r["res"].max() <= 1e-9 * normH


@pytest.mark.parametrize("precision", ["fp64", "mixed_df"])
def test_solve_harmonic_smallest_insulator_against_dense(precision):
    """Step 7 with harmonic Ritz pairs for the window centre: the same window
    eigenvalues as dense diagonalisation and as the oracle's harmonic run,
    residuals <= 1e-9 ||H||, unit vectors, in no more iterations than with
    ordinary Ritz pairs."""
    H = pkg.chebfd_matrix_create_lattice("topi", 8, 8, 8, t=1.0, m=1.0, W=0.5, seed=0,
                                         also_single=True)
    Ho = lattice.to_scipy(*lattice.topi_csr(8, 8, 8, t=1.0, m=1.0, W=0.5, seed=0))
    r = pkg.chebfd_solve(H, -0.1, 0.1, 64, 200, eps=1e-9, kernel="jackson", precision=precision,
                         extraction="harmonic")
    ritz = pkg.chebfd_solve(H, -0.1, 0.1, 64, 200, eps=1e-9, kernel="jackson",
                            precision=precision)
    ew, _ = _dense_window(Ho, -0.1, 0.1)
    normH = max(abs(r["a"]), abs(r["b"]))
    assert r["converged"] and r["nev"] == len(ew) > 0
    assert np.abs(np.sort(r["lam"]) - ew).max() <= 1e-10 * normH
    assert r["res"].max() <= 1e-9 * normH
    V = r["V"].cpu().numpy()
    assert np.abs(np.linalg.norm(V, axis=0) - 1.0).max() <= 1e-12
    assert np.abs(orr.residual_norms(Ho, V, r["lam"])).max() <= 1e-9 * normH
    assert r["iterations"] <= ritz["iterations"]
    ro = osolve.chebfd(Ho, r["a"], r["b"], -0.1, 0.1, 64, 200, 1e-9, kind="jackson", seed=0,
                       extraction="harmonic")
    assert np.abs(np.sort(ro["theta"]) - np.sort(r["lam"])).max() <= 1e-10 * normH


@pytest.mark.parametrize("precision", ["fp64", "mixed_df"])
def test_solve_inset_window_half_degree_against_dense(precision):
    """The filter window narrowed by half the target half-width with half
    the degree (N_p = 100, Lanczos): all window eigenvalues of the dense
    eigensolver, residuals <= 1e-9 ||H||, the oracle's eigenvalues."""
    H = pkg.chebfd_matrix_create_lattice("topi", 8, 8, 8, t=1.0, m=1.0, W=0.5, seed=0,
                                         also_single=True)
    Ho = lattice.to_scipy(*lattice.topi_csr(8, 8, 8, t=1.0, m=1.0, W=0.5, seed=0))
    r = pkg.chebfd_solve(H, -0.1, 0.1, 64, 100, eps=1e-9, kernel="lanczos", precision=precision,
                         window_inset=0.5)
    ew, _ = _dense_window(Ho, -0.1, 0.1)
    normH = max(abs(r["a"]), abs(r["b"]))
    assert r["converged"] and r["nev"] == len(ew) > 0
    assert np.abs(np.sort(r["lam"]) - ew).max() <= 1e-10 * normH
    assert r["res"].max() <= 1e-9 * normH
    ro = osolve.chebfd(Ho, r["a"], r["b"], -0.1, 0.1, 64, 100, 1e-9, seed=0, window_inset=0.5)
    assert np.abs(np.sort(ro["theta"]) - np.sort(r["lam"])).max() <= 1e-10 * normH
    with pytest.raises(pkg.ChebFDError):
        pkg.chebfd_solve(H, -0.1, 0.1, 64, 100, window_inset=1.0)


def test_solve_reports_no_convergence():
    H = pkg.chebfd_matrix_create_lattice("topi", 4, 4, 4, W=0.5, seed=0)
    r = pkg.chebfd_solve(H, -0.2, 0.2, 16, 20, eps=1e-12, kernel="jackson", max_iter=1)
    assert r["status"] == "ENOCONV" and not r["converged"] and r["iterations"] == 1


def test_solve_weak_filter_is_not_taken_for_an_empty_window():
    """The oracle's weak-filter case through the C ABI: flat-DOS diagonal H
    (D = 400), window [-0.02, 0.02] with 8 eigenvalues, N_p = 30, n_s = 64.
    The true pairs are ghost-flagged for several iterations; the solve must
    not stop with an empty "converged" window but find all 8 eigenvalues.
    With N_p = 20, n_s = 32 and a budget of 12 iterations it reports ENOCONV.
    A window inside a spectral gap still ends converged with no pairs."""
    import scipy.sparse as sp
    D = 400
    lam = -1.0 + 2.0 * np.arange(1, D + 1) / (D + 1)
    H = pkg.chebfd_matrix_create_csr(np.arange(D + 1), np.arange(D), lam)
    ew = lam[(lam >= -0.02) & (lam <= 0.02)]
    r = pkg.chebfd_solve(H, -0.02, 0.02, 64, 30, eps=1e-10, a=-1.001, b=1.001, max_iter=40)
    assert r["converged"] and r["nev"] == 8
    assert np.abs(np.sort(r["lam"]) - ew).max() <= 1e-10
    ro = osolve.chebfd(sp.diags(lam).tocsr(), -1.001, 1.001, -0.02, 0.02, 64, 30, 1e-10,
                       complex_values=False, max_iter=40)
    assert ro["converged"] and abs(ro["iterations"] - r["iterations"]) <= 2
    r = pkg.chebfd_solve(H, -0.02, 0.02, 32, 20, eps=1e-10, a=-1.001, b=1.001, max_iter=12)
    assert r["status"] == "ENOCONV" and not r["converged"] and r["iterations"] == 12
    gap = np.concatenate([np.linspace(-1, -0.2, 300), np.linspace(0.2, 1, 300)])
    G = pkg.chebfd_matrix_create_csr(np.arange(601), np.arange(600), gap)
    r = pkg.chebfd_solve(G, -0.05, 0.05, 16, 60, eps=1e-9, a=-1.01, b=1.01, max_iter=20)
    assert r["converged"] and r["nev"] == 0 and r["iterations"] <= 12


def test_solve_adaptive_degree_matches_oracle_rule():
    """Adaptive N_p (Sec. 6 with the rule of Sec. 2.4) through the C ABI on the
    oracle pin's linear-DOS diagonal (D = 4000, N_T = 100, N_S = 200, started at
    N_p = 300): the degree chosen from the first filter's moments agrees with
    the oracle's (same search vectors) within 2 %, later iterations use it, all
    100 eigenvalues are found, with fewer products than at the fixed degree.
    The smallest insulator (MIXED_DF, first filter in complex64) also finds
    every dense window eigenvalue."""
    import scipy.sparse as sp
    D, NS = 4000, 200
    delta = np.sqrt(100.0 / D)
    lam = lattice.linear_dos_eigs(D)
    H = pkg.chebfd_matrix_create_csr(np.arange(D + 1), np.arange(D), lam)
    r = pkg.chebfd_solve(H, -delta, delta, NS, 300, eps=1e-10, a=-1.0, b=1.0, adaptive=True)
    ro = osolve.chebfd(sp.diags(lam).tocsr(), -1.0, 1.0, -delta, delta, NS, 300, 1e-10,
                       complex_values=False, adaptive=True)
    Np = ro["adapted"][2]
    assert r["log"][0]["Np"] == 300
    assert all(abs(rec["Np"] - Np) <= 0.02 * Np for rec in r["log"][1:])
    exact = np.sort(lam[np.abs(lam) <= delta])
    assert r["converged"] and r["nev"] == len(exact) == 100
    assert np.abs(np.sort(r["lam"]) - exact).max() <= 1e-10
    fixed = pkg.chebfd_solve(H, -delta, delta, NS, 300, eps=1e-10, a=-1.0, b=1.0)
    assert r["n_mvm"] < fixed["n_mvm"]
    Ht = pkg.chebfd_matrix_create_lattice("topi", 8, 8, 8, t=1.0, m=1.0, W=0.5, seed=0,
                                          also_single=True)
    Ho = lattice.to_scipy(*lattice.topi_csr(8, 8, 8, t=1.0, m=1.0, W=0.5, seed=0))
    r = pkg.chebfd_solve(Ht, -0.1, 0.1, 64, 400, eps=1e-9, kernel="lanczos",
                         precision="mixed_df", adaptive=True)
    ew, _ = _dense_window(Ho, -0.1, 0.1)
    normH = max(abs(r["a"]), abs(r["b"]))
    assert r["converged"] and r["nev"] == len(ew) > 0
    assert np.abs(np.sort(r["lam"]) - ew).max() <= 1e-10 * normH
    assert r["log"][1]["Np"] != 400


@pytest.mark.parametrize("precision", ["fp64", "mixed_df"])
def test_solve_locking_matches_oracle(precision):
    """Hard locking (Sec. 6) through the C ABI on the oracle pin's linear-DOS
    diagonal (D = 4000, N_T = 100, N_S = 200, N_p = 95): pairs are locked four
    at a time, all 100 eigenvalues are found with orthonormal vectors, fewer
    products are needed than without locking (FP64: deflation with cuBLAS;
    MIXED_DF: on the tensor cores).  Harmonic pairs with locking: EINVAL."""
    D, NS, Np = 4000, 200, 95
    delta = np.sqrt(100.0 / D)
    lam = lattice.linear_dos_eigs(D)
    H = pkg.chebfd_matrix_create_csr(np.arange(D + 1), np.arange(D), lam, also_single=True)
    r = pkg.chebfd_solve(H, -delta, delta, NS, Np, eps=1e-10, a=-1.0, b=1.0,
                         precision=precision, locking=True)
    plain = pkg.chebfd_solve(H, -delta, delta, NS, Np, eps=1e-10, a=-1.0, b=1.0,
                             precision=precision)
    exact = np.sort(lam[np.abs(lam) <= delta])
    assert r["converged"] and r["nev"] == len(exact) == 100
    assert np.abs(r["lam"] - exact).max() <= 1e-10
    V = r["V"].cpu().numpy()
    assert np.abs(V.T @ V - np.eye(100)).max() <= 1e-10
    locked = max(rec["locked"] for rec in r["log"])
    assert locked >= 4 and locked % 4 == 0
    assert r["n_mvm"] < plain["n_mvm"]
    with pytest.raises(pkg.ChebFDError):
        pkg.chebfd_solve(H, -delta, delta, NS, Np, a=-1.0, b=1.0, locking=True,
                         extraction="harmonic")


def test_solve_locking_deflation_over_a_long_run():
    """The oracle pin's long locking run through the C ABI (linear-DOS
    diagonal, D = 4000, N_S = 200, N_p = 40, eps = 1e-13): pairs lock from the
    early iterations on and the run goes on for many more, so only the
    deflation of each filtered block against the locked vectors keeps their
    leftover components from returning as duplicate pairs.  Exactly the 100
    window eigenvalues, each once, with orthonormal vectors."""
    D, NS, Np = 4000, 200, 40
    delta = np.sqrt(100.0 / D)
    lam = lattice.linear_dos_eigs(D)
    H = pkg.chebfd_matrix_create_csr(np.arange(D + 1), np.arange(D), lam)
    r = pkg.chebfd_solve(H, -delta, delta, NS, Np, eps=1e-13, a=-1.0, b=1.0, locking=True,
                         max_iter=40)
    exact = np.sort(lam[np.abs(lam) <= delta])
    assert r["converged"] and r["nev"] == len(exact) == 100
    assert np.abs(np.sort(r["lam"]) - exact).max() <= 1e-12
    V = r["V"].cpu().numpy()
    assert np.abs(V.T @ V - np.eye(100)).max() <= 1e-10
    assert max(rec["locked"] for rec in r["log"]) >= 80
