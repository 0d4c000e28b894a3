"""Certificates, independent of the GPU, for the eigenpairs the library returns
at the benchmark workloads' full sizes, where dense diagonalisation is out of
reach (Sec. 3.1 step 8: a pair is converged when ||H v - lambda v|| <= eps ||H||).

For each returned pair the oracle recomputes the residual in FP64 with its own
CSR matrix (oracle.lattice) and a scipy product; the window set must be
+- paired (the insulator's chiral symmetry); two search-vector seeds must give
the same eigenvalues; the count must agree with the oracle's KPM estimate of
Eq. DOS:target within that estimate's stochastic and resolution error.  The
512-member disorder ensemble is solved in one batched call and every member is
certified the same way, the smallest members also against dense
diagonalisation."""
import numpy as np
import pytest
import torch

import paper_1510_04895_gb300 as pkg
from oracle import lattice
from paper_1510_04895_gb300 import workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _window(name):
    vals = {}
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def _oracle_residuals(Ho, V, lam):
    """||H v_k - lambda_k v_k|| by the oracle's CSR product, FP64."""
    R = Ho @ V - V * lam[None, :]
    return np.linalg.norm(R, axis=0)


def _kpm_count_tolerance(kpm_count, R, delta, S_w, M):
    """Three standard deviations of the stochastic trace over R probes
    (variance ~ N_T / R for a rank-N_T projector) plus the count that the
    Jackson kernel's resolution pi S_w / M smears across both window edges,
    with the linear DOS rho(delta) = 2 N_T / delta of the insulator and of
    graphene near zero energy."""
    return 3.0 * np.sqrt(kpm_count / R) + 2.0 * (2.0 * kpm_count / delta) * np.pi * S_w / M


def _certify(H, Ho, r, normH, chiral):
    V = r["V"].cpu().numpy()
    lam = r["lam"]
    res = _oracle_residuals(Ho, V, lam)
    assert res.max() <= 1e-9 * normH, res.max() / normH
    # the library's own residuals agree with the oracle's
    assert np.abs(res - r["res"]).max() <= 1e-11 * normH
    G = V.conj().T @ V
    assert np.abs(G - np.eye(len(lam))).max() <= 1e-10
    th = np.sort(lam)
    if chiral:
        assert np.abs(th + th[::-1]).max() <= 1e-10 * normH
    return th


def test_medium_insulator_solve_certified_by_oracle():
    """64x64x32x4 insulator (N = 524288), the benchmark's window (+-0.1401,
    oracle KPM count 100), n_s = 256, N_p = 309, MIXED_DF with the
    matrix-free steps: every returned pair has an oracle residual
    <= 1e-9 ||H||; +- pairing; seeds 0 and 1 give the same eigenvalues
    (within 1e-10 ||H||); the count is within the KPM estimate's error."""
    w = workloads.TOPI_MEDIUM
    g = _window("topi_64x64x32_window.txt")
    H = pkg.chebfd_matrix_create_lattice("topi", w["Lx"], w["Ly"], w["Lz"], t=w["t"], m=w["m"],
                                         W=w["W"], seed=w["seed"], also_single=True)
    H.set_matrix_free(True)
    Ho = lattice.to_scipy(*lattice.topi_csr(w["Lx"], w["Ly"], w["Lz"], t=w["t"], m=w["m"],
                                            W=w["W"], seed=w["seed"]))
    a, b, d = g["a"], g["b"], g["delta"]
    normH = max(abs(a), abs(b))
    found = []
    for seed in (0, 1):
        r = pkg.chebfd_solve(H, -d, d, 256, 309, eps=1e-9, kernel="lanczos", precision="mixed_df",
                             a=a, b=b, max_iter=40, seed=seed)
        assert r["converged"] and r["nev"] > 0
        found.append(_certify(H, Ho, r, normH, chiral=True))
        del r
        torch.cuda.empty_cache()
    assert len(found[0]) == len(found[1])
    assert np.abs(found[0] - found[1]).max() <= 1e-10 * normH
    tol = _kpm_count_tolerance(g["kpm_count"], g["R"], d, 0.5 * (b - a), g["M"])
    assert abs(len(found[0]) - g["kpm_count"]) <= tol, (len(found[0]), g["kpm_count"], tol)


def test_graphene_solve_certified_by_oracle():
    """1024x1024 graphene (N = 2097152), window +-0.01888 (oracle KPM count
    200), n_s = 512, N_p = 1779, MIXED_DF (FP32 filter until the residuals
    stall, double-float sweeps, FP64 Rayleigh-Ritz and residuals): every
    returned pair has an oracle residual <= 1e-9 ||H||, the count is within
    the KPM estimate's error.  (Graphene's spectrum is symmetric only without
    disorder, so there is no pairing check.)"""
    w = workloads.GRAPHENE
    g = _window("graphene_1024x1024_window.txt")
    H = pkg.chebfd_matrix_create_lattice("graphene", w["Lx"], w["Ly"], t=w["t"], W=w["W"],
                                         seed=w["seed"], also_single=True)
    Ho = lattice.to_scipy(*lattice.graphene_csr(w["Lx"], w["Ly"], t=w["t"], W=w["W"],
                                                seed=w["seed"]))
    a, b, d = g["a"], g["b"], g["delta"]
    normH = max(abs(a), abs(b))
    r = pkg.chebfd_solve(H, -d, d, 512, 1779, eps=1e-9, kernel="lanczos", precision="mixed_df",
                         a=a, b=b, max_iter=40, seed=0)
    assert r["converged"] and r["nev"] > 0
    _certify(H, Ho, r, normH, chiral=False)
    tol = _kpm_count_tolerance(g["kpm_count"], g["R"], d, 0.5 * (b - a), g["M"])
    assert abs(r["nev"] - g["kpm_count"]) <= tol, (r["nev"], g["kpm_count"], tol)


def test_ensemble_batched_solve_certified_by_oracle():
    """The 512-member disorder ensemble (L in U{10..20}, W in U[0.2, 2.0],
    seeds 100-611, window [-0.05, 0.05], n_s = 48, N_p = 300, Lanczos),
    solved in one chebfd_solve_batched call with MIXED precision: every member
    converges, every returned pair has an oracle residual <= 1e-9 ||H_i||,
    the windows are +- paired, and the first twelve members with L = 10
    (N = 4000) have exactly the window eigenvalues of dense diagonalisation."""
    e = workloads.ENSEMBLE
    members = workloads.ensemble_members(e["count"], e["first_seed"])
    mats, a, b = [], [], []
    for L, W, s in members:
        mats.append(pkg.chebfd_matrix_create_lattice("topi", L, L, L, t=e["t"], m=e["m"], W=W,
                                                     seed=s, also_single=True))
        bound = 1.01 * (abs(e["m"]) + 3 * e["t"] + W / 2)   # Weyl: clean radius plus W/2
        a.append(-bound)
        b.append(bound)
    n = sum(4 * L ** 3 for L, _, _ in members)
    X = torch.empty((n, e["ns"]), dtype=torch.complex64, device=DEV)
    E, _ = pkg.chebfd_ensemble_autotune(mats, X)
    del X
    lo, hi = e["window"]
    res, its = pkg.chebfd_solve_batched(E, mats, a, b, lo, hi, e["ns"], e["Np"], eps=1e-9,
                                        kernel=e["kernel"], precision="mixed", max_iter=40,
                                        vectors=True)
    dense_left = 12
    for i, (L, W, s) in enumerate(members):
        r = res[i]
        normH = max(abs(a[i]), abs(b[i]))
        assert r["converged"], (i, L, W, r["iterations"])
        Ho = lattice.to_scipy(*lattice.topi_csr(L, L, L, t=e["t"], m=e["m"], W=W, seed=s))
        if r["nev"]:
            _certify(None, Ho, r, normH, chiral=True)
        if L == 10 and dense_left > 0:
            dense_left -= 1
            ev = np.linalg.eigvalsh(Ho.toarray())
            exact = np.sort(ev[(ev >= lo) & (ev <= hi)])
            assert r["nev"] == len(exact), (i, r["nev"], len(exact))
            if len(exact):
                assert np.abs(np.sort(r["lam"]) - exact).max() <= 1e-10 * normH
    assert dense_left == 0


def _oracle_residuals_site_chunks(L, V, lam, chunk_sites=2_000_000):
    """||H v_k - lambda_k v_k|| for the columns of V with the oracle's rows of
    the insulator generated a block of sites at a time (the full CSR of 16e6
    rows would not fit beside V comfortably)."""
    Lx, Ly, Lz, t, m, W, seed = L
    nsite = Lx * Ly * Lz
    sq = np.zeros(V.shape[1])
    for s0 in range(0, nsite, chunk_sites):
        sites = np.arange(s0, min(nsite, s0 + chunk_sites), dtype=np.int64)
        rp, c, v = lattice.topi_csr(Lx, Ly, Lz, t=t, m=m, W=W, seed=seed, sites=sites)
        import scipy.sparse as sp
        rows = sp.csr_matrix((v, c, rp), shape=(4 * len(sites), 4 * nsite))
        R = rows @ V - V[4 * s0:4 * (s0 + len(sites))] * lam[None, :]
        sq += (np.abs(R) ** 2).sum(axis=0)
    return np.sqrt(sq)


@pytest.mark.skipif(__import__("os").environ.get("CHEBFD_LARGE_TESTS") != "1",
                    reason="the 16e6-row solve and its oracle certificate take about ten "
                           "minutes; opt in with CHEBFD_LARGE_TESTS=1")
def test_large_insulator_learned_solve_certified_by_oracle():
    """200x200x100x4 insulator (N = 16e6), window +-0.05305 (oracle KPM count
    100), MIXED_DF with the matrix-free steps and the MLP's (N_p, n_s,
    kernel): 12 returned pairs spread over the window get the oracle's FP64
    residual (its own rows of H, generated a block of sites at a time), each
    <= 1e-9 ||H|| and equal to the library's within 1e-11 ||H||; the window
    set is +- paired and its count within the KPM estimate's error."""
    import os
    from paper_1510_04895_gb300 import mlp_train
    w = workloads.TOPI_LARGE
    g = _window("topi_200x200x100_window.txt")
    H = pkg.chebfd_matrix_create_lattice("topi", w["Lx"], w["Ly"], w["Lz"], t=w["t"], m=w["m"],
                                         W=w["W"], seed=w["seed"], also_single=True)
    H.set_matrix_free(True)
    a, b, d = g["a"], g["b"], g["delta"]
    normH = max(abs(a), abs(b))
    net = pkg.MLP(mlp_train.N_IN, 128)
    net.set_params(np.load(os.path.join(os.path.dirname(pkg.__file__), "data",
                                        "mlp_weights.npy")).astype(np.float32))
    ns, Np, kern, _ = pkg.chebfd_choose_params(H, -d, d, mlp=net, a=a, b=b,
                                               m_feat=mlp_train.M_FEAT)
    r = pkg.chebfd_solve(H, -d, d, ns, Np, eps=1e-9, kernel=kern, precision="mixed_df", a=a, b=b,
                         max_iter=40, seed=0)
    assert r["converged"] and r["nev"] > 0
    lam = r["lam"]
    th = np.sort(lam)
    assert np.abs(th + th[::-1]).max() <= 1e-10 * normH
    tol = _kpm_count_tolerance(g["kpm_count"], g["R"], d, 0.5 * (b - a), g["M"])
    assert abs(r["nev"] - g["kpm_count"]) <= tol, (r["nev"], g["kpm_count"], tol)
    order = np.argsort(lam)
    pick = order[np.unique(np.linspace(0, len(lam) - 1, 12).round().astype(int))]
    V = r["V"][:, torch.from_numpy(pick).to(r["V"].device)].cpu().numpy()
    res = _oracle_residuals_site_chunks(
        (w["Lx"], w["Ly"], w["Lz"], w["t"], w["m"], w["W"], w["seed"]), V, lam[pick])
    assert res.max() <= 1e-9 * normH, res.max() / normH
    assert np.abs(res - r["res"][pick]).max() <= 1e-11 * normH
    G = V.conj().T @ V
    assert np.abs(G - np.eye(len(pick))).max() <= 1e-10
