"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself: a
value printed in the paper (fixtures under tests/golden/, each citing its
table or figure), a closed form, an invariant, brute force on a tiny case, or
a library routine that the definition reduces to.
"""
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.sparse as sp

from oracle import bounds, coeffs, filter as filt, kpm, lattice, quality, rng, rr, sell, solve, svqb

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


# ---------------------------------------------------------------- generator


def test_splitmix64_known_answers():
    want = [int(r[0], 16) for r in _rows("splitmix64_seed0.txt")]
    got = [int(x) for x in rng.words(0, 0, np.arange(len(want)))]
    assert got == want


def test_uniform_is_the_top_53_bits():
    """u = (word >> 11) 2^-53 on the published SplitMix64 outputs, in exact
    integer arithmetic."""
    want = [int(r[0], 16) for r in _rows("splitmix64_seed0.txt")]
    got = rng.uniform(0, 0, np.arange(len(want)))
    assert [float(x) for x in got] == [(w >> 11) / 2.0 ** 53 for w in want]


def test_uniform_range_and_streams_differ():
    u = rng.uniform(7, 0, np.arange(10000))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.02
    assert not np.array_equal(rng.words(7, 0, np.arange(8)), rng.words(7, 1, np.arange(8)))


# ---------------------------------------------------------------- coefficients


@pytest.mark.parametrize("window", [(-0.1, 0.1), (-0.3, 0.05), (0.2, 0.9)])
def test_window_coefficients_match_defining_integral(window):
    """c_n = (2 - delta_n0)/pi int_{-1}^{1} W T_n (1-x^2)^(-1/2) dx  (Sec. 2.1),
    integrated numerically in x = cos(theta) on [a, b] = [-2, 3]."""
    a, b = -2.0, 3.0
    lo, hi = window
    alpha, beta = coeffs.scaling(a, b)
    c = coeffs.window_cn(a, b, lo, hi, 40)
    for n in (0, 1, 2, 7, 40):
        # W((b-a)/2 x + (a+b)/2) is 1 for x in [alpha lo + beta, alpha hi + beta]
        x0, x1 = alpha * lo + beta, alpha * hi + beta
        f = lambda x: np.cos(n * np.arccos(x)) / np.sqrt(1 - x * x)
        val, _ = scipy.integrate.quad(f, x0, x1, limit=200)
        ref = (2.0 - (n == 0)) / np.pi * val
        assert abs(c[n] - ref) < 1e-10, (n, c[n], ref)


@pytest.mark.parametrize("a,b", [(-5.5, 5.5), (-2.0, 3.0), (0.5, 7.25), (-9.0, -1.0)])
def test_scaling_maps_interval(a, b):
    """alpha a + beta = -1 and alpha b + beta = 1 (Sec. 2.1), on symmetric and
    shifted intervals (beta = 0 only for the symmetric one)."""
    alpha, beta = coeffs.scaling(a, b)
    assert alpha * a + beta == pytest.approx(-1.0, abs=1e-15)
    assert alpha * b + beta == pytest.approx(1.0, abs=1e-15)


def test_kernel_factors_special_values():
    Np = 50
    for k in coeffs.KERNELS:
        assert coeffs.kernel_gn(k, Np)[0] == pytest.approx(1.0, abs=1e-14)
    j = coeffs.kernel_gn("jackson", Np)
    assert abs(j[Np]) < 1e-14 and abs(j[Np - 1]) < 1e-14
    f = coeffs.kernel_gn("fejer", Np)
    assert f[Np] == pytest.approx(1.0 / (Np + 1))
    l1 = coeffs.kernel_gn("lanczos", Np, mu=1.0)
    n = np.arange(1, Np + 1)
    assert np.allclose(l1[1:], np.sinc(n / (Np + 1.0)))
    assert np.allclose(coeffs.kernel_gn("lanczos", Np, mu=3.0)[1:], l1[1:] ** 3)


@pytest.mark.parametrize("kind", ["jackson", "fejer"])
def test_positive_kernels_have_no_gibbs_overshoot(kind):
    """Fejer and Jackson are positive kernels (WWAF06): the damped expansion of
    the window stays inside [0, 1]; the undamped one overshoots (Fig. filters)."""
    gc = coeffs.filter_coeffs(-1, 1, -0.01, 0.01, 200, kind)
    x = np.linspace(-1, 1, 20001)
    p = coeffs.eval_poly(gc, x)
    assert p.min() > -1e-12 and p.max() < 1 + 1e-12
    p_none = coeffs.eval_poly(coeffs.filter_coeffs(-1, 1, -0.01, 0.01, 200, "none"), x)
    assert p_none.min() < -0.01


def test_filter_is_about_one_inside_window():
    """p ~ 1 inside a wide window (Sec. 2.2) - pins the sign reading of c_n."""
    gc = coeffs.filter_coeffs(-1, 1, -0.2, 0.2, 400, "lanczos")
    assert coeffs.eval_poly(gc, np.array([0.0]))[0] == pytest.approx(1.0, abs=1e-3)


# ---------------------------------------------------------------- filter


def test_filter_on_diagonal_matches_cos_closed_form():
    """T_n(cos t) = cos(n t) (Sec. 2.1): for diagonal H and unit vectors the
    filtered entry i is sum_n gc_n cos(n arccos(alpha l_i + beta))."""
    lam = np.linspace(-1.9, 2.9, 300)
    H = sp.diags(lam).tocsr()
    a, b = -2.0, 3.0
    alpha, beta = coeffs.scaling(a, b)
    gc = coeffs.filter_coeffs(a, b, -0.3, 0.4, 250, "lanczos")
    X = np.eye(300)[:, :40] + 0.5 * np.eye(300)[:, 100:140]
    Y = filt.filter_block(H, alpha, beta, gc, X)
    th = np.arccos(alpha * lam + beta)
    n = np.arange(len(gc))
    p = np.cos(np.outer(th, n)) @ gc
    assert np.abs(Y - p[:, None] * X).max() <= 1e-13 * np.abs(gc).sum()


def test_filter_matches_dense_spectral_form_on_small_lattice():
    """p[H] X = V p(Lambda) V^H X with V, Lambda from a dense eigensolver."""
    rp, c, v = lattice.topi_csr(3, 4, 3, W=1.3, seed=11)
    H = lattice.to_scipy(rp, c, v)
    lam, V = np.linalg.eigh(H.toarray())
    a, b = lam[0] - 0.1, lam[-1] + 0.1
    alpha, beta = coeffs.scaling(a, b)
    gc = coeffs.filter_coeffs(a, b, -0.4, 0.4, 120, "jackson")
    rs = np.random.default_rng(3)
    X = rs.standard_normal((H.shape[0], 5)) + 1j * rs.standard_normal((H.shape[0], 5))
    Y = filt.filter_block(H, alpha, beta, gc, X)
    p = coeffs.eval_poly(gc, alpha * lam + beta)
    ref = V @ (p[:, None] * (V.conj().T @ X))
    assert np.linalg.norm(Y - ref) <= 1e-12 * np.linalg.norm(X)


def test_moments_on_diagonal_and_doubling_identities():
    lam = np.linspace(-0.95, 0.97, 64)
    H = sp.diags(lam).tocsr()
    rs = np.random.default_rng(0)
    X = rs.standard_normal((64, 3))
    mu = filt.moments(H, 1.0, 0.0, X, 30)
    th = np.arccos(lam)
    ref = np.array([(X * X * np.cos(n * th)[:, None]).sum(axis=0) for n in range(30)])
    assert np.allclose(mu, ref, atol=1e-12)
    T = filt.chebyshev_vectors(H, 1.0, 0.0, X, 14)
    for n in range(1, 14):
        assert np.allclose(mu[2 * n], 2 * (T[n] * T[n]).sum(0) - mu[0], atol=1e-11)
        assert np.allclose(mu[2 * n + 1], 2 * (T[n + 1] * T[n]).sum(0) - mu[1], atol=1e-11)


# ---------------------------------------------------------------- lattices


def test_topi_structure_hermitian_and_clean_spectrum():
    rp, c, v = lattice.topi_csr(4, 4, 6, W=0.0)
    assert np.all(np.diff(rp) == 13)                     # N_nzr = 13 (Sec. 4)
    for r in range(0, len(rp) - 1, 37):
        assert np.all(np.diff(c[rp[r]:rp[r + 1]]) > 0)
    H = lattice.to_scipy(rp, c, v)
    assert (H - H.conj().T).count_nonzero() == 0          # bitwise Hermitian
    e = np.linalg.eigvalsh(H.toarray())
    assert np.abs(e - lattice.topi_clean_spectrum(4, 4, 6)).max() < 1e-12
    assert np.sum(np.abs(e) < 1e-12) == 12                # Dirac points perm(0,0,pi)
    assert e.max() == pytest.approx(4.0)                  # m + 3t


def test_topi_disorder_chiral_symmetry():
    rp, c, v = lattice.topi_csr(3, 3, 4, W=2.0, seed=5)
    H = lattice.to_scipy(rp, c, v)
    assert (H - H.conj().T).count_nonzero() == 0
    e = np.linalg.eigvalsh(H.toarray())
    assert np.abs(e + e[::-1]).max() < 1e-12              # spec(H) = -spec(H)
    V = lattice.disorder(5, 36, 2.0)
    assert V.min() >= -1.0 and V.max() < 1.0
    d = H.diagonal().real
    assert np.array_equal(d[0::4], 1.0 + V) and np.array_equal(d[2::4], -(1.0 + V))


def test_topi_small_lattice_duplicates_summed():
    rp, c, v = lattice.topi_csr(2, 2, 2, W=0.3, seed=1)
    H = lattice.to_scipy(rp, c, v)
    assert (H - H.conj().T).count_nonzero() == 0
    big = lattice.to_scipy(*lattice.topi_csr(2, 2, 2, W=0.3, seed=1))
    # with edge 2, +e_j and -e_j reach the same site: T_j + T_j^dagger = -t Gamma1
    assert np.allclose(H.toarray()[0, 4 * 1 + 0], -1.0)
    assert np.array_equal(H.toarray(), big.toarray())


def test_graphene_disorder_on_the_diagonal():
    """Onsite disorder of the graphene generator: W (u - 1/2) per orbital, so
    the diagonal lies in [-W/2, W/2) with the uniform distribution's spread
    W / sqrt(12), changes with the seed, and vanishes at W = 0; the hopping
    entries stay -t whatever W."""
    Lx, Ly, W = 30, 20, 1.4
    rp, c, v = lattice.graphene_csr(Lx, Ly, t=1.0, W=W, seed=3)
    Hs = lattice.to_scipy(rp, c, v)
    d = Hs.diagonal()
    n = len(d)
    assert np.all(d >= -W / 2) and np.all(d < W / 2)
    assert abs(d.std() - W / np.sqrt(12.0)) <= 0.08 * W / np.sqrt(12.0)
    assert abs(d.mean()) <= 4 * W / np.sqrt(12.0 * n)
    off = (Hs - __import__("scipy").sparse.diags(d)).tocsr()
    off.eliminate_zeros()
    assert np.all(off.data == -1.0) and off.nnz == 3 * n
    d2 = lattice.to_scipy(*lattice.graphene_csr(Lx, Ly, t=1.0, W=W, seed=4)).diagonal()
    assert np.abs(d2 - d).max() > 0.1 * W
    d0 = lattice.to_scipy(*lattice.graphene_csr(Lx, Ly, t=1.0, W=0.0, seed=3)).diagonal()
    assert np.all(d0 == 0.0)


def test_graphene_structure_and_clean_spectrum():
    rp, c, v = lattice.graphene_csr(6, 9, W=0.0)
    assert np.all(np.diff(rp) == 4)
    H = lattice.to_scipy(rp, c, v)
    assert (H - H.T).count_nonzero() == 0
    e = np.linalg.eigvalsh(H.toarray())
    assert np.abs(e - lattice.graphene_clean_spectrum(6, 9)).max() < 1e-12
    rp, c, v = lattice.graphene_csr(5, 5, W=1.0, seed=2)
    d = lattice.to_scipy(rp, c, v).diagonal()
    assert d.min() >= -0.5 and d.max() < 0.5


def test_topi_rows_of_selected_sites_equal_full_matrix_rows():
    """The site-restricted generator (used for sampled checks at N = 16e6)
    gives exactly the rows of the full matrix."""
    full = lattice.to_scipy(*lattice.topi_csr(5, 4, 6, W=1.3, seed=7)).toarray()
    sites = np.array([0, 7, 33, 119])
    rp, c, v = lattice.topi_csr(5, 4, 6, W=1.3, seed=7, sites=sites)
    rows = (4 * sites[:, None] + np.arange(4)).ravel()
    dense = np.zeros((len(rows), full.shape[1]), complex)
    for i in range(len(rows)):
        for p in range(rp[i], rp[i + 1]):
            dense[i, c[p]] += v[p]
    assert np.array_equal(dense, full[rows])


def test_topi_slab_structure_and_clean_spectrum():
    """Eq. Ham on a slab: the clean spectrum equals the union over (k_x, k_y)
    of the layered chain built from the Bloch form (independent of the
    real-space generator); surface rows have 11 entries, bulk rows 13; the
    disorder sits on Gamma0 = 1, so tr H = 4 sum_s V_s (Gamma1 is traceless)."""
    for L in ((4, 3, 5), (3, 4, 2), (5, 5, 1)):
        rp, c, v = lattice.topi_slab_csr(*L, W=0.0)
        H = lattice.to_scipy(rp, c, v)
        assert (H - H.conj().T).count_nonzero() == 0
        e = np.linalg.eigvalsh(H.toarray())
        assert np.abs(e - lattice.topi_slab_clean_spectrum(*L)).max() < 1e-12
    rp, c, v = lattice.topi_slab_csr(4, 3, 5, W=0.0)
    lens = np.diff(rp).reshape(5, 3 * 4 * 4)           # rows grouped by layer z
    assert np.all(lens[0] == 11) and np.all(lens[-1] == 11) and np.all(lens[1:-1] == 13)
    rp, c, v = lattice.topi_slab_csr(4, 4, 6, m=2.0, W=2.0, seed=3)
    H = lattice.to_scipy(rp, c, v)
    V = lattice.disorder(3, 4 * 4 * 6, 2.0)
    assert abs(H.diagonal().sum() - 4 * V.sum()) < 1e-11
    d = H.diagonal().real.reshape(-1, 4)
    assert np.array_equal(d[:, 0], V + 2.0) and np.array_equal(d[:, 3], V - 2.0)


# ---------------------------------------------------------------- SELL


@pytest.mark.parametrize("C,sigma", [(1, 1), (4, 1), (4, 8), (32, 64), (3, 5)])
def test_sell_round_trip_and_sorting(C, sigma):
    rs = np.random.default_rng(C * 100 + sigma)
    n = 101
    lens = rs.integers(0, 9, n)
    rowptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    col = np.concatenate([np.sort(rs.choice(n, l, replace=False)) for l in lens]).astype(np.int32)
    val = rs.standard_normal(rowptr[-1])
    S = sell.sell_from_csr(rowptr, col, val, C, sigma)
    rows = sell.sell_to_dense_rows(S)
    for r in range(n):
        got = rows[r][:lens[r]]
        assert [g[0] for g in got] == list(col[rowptr[r]:rowptr[r + 1]])
        assert [g[1] for g in got] == list(val[rowptr[r]:rowptr[r + 1]])
        assert all(p[0] == r and p[1] == 0 for p in rows[r][lens[r]:])
    perm = S["perm"]
    assert sorted(perm) == list(range(n))
    for w0 in range(0, n, sigma):
        win = perm[w0:w0 + sigma]
        assert sorted(win) == list(range(w0, min(w0 + sigma, n)))
        key = [(-lens[r], r) for r in win]
        assert key == sorted(key)
    assert S["chunk_ptr"][-1] == sum(S["chunk_len"]) * C


def _keyed(name):
    out = {}
    for row in _rows(name):
        out[row[0]] = row[1:]
    return out


def test_sell_hand_worked_example():
    """SELL-C-sigma arrays of a 7-row matrix at C = 2, sigma = 4, written out by
    hand from the format's definition (tests/golden/sell_c2_sigma4.txt):
    sorting scope, chunk widths, column-major slots inside a chunk, padding
    column and value, the slot past the last row."""
    g = _keyed("sell_c2_sigma4.txt")
    rowptr = np.array(g["csr_rowptr"], dtype=np.int64)
    col = np.array(g["csr_col"], dtype=np.int32)
    val = np.array(g["csr_val"], dtype=np.float64)
    S = sell.sell_from_csr(rowptr, col, val, 2, 4)
    assert S["nchunks"] == 4
    assert S["perm"].tolist() == [int(v) for v in g["perm"]]
    assert S["chunk_len"].tolist() == [int(v) for v in g["chunk_len"]]
    assert S["chunk_ptr"].tolist() == [int(v) for v in g["chunk_ptr"]]
    assert S["col"].tolist() == [int(v) for v in g["col"]]
    assert S["val"].tolist() == [float(v) for v in g["val"]]


# ---------------------------------------------------------------- filter quality


def test_fig_polyeff1_optimal_degrees():
    for kind, want in _rows("fig_polyeff1.txt"):
        want = int(want)
        n_opt, _ = quality.optimal_Np(1e-3, 1e-3, kind=kind, n_lo=int(0.8 * want), n_hi=int(1.25 * want))
        assert abs(n_opt - want) <= 0.02 * want, (kind, n_opt, want)


def test_tab_lanczoskernel_scaling_constants():
    rows = _rows("tab_lanczoskernel.txt")
    for c, N0, eta0 in rows[::3]:
        c, N0, eta0 = float(c), float(N0), float(eta0)
        n_opt, e_opt = quality.optimal_Np(1e-3, 1e-3, c=c, n_lo=int(800 * N0), n_hi=int(1250 * N0))
        assert abs(n_opt / 1000.0 - N0) <= 0.02 * N0, (c, n_opt)
        assert abs(e_opt / 1000.0 - eta0) <= 0.02 * eta0, (c, e_opt)


def test_lanczos_N0_of_the_solver_follows_tab_lanczoskernel():
    """The N_0 the solver's degree rule uses (Sec. 2.4, adaptive degree) is
    Tab. lanczoskernel's at the printed interval centres, symmetric in the
    centre, between the neighbouring rows in between, and the last row's
    beyond c / S_w = 0.9."""
    rows = [(float(c), float(N0)) for c, N0, _ in _rows("tab_lanczoskernel.txt")]
    for c, N0 in rows:
        assert abs(solve.lanczos_N0(c) - N0) <= 1e-12, (c, N0)
        assert abs(solve.lanczos_N0(-c) - N0) <= 1e-12
    for (c0, n0), (c1, n1) in zip(rows, rows[1:]):
        v = solve.lanczos_N0(0.5 * (c0 + c1))
        assert min(n0, n1) <= v <= max(n0, n1)
    assert solve.lanczos_N0(0.97) == rows[-1][1]


def test_tab_num_optimal_degree_quality_and_effort():
    for dos, NS, dpd, Np, eta, est, num, nit, star in _rows("tab_num.txt")[::2]:
        NS, dpd, Np, eta, est = int(NS), float(dpd), int(Np), float(eta), float(est)
        delta = 2.5e-3 if dos == "flat" else 0.05
        margin = quality.margin_flat(NS, 100) if dos == "flat" else quality.margin_linear(NS, 100)
        assert abs(margin - dpd) <= 0.006
        # the table's N_p^opt follow from its printed (rounded) delta'/delta
        n_opt, e_opt = quality.optimal_Np(delta, dpd * delta, n_lo=int(0.8 * Np), n_hi=int(1.25 * Np) + 2)
        assert abs(n_opt - Np) <= max(0.02 * Np, 2), (dos, NS, n_opt, Np)
        assert abs(e_opt - eta) <= 0.02 * eta + 1, (dos, NS, e_opt, eta)
        # estimate column: N_MVM = eta N_S (-log10 eps), eps = 1e-12
        assert abs(e_opt * NS * 12 / 1e6 - est) <= 0.03 * est + 0.01


def test_effort_model_linear_minimum_at_four_NT():
    NS = np.linspace(110, 900, 2000)
    f = quality.effort_linear(2.58, 1.0, 0.05, 100, NS)
    assert abs(NS[np.argmin(f)] - 400) < 2
    assert f.min() == pytest.approx(4 * 2.58 / 0.05 * 100, rel=1e-4)
    g = quality.effort_flat(2.58, 1.0, 0.0025, 100, NS)
    assert np.all(np.diff(g) < 0)


def test_topi_effort_estimate_sec53():
    """Sec. 5.2: minimal effort 1.06e6 spMVMs for [a,b] = [-5.5, 5.5],
    I_T = [-0.06, 0.06], eps = 1e-9 (linear DOS, N_S = 4 N_T); the figure
    follows from the DOS estimate N_T ~ 124 quoted there (not the final 144)."""
    f = quality.effort_linear(2.58, 5.5, 0.06, 124, 4 * 124) * 9
    assert f == pytest.approx(1.06e6, rel=0.01)


# ---------------------------------------------------------------- search-space weight


def test_fig_filtermatrix_weight_bound():
    """Sec. 2.2: D = 1000, I_T = [-0.01, 0.01], N_S = 50, N_p = 200, Lanczos mu=2:
    after one filter step 1 - w_i <= ~1.5e-5 inside the target interval."""
    D = 1000
    lam = lattice.flat_dos_eigs(D)
    gc = coeffs.filter_coeffs(-1, 1, -0.01, 0.01, 200, "lanczos")
    p = coeffs.eval_poly(gc, lam)
    inw = np.abs(lam) <= 0.01
    assert inw.sum() == 10
    worst = []
    for seed in range(5):
        X = solve.search_vectors(seed, D, 50, False)
        Q, _, _ = svqb.svqb(p[:, None] * X)
        w = np.sqrt((np.abs(Q) ** 2).sum(axis=1))     # eigenvectors are unit vectors
        worst.append((1 - w[inw]).max())
    assert max(worst) <= 1e-4
    assert np.median(worst) <= 3e-5


# ---------------------------------------------------------------- KPM, bounds, SVQB, RR


def test_jackson_damped_kpm_dos_is_nonnegative():
    """The Jackson kernel is a positive kernel: the damped Chebyshev series of
    a density of states (a sum of delta peaks) is nowhere negative, while the
    undamped series oscillates below zero (the Gibbs oscillations the damping
    removes; Sec. 2.1, Tab. Kernel, and the KPM of Sec. 3.1 step 1).  Exact
    moments of a diagonal matrix, M = 128, on a fine grid."""
    lam = np.concatenate([np.linspace(-0.9, -0.2, 150), np.linspace(0.3, 0.8, 90)])
    a, b = -1.0, 1.0
    x = lam  # alpha = 1, beta = 0
    M = 128
    mu = np.cos(np.multiply.outer(np.arange(M), np.arccos(x))).mean(axis=1)
    grid = np.linspace(-0.999, 0.999, 4001)
    rho = kpm.dos(mu, len(lam), a, b, grid)
    assert rho.min() >= -1e-9 * rho.max()
    rho_plain = kpm.dos(mu, len(lam), a, b, grid, g=np.ones(M))
    assert rho_plain.min() < -1e-3 * rho_plain.max()
    # both integrate to the number of states
    for r in (rho, rho_plain):
        assert abs(np.trapezoid(r, grid) - len(lam)) <= 0.02 * len(lam)


def test_kpm_trace_exact_on_diagonal_and_count():
    lam = lattice.flat_dos_eigs(2000)
    H = sp.diags(lam).tocsr()
    mu = kpm.moments(H, 1.0, 0.0, 64, 3, seed=1, complex_values=False)
    ref = np.array([np.mean(np.cos(n * np.arccos(lam))) for n in range(64)])
    assert np.allclose(mu, ref, atol=1e-13)               # |r_i| = 1: exact trace
    cnt = kpm.count_in_window(kpm.moments(H, 1.0, 0.0, 512, 1, 1, False), 2000, -1, 1, -0.2, 0.2)
    assert abs(cnt - 400) < 8


def test_kpm_count_on_lattice_against_dense():
    rp, c, v = lattice.topi_csr(4, 4, 4, W=1.0, seed=4)
    H = lattice.to_scipy(rp, c, v)
    e = np.linalg.eigvalsh(H.toarray())
    a, b = e[0] - 0.05, e[-1] + 0.05
    alpha, beta = coeffs.scaling(a, b)
    mu = kpm.moments(H, alpha, beta, 256, 16, seed=3, complex_values=True)
    assert mu[0] == pytest.approx(1.0, abs=1e-12)
    cnt = kpm.count_in_window(mu, H.shape[0], a, b, -1.5, 1.5)
    assert abs(cnt - np.sum(np.abs(e) <= 1.5)) < 12



def test_residual_norms_two_state_closed_form():
    """For v = cos(phi) e_1 + e^{i psi} sin(phi) e_2 and H = diag(l1, l2, ...),
    theta = l1 cos^2 + l2 sin^2 and ||H v - theta v|| = |l1 - l2| |cos sin|
    (Sec. 3.1 step 7's residual, in closed form)."""
    import scipy.sparse as sps
    l = np.array([0.3, -1.1, 2.0, 0.7])
    H = sps.diags(l.astype(np.complex128)).tocsr()
    for phi, psi in ((0.0, 0.0), (0.3, 1.0), (np.pi / 4, -2.0), (1.2, 0.5)):
        v = np.zeros(4, np.complex128)
        v[0], v[1] = np.cos(phi), np.exp(1j * psi) * np.sin(phi)
        theta = l[0] * np.cos(phi) ** 2 + l[1] * np.sin(phi) ** 2
        res = rr.residual_norms(H, v[:, None], [theta])[0]
        want = abs(l[0] - l[1]) * abs(np.cos(phi) * np.sin(phi))
        assert abs(res - want) <= 1e-14


def test_lanczos_bounds_stay_inside_gershgorin():
    """The interval of Sec. 3.1 step 1 is widened by a margin but never beyond
    the Gershgorin discs: for a diagonal matrix the discs are the exact
    extremes, so [a, b] is exactly [min, max] of its eigenvalues."""
    lam = np.linspace(-1.0, 1.0, 400)
    H = lattice.to_scipy(*lattice.diagonal_csr(lam))
    a, b = bounds.lanczos_bounds(H, 30, seed=0)
    assert a == -1.0 and b == 1.0


@pytest.mark.parametrize("gen", ["topi", "graphene"])
def test_lanczos_bounds_enclose_spectrum(gen):
    if gen == "topi":
        H = lattice.to_scipy(*lattice.topi_csr(5, 4, 4, W=1.5, seed=2))
    else:
        H = lattice.to_scipy(*lattice.graphene_csr(12, 10, W=1.0, seed=2))
    e = np.linalg.eigvalsh(H.toarray())
    a, b = bounds.lanczos_bounds(H, 30, seed=1)
    assert a <= e[0] and b >= e[-1]
    assert (b - a) <= 1.06 * (e[-1] - e[0])
    g_lo, g_hi = bounds.gershgorin(H)
    assert g_lo <= a and b <= g_hi


def test_svqb_orthonormal_same_span_and_refill():
    rs = np.random.default_rng(1)
    Y = rs.standard_normal((500, 20)) + 1j * rs.standard_normal((500, 20))
    Y[:, 3] *= 1e-6
    Q, rank, cnt = svqb.svqb(Y)
    assert rank == 20 and cnt == 0
    assert np.abs(Q.conj().T @ Q - np.eye(20)).max() < 1e-12
    # same span: projecting Y onto span(Q) reproduces Y
    assert np.linalg.norm(Y - Q @ (Q.conj().T @ Y)) < 1e-10 * np.linalg.norm(Y)
    Z = np.concatenate([Y[:, :10], Y[:, :10] @ rs.standard_normal((10, 6))], axis=1)
    Q2, rank2, cnt2 = svqb.svqb(Z, seed=3)
    assert rank2 == 10 and cnt2 == 6 and Q2.shape == (500, 16)
    assert np.abs(Q2.conj().T @ Q2 - np.eye(16)).max() < 1e-12
    assert np.linalg.norm(Z[:, :10] - Q2 @ (Q2.conj().T @ Z[:, :10])) < 1e-9 * np.linalg.norm(Z)


def test_rayleigh_ritz_exact_on_invariant_subspace():
    H = lattice.to_scipy(*lattice.topi_csr(3, 3, 3, W=0.8, seed=9))
    lam, V = np.linalg.eigh(H.toarray())
    rs = np.random.default_rng(2)
    M = np.linalg.qr(rs.standard_normal((12, 12)) + 1j * rs.standard_normal((12, 12)))[0]
    Y = V[:, 40:52] @ M                                   # rotated invariant subspace
    theta, Vr, res = rr.rayleigh_ritz(H, Y)
    assert np.allclose(theta, lam[40:52], atol=1e-12)
    assert res.max() < 1e-12
    assert np.allclose(res, rr.residual_norms(H, Vr, theta), atol=1e-13)


def test_harmonic_ritz_exact_on_invariant_subspace():
    """On an invariant subspace the harmonic vectors are eigenvectors: Rayleigh
    quotients and harmonic values both equal the eigenvalues, residuals vanish."""
    H = lattice.to_scipy(*lattice.topi_csr(3, 3, 3, W=0.8, seed=9))
    lam, V = np.linalg.eigh(H.toarray())
    rs = np.random.default_rng(4)
    M = np.linalg.qr(rs.standard_normal((10, 10)) + 1j * rs.standard_normal((10, 10)))[0]
    Y = V[:, 50:60] @ M
    rho, Vh, res, theta_h = rr.harmonic_ritz(H, Y, 0.5 * (lam[50] + lam[59]) + 1e-3)
    assert np.allclose(rho, lam[50:60], atol=1e-12)
    assert np.allclose(np.sort(theta_h), lam[50:60], atol=1e-10)
    assert res.max() < 1e-12
    assert np.allclose(np.linalg.norm(Vh, axis=0), 1.0)


def test_harmonic_ritz_falls_back_to_ritz_pairs_when_singular():
    """tau equal to the eigenvalue of a basis vector makes Z^H Z singular:
    the ordinary Ritz pairs (here the exact eigenpairs) come back."""
    d = np.arange(64) / 8.0 - 3.0
    H = sp.diags(d).tocsr()
    E = np.zeros((64, 8))
    E[np.arange(8) * 5, np.arange(8)] = 1.0
    rho, V, res, _ = rr.harmonic_ritz(H, E, d[15])
    assert np.array_equal(rho, np.sort(d[np.arange(8) * 5]))
    assert res.max() == 0.0


def test_harmonic_values_are_inverse_ritz_values_of_the_shifted_inverse():
    """Harmonic Ritz values of H on span(Y) for target tau are tau + 1/mu with
    mu the Ritz values of (H - tau)^-1 on span((H - tau) Y) (Morgan 1991):
    checked against a dense inverse and an independent orthonormal basis."""
    H = lattice.to_scipy(*lattice.topi_csr(2, 3, 2, W=1.1, seed=3)).toarray()
    n = H.shape[0]
    rs = np.random.default_rng(6)
    Y = np.linalg.qr(rs.standard_normal((n, 7)) + 1j * rs.standard_normal((n, 7)))[0]
    tau = 0.137
    _, _, _, theta_h = rr.harmonic_ritz(H, Y, tau)
    Q = np.linalg.qr((H - tau * np.eye(n)) @ Y)[0]
    B = Q.conj().T @ np.linalg.inv(H - tau * np.eye(n)) @ Q
    mu = np.linalg.eigvalsh(0.5 * (B + B.conj().T))
    assert np.allclose(np.sort(theta_h), np.sort(tau + 1.0 / mu), rtol=1e-9, atol=1e-9)


# ---------------------------------------------------------------- whole iteration


@pytest.mark.parametrize("dos,NS,Np,want", [("linear", 200, 303, 5), ("flat", 200, 2500, 5),
                                            ("linear", 400, 124, 6), ("flat", 300, 1258, 6)])
def test_tab_num_iteration_counts(dos, NS, Np, want):
    """Tab. num: ChebFD on D = 40000 diagonal matrices finds all N_T = 100 target
    eigenpairs in N_iter iterations (+-1: the stars of the table).  For diagonal
    H, p[H] X = p(lambda) X exactly, which replaces the recurrence here."""
    D = 40000
    lam = lattice.flat_dos_eigs(D) if dos == "flat" else lattice.linear_dos_eigs(D)
    delta = 2.5e-3 if dos == "flat" else 0.05
    H = sp.diags(lam).tocsr()
    p = coeffs.eval_poly(coeffs.filter_coeffs(-1, 1, -delta, delta, Np, "lanczos"), lam)
    r = solve.chebfd(H, -1.0, 1.0, -delta, delta, NS, Np, 1e-12,
                     filter_fn=lambda X: p[:, None] * X, complex_values=False)
    assert r["converged"] and abs(r["iterations"] - want) <= 1
    exact = np.sort(lam[np.abs(lam) <= delta])
    assert len(exact) == 100 and len(r["theta"]) == 100
    assert np.abs(np.sort(r["theta"]) - exact).max() < 1e-12


def test_chebfd_small_topi_against_dense():
    """The smallest insulator workload: 8x8x8x4 (N = 2048), W = 0.5, window
    [-0.1, 0.1], n_s = 64, N_p = 200, Jackson; all window eigenvalues of the
    dense eigensolver within 1e-10 ||H||, residuals <= 1e-9 ||H||."""
    H = lattice.to_scipy(*lattice.topi_csr(8, 8, 8, t=1.0, m=1.0, W=0.5, seed=0))
    a, b = bounds.lanczos_bounds(H, 30, seed=0)
    e = np.linalg.eigvalsh(H.toarray())
    r = solve.chebfd(H, a, b, -0.1, 0.1, 64, 200, 1e-9, kind="jackson", seed=0)
    ew = e[np.abs(e) <= 0.1]
    assert r["converged"] and len(r["theta"]) == len(ew) > 0
    assert np.abs(np.sort(r["theta"]) - ew).max() <= 1e-10 * r["normH"]
    assert r["res"].max() <= 1e-9 * r["normH"]
    assert np.abs(r["V"].conj().T @ r["V"] - np.eye(len(ew))).max() < 1e-12
    th = np.sort(r["theta"])
    assert np.abs(th + th[::-1]).max() < 1e-10           # chiral +- pairing


# ---------------------------------------------------------------- MLP reference


def test_chebfd_harmonic_extraction_small_topi_against_dense():
    """Harmonic Ritz extraction (Sec. 6) on the smallest insulator workload:
    the same window eigenvalues as dense diagonalisation, residuals <= 1e-9
    ||H||, in no more iterations than ordinary Ritz pairs."""
    H = lattice.to_scipy(*lattice.topi_csr(8, 8, 8, t=1.0, m=1.0, W=0.5, seed=0))
    a, b = bounds.lanczos_bounds(H, 30, seed=0)
    e = np.linalg.eigvalsh(H.toarray())
    ew = e[np.abs(e) <= 0.1]
    r = solve.chebfd(H, a, b, -0.1, 0.1, 64, 200, 1e-9, kind="jackson", seed=0,
                     extraction="harmonic")
    assert r["converged"] and len(r["theta"]) == len(ew)
    assert np.abs(np.sort(r["theta"]) - ew).max() <= 1e-10 * r["normH"]
    assert r["res"].max() <= 1e-9 * r["normH"]
    ritz = solve.chebfd(H, a, b, -0.1, 0.1, 64, 200, 1e-9, kind="jackson", seed=0)
    assert r["iterations"] <= ritz["iterations"]


def test_chebfd_inset_window_halves_the_degree_small_topi():
    """A window narrowed by half the target half-width (W = 1 on [-0.05, 0.05]
    inside I_T = [-0.1, 0.1], Sec. 2.2) with half the degree (N_p = 100,
    Lanczos): all window eigenvalues of the dense eigensolver in as many
    iterations as the rectangular window at N_p = 200, half the spMVMs; the
    rectangular window at N_p = 100 needs more iterations."""
    H = lattice.to_scipy(*lattice.topi_csr(8, 8, 8, t=1.0, m=1.0, W=0.5, seed=0))
    a, b = bounds.lanczos_bounds(H, 30, seed=0)
    e = np.linalg.eigvalsh(H.toarray())
    ew = e[np.abs(e) <= 0.1]
    r = solve.chebfd(H, a, b, -0.1, 0.1, 64, 100, 1e-9, seed=0, window_inset=0.5)
    assert r["converged"] and len(r["theta"]) == len(ew)
    assert np.abs(np.sort(r["theta"]) - ew).max() <= 1e-10 * r["normH"]
    rect = solve.chebfd(H, a, b, -0.1, 0.1, 64, 200, 1e-9, seed=0)
    assert r["iterations"] <= rect["iterations"]


def test_inset_window_lowers_eta():
    """Sec. 2.3 quality measure at delta = delta' = 1e-2 on [-1, 1] (Lanczos
    mu = 2): the rectangular window reproduces Tab. lanczoskernel's centre
    value eta_0 = 2.58 / delta'; the window narrowed by half the half-width
    reaches eta <= 0.8 of it with N_p^opt <= 0.7 of the rectangular one."""
    n_r, e_r = quality.optimal_Np(1e-2, 1e-2, n_lo=400, n_hi=900)
    n_i, e_i = quality.optimal_Np(1e-2, 1e-2, n_lo=250, n_hi=700, inset=0.5)
    assert abs(e_r - 258.0) <= 0.02 * 258.0
    assert e_i <= 0.8 * e_r and n_i <= 0.7 * n_r


def test_mlp_gradient_matches_central_differences():
    from oracle import mlp
    rs = np.random.default_rng(0)
    P = mlp.init_params(7, 5, 3, seed=1)
    for k in P:
        P[k] = P[k] + 0.1 * rs.standard_normal(P[k].shape)
    X = rs.standard_normal((6, 7))
    T = np.c_[rs.standard_normal((6, 2)), rs.integers(0, 2, 6)]
    L0, G = mlp.loss_and_grad(P, X, T)
    assert L0 == pytest.approx(mlp.loss(P, X, T), rel=1e-14)
    h = 1e-6
    for k in P:
        flat = P[k].reshape(-1)
        for idx in range(flat.size):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(P, X, T)
            flat[idx] = old - h
            lm = mlp.loss(P, X, T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - G[k].reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx)


def test_mlp_adam_reduces_loss_on_a_fittable_target():
    from oracle import mlp
    rs = np.random.default_rng(3)
    X = rs.standard_normal((32, 4))
    T = np.c_[X[:, 0] * 0.5, np.tanh(X[:, 1]), (X[:, 2] > 0).astype(float)]
    P = mlp.init_params(4, 16, 3, seed=2)
    st = {}
    L_start = mlp.loss(P, X, T)
    for _ in range(300):
        _, G = mlp.loss_and_grad(P, X, T)
        mlp.adam_step(P, G, st, 1e-2)
    assert mlp.loss(P, X, T) < 0.2 * L_start


def test_adam_two_steps_known_answers():
    """Two Adam steps on three parameters against values worked by hand from
    Kingma and Ba's Algorithm 1 (tests/golden/adam_two_steps.txt): the
    bias-corrected moments and the parameters after each step."""
    from fractions import Fraction
    from oracle import mlp
    rows = _rows("adam_two_steps.txt")
    th0 = np.array([float(r[0]) for r in rows])
    g1 = np.array([float(r[1]) for r in rows])
    g2 = np.array([float(r[2]) for r in rows])
    P, st = {"theta": th0.copy()}, {}
    mlp.adam_step(P, {"theta": g1}, st, 0.1)
    mh1 = st["m_theta"] / (1 - 0.9)
    vh1 = st["v_theta"] / (1 - 0.999)
    for k, r in enumerate(rows):
        assert mh1[k] == pytest.approx(float(Fraction(r[3])), rel=1e-13)
        assert vh1[k] == pytest.approx(float(Fraction(r[4])), rel=1e-12)
        assert P["theta"][k] == pytest.approx(float(r[5]), rel=1e-14, abs=1e-15)
    mlp.adam_step(P, {"theta": g2}, st, 0.1)
    assert st["t"] == 2
    for k, r in enumerate(rows):
        assert P["theta"][k] == pytest.approx(float(r[8]), rel=1e-14, abs=1e-15)


def test_chebfd_empty_window_terminates():
    """A window inside a spectral gap holds no eigenvalue: the iteration stops
    with no pairs after two iterations without an accepted or converging
    in-window pair.  Spurious in-window Ritz values (mixtures of eigenvectors
    at both edges of the gap, ghost-flagged, residuals stagnating) may remain.
    The same on a gapped 5x5x5 insulator whose window [-0.3, 0.3] lies inside
    a gap of +-0.606 with many degenerate edge states: there the spurious
    values never leave the window, so the test must rest on their stagnation."""
    lam = np.concatenate([np.linspace(-1, -0.2, 300), np.linspace(0.2, 1, 300)])
    H = sp.diags(lam).tocsr()
    r = solve.chebfd(H, -1.01, 1.01, -0.05, 0.05, 16, 60, 1e-9, complex_values=False)
    assert r["converged"] and len(r["theta"]) == 0 and r["iterations"] <= 4
    assert r["log"][-1]["accepted"] == r["log"][-2]["accepted"] == 0
    Ho = lattice.to_scipy(*lattice.topi_csr(5, 5, 5, t=1.0, m=1.0, W=0.2, seed=104))
    assert np.abs(np.linalg.eigvalsh(Ho.toarray())).min() > 0.6
    bound = 1.01 * (1.0 + 3.0 + 0.1)
    r = solve.chebfd(Ho, -bound, bound, -0.3, 0.3, 32, 160, 1e-9, seed=0, max_iter=40)
    assert r["converged"] and len(r["theta"]) == 0 and r["iterations"] <= 4
    assert r["log"][-1]["in_window"] > 0


def test_chebfd_weak_filter_is_not_taken_for_an_empty_window():
    """A filter too weak for the ghost rule (Sec. 3.1 step 7): flat-DOS diagonal
    H (D = 400), window [-0.02, 0.02] with 8 eigenvalues, N_p = 30.  The
    residuals fall by less than 10x per iteration, so the true pairs are
    ghost-flagged for several successive iterations; that is no evidence of
    an empty window.  The iteration goes on until every window eigenvalue
    of the diagonal converges; with N_p = 20 and n_s = 32 it never converges
    within the budget and says so instead of returning an empty window."""
    D = 400
    lam = -1.0 + 2.0 * np.arange(1, D + 1) / (D + 1)
    H = sp.diags(lam).tocsr()
    ew = lam[(lam >= -0.02) & (lam <= 0.02)]
    assert len(ew) == 8
    r = solve.chebfd(H, -1.001, 1.001, -0.02, 0.02, 64, 30, 1e-10, complex_values=False,
                     max_iter=40)
    ghosted = [l for l in r["log"][1:] if l["accepted"] == 0 and l["in_window"] > 0]
    assert len(ghosted) >= 2
    assert r["converged"] and len(r["theta"]) == 8
    assert np.abs(np.sort(r["theta"]) - ew).max() <= 1e-10
    r = solve.chebfd(H, -1.001, 1.001, -0.02, 0.02, 32, 20, 1e-10, complex_values=False,
                     max_iter=12)
    assert not r["converged"] and r["iterations"] == 12


def test_adaptive_degree_follows_the_linear_dos_rule():
    """Adaptive N_p (Sec. 6 with the rule of Sec. 2.4): linear-DOS diagonal
    matrix, D = 4000, window +-0.158 (N_T = D delta^2 = 100), N_S = 200,
    started at N_p = 300.  The moments of the first filter give delta' close
    to the linear-DOS value (sqrt(N_S / N_T) - 1) delta (the construction of
    Tab. num) and N_p = N_0 / delta' with N_0 = 6.23 (Tab. lanczoskernel,
    centre); all 100 eigenvalues are found, with fewer products than the run
    that keeps N_p = 300."""
    D, NS = 4000, 200
    delta = np.sqrt(100.0 / D)
    lam = lattice.linear_dos_eigs(D)
    H = sp.diags(lam).tocsr()
    r = solve.chebfd(H, -1.0, 1.0, -delta, delta, NS, 300, 1e-10, complex_values=False,
                     adaptive=True)
    NT, dprime, Np = r["adapted"]
    want_dp = (np.sqrt(NS / 100.0) - 1.0) * delta
    assert abs(NT - 100) <= 10
    assert abs(dprime - want_dp) <= 0.1 * want_dp
    assert abs(Np - 6.23 / want_dp) <= 0.1 * 6.23 / want_dp and r["Np"] == Np
    exact = np.sort(lam[np.abs(lam) <= delta])
    assert r["converged"] and len(r["theta"]) == len(exact) == 100
    assert np.abs(np.sort(r["theta"]) - exact).max() < 1e-10
    fixed = solve.chebfd(H, -1.0, 1.0, -delta, delta, NS, 300, 1e-10, complex_values=False)
    assert fixed["converged"] and r["n_mvm"] < fixed["n_mvm"]


def test_chebfd_locking_deflation_over_a_long_run():
    """Hard locking with a weak filter and a tight eps (linear-DOS diagonal,
    D = 4000, N_T = 100, N_S = 200, N_p = 40, eps = 1e-13): pairs lock from
    the early iterations on and the run goes on for many more.  The locked
    vectors are accurate only to about eps, so the search block keeps small
    components along their eigenvectors, which the filter passes while it
    damps everything outside the window; only the deflation against the
    locked vectors keeps those components from growing into duplicate Ritz
    pairs.  The run converges to exactly the 100 window eigenvalues, each
    once, with orthonormal vectors."""
    D, NS, Np = 4000, 200, 40
    delta = np.sqrt(100.0 / D)
    lam = lattice.linear_dos_eigs(D)
    H = sp.diags(lam).tocsr()
    r = solve.chebfd(H, -1.0, 1.0, -delta, delta, NS, Np, 1e-13, complex_values=False,
                     locking=True, max_iter=40)
    exact = np.sort(lam[np.abs(lam) <= delta])
    assert r["converged"] and len(r["theta"]) == len(exact) == 100
    assert np.abs(np.sort(r["theta"]) - exact).max() <= 1e-12
    assert np.abs(r["V"].T @ r["V"] - np.eye(100)).max() <= 1e-10
    assert r["locked"] >= 80


def test_chebfd_locking_on_linear_dos():
    """Hard locking (Sec. 6) on the linear-DOS diagonal (D = 4000, window
    +-0.158 with N_T = 100, N_S = 200, N_p = 95): the eigenvalues near the
    window centre converge first and are locked, four at a time; the search
    block shrinks, the same 100 eigenvalues are found with orthonormal
    vectors, and fewer products are needed than without locking."""
    D, NS, Np = 4000, 200, 95
    delta = np.sqrt(100.0 / D)
    lam = lattice.linear_dos_eigs(D)
    H = sp.diags(lam).tocsr()
    plain = solve.chebfd(H, -1.0, 1.0, -delta, delta, NS, Np, 1e-10, complex_values=False)
    r = solve.chebfd(H, -1.0, 1.0, -delta, delta, NS, Np, 1e-10, complex_values=False,
                     locking=True)
    exact = np.sort(lam[np.abs(lam) <= delta])
    assert r["converged"] and len(r["theta"]) == len(exact) == 100
    assert np.abs(np.sort(r["theta"]) - exact).max() <= 1e-10
    assert np.abs(r["V"].T @ r["V"] - np.eye(100)).max() <= 1e-10
    assert r["locked"] >= 4 and r["locked"] % 4 == 0
    assert r["n_mvm"] < plain["n_mvm"]
