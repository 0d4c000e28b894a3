"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in the CPU oracle (a dropped term, a wrong sign,
an index off by one, a transposed operand, a wrong constant) by replacing one
oracle function or constant for the duration of the test, then runs the pins
of tests/test_oracle_pins.py that guard it: at least one of them must fail.
The mistakes live only here, on the CPU; the oracle itself is untouched.

Not listed, because no pin can tell them apart from the oracle's choice:
conventions that give a unitarily equivalent matrix (the sign of sigma_y in
Gamma3, the orientation of the graphene bonds, swapping T_j with T_j^dagger):
these mirror the lattice, leave every spectrum unchanged, and are fixed
between the oracle and the CUDA generators by the element-by-element parity
tests instead.
"""
import numpy as np
import pytest
import scipy.linalg

import test_oracle_pins as pins
from oracle import coeffs, filter as filt, kpm, lattice, mlp, quality, rng, rr, sell, svqb
from oracle import bounds, solve


# ---------------------------------------------------------------- mutants


def _wrap(module, name, fn):
    orig = getattr(module, name)

    def patch(mp):
        mp.setattr(module, name, fn(orig))
    return patch


def _filter_block(step_factor=2.0, gc_shift=0, last=None):
    """The Chebyshev filter sum with one planted change to the recurrence loop
    (n >= 3): the factor 2, the coefficient index, or the last degree."""
    def f(H, alpha, beta, gc, X):
        Np = len(gc) - 1
        t_prev = np.array(X, copy=True)
        t_cur = filt.apply_A(H, alpha, beta, t_prev)
        y = gc[0] * t_prev + gc[1] * t_cur
        for n in range(2, (Np if last is None else last) + 1):
            k = step_factor if n >= 3 else 2.0
            t_prev, t_cur = t_cur, k * filt.apply_A(H, alpha, beta, t_cur) - t_prev
            y = y + gc[n - (gc_shift if n >= 3 else 0)] * t_cur
        return y
    return f


def _kernel_gn(kind_bad, fn):
    """kernel_gn with one kernel's factors replaced by fn(Np, n, mu)."""
    def make(orig):
        def g(kind, Np, mu=2.0):
            if kind != kind_bad:
                return orig(kind, Np, mu)
            return fn(Np, np.arange(Np + 1, dtype=np.float64), mu)
        return g
    return make


def _jackson_np_plus_one(Np, n, mu):
    q = np.pi / (Np + 1)
    return ((Np + 1 - n) * np.cos(q * n) + np.sin(q * n) / np.tan(q)) / (Np + 1)


def _lanczos_over_np(Np, n, mu):
    g = np.ones(Np + 1)
    arg = np.pi * n[1:] / Np
    g[1:] = (np.sin(arg) / arg) ** mu
    return g


def _fejer_off_by_one(Np, n, mu):
    return (Np - n) / (Np + 1.0)


def _svqb_theta_power(power):
    """SVQB whose last scaling is Theta^(-power) instead of Theta^(-1/2)."""
    def make(orig):
        def f(Y, seed=0, refill_counter=0, max_pass=3, tol=1e-12):
            Y = np.array(Y, copy=True)
            D, ns = Y.shape
            S = Y.conj().T @ Y
            d = 1.0 / np.sqrt(np.real(np.diag(S)))
            theta, U = np.linalg.eigh(d[:, None] * S * d[None, :])
            keep = theta >= ns * 2.0 ** -52 * theta.max()
            Y = Y @ (d[:, None] * U[:, keep] / theta[keep][None, :] ** power)
            return Y, int(keep.sum()), refill_counter
        return f
    return make


def _svqb_no_diagonal_scaling(orig):
    def f(Y, seed=0, refill_counter=0, max_pass=3, tol=1e-12):
        Y = np.array(Y, copy=True)
        ns = Y.shape[1]
        theta, U = np.linalg.eigh(Y.conj().T @ Y)
        keep = theta >= ns * 2.0 ** -52 * theta.max()
        return Y @ (U[:, keep] / np.sqrt(theta[keep])[None, :]), int(keep.sum()), refill_counter
    return f


def _rr(transpose_only=False, rotate=True):
    def make(orig):
        def f(H, Y):
            HY = H @ Y
            G = (Y.T if transpose_only else Y.conj().T) @ HY
            G = 0.5 * (G + G.conj().T)
            theta, S = np.linalg.eigh(G)
            V = Y @ S if rotate else Y
            HV = HY @ S if rotate else HY
            return theta, V, np.linalg.norm(HV - V * theta[None, :], axis=0)
        return f
    return make


class _NumpyArgsort:
    """numpy with argsort replaced (for the SELL row sort)."""

    def __init__(self, argsort):
        self._argsort = argsort

    def __getattr__(self, k):
        return getattr(np, k)

    def argsort(self, a, kind=None):
        return self._argsort(np.asarray(a))


def _harmonic_unnormalised(orig):
    def f(H, Y, tau):
        HY = H @ Y
        Z = HY - tau * Y
        mu, S = scipy.linalg.eigh(Y.conj().T @ Z, Z.conj().T @ Z)
        V, HV = Y @ S, HY @ S
        rho = np.real(np.sum(V.conj() * HV, axis=0))
        o = np.argsort(rho)
        return rho[o], V[:, o], np.linalg.norm(HV - V * rho[None, :], axis=0)[o], tau + 1.0 / mu[o]
    return f


def _mix64_shift(orig):
    def f(z):
        z = np.asarray(z, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = (z ^ (z >> np.uint64(31))) * rng._M1
            z = (z ^ (z >> np.uint64(27))) * rng._M2
        return z ^ (z >> np.uint64(31))
    return f


def _words_from_zero(orig):
    def f(seed, stream, index):
        state = np.uint64((int(seed) * 256 + int(stream)) % (1 << 64))
        with np.errstate(over="ignore"):
            return rng.mix64(state + np.asarray(index, dtype=np.uint64) * rng.GAMMA)
    return f


def _uniform_low_bits(orig):
    def f(seed, stream, index):
        w = rng.words(seed, stream, index)
        return (w & np.uint64((1 << 53) - 1)).astype(np.float64) * (2.0 ** -53)
    return f


def _mlp_grad_sign(orig):
    def f(P, X, T):
        L, G = orig(P, X, T)
        k = sorted(G)[0]
        G = dict(G)
        G[k] = -G[k]
        return L, G
    return f


def _eta_natural_log(orig):
    def f(Np, delta, delta_p, **kw):
        s = quality.damping_sigma(Np, delta, delta_p, **kw)
        return np.inf if not s < 1.0 else -Np / np.log(s)
    return f


def _sell_layout(row_major=False, pad_col_zero=False):
    """sell_from_csr with a planted layout mistake, and a decoder that matches
    it (so the round-trip pin alone cannot see it): slots row-major inside a
    chunk (entry j of local row l at chunk_ptr + l*width + j), or padding
    slots pointing at column 0 instead of their own row."""
    def slot(S, k, l, j):
        wdt = S["chunk_len"][k]
        return S["chunk_ptr"][k] + (l * wdt + j if row_major else j * S["C"] + l)

    def patch(mp):
        orig = sell.sell_from_csr

        def build(rowptr, col, val, C, sigma):
            S = orig(rowptr, col, val, C, sigma)      # sort, widths, pointers kept
            scol, sval = np.zeros_like(S["col"]), np.zeros_like(S["val"])
            for k in range(S["nchunks"]):
                for l in range(C):
                    r = k * C + l
                    if r >= S["n"]:
                        continue
                    o = S["perm"][r]
                    b, e = rowptr[o], rowptr[o + 1]
                    for j in range(S["chunk_len"][k]):
                        pos = slot(S, k, l, j)
                        if j < e - b:
                            scol[pos], sval[pos] = col[b + j], val[b + j]
                        else:
                            scol[pos] = 0 if pad_col_zero else o
            S["col"], S["val"] = scol, sval
            return S

        def decode(S):
            rows = [[] for _ in range(S["n"])]
            for k in range(S["nchunks"]):
                for l in range(S["C"]):
                    r = k * S["C"] + l
                    if r < S["n"]:
                        for j in range(S["chunk_len"][k]):
                            pos = slot(S, k, l, j)
                            rows[S["perm"][r]].append((S["col"][pos], S["val"][pos]))
            return rows

        mp.setattr(sell, "sell_from_csr", build)
        mp.setattr(sell, "sell_to_dense_rows", decode)
    return patch


def _adam_without_bias_correction(orig):
    def f(P, G, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        state["t"] = state.get("t", 0) + 1
        for k in P:
            m = state.setdefault("m_" + k, np.zeros_like(P[k]))
            v = state.setdefault("v_" + k, np.zeros_like(P[k]))
            m[...] = beta1 * m + (1 - beta1) * G[k]
            v[...] = beta2 * v + (1 - beta2) * G[k] ** 2
            P[k] = P[k] - lr * m / (np.sqrt(v) + eps)
        return P
    return f


_pair = np.array([[0, 1], [1, 0]], dtype=np.complex128)

MUTANTS = {
    "c_n with the printed overall sign": (
        _wrap(coeffs, "window_cn", lambda o: lambda *a, **k: -o(*a, **k)),
        [pins.test_filter_is_about_one_inside_window,
         lambda: pins.test_window_coefficients_match_defining_integral((-0.1, 0.1))]),
    "c_0 with the factor 2 of c_n": (
        _wrap(coeffs, "window_cn",
              lambda o: lambda *a, **k: o(*a, **k) * np.r_[2.0, np.ones(a[4])]),
        [lambda: pins.test_window_coefficients_match_defining_integral((-0.3, 0.05))]),
    "sin(n theta_hi) and sin(n theta_lo) swapped in c_n (n >= 1)": (
        _wrap(coeffs, "window_cn",
              lambda o: lambda *a, **k: o(*a, **k) * np.r_[1.0, -np.ones(a[4])]),
        [pins.test_filter_is_about_one_inside_window,
         lambda: pins.test_window_coefficients_match_defining_integral((0.2, 0.9))]),
    "beta with the wrong sign": (
        _wrap(coeffs, "scaling", lambda o: lambda a, b: (2.0 / (b - a), (a + b) / (b - a))),
        [lambda: pins.test_scaling_maps_interval(-2.0, 3.0)]),
    "alpha without the factor 2": (
        _wrap(coeffs, "scaling", lambda o: lambda a, b: (1.0 / (b - a), (a + b) / (a - b))),
        [lambda: pins.test_scaling_maps_interval(-5.5, 5.5)]),
    "Jackson factors with N_p + 1": (
        _wrap(coeffs, "kernel_gn", _kernel_gn("jackson", _jackson_np_plus_one)),
        [pins.test_kernel_factors_special_values]),
    "Lanczos sigma factors over N_p": (
        _wrap(coeffs, "kernel_gn", _kernel_gn("lanczos", _lanczos_over_np)),
        [pins.test_kernel_factors_special_values]),
    "Fejer factors off by one": (
        _wrap(coeffs, "kernel_gn", _kernel_gn("fejer", _fejer_off_by_one)),
        [pins.test_kernel_factors_special_values]),
    "T_n sampled with sin": (
        _wrap(coeffs, "eval_poly", lambda o: lambda gc, x: np.sin(np.multiply.outer(
            np.arccos(np.clip(np.asarray(x, float), -1, 1)), np.arange(len(gc)))) @ gc),
        [pins.test_filter_is_about_one_inside_window]),
    "recurrence without the factor 2": (
        _wrap(filt, "filter_block", lambda o: _filter_block(step_factor=1.0)),
        [pins.test_filter_on_diagonal_matches_cos_closed_form]),
    "accumulation with g_{n-1} c_{n-1}": (
        _wrap(filt, "filter_block", lambda o: _filter_block(gc_shift=1)),
        [pins.test_filter_on_diagonal_matches_cos_closed_form]),
    "one Chebyshev step short": (
        _wrap(filt, "filter_block", lambda o: _filter_block(last=-1)),
        [pins.test_filter_on_diagonal_matches_cos_closed_form]),
    "A u without beta u": (
        _wrap(filt, "apply_A", lambda o: lambda H, alpha, beta, v: alpha * (H @ v)),
        [pins.test_filter_on_diagonal_matches_cos_closed_form]),
    "moments shifted by one degree": (
        _wrap(filt, "moments", lambda o: lambda H, al, be, X, count: o(H, al, be, X, count + 1)[1:]),
        [pins.test_moments_on_diagonal_and_doubling_identities]),
    "Gamma4 equal to Gamma2": (
        lambda mp: mp.setattr(lattice, "GAMMA", lattice.GAMMA[:3] + [lattice.GAMMA[1]]),
        [pins.test_topi_structure_hermitian_and_clean_spectrum]),
    "Gamma1 with the factors swapped (sigma_0 x sigma_z)": (
        lambda mp: mp.setattr(lattice, "GAMMA", [np.kron(np.eye(2), np.diag([1.0, -1.0]))
                                                 .astype(np.complex128)] + lattice.GAMMA[1:]),
        [pins.test_topi_disorder_chiral_symmetry]),
    "Gamma2 built from sigma_x x sigma_0": (
        lambda mp: mp.setattr(lattice, "GAMMA", [lattice.GAMMA[0], np.kron(_pair, np.eye(2))]
                              + lattice.GAMMA[2:]),
        [pins.test_topi_structure_hermitian_and_clean_spectrum]),
    "disorder uniform in [0, W)": (
        _wrap(lattice, "disorder", lambda o: lambda seed, count, W: o(seed, count, W) + 0.5 * W),
        [pins.test_topi_disorder_chiral_symmetry]),
    "SplitMix64 first shift 31": (
        _wrap(rng, "mix64", _mix64_shift),
        [pins.test_splitmix64_known_answers]),
    "SplitMix64 counter from 0": (
        _wrap(rng, "words", _words_from_zero),
        [pins.test_splitmix64_known_answers]),
    "uniform from the low 53 bits": (
        _wrap(rng, "uniform", _uniform_low_bits),
        [pins.test_uniform_is_the_top_53_bits]),
    "SELL rows sorted shortest first": (
        lambda mp: mp.setattr(sell, "np", _NumpyArgsort(lambda a: np.argsort(-a, kind="stable"))),
        [lambda: pins.test_sell_round_trip_and_sorting(4, 8)]),
    "SELL sort unstable on equal lengths": (
        lambda mp: mp.setattr(sell, "np", _NumpyArgsort(
            lambda a: np.lexsort((-np.arange(len(a)), a)))),   # ties: later row first
        [lambda: pins.test_sell_round_trip_and_sorting(32, 64)]),
    "SELL slots row-major inside a chunk (decoder to match)": (
        _sell_layout(row_major=True),
        [pins.test_sell_hand_worked_example]),
    "SELL padding slots pointing at column 0": (
        _sell_layout(pad_col_zero=True),
        [pins.test_sell_hand_worked_example]),
    "Adam without the bias correction": (
        _wrap(mlp, "adam_step", _adam_without_bias_correction),
        [pins.test_adam_two_steps_known_answers]),
    "SVQB scaled by Theta^-1": (
        _wrap(svqb, "svqb", _svqb_theta_power(1.0)),
        [pins.test_svqb_orthonormal_same_span_and_refill]),
    "SVQB without the diagonal scaling D": (
        _wrap(svqb, "svqb", _svqb_no_diagonal_scaling),
        [pins.test_svqb_orthonormal_same_span_and_refill]),
    "Rayleigh-Ritz with Y^T instead of Y^H": (
        _wrap(rr, "rayleigh_ritz", _rr(transpose_only=True)),
        [pins.test_rayleigh_ritz_exact_on_invariant_subspace]),
    "Ritz vectors not rotated (V = Y)": (
        _wrap(rr, "rayleigh_ritz", _rr(rotate=False)),
        [pins.test_rayleigh_ritz_exact_on_invariant_subspace]),
    "harmonic Ritz values tau - 1/mu": (
        _wrap(rr, "harmonic_ritz", lambda o: lambda H, Y, tau: (
            lambda r: (r[0], r[1], r[2], 2.0 * tau - r[3]))(o(H, Y, tau))),
        [pins.test_harmonic_values_are_inverse_ritz_values_of_the_shifted_inverse]),
    "harmonic vectors left K-normalised": (
        _wrap(rr, "harmonic_ritz", _harmonic_unnormalised),
        [pins.test_harmonic_ritz_exact_on_invariant_subspace]),
    "KPM moments without 1/R": (
        _wrap(kpm, "moments", lambda o: lambda H, alpha, beta, M, R, seed, complex_values:
              o(H, alpha, beta, M, R, seed, complex_values) * R),
        [pins.test_kpm_count_on_lattice_against_dense]),
    "KPM count without the factor D": (
        _wrap(kpm, "count_in_window", lambda o: lambda mu, D, *a, **k: o(mu, 1, *a, **k)),
        [pins.test_kpm_trace_exact_on_diagonal_and_count]),
    "inset window widened instead of narrowed": (
        _wrap(quality, "damping_sigma", lambda o: lambda *a, inset=0.0, **k: o(*a, inset=-inset, **k)),
        [pins.test_inset_window_lowers_eta]),
    "eta with the natural logarithm": (
        _wrap(quality, "eta", _eta_natural_log),
        [pins.test_tab_lanczoskernel_scaling_constants]),
    "linear-DOS margin with the flat-DOS rule": (
        _wrap(quality, "margin_linear", lambda o: quality.margin_flat),
        [pins.test_tab_num_optimal_degree_quality_and_effort]),
    "linear-DOS effort without the square root": (
        _wrap(quality, "effort_linear", lambda o: lambda eta0, S_w, delta, N_T, N_S:
              eta0 * S_w / delta * N_T * (N_S / N_T) / (1.0 - N_T / N_S)),
        [pins.test_effort_model_linear_minimum_at_four_NT]),
    "empty-window progress without converging pairs": (
        _wrap(solve, "converging", lambda o: lambda res, prev: False),
        [pins.test_chebfd_weak_filter_is_not_taken_for_an_empty_window]),
    "locking without deflation against the locked vectors": (
        _wrap(solve, "deflate", lambda o: lambda Y, L: Y),
        [pins.test_chebfd_locking_on_linear_dos,
         pins.test_chebfd_locking_deflation_over_a_long_run]),
    "adaptive margin where the search interval holds n_s / 2": (
        _wrap(solve, "degree_from_moments",
              lambda o: lambda mu, D, a, b, lo, hi, ns, Np0, **k: o(mu, D, a, b, lo, hi, ns // 2,
                                                                   Np0, **k)),
        [pins.test_adaptive_degree_follows_the_linear_dos_rule]),
    "adaptive degree without N_0": (
        _wrap(solve, "degree_from_moments",
              lambda o: lambda *a, **k: (lambda r: (r[0], r[1], max(2, int(round(r[2] / 6.23)))))(
                  o(*a, **k))),
        [pins.test_adaptive_degree_follows_the_linear_dos_rule]),
    "KPM without the Jackson damping": (
        _wrap(kpm, "jackson_kpm", lambda o: lambda M: np.ones(M)),
        [pins.test_jackson_damped_kpm_dos_is_nonnegative]),
    "onsite disorder left out": (
        _wrap(lattice, "disorder", lambda o: lambda seed, count, W: np.zeros(count)),
        [pins.test_graphene_disorder_on_the_diagonal]),
    "N_0 table read one row late": (
        lambda mp: mp.setattr(solve, "TAB_LANCZOS_N0",
                              solve.TAB_LANCZOS_N0[1:] + (solve.TAB_LANCZOS_N0[-1],)),
        [pins.test_lanczos_N0_of_the_solver_follows_tab_lanczoskernel]),
    "residual norms squared": (
        _wrap(rr, "residual_norms", lambda o: lambda H, V, th: o(H, V, th) ** 2),
        [pins.test_residual_norms_two_state_closed_form]),
    "Lanczos bounds not clamped to Gershgorin": (
        _wrap(bounds, "gershgorin", lambda o: lambda H: (-np.inf, np.inf)),
        [pins.test_lanczos_bounds_stay_inside_gershgorin]),
    "MLP gradient of one layer with the wrong sign": (
        _wrap(mlp, "loss_and_grad", _mlp_grad_sign),
        [pins.test_mlp_gradient_matches_central_differences]),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, monkeypatch):
    patch, checks = MUTANTS[name]
    patch(monkeypatch)
    caught = 0
    for check in checks:
        try:
            check()
        except AssertionError:
            caught += 1
    assert caught, "no pin caught the planted mistake: " + name
