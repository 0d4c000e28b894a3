"""Design findings reproduced on the CPU oracle (no GPU): each test reruns
one comparison quoted in the design notes, so the numbers there can be
regenerated from committed code."""
import numpy as np

from oracle import bounds, coeffs, filter as filt, lattice, solve


def _insulator_case(L=10, NT=60, NS=112):
    H = lattice.to_scipy(*lattice.topi_csr(L, L, L, t=1.0, m=1.0, W=1.0, seed=1))
    a, b = bounds.lanczos_bounds(H, 30, seed=0)
    e = np.linalg.eigvalsh(H.toarray())
    ae = np.sort(np.abs(e))
    delta = 0.5 * (ae[NT - 1] + ae[NT])          # a central window holding NT eigenvalues
    ratio = np.sqrt(NS / NT) - 1.0               # delta'/delta for a linear DOS (Sec. 2.4)
    Np = int(round(6.23 * 0.5 * (b - a) / (ratio * delta)))   # N_p = N_0 S_w / delta'
    return H, a, b, e[np.abs(e) <= delta], delta, NS, Np


def test_inset_window_halves_the_spmvms_on_a_10x10x10_insulator():
    """N = 4000, N_T = 60, N_S = 112 (delta'/delta = 0.37), Lanczos mu = 2:
    the window narrowed by half its half-width at half the degree finds every
    window eigenvalue in no more iterations than the rectangular window at
    the full degree (about half the spMVMs); the rectangular window at 0.6 of
    the degree is too weak for the ghost test for several iterations and
    needs more spMVMs than either."""
    H, a, b, ew, delta, NS, Np = _insulator_case()
    runs = {}
    for name, inset, scale in (("rect", 0.0, 1.0), ("inset", 0.5, 0.5), ("rect_short", 0.0, 0.6)):
        n = int(round(Np * scale))
        runs[name] = solve.chebfd(H, a, b, -delta, delta, NS, n, 1e-9, max_iter=25,
                                  complex_values=True, window_inset=inset)
        runs[name]["Np"] = n
    for name in ("rect", "inset"):
        r = runs[name]
        assert r["converged"] and len(r["theta"]) == len(ew) == 60
        assert np.abs(np.sort(r["theta"]) - ew).max() <= 1e-9 * r["normH"]
    assert runs["inset"]["iterations"] <= runs["rect"]["iterations"]
    mvm = {k: runs[k]["iterations"] * runs[k]["Np"] for k in ("rect", "inset")}
    assert mvm["inset"] <= 0.55 * mvm["rect"]
    short = runs["rect_short"]
    assert short["converged"] and len(short["theta"]) == 60
    assert short["iterations"] * short["Np"] > max(mvm["rect"], 2 * mvm["inset"])
