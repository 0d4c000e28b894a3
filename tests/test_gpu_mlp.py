"""The MLP's CUDA forward, loss, backward and Adam kernels against the FP64
oracle (tolerances of FP32 arithmetic), and the paper's parameter rule."""
import numpy as np
import pytest
import torch

import paper_1510_04895_gb300 as pkg
from oracle import lattice, mlp as omlp

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _setup(B=37, n_in=67, n_h=128, seed=0):
    rs = np.random.default_rng(seed)
    P = omlp.init_params(n_in, n_h, 3, seed=seed + 1)
    for k in P:
        P[k] = P[k] + 0.05 * rs.standard_normal(P[k].shape)
    flat = pkg.pack_params(P).astype(np.float32)
    P32 = pkg.unpack_params(flat.astype(np.float64), n_in, n_h)   # the weights the GPU sees
    X = rs.standard_normal((B, n_in)).astype(np.float32)
    T = np.c_[rs.standard_normal((B, 2)), rs.integers(0, 2, B)].astype(np.float32)
    net = pkg.MLP(n_in, n_h)
    net.set_params(flat)
    return net, P32, X, T


def test_mlp_forward_matches_oracle():
    net, P, X, T = _setup()
    Z = net.forward(torch.from_numpy(X).to(DEV)).cpu().numpy()
    Zo, _ = omlp.forward(P, X.astype(np.float64))
    assert np.abs(Z - Zo).max() <= 2e-5 * max(1.0, np.abs(Zo).max())


def test_mlp_loss_and_gradient_match_oracle():
    net, P, X, T = _setup(B=64, seed=3)
    loss = net.loss_grad(torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV))
    Lo, Go = omlp.loss_and_grad(P, X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - Lo) <= 1e-5 * max(1.0, abs(Lo))
    _, g = net.get_params()
    G = pkg.unpack_params(g.astype(np.float64), 67, 128)
    for k in Go:
        scale = max(np.abs(Go[k]).max(), 1e-3)
        assert np.abs(G[k] - Go[k]).max() <= 1e-5 * scale * 10, k


def test_mlp_adam_step_matches_oracle():
    net, P, X, T = _setup(B=16, seed=5)
    net.loss_grad(torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV))
    _, g = net.get_params()
    net.adam(1e-3)
    p_new, _ = net.get_params()
    G = pkg.unpack_params(g.astype(np.float64), 67, 128)
    Pn = omlp.adam_step({k: v.copy() for k, v in P.items()}, G, {}, 1e-3)
    ref = pkg.pack_params(Pn)
    assert np.abs(p_new - ref).max() <= 1e-6


def test_mlp_training_reduces_loss():
    rs = np.random.default_rng(9)
    X = rs.standard_normal((48, 10)).astype(np.float32)
    T = np.c_[0.5 * X[:, 0], np.tanh(X[:, 1]), (X[:, 2] > 0)].astype(np.float32)
    net = pkg.MLP(10, 32)
    P = omlp.init_params(10, 32, 3, seed=4)
    net.set_params(pkg.pack_params(P).astype(np.float32))
    Xd, Td = torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV)
    l0 = net.loss_grad(Xd, Td)
    for _ in range(400):
        net.loss_grad(Xd, Td)
        net.adam(1e-2)
    assert net.loss_grad(Xd, Td) < 0.2 * l0


def test_heuristic_parameters_on_smallest_insulator():
    """Paper's rule: N_T from the KPM DOS, n_s = 4 N_T, N_p = N_0 S_w / delta'.
    The KPM count is within its stochastic error of the exact count, and the
    chosen parameters solve the window completely."""
    H = pkg.chebfd_matrix_create_lattice("topi", 8, 8, 8, W=0.5, seed=0, also_single=True)
    e = np.linalg.eigvalsh(lattice.to_scipy(*lattice.topi_csr(8, 8, 8, W=0.5, seed=0)).toarray())
    exact = np.sort(e[np.abs(e) <= 0.1])
    ns, Np, kern, nt = pkg.chebfd_choose_params(H, -0.1, 0.1)
    assert abs(nt - len(exact)) <= 0.35 * len(exact) + 3
    assert ns % 8 == 0 and ns >= 16 and 8 <= Np <= 20000 and kern == "lanczos"
    f, nt2 = pkg.chebfd_param_features(H, -0.1, 0.1, 64)
    assert f.shape == (67,) and f[0] == pytest.approx(1.0, abs=1e-12) and nt2 == pytest.approx(nt)
    r = pkg.chebfd_solve(H, -0.1, 0.1, ns, Np, eps=1e-9, kernel=kern)
    assert r["converged"] and r["nev"] == len(exact)
    assert np.abs(np.sort(r["lam"]) - exact).max() <= 1e-10 * max(abs(r["a"]), abs(r["b"]))


def test_trained_mlp_gains_over_the_rule_on_held_out_insulators():
    """The MLP trained (on the GPU, by these kernels) on the method's own
    cost/convergence records chooses (N_p, n_s, kernel) for insulators it has
    not seen: small lattices (edge 6-8), disorder-ensemble members with the
    fixed window, and the two benchmark lattices' shapes reduced.  The cost
    is N_iter n_s N_p + 3 N_iter n_s^2 and the ground truth dense
    diagonalisation.  The rule finds every window eigenpair; the learned
    choice runs with a smaller margin and may miss on at most 2 instances of
    a family.  Its geometric-mean cost relative to the rule is below 1 on each
    family shaped like the benchmark workloads and over all instances
    together; on the small lattices, where the rule's margin is already
    small and the network trades fit for the larger families, it stays within
    10 % of the rule."""
    import os
    from paper_1510_04895_gb300 import mlp_train
    w = np.load(os.path.join(os.path.dirname(pkg.__file__), "data", "mlp_weights.npy"))
    logs = []
    for family, count in (("small", 16), ("ensemble", 10), ("medium_shape", 8),
                          ("large_shape", 8)):
        rows = mlp_train.evaluate(w, 1000, count, family=family)
        assert rows and all(r["heuristic"]["correct"] for r in rows)
        assert sum(r["mlp"]["correct"] for r in rows) >= len(rows) - 2
        ratio = np.log([r["mlp"]["cost"] / r["heuristic"]["cost"] for r in rows
                        if r["mlp"]["correct"]])
        gain = float(np.exp(ratio.mean()))
        print("MLP / rule geometric-mean cost, held-out %s: %.3f (%d instances)"
              % (family, gain, len(rows)))
        assert gain < (1.1 if family == "small" else 1.0), (family, gain)
        logs.extend(ratio)
    assert float(np.exp(np.mean(logs))) < 1.0


def test_mlp_retrains_from_committed_records():
    """Training from the committed records (all families) with the library's
    kernels reaches a small loss (the records are the method's own runs)."""
    import glob
    import os
    from paper_1510_04895_gb300 import mlp_train
    paths = sorted(glob.glob(os.path.join(os.path.dirname(pkg.__file__), "data",
                                          "mlp_records*.jsonl")))
    assert len(paths) == 4
    recs = [r for p in paths for r in mlp_train.load_records(p)]
    net, losses = mlp_train.train(recs, steps=1500)
    assert losses[-1] < 0.05 * losses[0]
