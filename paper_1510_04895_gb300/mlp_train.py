"""Training records, training and evaluation of the parameter-predicting MLP.

Records come from the method itself: disordered insulators are solved by
chebfd_solve with a grid of (N_p, n_s, kernel) around the paper's rule; each
run's cost and convergence are recorded, and the cheapest run that found
every eigenpair of the window is the label of that instance.  Four families
(see instance()): small lattices (FP64 solves), and, solved with MIXED_DF,
members of the disorder ensemble's kind with its fixed window and the two
benchmark insulators' shapes reduced.  The committed records are
data/mlp_records*.jsonl, the weights trained on all of them
data/mlp_weights.npy.

    python -m paper_1510_04895_gb300.mlp_train records --family ensemble \
        --precision mixed_df --count 64 --first 0 --out R.jsonl
    python -m paper_1510_04895_gb300.mlp_train train --records R1.jsonl R2.jsonl --out W.npy
    python -m paper_1510_04895_gb300.mlp_train evaluate --weights W.npy --family small

Cost of a run, in products with H (the paper's N_MVM unit, Sec. 3.3) plus
the dense work: N_iter n_s N_p + 3 N_iter n_s^2.  The factor 3 is the
measured ratio of FP64 Gram/Rayleigh-Ritz time to filter time per
(n_s x n_s)-vs-(n_s x N_p) unit on GB300 (FP64 GEMM 1.1 TFLOP/s against the
fused step's ~4.4 TB/s).
"""
import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

M_FEAT = 64
N_IN = M_FEAT + 3
EPS = 1e-9
NP_FACTORS = (0.5, 1.0, 2.0)
NS_FACTORS = (2.0, 4.0, 6.0)
KERNELS = ("jackson", "lanczos")


FAMILIES = ("small", "ensemble", "medium_shape", "large_shape")


def instance(k, family="small"):
    """Insulator k of a record family, from numpy's PCG64 seeded per family:
    small         edge L in {6, 7, 8}, Lz in {4..8}, W in U[0.3, 2.5],
                  N_T in U{6..30} (seed 7000 + k);
    ensemble      members of the disorder ensemble's kind: cubes of edge
                  L in {10, 11, 12}, W in U[0.2, 2.0], the fixed window
                  [-0.05, 0.05] (N_T = 0: the window is not sized from a
                  count; seed 20000 + k);
    medium_shape  the 64x64x32 benchmark lattice's shape reduced: Lx = Ly =
                  2 Lz with Lz in {5, 6, 7}, W = 1.0, N_T in U{10..60}
                  (seed 30000 + k);
    large_shape   the 200x200x100 lattice's shape reduced the same way,
                  W = 0.5, N_T in U{10..60} (seed 40000 + k)."""
    if family == "small":
        rs = np.random.default_rng(7000 + k)
        L = int(rs.integers(6, 9))
        Lz = int(rs.integers(4, 9))
        W = float(rs.uniform(0.3, 2.5))
        NT = int(rs.integers(6, 31))
        return dict(k=k, L=L, Lz=Lz, W=W, NT=NT, seed=7000 + k)
    if family == "ensemble":
        rs = np.random.default_rng(20000 + k)
        L = int(rs.integers(10, 13))
        return dict(k=k, family=family, L=L, Lz=L, W=float(rs.uniform(0.2, 2.0)), NT=0,
                    delta=0.05, seed=20000 + k)
    base = {"medium_shape": (30000, 1.0), "large_shape": (40000, 0.5)}[family]
    rs = np.random.default_rng(base[0] + k)
    Lz = int(rs.integers(5, 8))
    return dict(k=k, family=family, L=2 * Lz, Lz=Lz, W=base[1], NT=int(rs.integers(10, 61)),
                seed=base[0] + k)


def window_of(inst, eigs):
    """Half width of the instance's window: fixed, or sized to hold about N_T."""
    return inst["delta"] if inst.get("delta") else window_for(eigs, inst["NT"])


def dense_eigs(H):
    """Eigenvalues of a (small) library matrix by dense diagonalisation on the
    GPU (cuSOLVER through torch): the ground-truth window count of a record."""
    import torch
    A = torch.from_numpy(dense_of(H)).cuda()
    return torch.linalg.eigvalsh(A).cpu().numpy()


def cost_of(iterations, ns, Np):
    return iterations * ns * Np + 3 * iterations * ns * ns


def iteration_log(r):
    """The solve's per-iteration records (chebfd_result_iterations): precision
    phase, in-window / ghost / accepted counts, residual range and the seconds
    of the filter and of the dense steps, kept with each training run."""
    keys = ("fp64_filter", "in_window", "ghosts", "accepted", "res_min", "res_max", "Np",
            "seconds_filter", "seconds_dense")
    return [{k: rec[k] for k in keys} for rec in r["log"]]


def window_for(H_dense_eigs, NT):
    """Half width of a symmetric window holding about NT eigenvalues of
    smallest |lambda|: the cut is placed in the widest gap of |lambda| among the
    cut positions NT-4 .. NT+4 (the spectrum is +- paired and degenerate, so a
    cut at exactly NT may split a multiplet), half way across that gap."""
    e = np.sort(np.abs(H_dense_eigs))
    cuts = [n for n in range(max(2, NT - 4), min(len(e) - 1, NT + 5))]
    n = max(cuts, key=lambda c: (e[c] - e[c - 1]) / max(e[c], 1e-12))
    return 0.5 * (e[n - 1] + e[n])


def run_solve(pkg, H, lo, hi, ns, Np, kernel, a, b, precision="fp64", max_iter=25, seed=0):
    t0 = time.perf_counter()
    r = pkg.chebfd_solve(H, lo, hi, ns, Np, eps=EPS, kernel=kernel, precision=precision, a=a, b=b,
                         max_iter=max_iter, seed=seed)
    return r, time.perf_counter() - t0


def correct(r, exact, normH):
    if not r["converged"] or r["nev"] != len(exact):
        return False
    return bool(np.abs(np.sort(r["lam"]) - exact).max() <= 1e-8 * normH)


def make_records(count, first, out, family="small", precision="fp64"):
    import torch
    import paper_1510_04895_gb300 as pkg
    torch.cuda.set_device(0)
    with open(out, "w") as f:
        for k in range(first, first + count):
            inst = instance(k, family)
            L, Lz, W = inst["L"], inst["Lz"], inst["W"]
            H = pkg.chebfd_matrix_create_lattice("topi", L, L, Lz, t=1.0, m=1.0, W=W,
                                                 seed=inst["seed"], also_single=True)
            eigs = dense_eigs(H)                     # ground truth of the window count
            delta = window_of(inst, eigs)
            exact = np.sort(eigs[np.abs(eigs) <= delta])
            if len(exact) == 0:                      # a gapped member: nothing to learn
                print("instance %d: empty window, skipped" % k, flush=True)
                continue
            a, b, _, _ = pkg.chebfd_scale_bounds(H, 30, seed=0)
            normH = max(abs(a), abs(b))
            feats, nt_est = pkg.chebfd_param_features(H, -delta, delta, M_FEAT, a=a, b=b)
            ns_h, Np_h, _, _ = pkg.chebfd_choose_params(H, -delta, delta, a=a, b=b)
            runs = []
            for fp in NP_FACTORS:
                for fs in NS_FACTORS:
                    for kern in KERNELS:
                        Np = max(8, int(round(fp * Np_h)))
                        ns = max(16, int(np.ceil(fs * max(nt_est, 1.0) / 8.0)) * 8)
                        r, sec = run_solve(pkg, H, -delta, delta, ns, Np, kern, a, b,
                                           precision=precision)
                        ok = correct(r, exact, normH)
                        runs.append(dict(Np=Np, ns=ns, kernel=kern, converged=r["converged"],
                                         correct=ok, iterations=r["iterations"],
                                         n_mvm=r["n_mvm"], seconds=sec,
                                         cost=cost_of(r["iterations"], ns, Np),
                                         log=iteration_log(r)))
            rec = dict(instance=inst, precision=precision, delta=delta, a=a, b=b,
                       n_target_exact=len(exact),
                       n_target_kpm=nt_est, features=[float(x) for x in feats],
                       heuristic=dict(ns=ns_h, Np=Np_h), runs=runs)
            f.write(json.dumps(rec) + "\n")
            f.flush()
            print("instance %d: N=%d N_T=%d (kpm %.1f) best %s" % (
                k, 4 * L * L * Lz, len(exact), nt_est,
                min((r for r in runs if r["correct"]), key=lambda r: r["cost"], default=None)),
                flush=True)


def dense_of(H):
    """Dense matrix of a (small) library matrix, rebuilt from its exported SELL arrays."""
    S = H.export_sell()
    n, C = S["n"], S["C"]
    A = np.zeros((n, n), dtype=S["val"].dtype)
    for k in range(S["nchunks"]):
        for l in range(C):
            r = k * C + l
            if r >= n:
                continue
            row = S["perm"][r]
            for j in range(S["chunk_len"][k]):
                pos = S["chunk_ptr"][k] + j * C + l
                A[row, S["col"][pos]] += S["val"][pos]
    return A


def init_params(n_in, n_h, seed):
    """Uniform +-sqrt(3/fan_in) weights, zero biases, packed (W1 b1 W2 b2 W3 b3)."""
    rs = np.random.default_rng(seed)
    parts = [rs.uniform(-1, 1, (n_h, n_in)) * np.sqrt(3.0 / n_in), np.zeros(n_h),
             rs.uniform(-1, 1, (n_h, n_h)) * np.sqrt(3.0 / n_h), np.zeros(n_h),
             rs.uniform(-1, 1, (3, n_h)) * np.sqrt(3.0 / n_h), np.zeros(3)]
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)


def load_records(path):
    with open(path) as f:
        return [json.loads(l) for l in f if l.strip()]


def dataset(records):
    """Features and scale-free targets of the best correct run: log(N_p / N_p of
    the paper's rule), log(n_s / N_T estimate), 1 if the kernel is Lanczos."""
    X, T = [], []
    for rec in records:
        good = [r for r in rec["runs"] if r["correct"]]
        if not good:
            continue
        best = min(good, key=lambda r: r["cost"])
        X.append(rec["features"])
        T.append([np.log(best["Np"] / rec["heuristic"]["Np"]),
                  np.log(best["ns"] / max(rec["n_target_kpm"], 1.0)),
                  1.0 if best["kernel"] == "lanczos" else 0.0])
    return np.array(X, np.float32), np.array(T, np.float32)


def train(records, hidden=128, steps=3000, lr=3e-3, seed=0):
    """Train on the GPU with the library's MLP kernels; returns the MLP."""
    import torch
    import paper_1510_04895_gb300 as pkg
    X, T = dataset(records)
    net = pkg.MLP(N_IN, hidden)
    flat = init_params(N_IN, hidden, seed)
    # start the output bias at the target means
    flat[-3:] = T.mean(axis=0)
    flat[-1] = 0.0
    net.set_params(flat)
    Xd = torch.from_numpy(X).cuda()
    Td = torch.from_numpy(T).cuda()
    losses = []
    for it in range(steps):
        loss = net.loss_grad(Xd, Td)
        net.adam(lr)
        if it % 100 == 0 or it == steps - 1:
            losses.append(loss)
    return net, losses


def evaluate(weights, first, count, hidden=128, family="small"):
    """Solve fresh instances with the paper's rule and with the MLP; returns
    per-instance dicts (cost, correctness, seconds) for both."""
    import torch
    import paper_1510_04895_gb300 as pkg
    net = pkg.MLP(N_IN, hidden)
    net.set_params(np.asarray(weights, np.float32))
    out = []
    for k in range(first, first + count):
        inst = instance(k, family)
        L, Lz, W = inst["L"], inst["Lz"], inst["W"]
        H = pkg.chebfd_matrix_create_lattice("topi", L, L, Lz, t=1.0, m=1.0, W=W,
                                             seed=inst["seed"], also_single=True)
        eigs = dense_eigs(H)
        delta = window_of(inst, eigs)
        exact = np.sort(eigs[np.abs(eigs) <= delta])
        if len(exact) == 0:
            continue
        a, b, _, _ = pkg.chebfd_scale_bounds(H, 30, seed=0)
        normH = max(abs(a), abs(b))
        row = dict(instance=inst, n_target=len(exact))
        for name, model in (("heuristic", None), ("mlp", net)):
            ns, Np, kern, _ = pkg.chebfd_choose_params(H, -delta, delta, mlp=model, a=a, b=b,
                                                       m_feat=M_FEAT)
            r, sec = run_solve(pkg, H, -delta, delta, ns, Np, kern, a, b, max_iter=40)
            row[name] = dict(ns=ns, Np=Np, kernel=kern, iterations=r["iterations"],
                             correct=correct(r, exact, normH), seconds=sec,
                             cost=cost_of(r["iterations"], ns, Np), log=iteration_log(r))
        out.append(row)
    return out


def main():
    p = argparse.ArgumentParser()
    sub = p.add_subparsers(dest="cmd")
    r = sub.add_parser("records")
    r.add_argument("--out", required=True)
    r.add_argument("--count", type=int, default=64)
    r.add_argument("--first", type=int, default=0)
    r.add_argument("--family", default="small", choices=FAMILIES)
    r.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "mixed_df"])
    t = sub.add_parser("train")
    t.add_argument("--records", required=True, nargs="+")
    t.add_argument("--out", required=True)
    e = sub.add_parser("evaluate")
    e.add_argument("--weights", required=True)
    e.add_argument("--first", type=int, default=1000)
    e.add_argument("--count", type=int, default=16)
    e.add_argument("--family", default="small", choices=FAMILIES)
    e.add_argument("--out", required=True)
    a = p.parse_args()
    if a.cmd == "records":
        make_records(a.count, a.first, a.out, a.family, a.precision)
    elif a.cmd == "train":
        net, losses = train([rec for path in a.records for rec in load_records(path)])
        params, _ = net.get_params()
        np.save(a.out, params)
        print("losses", losses[::5], losses[-1])
    elif a.cmd == "evaluate":
        rows = evaluate(np.load(a.weights), a.first, a.count, family=a.family)
        with open(a.out, "w") as f:
            for row in rows:
                f.write(json.dumps(row) + "\n")
        ok = [r for r in rows if r["heuristic"]["correct"] and r["mlp"]["correct"]]
        ratio = [r["mlp"]["cost"] / r["heuristic"]["cost"] for r in ok]
        print("both correct %d/%d, mlp correct %d, heuristic correct %d, mean cost ratio "
              "mlp/heuristic %.3f, geo-mean %.3f" % (
                  len(ok), len(rows), sum(r["mlp"]["correct"] for r in rows),
                  sum(r["heuristic"]["correct"] for r in rows),
                  float(np.mean(ratio)) if ratio else float("nan"),
                  float(np.exp(np.mean(np.log(ratio)))) if ratio else float("nan")))


if __name__ == "__main__":
    main()
