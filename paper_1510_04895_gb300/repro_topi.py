"""The numerical experiment of Sec. 5.1 (Fig. ConvTopi, Fig. EffortTopi) on
the paper's own Hamiltonian, Eq. Ham: a 256 x 256 x 10 topological-insulator
slab (D = 5 * 2^19 = 2621440), t = 1, onsite V_n Gamma0 + 2 Gamma1 with
V_n uniform in [-V/2, V/2], V = 2, spectrum inside [a, b] = [-5.5, 5.5],
target interval [-0.06, 0.06], N_S = 256, N_p = 1438.  ChebFD runs until
every target vector has residual <= 1e-9 (the paper's absolute criterion;
1e-9 / 5.5 relative to ||H|| = 5.5) with the Jackson kernel and the Lanczos
kernel at mu = 1, 2, 3.  One JSON line per kernel: iterations, N_MVM =
iterations x N_S x N_p (the paper's effort unit; its best run, at N_S = 350,
needed 1.2e6 and the linear-DOS estimate is 1.06e6), eigenpairs found (the
paper finds N_T = 144 after a KPM estimate of 124), residuals and seconds.

    python -m paper_1510_04895_gb300.repro_topi [--precision mixed_df]
        [--kernels jackson lanczos1 lanczos2 lanczos3] [--L 256 256 10] [--seed 0]
        [--harmonic] [--inset F --Np-scale S]

--harmonic takes harmonic Ritz pairs for the window centre (Sec. 6);
--inset F filters with the window narrowed by F of its half-width (Sec. 2.2),
usually with --Np-scale 0.5 (N_p scaled by S).

The disorder realisation is this project's (SplitMix64 stream 0, seed 0);
the paper's is not published, so N_T and N_MVM agree only statistically.
"""
import argparse
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

KERNELS = {"jackson": ("jackson", 2.0), "lanczos1": ("lanczos", 1.0),
           "lanczos2": ("lanczos", 2.0), "lanczos3": ("lanczos", 3.0)}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--L", type=int, nargs=3, default=[256, 256, 10])
    p.add_argument("--V", type=float, default=2.0)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--ns", type=int, default=256)
    p.add_argument("--Np", type=int, default=1438)
    p.add_argument("--window", type=float, nargs=2, default=[-0.06, 0.06])
    p.add_argument("--ab", type=float, nargs=2, default=[-5.5, 5.5])
    p.add_argument("--eps-abs", dest="eps_abs", type=float, default=1e-9)
    p.add_argument("--precision", default="mixed_df", choices=["fp64", "mixed", "mixed_df"])
    p.add_argument("--kernels", nargs="+", default=list(KERNELS), choices=list(KERNELS))
    p.add_argument("--max-iter", dest="max_iter", type=int, default=30)
    p.add_argument("--harmonic", action="store_true")
    p.add_argument("--inset", type=float, default=0.0)
    p.add_argument("--Np-scale", dest="np_scale", type=float, default=1.0)
    args = p.parse_args(argv)

    import numpy as np
    import torch
    import paper_1510_04895_gb300 as pkg

    Lx, Ly, Lz = args.L
    t0 = time.perf_counter()
    H = pkg.chebfd_matrix_create_lattice("topi_slab", Lx, Ly, Lz, t=1.0, m=2.0, W=args.V,
                                         seed=args.seed, also_single=True)
    a_l, b_l, _, _ = pkg.chebfd_scale_bounds(H, 30, seed=0)
    a, b = args.ab
    lo, hi = args.window
    _, nt_kpm = pkg.chebfd_param_features(H, lo, hi, 64, a=a, b=b)
    norm = max(abs(a), abs(b))
    print(json.dumps({"matrix": "Eq. Ham slab %dx%dx%d (D = %d), V = %g, seed %d" % (
        Lx, Ly, Lz, H.n, args.V, args.seed), "lanczos_bounds": [a_l, b_l], "interval": [a, b],
        "bounds_inside_interval": bool(a <= a_l and b_l <= b), "kpm_n_target": nt_kpm,
        "setup_seconds": time.perf_counter() - t0}), flush=True)
    for name in args.kernels:
        kern, mu = KERNELS[name]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Np = max(8, int(round(args.Np * args.np_scale)))
        r = pkg.chebfd_solve(H, lo, hi, args.ns, Np, eps=args.eps_abs / norm, kernel=kern,
                             mu=mu, precision=args.precision, a=a, b=b, max_iter=args.max_iter,
                             seed=0, extraction="harmonic" if args.harmonic else "ritz",
                             window_inset=args.inset)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        lam = np.sort(r["lam"])
        print(json.dumps({
            "kernel": name, "precision": args.precision, "converged": r["converged"],
            "Np": Np, "harmonic": args.harmonic, "window_inset": args.inset,
            "iterations": r["iterations"], "fp64_filter_iterations": r["fp64_iterations"],
            "n_mvm": r["iterations"] * args.ns * Np, "n_target_found": r["nev"],
            "max_residual": float(r["res"].max()) if r["nev"] else None,
            "lambda_range": [float(lam[0]), float(lam[-1])] if r["nev"] else None,
            "seconds": sec, "seconds_filter": r["seconds_filter"],
            "seconds_dense": r["seconds_dense"]}), flush=True)
        del r
    return 0


if __name__ == "__main__":
    sys.exit(main())
