"""Profiling targets: small, self-contained launch sequences for ncu.

    python -m paper_1510_04895_gb300.profile_target [topi|graphene] [n_b] [c64|c128|r32|r64] [sell|free]
        five fused Chebyshev steps on one benchmark lattice (topi: the
        64x64x32x4 insulator, N = 524288; graphene: the 1024x1024 honeycomb
        lattice, N = 2097152); `sell` bypasses the insulator's blocked copy,
        `free` runs the matrix-free step.
    python -m paper_1510_04895_gb300.profile_target df [n_b] [free]
        one double-float filter of degree 8 on the insulator (n_b columns);
        `free` runs its step matrix-free.
    python -m paper_1510_04895_gb300.profile_target solve [fp64|mixed_df]
        one ChebFD iteration (filter of degree 20, SVQB + Rayleigh-Ritz) on a
        32x32x32x4 insulator (N = 131072, W = 1, seed 1) with n_s = 256: the
        dense steps' Gram and block products on a 0.5 GB block.
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import torch  # noqa: E402

import paper_1510_04895_gb300 as pkg  # noqa: E402
from paper_1510_04895_gb300 import workloads  # noqa: E402

kind = sys.argv[1] if len(sys.argv) > 1 else "topi"
w = workloads.GRAPHENE if kind == "graphene" else workloads.TOPI_MEDIUM
if kind == "solve":
    w = dict(w, Lx=32, Ly=32, Lz=32)
H = pkg.chebfd_matrix_create_lattice(w["kind"], w["Lx"], w["Ly"], w.get("Lz", 1), t=w["t"],
                                     m=w.get("m", 0.0), W=w["W"], seed=w["seed"], also_single=True)
if kind == "df":
    nb = int(sys.argv[2]) if len(sys.argv) > 2 else 32
    if len(sys.argv) > 3 and sys.argv[3] == "free":
        H.set_matrix_free(True)
    X = torch.empty((H.n, nb), dtype=torch.complex128, device="cuda")
    pkg.chebfd_random_block(X, ns_total=nb, seed=1)
    gc = pkg.chebfd_window_coeffs(-4.3, 4.3, -0.1, 0.1, 8, "lanczos", 2.0)
    pkg.chebfd_filter_block_df(H, 2.0 / 8.6, 0.0, gc, X)
elif kind == "solve":
    prec = sys.argv[2] if len(sys.argv) > 2 else "fp64"
    pkg.chebfd_solve(H, -0.14, 0.14, 256, 20, eps=1e-9, kernel="lanczos", precision=prec,
                     a=-4.2, b=4.2, max_iter=1, seed=0)
else:
    nb = int(sys.argv[2]) if len(sys.argv) > 2 else w["nb"]
    prec = sys.argv[3] if len(sys.argv) > 3 else ("c64" if kind == "topi" else "r32")
    dt = {"c64": torch.complex64, "c128": torch.complex128, "r32": torch.float32,
          "r64": torch.float64}[prec]
    if len(sys.argv) > 4 and sys.argv[4] == "sell" and H.blocked_width:
        H.set_blocked(False)            # row-wise SELL kernel instead of the blocked one
    if len(sys.argv) > 4 and sys.argv[4] == "free":
        H.set_matrix_free(True)         # entries rebuilt in registers
    U = torch.empty((H.n, nb), dtype=dt, device="cuda")
    W = torch.empty_like(U)
    Y = torch.zeros_like(U)
    pkg.chebfd_random_block(U, ns_total=nb, seed=1)
    pkg.chebfd_random_block(W, ns_total=nb, seed=2)
    for i in range(5):
        pkg.chebfd_chebyshev_step(H, 0.24, 0.0, 1e-3, U, W, Y)
torch.cuda.synchronize()
print("ok")
