"""Profiling target: five fused Chebyshev steps on one benchmark lattice.

Usage: python -m paper_1510_04895_gb300.profile_target [topi|graphene] [n_b] [c64|c128|r32|r64] [sell]
(a small, self-contained launch sequence for ncu: one matrix, three blocks).
topi: the 64x64x32x4 insulator (N = 524288); graphene: the 1024x1024
honeycomb lattice (N = 2097152).
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import torch
import paper_1510_04895_gb300 as pkg
from paper_1510_04895_gb300 import workloads

kind = sys.argv[1] if len(sys.argv) > 1 else "topi"
w = workloads.TOPI_MEDIUM if kind == "topi" else workloads.GRAPHENE
nb = int(sys.argv[2]) if len(sys.argv) > 2 else w["nb"]
prec = sys.argv[3] if len(sys.argv) > 3 else ("c64" if kind == "topi" else "r32")
dt = {"c64": torch.complex64, "c128": torch.complex128, "r32": torch.float32,
      "r64": torch.float64}[prec]
H = pkg.chebfd_matrix_create_lattice(kind, w["Lx"], w["Ly"], w.get("Lz", 1), t=w["t"],
                                     m=w.get("m", 0.0), W=w["W"], seed=w["seed"], also_single=True)
if len(sys.argv) > 4 and sys.argv[4] == "sell" and H.blocked_width:
    H.set_blocked(False)            # row-wise SELL kernel instead of the blocked one
U = torch.empty((H.n, nb), dtype=dt, device="cuda"); W = torch.empty_like(U); Y = torch.zeros_like(U)
pkg.chebfd_random_block(U, ns_total=nb, seed=1); pkg.chebfd_random_block(W, ns_total=nb, seed=2)
for i in range(5):
    pkg.chebfd_chebyshev_step(H, 0.24, 0.0, 1e-3, U, W, Y)
torch.cuda.synchronize()
print("ok")
