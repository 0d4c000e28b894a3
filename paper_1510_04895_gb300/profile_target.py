"""Profiling target: five fused Chebyshev steps on the 64x64x32x4 insulator.

Usage: python -m paper_1510_04895_gb300.profile_target [n_b] [c64|c128]
(a small, self-contained launch sequence for ncu: one matrix, three blocks).
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import torch
import paper_1510_04895_gb300 as pkg
nb = int(sys.argv[1]) if len(sys.argv) > 1 else 64
prec = sys.argv[2] if len(sys.argv) > 2 else "c64"
dt = torch.complex64 if prec == "c64" else torch.complex128
H = pkg.chebfd_matrix_create_lattice("topi", 64, 64, 32, t=1.0, m=1.0, W=1.0, seed=1, also_single=True)
U = torch.empty((H.n, nb), dtype=dt, device="cuda"); W = torch.empty_like(U); Y = torch.zeros_like(U)
pkg.chebfd_random_block(U, ns_total=nb, seed=1); pkg.chebfd_random_block(W, ns_total=nb, seed=2)
for i in range(5):
    pkg.chebfd_chebyshev_step(H, 0.24, 0.0, 1e-3, U, W, Y)
torch.cuda.synchronize()
print("ok")
