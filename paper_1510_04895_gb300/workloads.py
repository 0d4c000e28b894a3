"""Synthetic workloads: lattice sizes, seeds, windows and seeded random blocks.

This module holds no arithmetic of the method.  It names the workloads used by
the tests and the benchmark and draws seeded random input blocks (numpy
PCG64) that are handed unchanged to both the CUDA library and the CPU oracle.
"""
import numpy as np

# Topological insulator, 8x8x8 sites x 4 orbitals (N = 2048): the smallest case.
TOPI_SMALL = dict(kind="topi", Lx=8, Ly=8, Lz=8, t=1.0, m=1.0, W=0.5, seed=0,
                  window=(-0.1, 0.1), ns=64, nb=64, Np=200, kernel="jackson")

# Topological insulator, 64x64x32 x 4 (N = 524288), FP64 vs complex64 filter.
# The window half width is sized to hold about 100 eigenpairs (oracle KPM,
# tests/golden/topi_64x64x32_window.txt); Np follows from the Lanczos-kernel
# scaling N_p ~ N_0 S_w / delta' with N_0 = 6.23 (Tab. lanczoskernel).
TOPI_MEDIUM = dict(kind="topi", Lx=64, Ly=64, Lz=32, t=1.0, m=1.0, W=1.0, seed=1,
                   ns=256, nb=64, kernel="lanczos")

# Disordered graphene, 1024 x 1024 cells (N = 2097152), 4 stored entries per
# row, onsite disorder in [-0.5, 0.5]; central window with about 200
# eigenpairs (tests/golden/graphene_1024x1024_window.txt), n_s = 512 filtered
# in four blocks of 128.
GRAPHENE = dict(kind="graphene", Lx=1024, Ly=1024, Lz=1, t=1.0, m=0.0, W=1.0, seed=2, ns=512,
                nb=128, kernel="lanczos")

# Large insulator, 200x200x100 x 4 (N = 16e6), complex64 filter, 4 chunks of 64.
TOPI_LARGE = dict(kind="topi", Lx=200, Ly=200, Lz=100, t=1.0, m=1.0, W=0.5, seed=3,
                  ns=256, nb=64, kernel="lanczos")


def random_block(seed, n, nb, complex_values, dtype=None):
    """Seeded N x nb block with entries uniform in [-1, 1) (and imaginary parts)."""
    rs = np.random.default_rng(seed)
    X = rs.uniform(-1.0, 1.0, (n, nb))
    if complex_values:
        X = X + 1j * rs.uniform(-1.0, 1.0, (n, nb))
    return X.astype(dtype) if dtype is not None else X


# Disorder ensemble: 512 insulators, member i has seed 100 + i, lattice edge
# L_i uniform in {10..20} (N = 4 L^3 between 4000 and 32000) and disorder W_i
# uniform in [0.2, 2.0], both drawn from numpy's PCG64 seeded with 100 + i;
# window [-0.05, 0.05], n_s = 48, N_p = 300, Lanczos kernel (mu = 2).
ENSEMBLE = dict(count=512, first_seed=100, window=(-0.05, 0.05), ns=48, Np=300, t=1.0, m=1.0,
                kernel="lanczos")


def ensemble_members(count=512, first_seed=100):
    """[(L, W, seed)] of the disorder ensemble."""
    out = []
    for i in range(count):
        rs = np.random.default_rng(first_seed + i)
        L = int(rs.integers(10, 21))
        W = float(rs.uniform(0.2, 2.0))
        out.append((L, W, first_seed + i))
    return out
