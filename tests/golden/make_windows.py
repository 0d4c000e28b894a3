"""Write the central target windows of the larger insulator / graphene workloads.

Calls only the CPU oracle: Lanczos bounds [a, b], stochastic KPM moments
(Jackson-damped) and a bisection for the half width delta at which the KPM
count of Eq. DOS:target reaches the wanted number of eigenpairs.  The result
is frozen into a text file so that the CUDA path and the oracle filter with the
same window.  Usage: python tests/golden/make_windows.py <name> [M] [R]
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import bounds, coeffs, kpm, lattice  # noqa: E402

CASES = {
    "topi_64x64x32": dict(make=lambda: lattice.topi_csr(64, 64, 32, t=1.0, m=1.0, W=1.0, seed=1),
                          want=100),
    "graphene_1024x1024": dict(make=lambda: lattice.graphene_csr(1024, 1024, t=1.0, W=1.0, seed=2),
                               want=200),
    "topi_200x200x100": dict(make=lambda: lattice.topi_csr(200, 200, 100, t=1.0, m=1.0, W=0.5, seed=3),
                             want=100),
}


def main(name, M=2048, R=8):
    case = CASES[name]
    H = lattice.to_scipy(*case["make"]())
    D = H.shape[0]
    a, b = bounds.lanczos_bounds(H, 30, seed=0)
    alpha, beta = coeffs.scaling(a, b)
    mu = kpm.moments(H, alpha, beta, M, R, seed=0, complex_values=np.iscomplexobj(H.data))
    lo, hi = 1e-6, 1.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if kpm.count_in_window(mu, D, a, b, -mid, mid) < case["want"]:
            lo = mid
        else:
            hi = mid
    delta = 0.5 * (lo + hi)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), name + "_window.txt")
    with open(out, "w") as f:
        f.write("# Central target window [-delta, delta] holding ~%d eigenpairs, from the\n"
                "# oracle's Lanczos bounds and %d-moment, %d-probe Jackson-damped KPM DOS\n"
                "# (Sec. 3.1 steps 1-2, Eq. DOS:target); written by make_windows.py.\n" % (case["want"], M, R))
        f.write("a %.17g\nb %.17g\ndelta %.17g\nkpm_count %.6f\nM %d\nR %d\n"
                % (a, b, delta, kpm.count_in_window(mu, D, a, b, -delta, delta), M, R))
    print(open(out).read())


if __name__ == "__main__":
    args = sys.argv[1:]
    main(args[0], *(int(x) for x in args[1:]))
