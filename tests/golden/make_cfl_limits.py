"""Writes cfl_limits.txt: the one-dimensional von Neumann stability limit nu_N (largest Courant
number with amplification <= 1 + 1e-3 over all wavenumbers) of the oracle's ADER-DG scheme for
linear advection with the Rusanov flux, N = 1..6.  Sec. 3.4 states that CFL_N in Eq. (7) depends
on the order; these limits are what the workload CFL factors are measured against.  Calls only
the oracle.  Run:  python tests/golden/make_cfl_limits.py"""
import math
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle.aderdg import ADERDG, Grid  # noqa: E402
from oracle.pde import Advection  # noqa: E402


def amplification(N, nu, thetas=361):
    g = Grid((3,), (0.0,), (3.0,), [("periodic", "periodic")])
    s = ADERDG(Advection([1.0]), g, N)
    n = N + 1
    A = torch.zeros(3, n, n, dtype=torch.float64)
    for m in range(n):
        u = torch.zeros(3, n, 1, dtype=torch.float64)
        u[1, m, 0] = 1.0
        un = s.step(u, torch.tensor(nu, dtype=torch.float64))
        for c in range(3):
            A[c][:, m] = un[c, :, 0]
    A = A.to(torch.complex128)
    r = 0.0
    for th in np.linspace(0, math.pi, thetas):
        G = A[1] + A[0] * complex(math.cos(th), math.sin(th)) + A[2] * complex(math.cos(th), -math.sin(th))
        r = max(r, float(torch.linalg.eigvals(G).abs().max()))
    return r


def limit(N):
    lo, hi = 0.0, 1.0 / (2 * N + 1)
    for _ in range(24):
        mid = 0.5 * (lo + hi)
        if amplification(N, mid) <= 1 + 1e-3:
            lo = mid
        else:
            hi = mid
    return lo


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfl_limits.txt")
    with open(out, "w") as f:
        f.write("# N  nu_N (1-D von Neumann limit of the oracle scheme, Rusanov flux, N+1 Picard iterations)\n")
        f.write("# written by tests/golden/make_cfl_limits.py (oracle only); Sec. 3.4, Eq. (7)\n")
        for N in range(1, 7):
            f.write("%d %.6f\n" % (N, limit(N)))
    print(open(out).read())
