"""The benchmark's quadrature L2 norm of the density error (used for its convergence study)
against the oracle's own quadrature norm on the same states: a 2-D and a 3-D grid with uneven
cell counts, after a few oracle steps of the entropy wave (a state that is not the exact
solution, so every term of the norm is exercised)."""
import os
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import bench  # noqa: E402
from oracle.pde import Euler  # noqa: E402
from paper_1905_07987_gb300 import synth  # noqa: E402
from test_oracle_scheme import coords, l2_error, make  # noqa: E402


class _HostState:
    """What the norm reads from a context: the state size, the cell count, get_state()."""

    def __init__(self, u):
        self.u = u.reshape(-1)
        self.count = self.u.numel()
        self.cells = u.shape[0]

    def get_state(self, out):
        out.copy_(self.u)


@pytest.mark.parametrize("ncell,N", [((5, 3), 3), ((4, 3, 2), 2)])
def test_quadrature_norm_matches_the_oracle_norm(ncell, N):
    D = len(ncell)
    lo, hi = (0.0,) * D, (1.0, 0.75, 1.25)[:D]
    s = make(Euler(D), ncell, N, lo=lo, hi=hi)
    u = torch.tensor(synth.entropy_wave(coords(s)))
    for _ in range(3):
        u = s.step(u, s.cfl_dt(u))
    t = 0.0123
    ref = l2_error(s, u, lambda X: synth.entropy_wave(X, t)[..., 0])
    wl = dict(dim=D, order=N, ncell=ncell, lo=lo, hi=hi)
    got = bench.density_l2_quadrature(_HostState(u), wl, t, s.ref.x.numpy(), device="cpu")
    assert got == pytest.approx(ref, rel=1e-12), (got, ref)
    assert ref > 1e-4
