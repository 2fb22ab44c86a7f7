"""Shared helpers for the GPU parity tests: build the same case on the CUDA library (through the
C ABI) and on the CPU oracle from the same seeded synthetic inputs."""
import math

import numpy as np
import torch

from oracle.aderdg import ADERDG, Grid, PointSource
from oracle.pde import Advection, Elastic, Euler, ShallowWater
from paper_1905_07987_gb300 import ader, synth


def rel_linf(a, b):
    """max over variables of max|a - b| / max|b| (per-variable scale, floor 1e-300)."""
    a = np.asarray(a)
    b = np.asarray(b)
    nv = b.shape[-1]
    a = a.reshape(-1, nv)
    b = b.reshape(-1, nv)
    scale = np.maximum(np.abs(b).max(axis=0), 1e-300)
    return float((np.abs(a - b).max(axis=0) / scale).max())


class Case:
    def __init__(self, pde, dim, order, ncell, lo=None, hi=None, bc="periodic", cfl=None,
                 adv=(0.7, -0.4, 0.3), seed=1, material=None, picard_iters=0, limiter=False,
                 precision="fp64", predictor="picard", initial_guess="constant"):
        self.pde, self.dim, self.order = pde, dim, order
        self.ncell = tuple(ncell)
        self.lo = tuple(lo) if lo is not None else (0.0,) * dim
        self.hi = tuple(hi) if hi is not None else (1.0,) * dim
        self.bc = [(bc, bc)] * dim if isinstance(bc, str) else bc
        self.cfl = cfl if cfl is not None else synth.cfl_number(order)
        self.adv = adv[:dim]
        x, _ = ader.reference_nodes(order)
        self.nodes = x
        self.X = synth.node_coordinates(x, self.ncell, self.lo, self.hi)
        self.mat = material
        self.cfg = ader.make_config(pde, dim, order, self.ncell, self.lo, self.hi, self.bc, self.cfl,
                                    adv=self.adv, picard_iters=picard_iters, limiter=limiter,
                                    precision=precision, predictor=predictor,
                                    initial_guess=initial_guess)
        self.ctx = ader.Context(self.cfg)
        if pde == "euler":
            P = Euler(dim)
        elif pde == "advection":
            P = Advection(self.adv)
        elif pde == "swe":
            P = ShallowWater(9.81)
        else:
            P = Elastic()
        mat_t = torch.from_numpy(material) if material is not None else None
        self.oracle = ADERDG(P, Grid(self.ncell, self.lo, self.hi, self.bc), order, cfl=self.cfl,
                             picard_iters=picard_iters, material=mat_t, predictor=predictor,
                             initial_guess=initial_guess)
        if material is not None:
            self.ctx.set_material(torch.from_numpy(material.reshape(-1).copy()).cuda())
        self.shape = (self.ctx.cells,) + (order + 1,) * dim + (self.ctx.nvar,)

    def set(self, u):
        self.ctx.set_state(torch.from_numpy(np.ascontiguousarray(u).reshape(-1)).cuda())

    def get(self):
        out = torch.empty(self.ctx.count, dtype=torch.float64, device="cuda")
        self.ctx.get_state(out)
        torch.cuda.synchronize()
        return out.cpu().numpy().reshape(self.shape)

    def point_source(self, x0, M, f0, t0):
        self.ctx.set_point_source(x0, M, f0, t0)
        c, xi = synth.locate(x0, self.ncell, self.lo, self.hi)
        self.oracle.set_point_source(PointSource(c, xi, torch.tensor(M, dtype=torch.float64), f0, t0))

    def receivers(self, pts, max_steps):
        seismo = torch.zeros(max_steps, len(pts), 3, dtype=torch.float64, device="cuda")
        self.ctx.set_receivers(pts, seismo, max_steps)
        cells, xis = [], []
        for p in pts:
            c, xi = synth.locate(p, self.ncell, self.lo, self.hi)
            cells.append(c)
            xis.append(xi)
        self.oracle.set_receivers(cells, xis)
        return seismo

    def oracle_step(self, u, dt, t=0.0):
        return self.oracle.step(torch.from_numpy(np.ascontiguousarray(u)),
                                torch.tensor(dt, dtype=torch.float64), t).numpy()
