"""Pins for the oracle adjoint of the elastic step, with the Picard and with the
Cauchy-Kowalevski predictor (Sec. 3.3): the dot-product identity <A x, y> = <x, A^T y>, A^T
against a densely assembled A on a tiny grid, and central finite differences of the receiver
misfit with respect to the material and the moment tensor."""
import math

import numpy as np
import pytest
import torch

from oracle.adjoint import misfit, step_vjp
from oracle.aderdg import ADERDG, Grid, PointSource
from oracle.pde import Elastic
from paper_1905_07987_gb300 import synth

T = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float64)


def setup(ncell=(2, 2, 2), N=2, bc='absorbing', seed=3, source=True, predictor='picard'):
    mat = T(synth.elastic_material(ncell, seed=seed))
    g = Grid(ncell, (0, 0, 0), (1.0 * ncell[0] / 2, 1.0 * ncell[1] / 2, 1.0 * ncell[2] / 2), [(bc, bc)] * 3)
    s = ADERDG(Elastic(), g, N, cfl=synth.cfl_number(N), material=mat, predictor=predictor)
    if source:
        c, xi = synth.locate((0.4, 0.55, 0.6), ncell, (0, 0, 0), g.hi)
        s.set_point_source(PointSource(c, xi, T(synth.moment_tensor(seed=1)), 2.0, 0.5))
    return s


PREDICTORS = pytest.mark.parametrize("predictor", ["picard", "ck"])


@PREDICTORS
def test_dot_product_identity(predictor):
    s = setup(source=False, predictor=predictor)
    g = torch.Generator().manual_seed(0)
    shape = (s.grid.C,) + (s.n,) * 3 + (9,)
    x = torch.rand(shape, generator=g, dtype=torch.float64) - 0.5
    y = torch.rand(shape, generator=g, dtype=torch.float64) - 0.5
    dt = 0.01
    Ax = s.step(x, torch.tensor(dt, dtype=torch.float64))
    ATy, _, _ = step_vjp(s, x, y, dt)
    assert abs(float((Ax * y).sum() - (x * ATy).sum())) < 1e-12 * float((Ax * y).abs().sum())


@PREDICTORS
def test_transpose_matches_dense_operator(predictor):
    s = setup(ncell=(2, 1, 1), N=1, bc='periodic', source=False, predictor=predictor)
    shape = (s.grid.C,) + (s.n,) * 3 + (9,)
    m = int(np.prod(shape))
    dt = 0.02
    A = torch.zeros(m, m, dtype=torch.float64)
    for k in range(m):
        e = torch.zeros(m, dtype=torch.float64)
        e[k] = 1.0
        A[:, k] = s.step(e.reshape(shape), torch.tensor(dt, dtype=torch.float64)).reshape(-1)
    y = torch.rand(m, dtype=torch.float64)
    ATy, _, _ = step_vjp(s, torch.zeros(shape, dtype=torch.float64), y.reshape(shape), dt)
    assert torch.allclose(ATy.reshape(-1), A.T @ y, atol=1e-13)


def fd_setup(predictor='picard'):
    s = setup(ncell=(2, 2, 2), N=2, predictor=predictor)
    ncell = s.grid.ncell
    pts = np.array([[0.3, 0.7, 1.0], [0.8, 0.2, 1.0]])
    cells, xis = [], []
    for p in pts:
        c, xi = synth.locate(p, ncell, (0, 0, 0), s.grid.hi)
        cells.append(c)
        xis.append(xi)
    s.set_receivers(cells, xis)
    u0 = torch.zeros((s.grid.C,) + (s.n,) * 3 + (9,), dtype=torch.float64)
    dt = 0.6 * float(s.cfl_dt(u0 + 1.0))  # fixed dt from the initial material
    steps = 4
    obs = [0.01 * torch.ones(2, 3, dtype=torch.float64) * (k + 1) for k in range(steps)]
    return s, u0, dt, steps, obs


def adjoint_gradient(s, u0, dt, steps, obs):
    """Backward sweep: lambda^T = dJ/du^T, lambda^n = A^T lambda^{n+1} + dJ/du^n."""
    states = [u0]
    t = 0.5
    for k in range(steps):
        states.append(s.step(states[-1], torch.tensor(dt, dtype=torch.float64), t + k * dt))
    cells, phis, vars_ = s.receivers
    lam = torch.zeros_like(u0)
    gm = torch.zeros_like(s.mat)
    gM = torch.zeros(6, dtype=torch.float64)
    for n in range(steps, 0, -1):
        # dJ/du^n from the record of u^n (k = n-1)
        r = s.record(states[n]) - obs[n - 1]
        for i, (c, phi) in enumerate(zip(cells.tolist(), phis)):
            for a, v in enumerate(vars_):
                lam[c, ..., v] += dt * r[i, a] * phi
        lam, g1, g2 = step_vjp(s, states[n - 1], lam, dt, t + (n - 1) * dt)
        gm += g1
        gM += g2
    return gm, gM


@PREDICTORS
def test_gradients_match_central_finite_differences(predictor):
    s, u0, dt, steps, obs = fd_setup(predictor)
    gm, gM = adjoint_gradient(s, u0, dt, steps, obs)
    J = lambda: float(misfit(s, u0, steps, dt, obs, 0.5))
    mat0 = s.mat.clone()
    rng = np.random.default_rng(0)
    for trial in range(2):
        dirn = T(rng.standard_normal(mat0.shape)) * mat0
        eps = 1e-6
        s.mat = mat0 + eps * dirn
        Jp = J()
        s.mat = mat0 - eps * dirn
        Jm = J()
        s.mat = mat0
        fd = (Jp - Jm) / (2 * eps)
        ad = float((gm * dirn).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad) + 1e-18, (fd, ad)
    M0 = s.source.M.clone()
    for a in range(6):
        e = torch.zeros(6, dtype=torch.float64)
        e[a] = 1e-4
        s.source.M = M0 + e
        Jp = J()
        s.source.M = M0 - e
        Jm = J()
        s.source.M = M0
        fd = (Jp - Jm) / 2e-4
        assert abs(fd - float(gM[a])) <= 1e-6 * max(abs(float(gM[a])), 1e-12), (a, fd, float(gM[a]))
