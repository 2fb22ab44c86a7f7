"""Pins for the oracle's shallow water equations with bathymetry (Eq. (9), Sec. 2): a
state-dependent non-conservative product g h d(b + h)/dx_d and its path-conservative Rusanov
fluctuation.  Lake at rest (well balanced to round-off), order N+1 on a steady flow over a
periodic bump (exact by Bernoulli's law), and the x <-> y symmetry of a radial hump."""
import math

import numpy as np
import torch

from oracle.aderdg import ADERDG, Grid
from oracle.pde import ShallowWater
from paper_1905_07987_gb300 import synth

T = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float64)
G = 9.81


def coords(s):
    return synth.node_coordinates(s.ref.x.numpy(), s.grid.ncell, s.grid.lo, s.grid.hi)


def make(ncell, N, lo, hi, bc):
    g = Grid(ncell, lo, hi, [(bc, bc)] * 2)
    return ADERDG(ShallowWater(G), g, N, cfl=synth.cfl_number(N))


def state(h, hu, hv, b):
    return T(np.stack([h, hu, hv, b], axis=-1))


def test_lake_at_rest_is_preserved_to_round_off():
    """b = (x^2 + y^2)/10 (a polynomial the order-2 basis holds exactly, continuous across faces),
    h = 1 - b, no flow, reflecting walls: the free surface h + b = 1 stays flat, the flow stays
    zero, mass is conserved and b moves by round-off only."""
    s = make((5, 4), 2, (-1.0, -1.0), (1.0, 1.0), "wall")
    X = coords(s)
    b = 0.1 * (X[0] ** 2 + X[1] ** 2)
    u0 = state(1.0 - b, 0 * b, 0 * b, b)
    W = s.tensor_basis_weights()
    mass0 = float((u0[..., 0] * W).sum())
    u = u0
    for _ in range(5):
        u = s.step(u, s.cfl_dt(u))
    assert float((u - u0).abs().max()) < 1e-13
    assert abs(float((u[..., 0] * W).sum()) - mass0) < 1e-14 * mass0


def bernoulli_h(b, q=0.5, h0=1.0, b0=0.1):
    """Subcritical depth of the steady flow with discharge q over bathymetry b:
    q^2 / (2 h^2) + g (h + b) = q^2 / (2 h0^2) + g (h0 + b0), by Newton from h0."""
    E = q * q / (2 * h0 * h0) + G * (h0 + b0)
    h = np.full_like(b, h0)
    for _ in range(60):
        f = q * q / (2 * h * h) + G * (h + b) - E
        h = h - f / (G - q * q / h ** 3)
    return h


def l2_h(s, u, exact_fn):
    """L2 error of h with an (N+3)-point Gauss-Legendre rule per cell (no nodal superconvergence)."""
    from oracle.refelem import gauss_legendre
    xq, wq = gauss_legendre(s.N + 3)
    xq = np.array([float(v) for v in xq])
    wq = np.array([float(v) for v in wq])
    V = s.ref.values_at(list(xq))                       # [nq, n] basis values
    uq = u[..., 0]
    for d in range(2):
        ax = 1 + (1 - d)
        uq = torch.movedim(torch.tensordot(uq, V, dims=([ax], [1])), -1, ax)
    Xq = synth.node_coordinates(xq, s.grid.ncell, s.grid.lo, s.grid.hi)
    err = uq.numpy() - exact_fn(Xq)
    W = np.outer(wq, wq)
    vol = s.grid.h[0] * s.grid.h[1]
    return math.sqrt(float((W[None] * err ** 2).sum()) * vol)


def test_steady_flow_over_a_bump_converges_at_order_N_plus_1():
    """b = 0.1 + 0.05 sin(2 pi x), constant discharge 0.5, depth from Bernoulli's law: an exact
    steady solution (periodic in x, invariant in y).  After t = 0.05 the depth error falls at
    order N+1 = 3."""
    N = 2
    errs = []
    for nc in (8, 16):
        s = make((nc, 1), N, (0.0, 0.0), (1.0, 1.0 / nc), "periodic")
        X = coords(s)
        b = 0.1 + 0.05 * np.sin(2 * math.pi * X[0])
        h = bernoulli_h(b)
        u = state(h, 0.5 + 0 * h, 0 * h, b)
        u, t = s.run(u, None, t_end=0.05)
        errs.append(l2_h(s, u, lambda Xq: bernoulli_h(0.1 + 0.05 * np.sin(2 * math.pi * Xq[0]))))
    rate = math.log2(errs[0] / errs[1])
    assert rate > N + 1 - 0.5, (errs, rate)


def test_radial_hump_stays_symmetric_in_x_and_y():
    """A radial hump of water on a radial bottom in a square with reflecting walls: the solution
    keeps the x <-> y mirror symmetry, h(x, y) = h(y, x), hu(x, y) = hv(y, x)."""
    s = make((6, 6), 2, (-1.0, -1.0), (1.0, 1.0), "wall")
    X = coords(s)
    r2 = X[0] ** 2 + X[1] ** 2
    b = 0.05 * r2
    u = state(1.0 - b + 0.1 * np.exp(-8 * r2), 0 * b, 0 * b, b)
    for _ in range(4):
        u = s.step(u, s.cfl_dt(u))
    uu = u.reshape(6, 6, 3, 3, 4)                       # [cy, cx, ny, nx, var]
    ut = uu.transpose(0, 1).transpose(2, 3)             # x <-> y
    assert torch.allclose(uu[..., 0], ut[..., 0], atol=1e-13)
    assert torch.allclose(uu[..., 1], ut[..., 2], atol=1e-13)
    assert float(u[..., 1].abs().max()) > 1e-4           # the hump moves
