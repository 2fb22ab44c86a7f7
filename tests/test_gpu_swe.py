"""GPU parity of the shallow water equations with bathymetry (Eq. (9), Sec. 2) against the
oracle, through the C ABI: the state-dependent non-conservative product g h d(h + b)/dx_d node by
node in the predictor and its time average, the path-conservative Rusanov fluctuation at faces,
walls and periodic boundaries; the lake at rest to round-off."""

import numpy as np
import pytest
import torch

from cases import Case, rel_linf
from paper_1905_07987_gb300 import ader, synth

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(autouse=True, scope="module")
def _build():
    from paper_1905_07987_gb300 import build
    build.build()


# smooth periodic bathymetry with a moving, perturbed surface: every term of the system is active
# (non-zero flux, momentum in both directions, non-zero d(h + b)/dx)
flow_over_bump = synth.swe_flow_over_bump


@pytest.mark.parametrize("order,ncell", [(1, (7, 5)), (2, (6, 5)), (3, (5, 4)), (4, (4, 4)), (5, (3, 4))])
def test_swe_periodic_step(order, ncell):
    c = Case("swe", 2, order, ncell, bc="periodic")
    u0 = flow_over_bump(c.X)
    c.set(u0)
    c.ctx.step()
    dt = c.ctx.last_dt()
    assert rel_linf(c.get(), c.oracle_step(u0, dt)) <= TOL


@pytest.mark.parametrize("bc", ["wall", "absorbing"])
def test_swe_boundaries(bc):
    c = Case("swe", 2, 3, (6, 5), lo=(-1.0, -1.0), hi=(1.0, 1.0), bc=bc)
    x, y = c.X
    b = 0.1 * np.exp(-4 * ((x - 0.2) ** 2 + y ** 2))
    h = 1.0 - b + 0.05 * np.exp(-8 * ((x + 0.3) ** 2 + (y - 0.1) ** 2))
    u0 = np.stack([h, 0.1 * h, -0.05 * h, b], axis=-1)
    c.set(u0)
    c.ctx.step()
    dt = c.ctx.last_dt()
    assert rel_linf(c.get(), c.oracle_step(u0, dt)) <= TOL


def test_swe_free_run_matches_the_oracle():
    c = Case("swe", 2, 3, (8, 6), bc="periodic")
    u0 = flow_over_bump(c.X)
    c.set(u0)
    u = torch.from_numpy(u0)
    for _ in range(10):
        u = c.oracle.step(u, c.oracle.cfl_dt(u))
    c.ctx.run(10)
    assert rel_linf(c.get(), u.numpy()) <= 1e-11


def test_swe_lake_at_rest_is_preserved_to_round_off():
    """b = (x^2 + y^2)/10, h = 1 - b, no flow, walls: the free surface stays flat, the flow stays
    zero and the mass is conserved, to round-off, over 20 steps on the GPU."""
    c = Case("swe", 2, 2, (10, 8), lo=(-1.0, -1.0), hi=(1.0, 1.0), bc="wall")
    x, y = c.X
    b = 0.1 * (x ** 2 + y ** 2)
    u0 = np.stack([1.0 - b, 0 * b, 0 * b, b], axis=-1)
    c.set(u0)
    c.ctx.run(20)
    got = c.get()
    assert np.abs(got - u0).max() < 1e-13
    W = c.oracle.tensor_basis_weights().numpy()
    assert abs((got[..., 0] * W).sum() - (u0[..., 0] * W).sum()) < 1e-13 * (u0[..., 0] * W).sum()


def test_swe_options_beyond_the_kernels_are_rejected():
    for kw in (dict(precision="mixed"), dict(initial_guess="cerk"), dict(limiter=1)):
        cfg = ader.make_config("swe", 2, 3, (4, 4), (0, 0), (1, 1), "periodic", synth.cfl_number(3), **kw)
        with pytest.raises(ader.AderError) as e:
            ader.Context(cfg)
        assert e.value.status == ader.EUNSUPPORTED, kw


def test_swe_depth_loss_is_reported():
    """Shallow water has no limiter: a state whose depth reaches zero or below gives a non-finite
    wave speed sqrt(g h), latched by the CFL reduction as ADER_ENONFINITE; a wet state afterwards
    steps normally."""
    c = Case("swe", 2, 3, (6, 5), bc="periodic")
    u0 = flow_over_bump(c.X)
    for h in (0.0, -0.01):
        bad = u0.copy()
        bad[7, 1, 2, 0] = h
        c.set(bad)
        c.ctx.step()
        with pytest.raises(ader.AderError) as e:
            c.ctx.sync()
        assert e.value.status == ader.ENONFINITE, h
    c.set(u0)
    c.ctx.step()
    c.ctx.sync()
