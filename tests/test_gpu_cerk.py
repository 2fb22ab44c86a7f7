"""GPU parity of the continuous extension Runge-Kutta initial guess of the FP64 Picard predictor
(Sec. 5) against the oracle's, through the C ABI."""
import numpy as np
import pytest
import torch

from cases import Case, rel_linf
from paper_1905_07987_gb300 import ader, synth

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.mark.parametrize("dim,order,ncell,iters",
                         [(3, 4, (5, 4, 3), 1), (2, 3, (7, 5), 1), (3, 2, (3, 3, 3), 2), (2, 5, (4, 3), 3)])
def test_cerk_euler_step(dim, order, ncell, iters):
    c = Case("euler", dim, order, ncell, picard_iters=iters, initial_guess="cerk")
    u0 = synth.entropy_wave(c.X)
    c.set(u0)
    c.ctx.step()
    dt = c.ctx.last_dt()
    assert rel_linf(c.get(), c.oracle_step(u0, dt)) <= TOL


@pytest.mark.parametrize("order,iters", [(3, 1), (5, 2)])
def test_cerk_elastic_step_with_source(order, iters):
    ncell = (3, 4, 3)
    mat = synth.elastic_material(ncell, seed=order)
    c = Case("elastic", 3, order, ncell, hi=(1.5, 2.0, 1.5), bc="absorbing", material=mat,
             picard_iters=iters, initial_guess="cerk")
    rng = np.random.default_rng(order)
    u0 = rng.standard_normal(c.shape)
    c.point_source((0.75, 1.0, 0.75), synth.moment_tensor(seed=7), 2.0, 0.5)
    c.set(u0)
    c.ctx.set_time(0.37)
    c.ctx.step()
    dt = c.ctx.last_dt()
    assert rel_linf(c.get(), c.oracle_step(u0, dt, 0.37)) <= TOL


def test_cerk_advection_multistep():
    c = Case("advection", 3, 3, (4, 3, 3), picard_iters=1, initial_guess="cerk")
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal(c.shape)
    c.set(u0)
    u = torch.from_numpy(u0)
    t = 0.0
    for _ in range(4):
        dt = float(c.oracle.cfl_dt(u))
        u = c.oracle.step(u, torch.tensor(dt, dtype=torch.float64), t)
        t += dt
    c.ctx.run(4)
    assert rel_linf(c.get(), u.numpy()) <= 10 * TOL


def test_cerk_is_rejected_where_it_is_not_built():
    cfg = ader.make_config("elastic", 3, 3, (2, 2, 2), (0,) * 3, (1,) * 3, "absorbing",
                           synth.cfl_number(3), initial_guess="cerk")
    c = ader.Context(cfg)
    c.set_material(torch.from_numpy(synth.elastic_material((2, 2, 2), seed=1).reshape(-1).copy()).cuda())
    u = torch.zeros(c.count, dtype=torch.float64, device="cuda")
    lam = torch.zeros_like(u)
    gm = torch.zeros(8 * 3, dtype=torch.float64, device="cuda")
    gM = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(ader.AderError) as e:  # the adjoint differentiates the constant-guess step
        c.adjoint_step(0.0, 1e-3, u, lam, gm, gM)
    assert e.value.status == ader.EUNSUPPORTED
    c.close()
