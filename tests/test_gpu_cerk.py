"""GPU parity of the continuous extension Runge-Kutta initial guess of the Picard predictor
(Sec. 5) against the oracle's, through the C ABI: the FP64 form at 1e-12, the mixed form within
2e-6 of the step's change and within 1.1x the FP64 error against the exact solution."""
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


def change_rel(got, ref, u0):
    """max over variables of max|got - ref| / max|ref - u0| (error relative to the step's change)."""
    nv = ref.shape[-1]
    g, r = got.reshape(-1, nv), ref.reshape(-1, nv)
    d = np.abs(r - u0.reshape(-1, nv)).max(axis=0)
    return float((np.abs(g - r).max(axis=0) / np.maximum(d, 1e-300)).max())


@pytest.mark.parametrize("dim,order,ncell,iters",
                         [(3, 4, (5, 4, 3), 1), (2, 3, (7, 5), 1), (3, 3, (3, 4, 4), 2), (2, 5, (4, 3), 2)])
def test_mixed_cerk_euler_step(dim, order, ncell, iters):
    """Mixed predictor (binary32 stages and iterations on the increment) from the continuous
    extension Runge-Kutta guess: the step against the oracle's FP64 step with the same guess and
    iteration count, within 2e-6 of the step's change."""
    c = Case("euler", dim, order, ncell, picard_iters=iters, initial_guess="cerk", precision="mixed")
    u0 = synth.entropy_wave(c.X)
    c.set(u0)
    c.ctx.step()
    dt = c.ctx.last_dt()
    assert change_rel(c.get(), c.oracle_step(u0, dt), u0) < 2e-6


@pytest.mark.parametrize("order,iters", [(3, 1), (4, 2)])
def test_mixed_cerk_elastic_step_with_source(order, iters):
    ncell = (3, 4, 3)
    mat = synth.elastic_material(ncell, seed=order)
    c = Case("elastic", 3, order, ncell, hi=(1.5, 2.0, 1.5), bc="absorbing", material=mat,
             picard_iters=iters, initial_guess="cerk", precision="mixed")
    rng = np.random.default_rng(order)
    u0 = rng.standard_normal(c.shape)
    c.point_source((0.75, 1.0, 0.75), synth.moment_tensor(seed=7), 2.0, 0.5)
    c.set(u0)
    c.ctx.set_time(0.37)
    c.ctx.step()
    dt = c.ctx.last_dt()
    assert change_rel(c.get(), c.oracle_step(u0, dt, 0.37), u0) < 2e-6


def test_mixed_cerk_error_vs_exact_within_1p1_of_fp64():
    """3-D entropy wave, order 4 (the benchmark's scheme), 12^3 cells, 20 CFL steps: the mixed form
    with the CERK guess and one iteration has at most 1.1x the error of the FP64 form with the
    constant guess and N+1 iterations against the exact solution."""
    errs = {}
    for name, prec, guess, iters in (("fp64", "fp64", "constant", 0), ("mixed_cerk", "mixed", "cerk", 1)):
        c = Case("euler", 3, 4, (12, 12, 12), precision=prec, initial_guess=guess, picard_iters=iters)
        c.set(synth.entropy_wave(c.X))
        c.ctx.run(20)
        ex = synth.entropy_wave(c.X, c.ctx.time())
        errs[name] = float(np.sqrt(np.mean((c.get()[..., 0] - ex[..., 0]) ** 2)))
    assert errs["mixed_cerk"] <= 1.1 * errs["fp64"], errs


def test_mixed_cerk_full_size_sampled_cells_euler_81():
    """81^3 cells, order 4, mixed predictor from the CERK guess with one iteration (the
    benchmark's launch shape): sampled cells against the oracle's CERK step on their 3x3x3
    neighbourhood."""
    nc = (81, 81, 81)
    c = Case("euler", 3, 4, nc, precision="mixed", initial_guess="cerk", picard_iters=1)
    u0 = synth.entropy_wave(c.X)
    c.set(u0)
    c.ctx.step()
    dt = c.ctx.last_dt()
    got = c.get()
    from oracle.aderdg import ADERDG, Grid
    from oracle.pde import Euler
    sub = ADERDG(Euler(3), Grid((3, 3, 3), (0, 0, 0), (3 / 81,) * 3, [("periodic", "periodic")] * 3), 4,
                 cfl=c.cfl, picard_iters=1, initial_guess="cerk")
    rng = np.random.default_rng(5)
    samples = [(0, 0, 0), (80, 80, 80)] + [tuple(rng.integers(0, 81, 3)) for _ in range(4)]
    for (i, j, k) in samples:
        idx = [((i + di) % 81) + 81 * (((j + dj) % 81) + 81 * ((k + dk) % 81))
               for dk in (-1, 0, 1) for dj in (-1, 0, 1) for di in (-1, 0, 1)]
        out = sub.step(torch.from_numpy(u0[idx]), torch.tensor(dt, dtype=torch.float64)).numpy()
        centre = i + 81 * (j + 81 * k)
        assert change_rel(got[centre], out[13], u0[centre]) < 2e-6, (i, j, k)


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
