"""Mixed-precision predictor (binary32 increments over FP64 / float-float base terms) against the
FP64 oracle and the FP64 CUDA path.  The binary32 rounding only touches the O(dt) increment, so
the per-step difference is bounded relative to the per-step CHANGE of the solution, and the
error against an exact solution must stay within 1.1x the FP64 discretisation error."""
import math

import numpy as np
import pytest
import torch

from paper_1905_07987_gb300 import synth
from cases import Case, rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _build():
    from paper_1905_07987_gb300 import build
    build.build()


def change_rel(got, ref, u0):
    """max over variables of max|got - ref| / max|ref - u0| (error relative to the step's change)."""
    nv = ref.shape[-1]
    g = got.reshape(-1, nv)
    r = ref.reshape(-1, nv)
    d = np.abs(r - u0.reshape(-1, nv)).max(axis=0)
    return float((np.abs(g - r).max(axis=0) / np.maximum(d, 1e-300)).max())


@pytest.mark.parametrize("dim,order,ncell", [(3, 4, (5, 4, 3)), (2, 3, (7, 5)), (3, 3, (3, 4, 4))])
def test_mixed_euler_step_close_to_fp64(dim, order, ncell):
    c = Case("euler", dim, order, ncell, precision="mixed")
    X = c.X
    rho = 1.0 + 0.2 * np.sin(2 * math.pi * sum(X))
    u0 = synth.euler_conserved(rho, [0.5 + 0.1 * np.cos(2 * math.pi * X[0])] + [0.3] * (dim - 1),
                               1.0 + 0.1 * rho)
    c.set(u0)
    c.ctx.step()
    dt = c.ctx.last_dt()
    ref = c.oracle_step(u0, dt)
    got = c.get()
    assert change_rel(got, ref, u0) < 2e-6
    assert rel_linf(got, ref) < 1e-9


def test_mixed_euler_wall_boundary():
    c = Case("euler", 3, 3, (4, 3, 4), lo=(-1, -1, -1), hi=(1, 1, 1), bc="wall", precision="mixed")
    r2 = sum(x * x for x in c.X)
    u0 = synth.euler_conserved(1.0 + 0.3 * np.exp(-4 * r2), [0.0] * 3, 1.0 + 0.5 * np.exp(-4 * r2))
    c.set(u0)
    c.ctx.step()
    ref = c.oracle_step(u0, c.ctx.last_dt())
    assert change_rel(c.get(), ref, u0) < 2e-6


@pytest.mark.parametrize("order", [2, 3, 5])
def test_mixed_elastic_step_with_source(order):
    ncell = (3, 3, 4)
    mat = synth.elastic_material(ncell, seed=order)
    c = Case("elastic", 3, order, ncell, hi=(1.5, 1.5, 2.0), bc="absorbing", material=mat,
             precision="mixed")
    rng = np.random.default_rng(order)
    u0 = rng.standard_normal(c.shape)
    c.point_source((0.75, 0.75, 1.0), synth.moment_tensor(seed=3), 2.0, 0.5)
    c.set(u0)
    c.ctx.set_time(0.41)
    c.ctx.step()
    ref = c.oracle_step(u0, c.ctx.last_dt(), 0.41)
    assert change_rel(c.get(), ref, u0) < 2e-6


def test_mixed_advection():
    c = Case("advection", 3, 2, (3, 3, 2), precision="mixed")
    rng = np.random.default_rng(0)
    u0 = rng.standard_normal(c.shape)
    c.set(u0)
    c.ctx.step()
    ref = c.oracle_step(u0, c.ctx.last_dt())
    assert change_rel(c.get(), ref, u0) < 2e-6


def test_mixed_error_vs_exact_within_1p1_of_fp64():
    """2-D entropy wave, order 3, 24^2 cells to t = 0.25: error of the mixed form against the exact
    solution is at most 1.1 x the FP64 form's."""
    errs = {}
    for prec in ("fp64", "mixed"):
        c = Case("euler", 2, 3, (24, 24), precision=prec)
        c.set(synth.entropy_wave(c.X))
        c.ctx.run(0, 0.0)
        n = 0
        while c.ctx.time() < 0.25 - 1e-14 and n < 10000:
            c.ctx.run(10, t_end=0.25)
            n += 10
        t = c.ctx.time()
        ex = synth.entropy_wave(c.X, t)
        errs[prec] = float(np.sqrt(np.mean((c.get()[..., 0] - ex[..., 0]) ** 2)))
    assert errs["mixed"] <= 1.1 * errs["fp64"], errs


def test_mixed_full_size_sampled_cells_euler_81():
    """The benchmark's configuration (81^3 cells, order 4, entropy wave, mixed predictor, the same
    launch shapes): sampled cells against the FP64 oracle on their 3x3x3 neighbourhood (a cell's
    update depends only on itself and its face neighbours)."""
    nc = (81, 81, 81)
    c = Case("euler", 3, 4, nc, precision="mixed")
    u0 = synth.entropy_wave(c.X)
    c.set(u0)
    c.ctx.step()
    dt = c.ctx.last_dt()
    got = c.get()
    from oracle.aderdg import ADERDG, Grid
    from oracle.pde import Euler
    sub = ADERDG(Euler(3), Grid((3, 3, 3), (0, 0, 0), (3 / 81,) * 3, [("periodic", "periodic")] * 3), 4,
                 cfl=c.cfl)
    rng = np.random.default_rng(1)
    samples = [(0, 0, 0), (80, 80, 80), (13, 52, 71)] + [tuple(rng.integers(0, 81, 3)) for _ in range(5)]
    for (i, j, k) in samples:
        idx = [((i + di) % 81) + 81 * (((j + dj) % 81) + 81 * ((k + dk) % 81))
               for dk in (-1, 0, 1) for dj in (-1, 0, 1) for di in (-1, 0, 1)]
        out = sub.step(torch.from_numpy(u0[idx]), torch.tensor(dt, dtype=torch.float64)).numpy()
        centre = i + 81 * (j + 81 * k)
        assert change_rel(got[centre], out[13], u0[centre]) < 2e-6, (i, j, k)
        assert rel_linf(got[centre], out[13]) < 1e-9, (i, j, k)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_uniform_flow_is_preserved(prec):
    """Degenerate case: a constant state with non-zero velocity is an exact solution; every flux
    derivative and increment vanishes up to rounding."""
    c = Case("euler", 3, 3, (4, 5, 3), precision=prec)
    u0 = synth.euler_conserved(np.full_like(c.X[0], 1.3), [np.full_like(c.X[0], 0.4), -0.2, 0.7],
                               np.full_like(c.X[0], 2.1))
    c.set(u0)
    for _ in range(3):
        c.ctx.step()
    assert rel_linf(c.get(), u0) < 1e-13


@pytest.mark.parametrize("case", ["entropy_wave", "explosion"])
def test_mixed_cfl_dt_equals_fp64(case):
    """The mixed form evaluates the CFL eigenvalue maximum in FP64 (its binary32 enclosures only
    decide which nodes need it), so on the same state its dt is the FP64 form's, bit for bit; the
    explosion's piecewise-constant regions make most nodes candidates of the filter."""
    dts = {}
    for prec in ("fp64", "mixed"):
        if case == "entropy_wave":
            c = Case("euler", 3, 4, (14, 13, 12), precision=prec)
            u0 = synth.entropy_wave(c.X)
        else:
            c = Case("euler", 3, 3, (17, 16, 16), lo=(-1,) * 3, hi=(1,) * 3, bc="wall",
                     precision=prec)
            u0 = synth.explosion(c.X)
        c.set(u0)
        c.ctx.step()
        dts[prec] = c.ctx.last_dt()
    assert dts["mixed"] == dts["fp64"], dts


def test_mixed_nonfinite_state_is_reported():
    """A NaN in the state reaches the filtered CFL kernel as a candidate and is latched as
    ENONFINITE, as in the FP64 form; a clean state afterwards steps normally."""
    from paper_1905_07987_gb300 import ader
    c = Case("euler", 3, 3, (4, 3, 4), precision="mixed")
    u0 = synth.entropy_wave(c.X)
    bad = u0.copy()
    bad[5, 1, 2, 0, 4] = np.nan
    c.set(bad)
    c.ctx.step()
    with pytest.raises(ader.AderError) as e:
        c.ctx.sync()
    assert e.value.status == ader.ENONFINITE
    c.set(u0)
    c.ctx.step()
    c.ctx.sync()
