"""GPU parity of the FP64 CUDA path against the CPU oracle (same seeded inputs, element by
element).  Tolerance: relative L-infinity <= 1e-12 per variable (scaled by max|u_var|)."""
import math

import numpy as np
import pytest
import torch

from paper_1905_07987_gb300 import ader, synth
from cases import Case, rel_linf

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(autouse=True, scope="module")
def _build():
    from paper_1905_07987_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def euler_data(c, kind="wave", seed=0):
    if kind == "wave":
        return synth.entropy_wave(c.X)
    rng = np.random.default_rng(seed)
    X = c.X
    D = c.dim
    bump = np.exp(-6 * sum((x - 0.5 * (lo + hi)) ** 2 for x, lo, hi in zip(X, c.lo, c.hi)))
    rho = 1.0 + 0.4 * bump + 0.02 * rng.standard_normal(X[0].shape)
    vel = [0.3 * np.sin(2 * math.pi * X[(d + 1) % D]) + 0.1 * d for d in range(D)]
    p = 1.0 + 0.5 * bump
    return synth.euler_conserved(rho, vel, p)


@pytest.mark.parametrize("dim,order,ncell", [(2, 3, (7, 5)), (2, 1, (3, 4)), (3, 4, (5, 4, 3)),
                                             (3, 2, (3, 3, 4)), (3, 3, (4, 3, 2))])
def test_euler_periodic_step(dim, order, ncell):
    c = Case("euler", dim, order, ncell)
    u0 = euler_data(c, "random", seed=order)
    c.set(u0)
    c.ctx.step()
    dt = c.ctx.last_dt()
    ref_dt = float(c.oracle.cfl_dt(torch.from_numpy(u0)))
    assert abs(dt - ref_dt) <= 1e-14 * ref_dt
    assert rel_linf(c.get(), c.oracle_step(u0, dt)) <= TOL


@pytest.mark.parametrize("bc", ["wall", "absorbing"])
def test_euler_boundaries(bc):
    c = Case("euler", 3, 3, (4, 3, 5), lo=(-1, -1, -1), hi=(1, 1, 1), bc=bc)
    u0 = euler_data(c, "random", seed=3)
    c.set(u0)
    c.ctx.step()
    dt = c.ctx.last_dt()
    assert rel_linf(c.get(), c.oracle_step(u0, dt)) <= TOL


def test_euler_2d_mixed_boundaries():
    bc = [("wall", "absorbing"), ("periodic", "periodic")]
    c = Case("euler", 2, 3, (6, 5), bc=bc)
    u0 = euler_data(c, "random", seed=5)
    c.set(u0)
    c.ctx.step()
    assert rel_linf(c.get(), c.oracle_step(u0, c.ctx.last_dt())) <= TOL


@pytest.mark.parametrize("order", range(1, 7))
def test_advection_all_orders(order):
    for dim, nc in ((2, (3, 4)), (3, (3, 2, 2))):
        c = Case("advection", dim, order, nc, bc="absorbing" if order % 2 else "periodic")
        rng = np.random.default_rng(order)
        u0 = rng.standard_normal(c.shape)
        c.set(u0)
        c.ctx.step()
        assert rel_linf(c.get(), c.oracle_step(u0, c.ctx.last_dt())) <= TOL


@pytest.mark.parametrize("order", [2, 3, 4, 5])
def test_elastic_step_with_source(order):
    ncell = (3, 4, 3)
    mat = synth.elastic_material(ncell, seed=order)
    c = Case("elastic", 3, order, ncell, hi=(1.5, 2.0, 1.5), bc="absorbing", material=mat)
    rng = np.random.default_rng(order)
    u0 = rng.standard_normal(c.shape)
    M = synth.moment_tensor(seed=7)
    c.point_source((0.75, 1.0, 0.75), M, 2.0, 0.5)
    c.set(u0)
    c.ctx.set_time(0.37)
    c.ctx.step()
    dt = c.ctx.last_dt()
    assert rel_linf(c.get(), c.oracle_step(u0, dt, 0.37)) <= TOL


def test_elastic_periodic_multistep_and_receivers():
    ncell = (4, 3, 3)
    mat = synth.elastic_material(ncell, seed=11)
    c = Case("elastic", 3, 3, ncell, hi=(2.0, 1.5, 1.5), bc="periodic", material=mat)
    u0 = synth.plane_wave_elastic(c.X, [2.7, 30.0, 25.0], L=2.0)
    pts = synth.receivers_top(ncell, c.lo, c.hi, nside=3)
    seismo = c.receivers(pts, 8)
    c.set(u0)
    u = torch.from_numpy(u0)
    t = 0.0
    rec = []
    for k in range(5):
        dt = float(c.oracle.cfl_dt(u))
        u = c.oracle.step(u, torch.tensor(dt, dtype=torch.float64), t)
        t += dt
        rec.append(c.oracle.record(u).numpy())
    c.ctx.run(5)
    assert rel_linf(c.get(), u.numpy()) <= 10 * TOL
    got = seismo[:5].cpu().numpy()
    ref = np.stack(rec)
    assert np.abs(got - ref).max() <= 10 * TOL * np.abs(ref).max()
    assert abs(c.ctx.time() - t) <= 1e-13 * t


def test_euler_free_running_matches_oracle_over_many_steps():
    c = Case("euler", 2, 3, (9, 8))
    u0 = synth.entropy_wave(c.X)
    c.set(u0)
    u, t = c.oracle.run(torch.from_numpy(u0), 20)
    c.ctx.run(20)
    assert rel_linf(c.get(), u.numpy()) <= 20 * TOL
    assert abs(c.ctx.time() - t) <= 1e-13 * t


def test_t_end_clipping_and_fixed_dt():
    c = Case("euler", 2, 2, (5, 5))
    u0 = synth.entropy_wave(c.X)
    c.set(u0)
    c.ctx.step(dt=0.004)
    assert c.ctx.last_dt() == 0.004
    assert rel_linf(c.get(), c.oracle_step(u0, 0.004)) <= TOL
    c.ctx.set_time(0.0)
    c.set(u0)
    c.ctx.run(3, t_end=0.01)
    assert abs(c.ctx.time() - 0.01) < 1e-16
    u, t = c.oracle.run(torch.from_numpy(u0), None, t_end=0.01)
    assert rel_linf(c.get(), u.numpy()) <= 10 * TOL
    # a further step at t = t_end leaves the state unchanged
    before = c.get()
    c.ctx.step(t_end=0.01)
    assert c.ctx.last_dt() == 0.0
    assert np.array_equal(c.get(), before)


def test_graph_replay_equals_step_loop():
    c1 = Case("euler", 3, 3, (4, 4, 3))
    c2 = Case("euler", 3, 3, (4, 4, 3))
    u0 = synth.entropy_wave(c1.X)
    c1.set(u0)
    c2.set(u0)
    c1.ctx.run(6)
    c2.ctx.run_graph(2, 3)
    c2.ctx.sync()
    assert np.array_equal(c1.get(), c2.get())


def test_errors_are_reported():
    c = Case("euler", 2, 2, (3, 3))
    with pytest.raises(ader.AderError) as e:
        c.ctx.step()
    assert e.value.status == ader.ESTATE
    with pytest.raises(ader.AderError):
        c.ctx.set_state(torch.zeros(5, dtype=torch.float64, device="cuda"))
    u0 = synth.entropy_wave(c.X)
    u0[4, 1, 2, 0] = np.nan
    c.set(u0)
    c.ctx.step()
    with pytest.raises(ader.AderError) as e:
        c.ctx.sync()
    assert e.value.status == ader.ENONFINITE
    c.set(synth.entropy_wave(c.X))
    c.ctx.step()
    c.ctx.sync()  # status was cleared


def test_full_size_sampled_cells_euler_81():
    """Full-size entropy wave (81^3 cells, p=4) in the launch configuration the benchmark times;
    sampled cells checked against the oracle on their 3x3x3 neighbourhood (the update of a cell
    depends only on itself and its face neighbours)."""
    nc = (81, 81, 81)
    c = Case("euler", 3, 4, nc)
    u0 = synth.entropy_wave(c.X)
    c.set(u0)
    c.ctx.step()
    dt = c.ctx.last_dt()
    got = c.get()
    from oracle.aderdg import ADERDG, Grid
    from oracle.pde import Euler
    sub = ADERDG(Euler(3), Grid((3, 3, 3), (0, 0, 0), (3 / 81,) * 3, [("periodic", "periodic")] * 3), 4,
                 cfl=c.cfl)
    rng = np.random.default_rng(0)
    samples = [(0, 0, 0), (80, 80, 80), (40, 7, 63)] + [tuple(rng.integers(0, 81, 3)) for _ in range(5)]
    for (i, j, k) in samples:
        idx = []
        for dk in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    idx.append(((i + di) % 81) + 81 * (((j + dj) % 81) + 81 * ((k + dk) % 81)))
        loc = u0[idx]
        out = sub.step(torch.from_numpy(loc), torch.tensor(dt, dtype=torch.float64)).numpy()
        centre = i + 81 * (j + 81 * k)
        assert rel_linf(got[centre], out[13]) <= TOL, (i, j, k)


@pytest.mark.parametrize("ncell,bc", [((1, 1, 1), "periodic"), ((1, 3, 2), "wall"),
                                       ((4, 1, 1), "absorbing"), ((1, 1), "periodic"),
                                       ((1, 5), "wall"), ((3, 1), [("periodic", "periodic"), ("wall", "absorbing")])])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grids_one_cell_thick(ncell, bc, prec):
    """Degenerate grids one cell thick in some direction: a periodic cell is its own face
    neighbour (both faces of the line are the same face), a wall cell has walls on both sides.
    One Euler step against the oracle (FP64 1e-12; mixed within 2e-6 of the step's change)."""
    dim = len(ncell)
    c = Case("euler", dim, 3, ncell, lo=(-1.0,) * dim, hi=(1.0,) * dim, bc=bc, precision=prec)
    u0 = synth.entropy_wave(c.X)
    c.set(u0)
    c.ctx.step()
    dt = c.ctx.last_dt()
    ref = c.oracle_step(u0, dt)
    if prec == "fp64":
        assert rel_linf(c.get(), ref) <= TOL
    else:
        assert np.abs(c.get() - ref).max() <= 2e-6 * np.abs(ref - u0).max()


@pytest.mark.parametrize("ncell", [(1, 1, 1), (1, 2, 3), (3, 1, 1)])
def test_elastic_ck_on_grids_one_cell_thick(ncell):
    """The Cauchy-Kowalevski elastic step (absorbing boundaries) on grids one cell thick."""
    mat = synth.elastic_material(ncell, seed=7)
    c = Case("elastic", 3, 3, ncell, lo=(0.0,) * 3, hi=tuple(0.5 * n for n in ncell), bc="absorbing",
             material=mat, predictor="ck")
    m, L = (2.7, 30.0, 25.0), 0.5 * max(ncell)
    # four superposed plane waves: all nine components vary (none is zero up to round-off)
    u0 = (synth.plane_wave_elastic(c.X, m, kind='p', L=L)
          + synth.plane_wave_elastic(c.X, m, kind='s', L=L / 2)
          + synth.plane_wave_elastic(c.X, m, kind='s', direction=(0.0, 1.0, 0.0), L=L / 3)
          + synth.plane_wave_elastic(c.X, m, kind='s', direction=(0.0, 0.0, 1.0), L=L / 2))
    c.set(u0)
    c.ctx.step()
    dt = c.ctx.last_dt()
    assert rel_linf(c.get(), c.oracle_step(u0, dt)) <= TOL


def test_configurations_beyond_the_kernels_are_rejected_at_create():
    """The 3-D Euler mixed predictor at order 6 needs more shared memory than a block has: the
    context is refused up front instead of failing at the first step."""
    cfg = ader.make_config("euler", 3, 6, (2, 2, 2), (0,) * 3, (1,) * 3, "periodic",
                           synth.cfl_number(6), precision="mixed")
    with pytest.raises(ader.AderError) as e:
        ader.Context(cfg)
    assert e.value.status == ader.EUNSUPPORTED
    cfg = ader.make_config("euler", 3, 6, (2, 2, 2), (0,) * 3, (1,) * 3, "periodic",
                           synth.cfl_number(6), precision="fp64")
    ader.Context(cfg)  # the FP64 kernel fits


@pytest.mark.parametrize("state", ["entropy_wave", "explosion", "uniform", "spike"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cfl_dt_matches_the_oracle(state, prec):
    """On grids of 2^18 nodes and more the CFL kernel evaluates speeds in FP64 only where binary32
    enclosures cannot rule a node out; its dt must equal the oracle's FP64 maximum over every node
    (to FP64 rounding of the speed formula): smooth data, piecewise-constant data, a uniform state
    where every node ties, and a single node far faster than the rest (17 x 16 x 16 cells of
    order 3: 278 528 nodes)."""
    c = Case("euler", 3, 3, (17, 16, 16), lo=(-1,) * 3, hi=(1,) * 3, bc="wall", precision=prec)
    if state == "entropy_wave":
        u0 = synth.entropy_wave(c.X)
    elif state == "explosion":
        u0 = synth.explosion(c.X)
    else:
        u0 = synth.euler_conserved(np.full_like(c.X[0], 1.1), [np.full_like(c.X[0], 0.3), 0.2, -0.1],
                                   np.full_like(c.X[0], 0.9))
        if state == "spike":
            u0 = u0.copy()
            u0[2377, 2, 1, 3] = synth.euler_conserved(np.array(0.9), [np.array(4.0), 0.0, 0.0],
                                                    np.array(3.0))
    c.set(u0)
    c.ctx.step()
    dt = c.ctx.last_dt()
    ref = float(c.oracle.cfl_dt(torch.from_numpy(u0)))
    assert abs(dt - ref) <= 2e-15 * ref, (dt, ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_host_batch_equals_the_step_loop(precision):
    """ader_step_host_batch (host states in and out, copies overlapped on copy streams) gives, for
    every state, the bits of set_state / step / get_state from the same time; the context ends
    with the last result."""
    c = Case("euler", 3, 3, (6, 5, 4), precision=precision)
    x, _ = ader.reference_nodes(3)
    base = synth.entropy_wave(c.X)
    rng = np.random.default_rng(5)
    ins = [torch.from_numpy((base * (1.0 + 0.01 * k) + 0.001 * rng.standard_normal(c.shape))
                            .reshape(-1).copy()).pin_memory() for k in range(4)]
    outs = [torch.empty(c.ctx.count, dtype=torch.float64).pin_memory() for _ in ins]
    c.ctx.set_time(0.25)
    c.ctx.step_host_batch(ins, outs)
    last = torch.empty(c.ctx.count, dtype=torch.float64, device="cuda")
    c.ctx.get_state(last)
    for k, u in enumerate(ins):
        c.ctx.set_state(u.cuda())
        c.ctx.set_time(0.25)
        c.ctx.step()
        ref = torch.empty(c.ctx.count, dtype=torch.float64, device="cuda")
        c.ctx.get_state(ref)
        torch.cuda.synchronize()
        assert torch.equal(outs[k], ref.cpu()), k
    assert torch.equal(last.cpu(), outs[-1])
