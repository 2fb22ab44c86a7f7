"""Ensembles of uneven elastic grids advanced by one CUDA graph: identical to stepping every run
on its own, for every launch shape the autotuner may choose, and each run against the oracle."""
import numpy as np
import pytest
import torch

from paper_1905_07987_gb300 import ader, synth
from cases import rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _build():
    from paper_1905_07987_gb300 import build
    build.build()


def member_configs(sides, order, precision="fp64", predictor="picard"):
    cfgs = []
    for s in sides:
        cfgs.append(ader.make_config("elastic", 3, order, (s, s, s), (0, 0, 0), (0.5 * s,) * 3,
                                     "absorbing", synth.cfl_number(order), precision=precision,
                                     predictor=predictor))
    return cfgs


def setup_member(ctx, side, order, seed):
    x, _ = ader.reference_nodes(order)
    X = synth.node_coordinates(x, (side,) * 3, (0, 0, 0), (0.5 * side,) * 3)
    mat = synth.elastic_material((side,) * 3, seed=seed)
    ctx.set_material(torch.from_numpy(mat.reshape(-1).copy()).cuda())
    c = 0.25 * side
    bump = np.exp(-4 * ((X[0] - c) ** 2 + (X[1] - c) ** 2 + (X[2] - c) ** 2))
    u0 = np.stack([bump, 0 * bump, -bump] + [0.1 * bump] * 6, -1)
    ctx.set_state(torch.from_numpy(u0.reshape(-1).copy()).cuda())
    ctx.set_point_source((0.2 * side, 0.3 * side, 0.25 * side), synth.moment_tensor(seed=seed), 2.0, 0.5)
    return u0, mat


def states(ctxs):
    out = []
    for c in ctxs:
        t = torch.empty(c.count, dtype=torch.float64, device="cuda")
        c.get_state(t)
        out.append(t)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in out]


@pytest.mark.parametrize("branches,spg,bps,prec", [(1, 2, 1, "fp64"), (2, 4, 1, "fp64"),
                                                   (3, 2, 1, "fp64"), (0, 2, 1, "fp64"),
                                                   (0, 4, 2, "fp64"), (0, 2, 1, "mixed"),
                                                   (0, 4, 3, "mixed"), (-1, 2, 1, "fp64"),
                                                   (-1, 4, 2, "fp64"), (-1, 2, 1, "mixed"),
                                                   (-1, 4, 2, "mixed")])
def test_ensemble_graph_equals_separate_runs(branches, spg, bps, prec):
    """Every launch shape, including the persistent launches shared by all runs (branches 0: one
    per phase; -1: one cooperative launch for all steps of a graph, grid-wide barriers between the
    phases), gives each run exactly the result of stepping it on its own."""
    sides, order = [3, 5, 4, 2], 2
    ens = ader.Ensemble(member_configs(sides, order, precision=prec))
    singles = [ader.Context(c) for c in member_configs(sides, order, precision=prec)]
    for i, s in enumerate(sides):
        setup_member(ens.runs[i], s, order, seed=i)
        setup_member(singles[i], s, order, seed=i)
    ens.set_launch(branches, spg, bps)
    dt = 1e-3
    ens.step(7, dt=dt)
    ens.sync()
    for c in singles:
        c.run(7, dt=dt)
    for a, b in zip(states(ens.runs), states(singles)):
        assert np.array_equal(a, b)
    ens.close()


@pytest.mark.parametrize("sides,order,launch", [([2, 3], 3, None), ([8, 10, 9], 3, None),
                                                ([8, 10, 9], 3, (0, 2, 2)), ([12, 8], 4, (0, 2, 1)),
                                                ([12, 8, 10], 4, (-1, 2, 1))])
def test_ensemble_members_match_the_oracle(sides, order, launch):
    """Each run of the ensemble against the oracle run on its own grid: the per-run kernels and
    the persistent launches shared by all runs (many blocks per run at sides 8..12)."""
    from oracle.aderdg import ADERDG, Grid, PointSource
    from oracle.pde import Elastic
    ens = ader.Ensemble(member_configs(sides, order))
    dt = None  # CFL steps per run (the per-run kernels); the persistent launches need a fixed dt
    if launch is not None:
        ens.set_launch(*launch)
        dt = 1e-3
    refs = []
    for i, s in enumerate(sides):
        u0, mat = setup_member(ens.runs[i], s, order, seed=10 + i)
        g = Grid((s,) * 3, (0, 0, 0), (0.5 * s,) * 3, [("absorbing", "absorbing")] * 3)
        o = ADERDG(Elastic(), g, order, cfl=synth.cfl_number(order), material=torch.from_numpy(mat))
        cell, xi = synth.locate((0.2 * s, 0.3 * s, 0.25 * s), (s,) * 3, (0, 0, 0), (0.5 * s,) * 3)
        o.set_point_source(PointSource(cell, xi, torch.from_numpy(synth.moment_tensor(seed=10 + i)), 2.0, 0.5))
        u, t = o.run(torch.from_numpy(u0), 4, dt=dt)
        refs.append(u.numpy())
    ens.step(4, dt=dt or 0.0)
    ens.sync()
    for a, r in zip(states(ens.runs), refs):
        assert rel_linf(a.reshape(r.shape), r) <= 1e-11
    ens.close()


def test_autotune_keeps_results_and_picks_a_valid_shape():
    sides, order = [4, 3, 5], 2
    ens = ader.Ensemble(member_configs(sides, order, precision="mixed"))
    for i, s in enumerate(sides):
        setup_member(ens.runs[i], s, order, seed=i)
    before = states(ens.runs)
    b, spg, bps, ms = ens.autotune(1e-3)
    assert b in (0, 1, 2, 4) and spg in (2, 4) and ms > 0
    assert (bps in (1, 2)) if b == 0 else bps == 0
    after = states(ens.runs)
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    ens.step(6, dt=1e-3)
    ens.sync()
    ens.close()


def test_persistent_launch_falls_back_when_the_runs_differ():
    """Runs with different cell sizes cannot share the persistent launches' tables: the step falls
    back to per-run kernels and still matches separate runs."""
    sides, order = [3, 4], 2
    cfgs = member_configs(sides, order)
    cfgs[1] = ader.make_config("elastic", 3, order, (4, 4, 4), (0, 0, 0), (3.0,) * 3, "absorbing",
                               synth.cfl_number(order))
    ens = ader.Ensemble(cfgs)
    singles = [ader.Context(c) for c in cfgs]
    for i, s in enumerate(sides):
        setup_member(ens.runs[i], s, order, seed=i)
        setup_member(singles[i], s, order, seed=i)
    ens.set_launch(0, 2, 1)
    ens.step(4, dt=1e-3)
    ens.sync()
    for c in singles:
        c.run(4, dt=1e-3)
    for a, b in zip(states(ens.runs), states(singles)):
        assert np.array_equal(a, b)
    ens.close()


def test_persistent_launch_order_four_mixed_uneven_sizes():
    """The benchmark's kind of ensemble (order 4, mixed predictor, uneven cube sides) on the
    persistent launches equals separate runs."""
    sides, order = [6, 3, 5, 2, 4], 4
    ens = ader.Ensemble(member_configs(sides, order, precision="mixed"))
    singles = [ader.Context(c) for c in member_configs(sides, order, precision="mixed")]
    for i, s in enumerate(sides):
        setup_member(ens.runs[i], s, order, seed=30 + i)
        setup_member(singles[i], s, order, seed=30 + i)
    ens.set_launch(0, 2, 2)
    ens.step(5, dt=1e-3)
    ens.sync()
    for c in singles:
        c.run(5, dt=1e-3)
    for a, b in zip(states(ens.runs), states(singles)):
        assert np.array_equal(a, b)
    ens.close()


def test_fused_launch_barrier_timeout_is_reported_and_recoverable():
    """The fused launch's grid-wide barrier waits are bounded: with the limit at 0 polls a wait
    runs out, every run's status latches ADER_ETIMEOUT and ader_ensemble_sync returns it (no hang,
    no fault); with the limit restored the ensemble steps correctly again."""
    sides, order = [4, 5, 3], 2
    ens = ader.Ensemble(member_configs(sides, order))
    singles = [ader.Context(c) for c in member_configs(sides, order)]
    for i, s in enumerate(sides):
        setup_member(ens.runs[i], s, order, seed=50 + i)
        setup_member(singles[i], s, order, seed=50 + i)
    ens.set_launch(-1, 2, 1)
    ens.set_wait_limit(0)
    ens.step(2, dt=1e-3)
    with pytest.raises(ader.AderError) as e:
        ens.sync()
    assert e.value.status == ader.ETIMEOUT
    ens.set_wait_limit(1 << 24)
    for i, s in enumerate(sides):  # the timed-out launch left the states undefined: set again
        setup_member(ens.runs[i], s, order, seed=50 + i)
        ens.runs[i].set_time(0.0)
    ens.step(4, dt=1e-3)
    ens.sync()
    for c in singles:
        c.run(4, dt=1e-3)
    for a, b in zip(states(ens.runs), states(singles)):
        assert np.array_equal(a, b)
    ens.close()


@pytest.mark.parametrize("order,prec,launch", [(4, "fp64", (0, 2, 1)), (4, "mixed", (0, 2, 1)),
                                               (5, "mixed", (0, 4, 1)), (4, "mixed", (2, 2, 1))])
def test_ck_ensemble_equals_separate_runs(order, prec, launch):
    """Runs with the Cauchy-Kowalevski predictor: the persistent launch over all runs' cells
    (branches 0, orders 4 and 5) and the per-run branches give each run exactly the result of
    stepping it on its own."""
    sides = [3, 5, 4, 2]
    ens = ader.Ensemble(member_configs(sides, order, precision=prec, predictor="ck"))
    singles = [ader.Context(c) for c in member_configs(sides, order, precision=prec, predictor="ck")]
    for i, s in enumerate(sides):
        setup_member(ens.runs[i], s, order, seed=i)
        setup_member(singles[i], s, order, seed=i)
    ens.set_launch(*launch)
    ens.step(5, dt=1e-3)
    ens.sync()
    for c in singles:
        c.run(5, dt=1e-3)
    for a, b in zip(states(ens.runs), states(singles)):
        assert np.array_equal(a, b)
    ens.close()
