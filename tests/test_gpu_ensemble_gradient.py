"""Batched adjoint of an ensemble of uneven elastic runs (ader_ensemble_misfit_gradient), with the
Picard and with the Cauchy-Kowalevski predictor: every run's misfit and gradient equal the
single-context checkpointed gradient of the same run, in any grouping of the runs, and match
central finite differences; the mixed-precision forward sweep gives the FP64 gradient up to the
mixed form's forward error.  The source sits three cells below
the top face so that the receivers record signal within the few steps of the test."""
import numpy as np
import pytest
import torch

from paper_1905_07987_gb300 import ader, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _build():
    from paper_1905_07987_gb300 import build
    build.build()


def cfg(side, order, precision="fp64", predictor="picard"):
    return ader.make_config("elastic", 3, order, (side,) * 3, (0, 0, 0), (0.5 * side,) * 3, "absorbing",
                            synth.cfl_number(order), precision=precision, predictor=predictor)


def setup(ctx, side, seed, steps):
    L = 0.5 * side
    ctx.set_material(torch.from_numpy(synth.elastic_material((side,) * 3, seed=seed).reshape(-1).copy()).cuda())
    # source three cells below the centre of the top face
    ctx.set_point_source((0.5 * L, 0.5 * L, L - 3 * 0.5 + 0.25), synth.moment_tensor(seed=seed), 2.0, 0.5)
    seismo = torch.zeros(steps + 2, 16, 3, dtype=torch.float64, device="cuda")
    ctx.set_receivers(synth.receivers_top((side,) * 3, (0, 0, 0), (L,) * 3, nside=4), seismo, steps + 2)
    return seismo


def problem(sides, order, steps, precision="fp64", predictor="picard"):
    ens = ader.Ensemble([cfg(s, order, precision, predictor) for s in sides])
    keep = [setup(ens.runs[i], s, 10 + i, steps) for i, s in enumerate(sides)]
    u0 = [torch.zeros(r.count, dtype=torch.float64, device="cuda") for r in ens.runs]
    rng = np.random.default_rng(5)
    obs = [torch.from_numpy(1e-4 * rng.standard_normal(steps * 16 * 3)).cuda() for _ in sides]
    return ens, keep, u0, obs


def grads(ens):
    gm = [torch.zeros(r.cells * 3, dtype=torch.float64, device="cuda") for r in ens.runs]
    gM = [torch.zeros(6, dtype=torch.float64, device="cuda") for r in ens.runs]
    return gm, gM


PREDICTORS = pytest.mark.parametrize("predictor", ["picard", "ck"])


@PREDICTORS
def test_batched_gradient_equals_single_context_gradients(predictor):
    sides, order, steps, k, dt = [4, 3, 5], 3, 7, 3, 4e-3
    ens, keep, u0, obs = problem(sides, order, steps, predictor=predictor)
    gm, gM = grads(ens)
    J = ens.misfit_gradient(u0, 0.45, dt, steps, k, obs, gm, gM)
    # each run alone through the single-context entry point
    for i, s in enumerate(sides):
        c = ader.Context(cfg(s, order, predictor=predictor))
        kk = setup(c, s, 10 + i, steps)
        g1 = torch.zeros(c.cells * 3, dtype=torch.float64, device="cuda")
        M1 = torch.zeros(6, dtype=torch.float64, device="cuda")
        J1 = c.misfit_gradient(u0[i], 0.45, dt, steps, k, obs[i], g1, M1)
        assert J1 > 0
        assert J[i] == J1, (i, J[i], J1)
        assert torch.equal(gm[i], g1) and torch.equal(gM[i], M1), i
        c.close()
        del kk
    # any grouping: one run per group (a budget of one byte)
    gm2, gM2 = grads(ens)
    J2 = ens.misfit_gradient(u0, 0.45, dt, steps, k, obs, gm2, gM2, mem_budget=1)
    assert J2 == J
    for a, b in zip(gm + gM, gm2 + gM2):
        assert torch.equal(a, b)
    ens.close()


@PREDICTORS
def test_batched_gradient_matches_central_differences(predictor):
    sides, order, steps, k, dt = [3, 4], 2, 6, 2, 4e-3
    ens, keep, u0, obs = problem(sides, order, steps, predictor=predictor)
    gm, gM = grads(ens)
    J = ens.misfit_gradient(u0, 0.45, dt, steps, k, obs, gm, gM)
    i = 1
    side = sides[i]
    mat = synth.elastic_material((side,) * 3, seed=10 + i)
    rng = np.random.default_rng(7)
    dirn = rng.standard_normal(mat.shape) * mat
    eps = 1e-6
    Js = []
    for sgn in (1, -1):
        ens.runs[i].set_material(torch.from_numpy((mat + sgn * eps * dirn).reshape(-1).copy()).cuda())
        Js.append(ens.misfit_gradient(u0, 0.45, dt, steps, k, obs)[i])
    ens.runs[i].set_material(torch.from_numpy(mat.reshape(-1).copy()).cuda())
    fd = (Js[0] - Js[1]) / (2 * eps)
    ad = float((gm[i].cpu().numpy().reshape(-1, 3) * dirn).sum())
    assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
    ens.close()


@PREDICTORS
def test_mixed_forward_gradient_is_close_to_fp64(predictor):
    """The mixed-precision forward sweep (the batched-adjoint workload's form) with the FP64
    adjoint: the gradient differs from the all-FP64 one by the mixed form's forward error only."""
    sides, order, steps, k, dt = [4, 5], 4, 6, 3, 3e-3
    out = {}
    for prec in ("fp64", "mixed"):
        ens, keep, u0, obs = problem(sides, order, steps, precision=prec, predictor=predictor)
        gm, gM = grads(ens)
        J = ens.misfit_gradient(u0, 0.45, dt, steps, k, obs, gm, gM)
        out[prec] = (J, [g.cpu().numpy() for g in gm], [g.cpu().numpy() for g in gM])
        ens.close()
    for i in range(len(sides)):
        assert abs(out["mixed"][0][i] - out["fp64"][0][i]) <= 1e-6 * abs(out["fp64"][0][i])
        a, b = out["mixed"][1][i], out["fp64"][1][i]
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()
