"""Gradient of the receiver misfit through the checkpointed adjoint sweep of the library (Picard
and Cauchy-Kowalevski predictors): against the oracle's adjoint sweep, against central finite
differences of the GPU forward solver (relative <= 1e-6), and through torch.autograd."""
import numpy as np
import pytest
import torch

from oracle.adjoint import misfit
from oracle.aderdg import PointSource
from paper_1905_07987_gb300 import synth
from paper_1905_07987_gb300.autograd import receiver_misfit
from cases import Case

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _build():
    from paper_1905_07987_gb300 import build
    build.build()


def problem(order=2, ncell=(3, 2, 3), steps=9, k=4, bc="absorbing", predictor="picard",
            precision="fp64"):
    mat = synth.elastic_material(ncell, seed=7)
    hi = tuple(0.5 * n for n in ncell)
    c = Case("elastic", 3, order, ncell, hi=hi, bc=bc, material=mat, predictor=predictor,
             precision=precision)
    x0 = (0.41 * hi[0], 0.52 * hi[1], 0.47 * hi[2])
    M = synth.moment_tensor(seed=4)
    c.point_source(x0, M, 2.0, 0.5)
    c.ctx.src_x0, c.ctx.src_f0, c.ctx.src_t0 = x0, 2.0, 0.5
    pts = np.array([[0.3 * hi[0], 0.6 * hi[1], hi[2]], [0.8 * hi[0], 0.25 * hi[1], hi[2]],
                    [0.55 * hi[0], 0.5 * hi[1], hi[2]]])
    c.receivers(pts, steps + 2)
    u0 = np.zeros(c.shape)
    dt = 0.8 * float(c.oracle.cfl_dt(torch.ones(c.shape, dtype=torch.float64)))
    obs = 1e-3 * np.random.default_rng(1).standard_normal((steps, len(pts), 3))
    return c, mat, M, u0, dt, steps, k, obs


def gpu_J(c, mat, M, u0, dt, steps, k, obs, grads=False):
    c.ctx.set_material(torch.from_numpy(mat.reshape(-1).copy()).cuda())
    c.ctx.set_point_source(c.ctx.src_x0, M, 2.0, 0.5)
    gm = torch.zeros(c.ctx.cells * 3, dtype=torch.float64, device="cuda") if grads else None
    gM = torch.zeros(6, dtype=torch.float64, device="cuda") if grads else None
    J = c.ctx.misfit_gradient(torch.from_numpy(u0.reshape(-1).copy()).cuda(), 0.5, dt, steps, k,
                              torch.from_numpy(obs.reshape(-1).copy()).cuda(), gm, gM)
    if grads:
        return J, gm.cpu().numpy().reshape(-1, 3), gM.cpu().numpy()
    return J


PREDICTORS = pytest.mark.parametrize("predictor", ["picard", "ck"])


@PREDICTORS
def test_misfit_and_gradient_match_the_oracle(predictor):
    c, mat, M, u0, dt, steps, k, obs = problem(predictor=predictor)
    J, gm, gM = gpu_J(c, mat, M, u0, dt, steps, k, obs, grads=True)
    s = c.oracle
    matt = torch.from_numpy(mat).requires_grad_(True)
    Mt = torch.from_numpy(M).requires_grad_(True)
    s.mat = matt
    src = s.source
    s.source = PointSource(src.cell, src.xi, Mt, src.f0, src.t0)
    Jo = misfit(s, torch.from_numpy(u0), steps, dt, [torch.from_numpy(o) for o in obs], 0.5)
    go_m, go_M = torch.autograd.grad(Jo, [matt, Mt])
    jo = float(Jo.detach())
    assert abs(J - jo) <= 1e-12 * abs(jo)
    assert np.abs(gm - go_m.numpy()).max() <= 1e-10 * np.abs(go_m.numpy()).max()
    assert np.abs(gM - go_M.numpy()).max() <= 1e-10 * np.abs(go_M.numpy()).max()


@PREDICTORS
def test_gradient_matches_central_finite_differences(predictor):
    c, mat, M, u0, dt, steps, k, obs = problem(order=3, ncell=(2, 3, 2), steps=8, k=3,
                                               predictor=predictor)
    J, gm, gM = gpu_J(c, mat, M, u0, dt, steps, k, obs, grads=True)
    rng = np.random.default_rng(3)
    for _ in range(2):
        dirn = rng.standard_normal(mat.shape) * mat
        eps = 1e-6
        Jp = gpu_J(c, mat + eps * dirn, M, u0, dt, steps, k, obs)
        Jm = gpu_J(c, mat - eps * dirn, M, u0, dt, steps, k, obs)
        fd = (Jp - Jm) / (2 * eps)
        ad = float((gm * dirn).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
    for a in range(6):
        e = np.zeros(6)
        e[a] = 1e-4
        fd = (gpu_J(c, mat, M + e, u0, dt, steps, k, obs) - gpu_J(c, mat, M - e, u0, dt, steps, k, obs)) / 2e-4
        assert abs(fd - gM[a]) <= 1e-6 * max(abs(gM[a]), 1e-30), (a, fd, gM[a])


def test_autograd_function():
    c, mat, M, u0, dt, steps, k, obs = problem(steps=6, k=2)
    J0, gm, gM = gpu_J(c, mat, M, u0, dt, steps, k, obs, grads=True)
    m = torch.from_numpy(mat.copy()).cuda().requires_grad_(True)
    Mt = torch.from_numpy(M.copy()).cuda().requires_grad_(True)
    J = receiver_misfit(m, Mt, c.ctx, torch.from_numpy(u0).cuda(), 0.5, dt, steps, k,
                        torch.from_numpy(obs).cuda())
    (2.0 * J).backward()
    assert abs(float(J.detach()) - J0) <= 1e-14 * abs(J0)
    assert np.allclose(m.grad.cpu().numpy(), 2 * gm, rtol=1e-13, atol=0)
    assert np.allclose(Mt.grad.cpu().numpy(), 2 * gM, rtol=1e-13, atol=0)


def test_ck_gradient_with_mixed_forward_is_close_to_fp64():
    """Order 4 with the mixed-precision Cauchy-Kowalevski forward sweep (the adjoint runs in FP64
    on the recomputed states): the misfit and gradients stay within 1e-6 of the FP64 form."""
    out = {}
    for prec in ("fp64", "mixed"):
        c, mat, M, u0, dt, steps, k, obs = problem(order=4, ncell=(3, 3, 2), steps=6, k=3,
                                                   predictor="ck", precision=prec)
        u0 = 1e-3 * np.random.default_rng(2).standard_normal(c.shape)
        out[prec] = gpu_J(c, mat, M, u0, dt, steps, k, obs, grads=True)
    (Jf, gmf, gMf), (Jm, gmm, gMm) = out["fp64"], out["mixed"]
    assert abs(Jm - Jf) <= 1e-6 * abs(Jf)
    assert np.abs(gmm - gmf).max() <= 1e-6 * np.abs(gmf).max()
    assert np.abs(gMm - gMf).max() <= 1e-6 * np.abs(gMf).max()


def test_mixed_ck_gradient_matches_fp64_central_differences():
    """The gradient of a mixed CK context (mixed forward sweep, mixed-precision adjoint) against
    central differences of the FP64 CK forward solver: relative 1e-6."""
    c, mat, M, u0, dt, steps, k, obs = problem(order=4, ncell=(2, 3, 2), steps=8, k=3,
                                               predictor="ck", precision="mixed")
    J, gm, gM = gpu_J(c, mat, M, u0, dt, steps, k, obs, grads=True)
    f, *_ = problem(order=4, ncell=(2, 3, 2), steps=8, k=3, predictor="ck")
    rng = np.random.default_rng(3)
    for _ in range(2):
        dirn = rng.standard_normal(mat.shape) * mat
        eps = 1e-6
        Jp = gpu_J(f, mat + eps * dirn, M, u0, dt, steps, k, obs)
        Jm = gpu_J(f, mat - eps * dirn, M, u0, dt, steps, k, obs)
        fd = (Jp - Jm) / (2 * eps)
        ad = float((gm * dirn).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
    for a in range(6):
        e = np.zeros(6)
        e[a] = 1e-4
        fd = (gpu_J(f, mat, M + e, u0, dt, steps, k, obs) - gpu_J(f, mat, M - e, u0, dt, steps, k, obs)) / 2e-4
        assert abs(fd - gM[a]) <= 1e-6 * max(abs(gM[a]), 1e-30), (a, fd, gM[a])
