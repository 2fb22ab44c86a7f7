"""GPU parity of the hand-written adjoint of the elastic step (Picard and Cauchy-Kowalevski
predictors) against the oracle's reverse-mode derivative of its own step: lambda^n, the per-cell
material gradient and the moment-tensor gradient, relative 1e-12."""
import numpy as np
import pytest
import torch

from oracle.adjoint import step_vjp
from paper_1905_07987_gb300 import synth
from cases import Case, rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _build():
    from paper_1905_07987_gb300 import build
    build.build()


def close(a, b, tol=1e-12):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1e-300)


CASES = [(2, "absorbing", (3, 2, 3)), (3, "periodic", (2, 3, 2)), (4, "absorbing", (2, 2, 3)),
         (5, "absorbing", (2, 2, 2)), (1, "periodic", (4, 3, 2))]


@pytest.mark.parametrize("predictor", ["picard", "ck"])
@pytest.mark.parametrize("order,bc,ncell", CASES)
def test_adjoint_step_matches_oracle(order, bc, ncell, predictor):
    """Picard form: the adjoint of the Picard iteration; Cauchy-Kowalevski form: the adjoint of
    the Taylor recursion (Sec. 3.3), each against the oracle's derivative of its own step."""
    mat = synth.elastic_material(ncell, seed=order + 10)
    hi = tuple(0.5 * n for n in ncell)
    c = Case("elastic", 3, order, ncell, hi=hi, bc=bc, material=mat, predictor=predictor)
    c.point_source(tuple(0.37 * h for h in hi), synth.moment_tensor(seed=2), 2.0, 0.5)
    rng = np.random.default_rng(order)
    u_n = rng.standard_normal(c.shape)
    lam = rng.standard_normal(c.shape)
    dt = 0.7 * float(c.oracle.cfl_dt(torch.from_numpy(u_n)))
    t_n = 0.43
    lam_ref, gm_ref, gM_ref = step_vjp(c.oracle, torch.from_numpy(u_n), torch.from_numpy(lam), dt, t_n)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()
    lam_d = dev(lam)
    gm = torch.zeros(c.ctx.cells * 3, dtype=torch.float64, device="cuda")
    gM = torch.zeros(6, dtype=torch.float64, device="cuda")
    c.ctx.adjoint_step(t_n, dt, dev(u_n), lam_d, gm, gM)
    torch.cuda.synchronize()
    assert rel_linf(lam_d.cpu().numpy().reshape(c.shape), lam_ref.numpy()) <= 1e-12
    assert close(gm.cpu().numpy(), gm_ref.numpy())
    assert close(gM.cpu().numpy(), gM_ref.numpy())


def test_adjoint_adds_dJdu_and_accumulates():
    ncell = (2, 2, 2)
    mat = synth.elastic_material(ncell, seed=1)
    c = Case("elastic", 3, 2, ncell, bc="absorbing", material=mat)
    rng = np.random.default_rng(5)
    u_n = torch.from_numpy(rng.standard_normal(c.shape).reshape(-1)).cuda()
    lam0 = torch.from_numpy(rng.standard_normal(c.shape).reshape(-1)).cuda()
    dJ = torch.from_numpy(rng.standard_normal(c.shape).reshape(-1)).cuda()
    gm = torch.zeros(24, dtype=torch.float64, device="cuda")
    gM = torch.zeros(6, dtype=torch.float64, device="cuda")
    l1 = lam0.clone()
    c.ctx.adjoint_step(0.0, 1e-3, u_n, l1, gm, gM)
    l2 = lam0.clone()
    gm2 = gm.clone()
    c.ctx.adjoint_step(0.0, 1e-3, u_n, l2, gm2, gM, dJdu=dJ)
    torch.cuda.synchronize()
    assert torch.allclose(l2, l1 + dJ, rtol=0, atol=1e-13)
    assert torch.allclose(gm2, 2 * gm, rtol=1e-13, atol=0)


def test_receiver_adjoint_is_the_transpose_of_the_read_out():
    ncell = (3, 3, 2)
    mat = synth.elastic_material(ncell, seed=2)
    c = Case("elastic", 3, 3, ncell, hi=(1.5, 1.5, 1.0), bc="absorbing", material=mat)
    pts = np.array([[0.2, 0.3, 1.0], [1.1, 0.7, 1.0], [0.25, 0.35, 1.0]])
    seismo = c.receivers(pts, 2)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(c.shape)
    y = rng.standard_normal((3, 3))
    c.set(x)
    c.ctx.run(1, dt=1e-12)  # records v(x_r) of (practically) x into row 0
    Rx = seismo[0].cpu().numpy()
    dJ = torch.zeros(c.ctx.count, dtype=torch.float64, device="cuda")
    c.ctx.receivers_adjoint(torch.from_numpy(y.reshape(-1).copy()).cuda(), 1.0, dJ)
    torch.cuda.synchronize()
    xr = c.get()
    lhs = float((c.oracle.record(torch.from_numpy(xr)).numpy() * y).sum())
    rhs = float((xr.reshape(-1) * dJ.cpu().numpy()).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert np.allclose(Rx, c.oracle.record(torch.from_numpy(xr)).numpy(), atol=1e-12)


@pytest.mark.parametrize("static", [False, True])
def test_nonfinite_forward_state_is_reported(static):
    """A NaN in the forward state u_n makes the material gradient non-finite: both adjoint entry
    points latch it on the device and the next ader_sync returns ADER_ENONFINITE; the call after
    that starts clean."""
    from paper_1905_07987_gb300 import ader
    ncell = (2, 2, 2)
    mat = synth.elastic_material(ncell, seed=3)
    c = Case("elastic", 3, 2, ncell, bc="absorbing", material=mat)
    rng = np.random.default_rng(11)
    u = rng.standard_normal(c.ctx.count)
    u[5] = np.nan
    u_n = torch.from_numpy(u).cuda()
    lam = torch.from_numpy(rng.standard_normal(c.ctx.count)).cuda()
    gm = torch.zeros(c.ctx.cells * 3, dtype=torch.float64, device="cuda")
    gM = torch.zeros(6, dtype=torch.float64, device="cuda")
    c.ctx.adjoint_step(0.0, 1e-3, u_n, lam, gm, gM, static=static)
    with pytest.raises(ader.AderError) as e:
        c.ctx.sync()
    assert e.value.status == ader.ENONFINITE
    # a finite call afterwards reports nothing
    u_ok = torch.from_numpy(rng.standard_normal(c.ctx.count)).cuda()
    gm.zero_()
    c.ctx.adjoint_step(0.0, 1e-3, u_ok, lam.nan_to_num(0.0), gm, gM.zero_(), static=static)
    c.ctx.sync()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("order,ncell", [(4, (5, 4, 3)), (2, (7, 3, 5)), (3, (3, 5, 4))])
def test_ck_adjoint_static_and_repeatable(order, ncell, precision):
    """The Cauchy-Kowalevski adjoint through both entry points (work memory allocated by the
    context, and the fixed device array) gives identical bits, and so does a repeated call
    (fixed-order reductions); several cells per block at orders 2-3 with a ragged last block."""
    mat = synth.elastic_material(ncell, seed=7)
    hi = tuple(0.5 * n for n in ncell)
    c = Case("elastic", 3, order, ncell, hi=hi, bc="absorbing", material=mat, predictor="ck",
             precision=precision)
    c.point_source(tuple(0.61 * h for h in hi), synth.moment_tensor(seed=4), 2.0, 0.5)
    rng = np.random.default_rng(11)
    u_n = torch.from_numpy(rng.standard_normal(c.shape).reshape(-1)).cuda()
    lam0 = torch.from_numpy(rng.standard_normal(c.shape).reshape(-1)).cuda()
    dt = 0.6 * float(c.oracle.cfl_dt(torch.from_numpy(u_n.cpu().numpy().reshape(c.shape))))
    outs = []
    for static in (False, True, False):
        lam = lam0.clone()
        gm = torch.zeros(c.ctx.cells * 3, dtype=torch.float64, device="cuda")
        gM = torch.zeros(6, dtype=torch.float64, device="cuda")
        c.ctx.adjoint_step(0.31, dt, u_n, lam, gm, gM, static=static)
        torch.cuda.synchronize()
        outs.append((lam.cpu(), gm.cpu(), gM.cpu()))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert torch.equal(a, b)
    lam_ref, gm_ref, gM_ref = step_vjp(c.oracle, torch.from_numpy(u_n.cpu().numpy().reshape(c.shape)),
                                       torch.from_numpy(lam0.cpu().numpy().reshape(c.shape)), dt, 0.31)
    tol = 1e-12 if precision == "fp64" else MIXED_TOL
    assert rel_linf(outs[0][0].numpy().reshape(c.shape), lam_ref.numpy()) <= tol
    assert close(outs[0][1].numpy(), gm_ref.numpy(), tol)
    assert close(outs[0][2].numpy(), gM_ref.numpy(), tol)


# Mixed-precision CK adjoint against the FP64 derivative: the binary32 parts are the level
# corrections dt L^T mu_{k+1} (unit roundoff 6e-8 times |dt L^T| |mu|, and |mu| <= |dt L^T| |lambda|
# + |F|) and the pairings of the levels k >= 1.  On these random (not smooth) states |dt L^T| is
# O(1) rather than O(CFL), so the bound is a few unit roundoffs of binary32 relative to the
# largest value: 2e-6 leaves room for the N levels and the sums over nodes.
MIXED_TOL = 2e-6


@pytest.mark.parametrize("order,bc,ncell", CASES)
def test_mixed_ck_adjoint_step_close_to_oracle(order, bc, ncell):
    """The mixed-precision adjoint of a mixed CK context against the oracle's FP64 derivative of
    the CK step (the tolerance above)."""
    mat = synth.elastic_material(ncell, seed=order + 10)
    hi = tuple(0.5 * n for n in ncell)
    c = Case("elastic", 3, order, ncell, hi=hi, bc=bc, material=mat, predictor="ck",
             precision="mixed")
    c.point_source(tuple(0.37 * h for h in hi), synth.moment_tensor(seed=2), 2.0, 0.5)
    rng = np.random.default_rng(order)
    u_n = rng.standard_normal(c.shape)
    lam = rng.standard_normal(c.shape)
    dt = 0.7 * float(c.oracle.cfl_dt(torch.from_numpy(u_n)))
    t_n = 0.43
    lam_ref, gm_ref, gM_ref = step_vjp(c.oracle, torch.from_numpy(u_n), torch.from_numpy(lam), dt, t_n)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()
    lam_d = dev(lam)
    gm = torch.zeros(c.ctx.cells * 3, dtype=torch.float64, device="cuda")
    gM = torch.zeros(6, dtype=torch.float64, device="cuda")
    c.ctx.adjoint_step(t_n, dt, dev(u_n), lam_d, gm, gM)
    torch.cuda.synchronize()
    err = rel_linf(lam_d.cpu().numpy().reshape(c.shape), lam_ref.numpy())
    assert err <= MIXED_TOL, err
    assert close(gm.cpu().numpy(), gm_ref.numpy(), MIXED_TOL)
    assert close(gM.cpu().numpy(), gM_ref.numpy(), MIXED_TOL)
