"""GPU parity of the a-posteriori subcell limiter (Sec. 3.5) against the oracle: troubled-cell
flags bit-identical, states within relative 1e-12 per step (teacher forcing: both sides start
every step from the oracle's state and representation), free-running runs, the pure FV mode,
and conservation."""
import numpy as np
import pytest
import torch

from oracle.limiter import Limiter
from paper_1905_07987_gb300 import ader, synth
from cases import Case, rel_linf

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(autouse=True, scope="module")
def _build():
    from paper_1905_07987_gb300 import build
    build.build()


def explosion_case(ncell, order, limiter=1, bc="wall", precision="fp64", initial_guess="constant",
                   picard_iters=0):
    dim = len(ncell)
    c = Case("euler", dim, order, ncell, lo=(-1.0,) * dim, hi=(1.0,) * dim, bc=bc, limiter=limiter,
             precision=precision, initial_guess=initial_guess, picard_iters=picard_iters)
    lim = Limiter(c.oracle)
    u0 = synth.explosion(c.X)
    Us = synth.explosion(synth.subcell_centres(lim.ns, c.ncell, c.lo, c.hi))
    flags = synth.discontinuous_cells(Us)
    u, rep = lim.initial_rep(torch.from_numpy(u0), torch.from_numpy(Us), torch.from_numpy(flags))
    return c, lim, u0, Us, flags, u, rep


def gpu_set(c, u_nodal_before_init, Us, flags):
    c.set(u_nodal_before_init)
    c.ctx.set_subcell_state(torch.from_numpy(np.ascontiguousarray(Us).reshape(-1)).cuda(),
                            torch.from_numpy(flags.astype(np.uint8)).cuda())


def gpu_rep(c, lim):
    out = torch.empty(c.ctx.cells * lim.ns ** c.dim * c.ctx.nvar, dtype=torch.float64, device="cuda")
    c.ctx.get_subcell_state(out)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape((c.ctx.cells,) + (lim.ns,) * c.dim + (c.ctx.nvar,))


@pytest.mark.parametrize("dim,ncell,order", [(2, (10, 10), 2), (2, (9, 8), 3), (3, (6, 6, 6), 3),
                                             (3, (5, 4, 6), 2), (3, (4, 4, 4), 4),
                                             # one cell thick: the FV halo reflects inside the cell
                                             (2, (1, 8), 2), (3, (1, 5, 4), 2), (2, (6, 1), 3)])
def test_limited_steps_teacher_forced(dim, ncell, order):
    c, lim, u0, Us, flags, u, rep = explosion_case(ncell, order)
    gpu_set(c, u0, Us, flags)
    # the initial FV cells: identical state and representation on both sides
    assert rel_linf(c.get(), u.numpy()) <= TOL
    assert rel_linf(gpu_rep(c, lim), rep.numpy()) <= TOL
    prev = torch.from_numpy(flags)
    t = 0.0
    for step in range(3):
        if step > 0:  # teacher forcing: restart the GPU from the oracle's state
            gpu_set(c, u.numpy(), rep.numpy(), prev.numpy())
            # set_state reset u of flagged cells to R(rep): same as the oracle's u for those cells
        c.ctx.set_time(t)
        c.ctx.step()
        dt = c.ctx.last_dt()
        u, tr, rep, ok = lim.step(u, rep, torch.tensor(dt, dtype=torch.float64), t)
        assert ok
        fl = np.zeros(c.ctx.cells, dtype=np.uint8)
        fl[:] = c.ctx.flags()
        assert np.array_equal(fl.astype(bool), tr.numpy()), step
        assert c.ctx.troubled_count() == int(tr.sum())
        assert rel_linf(c.get(), u.numpy()) <= TOL, step
        assert rel_linf(gpu_rep(c, lim), rep.numpy()) <= TOL, step
        prev = tr
        t += dt


def test_limited_free_run_flags_identical_every_step():
    c, lim, u0, Us, flags, u, rep = explosion_case((12, 12), 3)
    gpu_set(c, u0, Us, flags)
    for step in range(12):
        c.ctx.step()
        dt = c.ctx.last_dt()
        u, tr, rep, ok = lim.step(u, rep, torch.tensor(dt, dtype=torch.float64))
        assert np.array_equal(c.ctx.flags().astype(bool), tr.numpy()), step
    assert rel_linf(c.get(), u.numpy()) <= 1e-11


@pytest.mark.parametrize("ncell", [(12, 12), (6, 5, 6)])
def test_limited_run_with_the_cerk_guess(ncell):
    """The limiter after the predictor started from the continuous extension Runge-Kutta guess
    (Sec. 5) with one Picard iteration: troubled flags identical to the oracle's every step of a
    free run, state 1e-11."""
    c, lim, u0, Us, flags, u, rep = explosion_case(ncell, 3, initial_guess="cerk", picard_iters=1)
    gpu_set(c, u0, Us, flags)
    for step in range(8):
        c.ctx.step()
        dt = c.ctx.last_dt()
        u, tr, rep, ok = lim.step(u, rep, torch.tensor(dt, dtype=torch.float64))
        assert np.array_equal(c.ctx.flags().astype(bool), tr.numpy()), step
    assert rel_linf(c.get(), u.numpy()) <= 1e-11


def test_pure_fv_mode_matches_forced_oracle():
    c, lim, u0, Us, flags, u, rep = explosion_case((6, 5, 4), 2, limiter=2)
    gpu_set(c, u0, Us, flags)
    c.ctx.step()
    dt = c.ctx.last_dt()
    u1, tr, rep1, ok = lim.step(u, rep, torch.tensor(dt, dtype=torch.float64), force=True)
    assert c.ctx.flags().all() and tr.all()
    assert rel_linf(c.get(), u1.numpy()) <= TOL
    assert rel_linf(gpu_rep(c, lim), rep1.numpy()) <= TOL


def test_limited_run_conserves_mass_and_energy():
    c, lim, u0, Us, flags, u, rep = explosion_case((8, 8, 8), 3)
    gpu_set(c, u0, Us, flags)
    W = c.oracle.tensor_basis_weights().numpy()
    vol = np.prod(c.oracle.grid.h)

    def tot(x):
        return (x * W[None, ..., None]).reshape(-1, x.shape[-1]).sum(0) * vol

    m0 = tot(c.get())
    c.ctx.run(10)
    m1 = tot(c.get())
    assert abs(m1[0] - m0[0]) < 1e-13 * abs(m0[0])
    assert abs(m1[4] - m0[4]) < 1e-13 * abs(m0[4])
    assert c.ctx.troubled_count() > 0


def test_mixed_limited_run_conserves_and_tracks_fp64():
    """Mixed predictor (binary32 increments and wave speeds) with the limiter on: mass and energy
    are conserved to round-off, the state stays admissible, and after the same number of steps it
    is close to the FP64 limited run (the two may differ where a flag flips)."""
    out = {}
    for prec in ("fp64", "mixed"):
        c, lim, u0, Us, flags, u, rep = explosion_case((8, 8, 8), 3, precision=prec)
        gpu_set(c, u0, Us, flags)
        W = c.oracle.tensor_basis_weights().numpy()
        vol = np.prod(c.oracle.grid.h)

        def tot(x):
            return (x * W[None, ..., None]).reshape(-1, x.shape[-1]).sum(0) * vol

        m0 = tot(c.get())
        c.ctx.run(6)
        got = c.get()
        m1 = tot(got)
        assert abs(m1[0] - m0[0]) < 1e-13 * abs(m0[0]), prec
        assert abs(m1[4] - m0[4]) < 1e-13 * abs(m0[4]), prec
        assert np.isfinite(got).all() and got[..., 0].min() > 0, prec
        assert c.ctx.troubled_count() > 0
        out[prec] = got
    diff = np.abs(out["mixed"] - out["fp64"]).max(axis=tuple(range(out["fp64"].ndim - 1)))
    scale = np.abs(out["fp64"]).max(axis=tuple(range(out["fp64"].ndim - 1)))
    assert (diff <= 1e-3 * scale).all(), diff / scale


def shifted_explosion_case(ncell, order, lo, hi, bc, limiter=3):
    """Explosion on a box that cuts the sphere, so that cells along the discontinuity touch the
    domain boundary (and, periodic, wrap around it)."""
    dim = len(ncell)
    c = Case("euler", dim, order, ncell, lo=lo, hi=hi, bc=bc, limiter=limiter)
    lim = Limiter(c.oracle)
    u0 = synth.explosion(c.X)
    Us = synth.explosion(synth.subcell_centres(lim.ns, c.ncell, c.lo, c.hi))
    flags = synth.discontinuous_cells(Us)
    u, rep = lim.initial_rep(torch.from_numpy(u0), torch.from_numpy(Us), torch.from_numpy(flags))
    return c, lim, u0, Us, flags, u, rep


@pytest.mark.parametrize("ncell,order,steps,box", [
    ((10, 10), 2, 6, None), ((6, 6, 5), 2, 3, None),
    # periodic, the sphere cut by the lower x face: FV cells on both wrapped boundaries
    ((10, 10), 2, 5, ((-0.45, -1.0), (1.55, 1.0), "periodic")),
    ((6, 5, 6), 2, 3, ((-0.45, -1.0, -1.0), (1.55, 1.0, 1.0), "periodic"))])
def test_hybrid_status_run_matches_the_oracle(ncell, order, steps, box):
    """limiter = 3 (troubled cells stay FV two more steps, face neighbours compute with FV; the
    cells put into the FV space at the start count as troubled at t^0): the FV set and the state
    against the oracle's hybrid step, every step."""
    if box is None:
        c, lim, u0, Us, flags, u, rep = explosion_case(ncell, order, limiter=3)
    else:
        c, lim, u0, Us, flags, u, rep = shifted_explosion_case(ncell, order, *box)
        # the FV set reaches the periodic boundary in the direction that wraps
        fl = flags.reshape(tuple(reversed(ncell)))
        assert fl[..., 0].any()
    gpu_set(c, u0, Us, flags)
    status = lim.initial_status(torch.from_numpy(flags), persist=2)
    for step in range(steps):
        c.ctx.step()
        dt = c.ctx.last_dt()
        u, fv, rep, ok, status = lim.step_hybrid(u, rep, status, torch.tensor(dt, dtype=torch.float64),
                                                 persist=2, layer=True)
        got = c.ctx.flags().astype(bool)
        assert np.array_equal(got, fv.numpy()), step
        if step < 2:  # the initial FV cells keep their two FV steps
            assert got[flags].all(), step
    assert rel_linf(c.get(), u.numpy()) <= 1e-11


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hybrid_with_every_cell_counting_is_the_pure_fv_step(precision):
    """Every cell put into the FV space at the start (each counts `persist` FV steps): no cell is
    checked and no DG result is kept, so the hybrid step is the oracle's pure FV step, whatever
    the predictor's precision (the GPU skips every cell's predictor)."""
    c, lim, u0, Us, flags, u, rep = explosion_case((6, 5, 4), 2, limiter=3, precision=precision)
    every = np.ones_like(flags)
    gpu_set(c, u0, Us, every)
    u, rep = lim.initial_rep(torch.from_numpy(u0), torch.from_numpy(Us), torch.from_numpy(every))
    status = lim.initial_status(torch.from_numpy(every), persist=2)
    c.ctx.step()
    dt = torch.tensor(c.ctx.last_dt(), dtype=torch.float64)
    u1, fv, rep1, ok, status = lim.step_hybrid(u, rep, status, dt, persist=2)
    U_all, _ = lim.fv_global(rep, dt)
    assert fv.all() and torch.equal(rep1, U_all)
    assert c.ctx.flags().astype(bool).all()
    assert rel_linf(c.get(), u1.numpy()) <= TOL
    assert np.abs(gpu_rep(c, lim) - rep1.numpy()).max() <= TOL * np.abs(rep1.numpy()).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hybrid_skips_the_predictor_of_counting_cells(precision):
    """The predictor launch of a step in which every cell counts FV steps does no work: its time
    is a small fraction of the same launch with every cell in DG (24^3 cells, order 3)."""
    n = 24
    c, lim, u0, Us, flags, u, rep = explosion_case((n, n, n), 3, limiter=3, precision=precision)
    every = np.ones_like(flags)

    def predictor_ms(fl):
        gpu_set(c, u0, Us, fl)
        c.ctx.step()          # warm-up (the counts go from 2 to 1)
        gpu_set(c, u0, Us, fl)
        c.ctx.enable_timing(True)
        c.ctx.step()
        ph, nrec = c.ctx.phase_times()
        c.ctx.enable_timing(False)
        assert nrec == 1
        return ph["predictor"]

    full = predictor_ms(np.zeros_like(flags))
    skipped = predictor_ms(every)
    assert skipped < 0.2 * full, (skipped, full)


def rel_linf_floored(a, b):
    """rel_linf with a variable that is zero up to round-off (its largest value below 1e-8 of the
    state's) measured against the size of the state."""
    nv = b.shape[-1]
    a, b = np.asarray(a).reshape(-1, nv), np.asarray(b).reshape(-1, nv)
    g = np.abs(b).max()
    scale = np.abs(b).max(axis=0)
    scale = np.where(scale > 1e-8 * g, scale, g)
    return float((np.abs(a - b).max(axis=0) / scale).max())


def rarefaction_case(floor):
    """rho = 1, p = 0.4, u = -3 / +3 left / right of x = 0 on 8 x 4 cells, order 2, walls, and an
    admissibility floor on density and pressure (Table 2 isPhysicallyAdmissable)."""
    nc, lo, hi = (8, 4), (-1.0, -0.5), (1.0, 0.5)
    c = Case("euler", 2, 2, nc, lo=lo, hi=hi, bc="wall", limiter=1)
    c.ctx.close()
    c.cfg = ader.make_config("euler", 2, 2, nc, lo, hi, "wall", c.cfl, limiter=1, adm_floor=floor)
    c.ctx = ader.Context(c.cfg)
    lim = Limiter(c.oracle, floor=floor)
    Xs = synth.subcell_centres(lim.ns, nc, lo, hi)
    Us = synth.euler_conserved(np.ones_like(Xs[0]), [np.where(Xs[0] < 0, -3.0, 3.0), 0 * Xs[0]],
                               np.full_like(Xs[0], 0.4))
    u0 = synth.euler_conserved(np.ones_like(c.X[0]), [np.where(c.X[0] < 0, -3.0, 3.0), 0 * c.X[0]],
                               np.full_like(c.X[0], 0.4))
    flags = synth.discontinuous_cells(Us)
    u, rep = lim.initial_rep(torch.from_numpy(u0), torch.from_numpy(Us), torch.from_numpy(flags))
    return c, lim, u0, Us, flags, u, rep


def test_first_order_fallback_matches_the_oracle():
    """Floor 0.1: the MUSCL-Hancock recompute of the third step falls below it, the step is redone
    with the first-order scheme for every troubled cell (a second, conditional launch); flags,
    state and representation equal the oracle's every step, and no error is reported."""
    from paper_1905_07987_gb300 import ader as _a  # noqa: F401
    c, lim, u0, Us, flags, u, rep = rarefaction_case(0.1)
    gpu_set(c, u0, Us, flags)
    used = []
    for step in range(3):
        c.ctx.step()
        dt = c.ctx.last_dt()  # raises on a latched error
        u, tr, rep, ok = lim.step(u, rep, torch.tensor(dt, dtype=torch.float64))
        used.append(lim.last_fallback)
        assert ok
        assert np.array_equal(c.ctx.flags().astype(bool), tr.numpy()), step
        # the y momentum of this flow is zero up to round-off: variable scales are floored at the
        # size of the state
        assert rel_linf_floored(c.get(), u.numpy()) <= TOL, step
        assert rel_linf_floored(gpu_rep(c, lim), rep.numpy()) <= TOL, step
    assert used == [False, False, True]


def test_fallback_that_is_still_inadmissible_is_reported():
    c, lim, u0, Us, flags, u, rep = rarefaction_case(0.39)
    gpu_set(c, u0, Us, flags)
    c.ctx.step()
    c.ctx.step()
    c.ctx.sync()
    c.ctx.step()
    with pytest.raises(ader.AderError) as e:
        c.ctx.sync()
    assert e.value.status == ader.EADMISSIBLE


def test_host_batch_with_the_limiter_equals_the_step_loop():
    """ader_step_host_batch on a limited context: every host state gets the limiter data of
    ader_set_state (fresh DMP bounds from its own projection), so each result equals set_state /
    step / get_state bit for bit."""
    c, lim, u0, Us, flags, u, rep = explosion_case((8, 7), 3)
    ins = [torch.from_numpy((u0 * (1.0 + 0.02 * k)).reshape(-1).copy()).pin_memory() for k in range(3)]
    outs = [torch.empty(c.ctx.count, dtype=torch.float64).pin_memory() for _ in ins]
    c.ctx.set_time(0.0)
    c.ctx.step_host_batch(ins, outs)
    for k, x in enumerate(ins):
        c.ctx.set_state(x.cuda())
        c.ctx.set_time(0.0)
        c.ctx.step()
        assert np.array_equal(c.get().reshape(-1), outs[k].numpy()), k
