"""Pins for the oracle's a-posteriori subcell limiter (Sec. 3.5): Godunov limit of the FV scheme,
the exact Sod solution, conservation through troubled cells and neighbour fixes, no troubled
cells on smooth data, symmetry of the explosion, and detection of non-finite states."""
import math

import numpy as np
import pytest
import torch

from oracle.aderdg import ADERDG, Grid
from oracle.limiter import Limiter
from oracle.pde import Euler
from paper_1905_07987_gb300 import synth
from sod_exact import sample, star_state

T = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float64)


def make(ncell, N, lo, hi, bc):
    dim = len(ncell)
    g = Grid(ncell, lo, hi, [(bc, bc)] * dim if isinstance(bc, str) else bc)
    s = ADERDG(Euler(dim), g, N, cfl=synth.cfl_number(N))
    return s, Limiter(s)


def coords(s):
    return synth.node_coordinates(s.ref.x.numpy(), s.grid.ncell, s.grid.lo, s.grid.hi)


def test_exact_riemann_solver_reproduces_the_textbook_sod_star_state():
    ps, us = star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(ps - 0.30313) < 1e-5 and abs(us - 0.92745) < 1e-5


def test_fv_without_slopes_is_first_order_godunov_rusanov():
    s, lim = make((3, 2), 2, (0, 0), (1, 1), 'periodic')
    rng = np.random.default_rng(0)
    rep = T(synth.euler_conserved(1 + 0.3 * rng.random((6, 5, 5)), [0.2 * rng.random((6, 5, 5)), -0.1],
                                  1 + 0.2 * rng.random((6, 5, 5))))
    dt = 0.003
    U_new, _ = lim.fv_global(rep, dt, slopes=False)
    G = lim.to_global(rep)  # [10 (y), 15 (x), 4]
    pde = Euler(2)
    dx = [1 / 15, 1 / 10]
    out = G.clone()
    for d, ax in ((0, 1), (1, 0)):
        Ur = torch.roll(G, -1, dims=ax)
        s_ = torch.maximum(pde.max_speed(G, d), pde.max_speed(Ur, d))[..., None]
        f = 0.5 * (pde.flux(G, d) + pde.flux(Ur, d)) - 0.5 * s_ * (Ur - G)  # right faces
        out = out - dt / dx[d] * (f - torch.roll(f, 1, dims=ax))
    assert torch.allclose(lim.to_global(U_new), out, atol=1e-14)


def sod_run(nc, t_end=0.15):
    s, lim = make((nc, 1), 2, (0, 0), (1, 1.0 / nc), [('absorbing', 'absorbing'), ('periodic', 'periodic')])
    X = coords(s)
    left = X[0] < 0.5
    u = T(synth.euler_conserved(np.where(left, 1.0, 0.125), [0.0, 0.0], np.where(left, 1.0, 0.1)))
    Xs = synth.subcell_centres(lim.ns, s.grid.ncell, s.grid.lo, s.grid.hi)
    ls = Xs[0] < 0.5
    Us = synth.euler_conserved(np.where(ls, 1.0, 0.125), [0.0, 0.0], np.where(ls, 1.0, 0.1))
    u, rep = lim.initial_rep(u, T(Us), torch.from_numpy(synth.discontinuous_cells(Us)))
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(float(s.cfl_dt(u)), t_end - t)
        u, tr, rep, ok = lim.step(u, rep, torch.tensor(dt, dtype=torch.float64), t, force=True)
        assert ok
        t += dt
    # L1 error of the subcell averages (the FV representation) against the exact solution
    G = lim.to_global(rep)[0, :, 0].numpy()
    ns = lim.ns
    xs = (np.arange(nc * ns) + 0.5) / (nc * ns)
    ex = np.array([sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (x - 0.5) / t)[0] for x in xs])
    return np.mean(np.abs(G - ex))


def test_pure_fv_scheme_converges_to_the_exact_sod_solution():
    e1 = sod_run(8)
    e2 = sod_run(16)
    assert e2 < 0.65 * e1, (e1, e2)
    assert e2 < 0.02


def explosion(ncell, N, lo=-1.0, hi=1.0):
    """Explosion data; cells cut by the initial sphere start with FV subcell averages."""
    dim = len(ncell)
    s, lim = make(ncell, N, (lo,) * dim, (hi,) * dim, 'wall')
    u = T(synth.explosion(coords(s)))
    Us = synth.explosion(synth.subcell_centres(lim.ns, s.grid.ncell, s.grid.lo, s.grid.hi))
    flags = torch.from_numpy(synth.discontinuous_cells(Us))
    u, rep = lim.initial_rep(u, T(Us), flags)
    return s, lim, u, rep


def totals(s, u):
    W = s.tensor_basis_weights()
    vol = 1.0
    for h in s.grid.h:
        vol *= h
    return (u * W[None, ..., None]).sum(dim=tuple(range(0, s.D + 1))) * vol


def test_limited_explosion_conserves_mass_and_energy_and_flags_the_front():
    s, lim, u, rep = explosion((10, 10), 2)
    m0 = totals(s, u)
    n_tr = []
    for _ in range(4):
        u, tr, rep, ok = lim.step(u, rep, s.cfl_dt(u))
        assert ok
        n_tr.append(int(tr.sum()))
    m1 = totals(s, u)
    assert abs(float(m1[0] - m0[0])) < 1e-13 * float(m0[0])
    assert abs(float(m1[3] - m0[3])) < 1e-13 * float(m0[3])
    assert min(n_tr) > 0 and max(n_tr) < 100


def test_explosion_flags_and_state_are_symmetric():
    s, lim, u, rep = explosion((8, 8), 2)
    for _ in range(3):
        u, tr, rep, ok = lim.step(u, rep, s.cfl_dt(u))
    F = tr.reshape(8, 8)
    assert torch.equal(F, F.flip(0)) and torch.equal(F, F.flip(1)) and torch.equal(F, F.T)
    uu = u.reshape(8, 8, 3, 3, 4)
    assert torch.allclose(uu[..., 0], uu.flip(1).flip(3)[..., 0], atol=1e-12)
    assert torch.allclose(uu[..., 0], uu.transpose(0, 1).transpose(2, 3)[..., 0], atol=1e-12)


def test_smooth_flow_has_no_troubled_cells():
    """A smooth wave of small amplitude stays inside the relaxed DMP (delta0 = 1e-4)."""
    s, lim = make((8, 8), 3, (0, 0), (1, 1), 'periodic')
    u = T(synth.entropy_wave(coords(s), amp=1e-3))
    u, rep = lim.initial_rep(u)
    for _ in range(3):
        u, tr, rep, ok = lim.step(u, rep, s.cfl_dt(u))
        assert not tr.any()


def test_forced_recompute_equals_pure_fv_and_is_conservative():
    s, lim, u, rep = explosion((6, 6), 2)
    dt = s.cfl_dt(u)
    u1, tr, rep1, ok = lim.step(u, rep, dt, force=True)
    U_all, _ = lim.fv_global(rep, dt)
    assert tr.all() and torch.allclose(rep1, U_all, atol=0)
    assert torch.allclose(u1, lim.reconstruct(U_all), atol=0)
    m0, m1 = totals(s, u), totals(s, u1)
    assert abs(float(m1[0] - m0[0])) < 1e-14


def test_non_finite_candidate_is_troubled():
    s, lim = make((4, 4), 2, (0, 0), (1, 1), 'periodic')
    u = T(synth.entropy_wave(coords(s)))
    u, rep = lim.initial_rep(u)
    bad = u.clone()
    bad[5, 1, 1, 2] = float('nan')
    tr, _ = lim.detect(bad, rep)
    assert bool(tr[5]) and int(tr.sum()) == 1


# ---- the relaxed DMP band and positivity, on cell-wise constant states (subcell averages of a
# constant cell are that constant) ----------------------------------------------------------------

def _constant_cells(s, values):
    """[C, n, n, 4] with the conserved state values[c] (rho, jx, jy, E) in every node of cell c."""
    n = s.n
    v = torch.as_tensor(values, dtype=torch.float64)
    return v[:, None, None, :].expand(v.shape[0], n, n, 4).clone()


def _flat(C, rho=1.0, E=2.5):
    return [[rho, 0.0, 0.0, E] for _ in range(C)]


def test_dmp_band_is_delta0_on_a_flat_neighbourhood():
    """m = M everywhere: the band is delta0 = 1e-4 on both sides, only the raised cell flips."""
    s, lim = make((4, 4), 2, (0, 0), (1, 1), 'periodic')
    base = _constant_cells(s, _flat(16))
    rep = lim.project(base)
    for shift, troubled in ((0.9e-4, False), (1.1e-4, True), (-0.9e-4, False), (-1.1e-4, True)):
        cand = base.clone()
        cand[5, ..., 0] += shift
        tr, _ = lim.detect(cand, rep)
        assert bool(tr[5]) == troubled, shift
        assert int(tr.sum()) == int(troubled)


def test_dmp_band_scales_with_the_face_neighbourhood_range():
    """A face neighbour at rho = 2 makes the range 1 and the band 1e-3 (M - m) = 1e-3 > delta0;
    a diagonal neighbour at rho = 2 does not widen the band (face neighbourhood)."""
    s, lim = make((4, 4), 2, (0, 0), (1, 1), 'periodic')
    vals = _flat(16)
    vals[6][0] = 2.0                         # (2, 1): face neighbour of cell 5 = (1, 1)
    rep = lim.project(_constant_cells(s, vals))
    for rho, troubled in ((2.0 + 0.9e-3, False), (2.0 + 1.1e-3, True), (1.0 - 0.9e-3, False)):
        cand_vals = [list(v) for v in vals]
        cand_vals[5][0] = rho
        tr, _ = lim.detect(_constant_cells(s, cand_vals), rep)
        assert bool(tr[5]) == troubled, rho
    vals = _flat(16)
    vals[10][0] = 2.0                        # (2, 2): diagonal to cell 5
    rep = lim.project(_constant_cells(s, vals))
    cand_vals = [list(v) for v in vals]
    cand_vals[5][0] = 1.5
    tr, _ = lim.detect(_constant_cells(s, cand_vals), rep)
    assert bool(tr[5])


def test_positivity_is_checked_inside_the_dmp_band():
    """Neighbourhood bands jx in [-2, 2], E in [1.5, 2.5], rho = 1: the candidate (1, 1.9, 0, 1.5)
    is inside every band but has p = 0.4 (1.5 - 1.9^2 / 2) < 0, so it is troubled; (1, 1, 0, 1.5)
    (p = 0.4) is not."""
    s, lim = make((4, 4), 2, (0, 0), (1, 1), 'periodic')
    vals = _flat(16)
    vals[5] = [1.0, 2.0, 0.0, 2.5]
    vals[6] = [1.0, -2.0, 0.0, 2.5]
    vals[9] = [1.0, 0.0, 0.0, 1.5]
    rep = lim.project(_constant_cells(s, vals))
    for jx, troubled in ((1.9, True), (1.0, False)):
        cand_vals = [list(v) for v in vals]
        cand_vals[5] = [1.0, jx, 0.0, 1.5]
        tr, _ = lim.detect(_constant_cells(s, cand_vals), rep)
        assert bool(tr[5]) == troubled, jx


# ---- hybrid ADER-DG / FV status (cells stay FV for several steps, FV interface layer) ---------

def test_hybrid_without_persistence_or_layer_is_the_per_step_limiter():
    s, lim, u, rep = explosion((8, 8), 2)
    u2, rep2 = u.clone(), rep.clone()
    status = torch.zeros(64, dtype=torch.long)
    for _ in range(3):
        dt = s.cfl_dt(u)
        u, tr, rep, ok = lim.step(u, rep, dt)
        u2, fv, rep2, ok2, status = lim.step_hybrid(u2, rep2, status, dt, persist=0, layer=False)
        assert torch.equal(tr, fv) and torch.equal(u, u2) and torch.equal(rep, rep2)
        assert not status.any()


def test_hybrid_conserves_mass_and_energy_and_keeps_the_symmetry():
    s, lim, u, rep = explosion((8, 8), 2)
    m0 = totals(s, u)
    status = torch.zeros(64, dtype=torch.long)
    for _ in range(4):
        u, fv, rep, ok, status = lim.step_hybrid(u, rep, status, s.cfl_dt(u), persist=2, layer=True)
        assert ok
    m1 = totals(s, u)
    assert abs(float(m1[0] - m0[0])) < 1e-13 * float(m0[0])
    assert abs(float(m1[3] - m0[3])) < 1e-13 * float(m0[3])
    F = fv.reshape(8, 8)
    assert torch.equal(F, F.flip(0)) and torch.equal(F, F.flip(1)) and torch.equal(F, F.T)
    uu = u.reshape(8, 8, 3, 3, 4)
    assert torch.allclose(uu[..., 0], uu.transpose(0, 1).transpose(2, 3)[..., 0], atol=1e-12)


def test_hybrid_status_counts_down_with_its_interface_layer():
    """Smooth data (nothing detected): a cell given two FV steps is FV with its four face
    neighbours for two steps, then the whole grid is DG again."""
    s, lim = make((6, 6), 2, (0, 0), (1, 1), 'periodic')
    u = T(synth.entropy_wave(coords(s), amp=1e-3))
    u, rep = lim.initial_rep(u)
    status = torch.zeros(36, dtype=torch.long)
    status[14] = 2                                   # cell (2, 2)
    layer = {14, 13, 15, 8, 20}
    for k, expect in enumerate((layer, layer, set())):
        u, fv, rep, ok, status = lim.step_hybrid(u, rep, status, s.cfl_dt(u), persist=2)
        assert set(torch.nonzero(fv).flatten().tolist()) == expect, k
        assert ok


def test_initial_fv_cells_keep_their_fv_steps():
    """Cells that start in the FV space along the initial discontinuity count as troubled at
    t^0 (Sec. 3.5): on data where nothing is detected they stay FV, with their interface layer,
    for exactly `persist` steps."""
    s, lim = make((6, 6), 2, (0, 0), (1, 1), 'periodic')
    u = T(synth.entropy_wave(coords(s), amp=1e-3))
    flags = torch.zeros(36, dtype=torch.bool)
    flags[[14, 27]] = True                           # cells (2, 2) and (3, 4)
    U = lim.project(u)
    u, rep = lim.initial_rep(u, U, flags)
    status = lim.initial_status(flags, persist=3)
    assert status.tolist().count(3) == 2 and int(status.sum()) == 6
    layer = {14, 13, 15, 8, 20, 27, 26, 28, 21, 33}
    for k, expect in enumerate((layer, layer, layer, set())):
        u, fv, rep, ok, status = lim.step_hybrid(u, rep, status, s.cfl_dt(u), persist=3)
        assert set(torch.nonzero(fv).flatten().tolist()) == expect, k
        assert ok


def test_hybrid_with_every_cell_fv_is_the_pure_fv_scheme():
    s, lim, u, rep = explosion((6, 6), 2)
    dt = s.cfl_dt(u)
    status = torch.ones(36, dtype=torch.long)
    u1, fv, rep1, ok, _ = lim.step_hybrid(u, rep, status, dt)
    U_all, _ = lim.fv_global(rep, dt)
    assert fv.all() and torch.equal(rep1, U_all)
    assert torch.equal(u1, lim.reconstruct(U_all))


def test_hybrid_does_not_use_the_dg_predictor_of_counting_cells():
    """A cell with FV steps left computes with FV, and with the interface layer so do its face
    neighbours, whose DG candidates are not checked either: its predictor's output reaches
    nothing that is kept.  Replacing that output by NaN leaves the hybrid step bit-identical
    (the GPU skips those cells' predictor)."""
    s, lim, u, rep = explosion((8, 8), 2)
    status = torch.zeros(64, dtype=torch.long)
    for _ in range(2):
        u, fv, rep, ok, status = lim.step_hybrid(u, rep, status, s.cfl_dt(u), persist=2)
    counting = status > 0
    assert counting.any() and not counting.all()
    dt = s.cfl_dt(u)
    ref = lim.step_hybrid(u, rep, status, dt, persist=2)
    plain = s.predictor

    def broken(uu, dtt, t=0.0, **kw):
        q = plain(uu, dtt, t, **kw)
        q[counting] = float("nan")
        return q

    s.predictor = broken
    try:
        got = lim.step_hybrid(u, rep, status, dt, persist=2)
    finally:
        del s.predictor
    assert torch.isnan(broken(u, dt)).any()
    for a, b in zip(ref, got):
        assert torch.equal(a, b) if torch.is_tensor(a) else a == b


# ---- first-order fallback of the FV recompute (Table 1: Godunov beside MUSCL-Hancock) --------

def double_rarefaction(s, lim, nc, lo, hi, ul=-3.0, p=0.4):
    """rho = 1, p = 0.4, u = -3 / +3 left / right of x = 0: two strong rarefactions that deepen
    the density and pressure minimum at the centre (the cells along x = 0 start in FV)."""
    Xs = synth.subcell_centres(lim.ns, nc, lo, hi)
    Us = synth.euler_conserved(np.ones_like(Xs[0]), [np.where(Xs[0] < 0, ul, -ul), 0 * Xs[0]],
                               np.full_like(Xs[0], p))
    X = coords(s)
    u0 = synth.euler_conserved(np.ones_like(X[0]), [np.where(X[0] < 0, ul, -ul), 0 * X[0]],
                               np.full_like(X[0], p))
    fl = synth.discontinuous_cells(Us)
    return lim.initial_rep(T(u0), T(Us), torch.from_numpy(fl))


def test_fallback_is_the_first_order_scheme_where_muscl_falls_below_the_floor():
    """With an admissibility floor of 0.1 on density and pressure the MUSCL-Hancock recompute of
    the third step dips to p ~ 0.015 at the centre while the zero-slope scheme stays near 0.33:
    that step is redone first order for every troubled cell (its result equals the step with
    the zero-slope scheme), it is admissible, and mass and energy stay conserved."""
    nc, lo, hi = (8, 4), (-1.0, -0.5), (1.0, 0.5)
    s, _ = make(nc, 2, lo, hi, 'wall')
    lim = Limiter(s, floor=0.1)
    u, rep = double_rarefaction(s, lim, nc, lo, hi)
    m0 = totals(s, u)
    used = []
    for _ in range(3):
        dt = s.cfl_dt(u)
        U_muscl, _ = lim.fv_global(rep, dt)
        U_god, _ = lim.fv_global(rep, dt, slopes=False)
        u_prev, rep_prev = u, rep
        u, tr, rep, ok = lim.step(u, rep, dt)
        used.append(lim.last_fallback)
        assert ok
        if lim.last_fallback:
            assert not bool(lim.admissible(U_muscl[tr]).all())
            assert torch.equal(rep[tr], U_god[tr])
        else:
            assert torch.equal(rep[tr], U_muscl[tr])
    assert used == [False, False, True]
    m1 = totals(s, u)
    assert abs(float(m1[0] - m0[0])) < 1e-13 * float(m0[0])
    assert abs(float(m1[3] - m0[3])) < 1e-13 * float(m0[3])


def test_fallback_that_is_still_inadmissible_is_reported():
    nc, lo, hi = (8, 4), (-1.0, -0.5), (1.0, 0.5)
    s, _ = make(nc, 2, lo, hi, 'wall')
    lim = Limiter(s, floor=0.39)  # above the zero-slope scheme's minimum pressure at step 3
    u, rep = double_rarefaction(s, lim, nc, lo, hi)
    oks = []
    for _ in range(3):
        u, tr, rep, ok = lim.step(u, rep, s.cfl_dt(u))
        oks.append(ok)
    assert not all(oks) and lim.last_fallback
