"""Pins for the oracle's whole ADER-DG step (Sec. 3.3-3.4): weak = strong corrector, exact upwind
limits, free-stream preservation, conservation, symmetry, convergence order N+1 on exact
solutions, energy decay with absorbing boundaries, von Neumann stability of the chosen CFL
factors, and closed forms for the point source and the receivers."""
import math

import numpy as np
import pytest
import torch

from oracle.aderdg import ADERDG, Grid, PointSource
from oracle.pde import Advection, AdvectionNCP, Elastic, Euler
from oracle.refelem import gauss_legendre
from paper_1905_07987_gb300 import synth

T = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float64)


def periodic(dim):
    return [('periodic', 'periodic')] * dim


def make(pde, ncell, N, lo=None, hi=None, bc=None, mat=None, cfl=None):
    dim = len(ncell)
    lo = lo or (0.0,) * dim
    hi = hi or (1.0,) * dim
    g = Grid(ncell, lo, hi, bc or periodic(dim))
    return ADERDG(pde, g, N, cfl=cfl if cfl is not None else synth.cfl_number(N), material=mat)


def coords(s):
    return synth.node_coordinates(s.ref.x.numpy(), s.grid.ncell, s.grid.lo, s.grid.hi)


def test_synth_coordinates_follow_the_state_layout():
    s = make(Euler(3), (3, 2, 2), 2)
    Xo = s.node_coords()
    Xs = coords(s)
    for d in range(3):
        assert np.allclose(Xo[d].numpy(), Xs[d])


def cell_integral(s, u):
    W = s.tensor_basis_weights()
    vol = 1.0
    for h in s.grid.h:
        vol *= h
    return (u * W[None, ..., None]).sum(dim=tuple(range(0, s.D + 1))) * vol


@pytest.mark.parametrize("dim,N", [(2, 3), (3, 2)])
def test_free_stream_preserved(dim, N):
    s = make(Euler(dim), (3,) * dim, N)
    u = T(synth.constant_state(coords(s)))
    u1 = s.step(u, s.cfl_dt(u))
    assert torch.allclose(u1, u, atol=2e-15 * float(u.abs().max()), rtol=0)
    # and at a reflecting wall the at-rest state is preserved
    s = make(Euler(dim), (3,) * dim, N, bc=[('wall', 'wall')] * dim)
    u = T(synth.constant_state(coords(s), vel=[0.0] * dim))
    u1 = s.step(u, s.cfl_dt(u))
    assert torch.allclose(u1, u, atol=2e-15 * float(u.abs().max()), rtol=0)


def test_weak_form_equals_strong_form():
    """Eq. (6) integrated by parts once more: the nodal strong form the oracle uses must equal
    the weak form  w_j du_j = dt/h sum_d [ sum_m w_m D[m, j_d] Fbar(m) - e1_j G+ + e0_j G- ]."""
    s = make(Euler(2), (4, 3), 3)
    X = coords(s)
    rho = 1.0 + 0.3 * np.sin(2 * math.pi * X[0]) * np.cos(2 * math.pi * X[1])
    u = T(synth.euler_conserved(rho, [0.4 + 0.1 * np.cos(2 * math.pi * X[1]), -0.3], 1.0 + 0.2 * rho))
    dt = s.cfl_dt(u)
    u1, info = s.step(u, dt, details=True)
    ref = s.ref
    weak = torch.zeros_like(u)
    for d in range(2):
        ax = s.sax(d)
        Fb = info['Fbar'][d]
        # sum_m w_m D[m, j] F(m) along axis ax
        M = (ref.D * ref.w[:, None]).T  # M[j, m] = w_m D[m, j]
        vol = torch.movedim(torch.tensordot(Fb, M, dims=([ax], [1])), -1, ax)
        PhiL, PhiR = info['fluxes'][d]
        shape = [1] * (s.D + 2)
        shape[ax] = s.n
        face = ref.e1.reshape(shape) * PhiL.unsqueeze(ax) - ref.e0.reshape(shape) * PhiR.unsqueeze(ax)
        weak = weak + dt / s.grid.h[d] * (vol - face) / ref.w.reshape(shape)
    assert torch.allclose(u1 - u, weak, atol=1e-13, rtol=0)


def test_rusanov_is_exact_upwind_for_advection():
    s = make(Advection([0.7, 0.0]), (4, 1), 2)
    qL = torch.rand(5, 3, 1, dtype=torch.float64)
    qR = torch.rand(5, 3, 1, dtype=torch.float64)
    GL, GR = s.riemann(0, qL, qR, 0.7 * qL, 0.7 * qR)
    assert torch.allclose(GL, 0.7 * qL, atol=1e-15) and torch.allclose(GR, GL)


def test_ncp_fluctuations_are_exact_upwind():
    s = make(AdvectionNCP([0.6, 0.0]), (4, 1), 2)
    qL = torch.rand(5, 3, 1, dtype=torch.float64)
    qR = torch.rand(5, 3, 1, dtype=torch.float64)
    z = torch.zeros_like(qL)
    PhiL, PhiR = s.riemann(0, qL, qR, z, z, torch.zeros(5, 1, dtype=torch.float64),
                           torch.zeros(5, 1, dtype=torch.float64))
    assert torch.allclose(PhiL, z, atol=1e-15)              # nothing to the upwind cell
    assert torch.allclose(-PhiR, 0.6 * (qR - qL), atol=1e-15)  # a dq to the downwind cell


@pytest.mark.parametrize("N", [1, 3])
def test_ncp_scheme_equals_conservative_scheme_for_constant_speed(N):
    a = [0.8, -0.5]
    s1 = make(Advection(a), (4, 3), N)
    s2 = make(AdvectionNCP(a), (4, 3), N)
    X = coords(s1)
    u = T(np.sin(2 * math.pi * X[0]) * np.cos(2 * math.pi * X[1]))[..., None]
    dt = s1.cfl_dt(u)
    assert torch.allclose(s1.step(u, dt), s2.step(u, dt), atol=1e-14)


def test_elastic_fluctuations_sum_to_the_jump_term_homogeneous():
    s = make(Elastic(), (2, 2, 2), 2, mat=T(np.tile([2.7, 30.0, 25.0], (8, 1))))
    m = T(np.tile([2.7, 30.0, 25.0], (6, 1)))
    qL = torch.rand(6, 3, 3, 9, dtype=torch.float64)
    qR = torch.rand(6, 3, 3, 9, dtype=torch.float64)
    z = torch.zeros_like(qL)
    for d in range(3):
        PhiL, PhiR = s.riemann(d, qL, qR, z, z, m, m)
        B = Elastic().ncp_matrix(m, d)
        jump = torch.einsum('cij,c...j->c...i', B, qR - qL)
        assert torch.allclose(PhiL - PhiR, jump, atol=1e-12)


def test_conservation_periodic_euler():
    s = make(Euler(2), (5, 4), 3)
    X = coords(s)
    g = np.random.default_rng(1)
    rho = 1.0 + 0.2 * np.sin(2 * math.pi * X[0] + 1.0) + 0.05 * g.standard_normal(X[0].shape)
    u = T(synth.euler_conserved(rho, [0.5 + 0.1 * np.sin(2 * math.pi * X[1]), 0.2], 1.0))
    m0 = cell_integral(s, u)
    t = 0.0
    for _ in range(5):
        dt = s.cfl_dt(u)
        u = s.step(u, dt, t)
        t += float(dt)
    m1 = cell_integral(s, u)
    assert torch.allclose(m0, m1, atol=1e-14 * float(m0.abs().max()), rtol=0)


def test_wall_conserves_mass_energy_and_keeps_mirror_symmetry():
    s = make(Euler(2), (6, 6), 2, lo=(-1, -1), hi=(1, 1), bc=[('wall', 'wall')] * 2)
    X = coords(s)
    r2 = X[0] ** 2 + X[1] ** 2
    u = T(synth.euler_conserved(1.0 + 0.5 * np.exp(-8 * r2), [0.0, 0.0], 1.0 + np.exp(-8 * r2)))
    m0 = cell_integral(s, u)
    for _ in range(4):
        u = s.step(u, s.cfl_dt(u))
    m1 = cell_integral(s, u)
    for v in (0, 3):
        assert abs(float(m1[v] - m0[v])) < 1e-13 * abs(float(m0[v]))
    # mirror x -> -x: rho symmetric, jx antisymmetric
    uu = u.reshape(6, 6, 3, 3, 4)  # [cy, cx, ny, nx, v]
    flip = uu.flip(1).flip(3)
    assert torch.allclose(uu[..., 0], flip[..., 0], atol=1e-13)
    assert torch.allclose(uu[..., 1], -flip[..., 1], atol=1e-13)


def test_diagonal_wave_is_symmetric_in_x_and_y():
    s = make(Euler(2), (5, 5), 2)
    u = T(synth.entropy_wave(coords(s)))
    for _ in range(3):
        u = s.step(u, s.cfl_dt(u))
    uu = u.reshape(5, 5, 3, 3, 4)
    sw = uu.transpose(0, 1).transpose(2, 3)
    assert torch.allclose(uu[..., 0], sw[..., 0], atol=1e-13)
    assert torch.allclose(uu[..., 1], sw[..., 2], atol=1e-13)


def l2_error(s, u, exact_fn, var=0):
    """L2 error with (N+2)-point Gauss-Legendre quadrature per cell (avoids nodal superconvergence)."""
    xq, wq = gauss_legendre(s.N + 2)
    xq = xq.astype(float)
    wq = T(wq.astype(float))
    V = s.ref.values_at(xq)
    uq = u[..., var]
    for d in range(s.D):
        uq = torch.movedim(torch.tensordot(uq, V, dims=([s.sax(d)], [1])), -1, s.sax(d))
    Xq = synth.node_coordinates(xq, s.grid.ncell, s.grid.lo, s.grid.hi)
    ex = T(exact_fn(Xq))
    W = None
    for d in reversed(range(s.D)):
        W = wq if W is None else torch.einsum('...,m->...m', W, wq)
    vol = 1.0
    for h in s.grid.h:
        vol *= h
    return math.sqrt(float((W * (uq - ex) ** 2).sum()) * vol)


@pytest.mark.parametrize("N,grids,min_rate", [(1, (8, 16), 1.8), (2, (8, 16), 2.6), (3, (6, 12), 3.6)])
def test_euler_2d_converges_at_order_N_plus_1(N, grids, min_rate):
    errs = []
    for nc in grids:
        s = make(Euler(2), (nc, nc), N)
        u = T(synth.entropy_wave(coords(s)))
        u, t = s.run(u, None, t_end=0.1)
        errs.append(l2_error(s, u, lambda X: synth.entropy_wave(X, t)[..., 0]))
    rate = math.log2(errs[0] / errs[1])
    assert rate > min_rate, (errs, rate)


def test_euler_3d_converges():
    errs = []
    for nc in (4, 8):
        s = make(Euler(3), (nc,) * 3, 3)
        u = T(synth.entropy_wave(coords(s)))
        u, t = s.run(u, None, t_end=0.05)
        errs.append(l2_error(s, u, lambda X: synth.entropy_wave(X, t)[..., 0]))
    assert math.log2(errs[0] / errs[1]) > 3.6, errs


@pytest.mark.parametrize("kind", ['p', 's'])
def test_elastic_plane_wave_converges(kind):
    mat = [2.7, 30.0, 25.0]
    errs = []
    for nc in (4, 8):
        s = make(Elastic(), (nc, 1, 1), 2, hi=(1.0, 1.0 / nc, 1.0 / nc),
                 mat=T(np.tile(mat, (nc, 1))))
        u = T(synth.plane_wave_elastic(coords(s), mat, kind=kind))
        u, t = s.run(u, None, t_end=0.05)
        errs.append(l2_error(s, u, lambda X: synth.plane_wave_elastic(X, mat, t, kind=kind)[..., 0 if kind == 'p' else 1],
                             var=0 if kind == 'p' else 1))
    assert math.log2(errs[0] / errs[1]) > 2.5, errs


def test_elastic_energy_does_not_grow_with_absorbing_boundaries():
    ncell = (3, 3, 3)
    mat = T(synth.elastic_material(ncell, seed=4))
    s = make(Elastic(), ncell, 2, hi=(1.5, 1.5, 1.5), bc=[('absorbing', 'absorbing')] * 3, mat=mat)
    X = coords(s)
    bump = np.exp(-10 * ((X[0] - 0.75) ** 2 + (X[1] - 0.7) ** 2 + (X[2] - 0.8) ** 2))
    u = T(np.stack([bump, 0.5 * bump, 0 * bump] + [0.3 * bump] * 6, -1))
    W = s.tensor_basis_weights()

    def energy(u):
        m = mat.reshape(-1, 1, 1, 1, 3).expand(-1, 3, 3, 3, 3)
        return float((Elastic.energy_density(u, m) * W).sum())

    e = [energy(u)]
    for _ in range(12):
        u = s.step(u, s.cfl_dt(u))
        e.append(energy(u))
    assert all(e[i + 1] <= e[i] * (1 + 1e-12) for i in range(len(e) - 1)), e
    assert e[-1] < e[0]


def amplification(N, nu):
    """Largest |eigenvalue| over wavenumbers of the one-step operator of 1-D advection at Courant
    number nu (von Neumann analysis from the oracle's own step applied to unit vectors)."""
    g = Grid((3,), (0.0,), (3.0,), periodic(1))
    s = ADERDG(Advection([1.0]), g, N)
    n = N + 1
    A = torch.zeros(3, n, n, dtype=torch.float64)
    for m in range(n):
        u = torch.zeros(3, n, 1, dtype=torch.float64)
        u[1, m, 0] = 1.0
        un = s.step(u, torch.tensor(nu, dtype=torch.float64))
        for c in range(3):
            A[c][:, m] = un[c, :, 0]
    A = A.to(torch.complex128)
    r = 0.0
    for th in np.linspace(0, math.pi, 181):
        G = A[1] + A[0] * complex(math.cos(th), math.sin(th)) + A[2] * complex(math.cos(th), -math.sin(th))
        r = max(r, float(torch.linalg.eigvals(G).abs().max()))
    return r


@pytest.mark.parametrize("N", [1, 2, 3])
def test_cfl_factor_is_stable_and_literal_eq7_is_not(N):
    """The workloads' time-step factor (0.9 KAPPA[N] in Eq. (7)) is von Neumann stable; for N >= 2
    Eq. (7) with CFL_N = 0.9 and no order-dependent factor is not."""
    nu = synth.cfl_number(N) / (2 * N + 1)
    assert amplification(N, nu) <= 1 + 1e-12
    if N >= 2:
        assert amplification(N, 0.9 / (2 * N + 1)) > 1 + 1e-3


def test_point_source_injects_the_time_integral_of_the_wavelet():
    """Testing the delta source against the basis: the integral of the update over the domain is
    -M_a times the integral of the Ricker wavelet over the step, int R = [tau exp(-pi^2 f0^2 tau^2)]."""
    ncell = (2, 2, 2)
    mat = T(np.tile([2.7, 30.0, 25.0], (8, 1)))
    s = make(Elastic(), ncell, 3, hi=(1.0, 1.0, 1.0), mat=mat)
    M = T([1.0, -0.5, 0.25, 0.7, -0.3, 0.2])
    s.set_point_source(PointSource(cell=5, xi=(0.3, 0.6, 0.45), M=M, f0=2.0, t0=0.5))
    u = torch.zeros([8, 4, 4, 4, 9], dtype=torch.float64)
    t, dt = 0.41, 0.02
    u1 = s.step(u, torch.tensor(dt, dtype=torch.float64), t)
    tot = cell_integral(s, u1)
    a = (math.pi * 2.0) ** 2
    F = lambda x: (x - 0.5) * math.exp(-a * (x - 0.5) ** 2)
    integral = F(t + dt) - F(t)
    for k, var in enumerate(range(3, 9)):
        assert abs(float(tot[var]) - (-float(M[k]) * integral)) < 1e-10
    assert float(tot[:3].abs().max()) < 1e-15


def test_receiver_reads_the_polynomial():
    ncell = (2, 2, 2)
    s = make(Elastic(), ncell, 3, mat=T(np.tile([2.7, 30.0, 25.0], (8, 1))))
    X = coords(s)
    f = lambda x, y, z: 1 + x - 2 * y * y + x * y * z + z ** 3
    u = np.zeros(X[0].shape + (9,))
    u[..., 0] = f(X[0], X[1], X[2])
    u[..., 2] = 2 * f(X[0], X[1], X[2])
    pts = [(0.3, 0.8, 1.0), (0.9, 0.1, 0.45)]
    cells, xis = [], []
    for p in pts:
        c, xi = synth.locate(p, ncell, (0, 0, 0), (1, 1, 1))
        cells.append(c)
        xis.append(xi)
    s.set_receivers(cells, xis)
    rec = s.record(T(u))
    for i, p in enumerate(pts):
        assert abs(float(rec[i, 0]) - f(*p)) < 1e-13
        assert abs(float(rec[i, 2]) - 2 * f(*p)) < 1e-13


def test_cfl_time_step_closed_form():
    s = make(Euler(3), (4, 4, 4), 4)
    u = T(synth.constant_state(coords(s), rho=1.3, vel=[0.5, -0.9, 0.2], p=0.8))
    c = math.sqrt(1.4 * 0.8 / 1.3)
    lam = 0.9 + c
    assert abs(float(s.cfl_dt(u)) - synth.cfl_number(4) / (3 * 9) * 0.25 / lam) < 1e-15


def test_elastic_plane_wave_converges_with_the_ck_predictor():
    """The Cauchy-Kowalevski form of the scheme keeps order N+1 on an exact plane P wave."""
    mat = [2.7, 30.0, 25.0]
    errs = []
    for nc in (4, 8):
        g = Grid((nc, 1, 1), (0.0,) * 3, (1.0, 1.0 / nc, 1.0 / nc), periodic(3))
        s = ADERDG(Elastic(), g, 2, cfl=synth.cfl_number(2), material=T(np.tile(mat, (nc, 1))),
                   predictor="ck")
        u = T(synth.plane_wave_elastic(coords(s), mat, kind='p'))
        u, t = s.run(u, None, t_end=0.05)
        errs.append(l2_error(s, u, lambda X: synth.plane_wave_elastic(X, mat, t, kind='p')[..., 0], var=0))
    assert math.log2(errs[0] / errs[1]) > 2.5, errs


def test_euler_2d_with_the_cerk_guess_and_one_iteration_keeps_order_N_plus_1():
    """Order 3 (N+1 = 4) with the continuous extension Runge-Kutta guess (order 4 in dt) and a
    single Picard iteration instead of N+1 = 4."""
    errs = []
    for nc in (6, 12):
        g = Grid((nc, nc), (0.0, 0.0), (1.0, 1.0), periodic(2))
        s = ADERDG(Euler(2), g, 3, cfl=synth.cfl_number(3), picard_iters=1, initial_guess="cerk")
        u = T(synth.entropy_wave(coords(s)))
        u, t = s.run(u, None, t_end=0.1)
        errs.append(l2_error(s, u, lambda X: synth.entropy_wave(X, t)[..., 0]))
    rate = math.log2(errs[0] / errs[1])
    assert rate > 3.6, (errs, rate)
