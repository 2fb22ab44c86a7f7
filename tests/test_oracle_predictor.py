"""Pins for the oracle's space-time predictor (Eq. (5), Sec. 3.3): exact polynomial solutions,
the dense direct solve of the same system, and an independent Cauchy-Kowalevski expansion."""
import math

import pytest
import torch

from oracle.aderdg import ADERDG, Grid
from oracle.ck import ck_predictor, dense_spacetime_solve, spatial_operator
from oracle.pde import Advection, AdvectionNCP, Elastic
from paper_1905_07987_gb300 import synth


def poly(X, N, seed):
    """A random polynomial of total degree <= N in the node coordinates."""
    g = torch.Generator().manual_seed(seed)
    D = len(X)
    out = torch.zeros_like(X[0])
    import itertools
    for exps in itertools.product(range(N + 1), repeat=D):
        if sum(exps) <= N:
            c = float(torch.rand(1, generator=g)) * 2 - 1
            term = torch.ones_like(X[0])
            for d in range(D):
                term = term * X[d] ** exps[d]
            out = out + c * term
    return out


@pytest.mark.parametrize("dim,N", [(2, 1), (2, 3), (3, 2), (3, 4)])
def test_picard_exact_for_polynomial_data(dim, N):
    """Linear constant-coefficient PDE and data of total degree <= N: the exact solution is a
    degree-N polynomial in time, which the collocated time weak form reproduces exactly; the
    default N+1 Picard iterations reach it at every space-time node."""
    a = [0.7, -0.4, 0.25][:dim]
    g = Grid((2,) * dim, (0.0,) * dim, (1.0,) * dim, [('periodic', 'periodic')] * dim)
    s = ADERDG(Advection(a), g, N)
    X = s.node_coords()
    u = poly(X, N, 7)[..., None]
    dt = 0.03
    q = s.predictor(u, dt)
    for k in range(N + 1):
        t = float(s.ref.x[k]) * dt
        Xs = [X[d] - a[d] * t for d in range(dim)]
        assert torch.allclose(q[:, k, ..., 0], poly(Xs, N, 7), atol=1e-12)
    # each iteration adds one degree in time: N-1 iterations are not exact
    q_short = s.predictor(u, dt, iters=N - 1)
    assert (q_short - q).abs().max() > 1e-10


def _cell_ops(N, dim, pde, mat=None, h=0.5):
    s = ADERDG(pde, Grid((1,) * dim, (0.0,) * dim, (h,) * dim, [('periodic', 'periodic')] * dim), N,
               material=mat)
    if isinstance(pde, Elastic):
        A = [pde.ncp_matrix(mat, d)[0] for d in range(dim)]
    else:
        A = [torch.tensor([[pde.a[d]]], dtype=torch.float64) for d in range(dim)]
    L = spatial_operator(s.ref.D, A, [h] * dim)
    return s, L


@pytest.mark.parametrize("N", [2, 3])
def test_picard_converges_to_dense_solve_elastic(N):
    mat = torch.tensor([[2.7, 30.0, 25.0]], dtype=torch.float64)
    s, L = _cell_ops(N, 3, Elastic(), mat)
    g = torch.Generator().manual_seed(3)
    u = torch.rand([1] + [N + 1] * 3 + [9], generator=g, dtype=torch.float64) - 0.5
    dt = 0.02 * 0.5 / 5.0
    q = s.predictor(u, dt, iters=60)
    qd = dense_spacetime_solve(s.ref.K1, s.ref.w, s.ref.e0, L, u.reshape(-1), dt)
    assert torch.allclose(q.reshape(N + 1, -1), qd, atol=1e-13 * float(u.abs().max()) * 10)


@pytest.mark.parametrize("N", [2, 4])
def test_ck_equals_picard_for_polynomial_data(N):
    a = [0.6, -0.3]
    s, L = _cell_ops(N, 2, Advection(a), h=1.0)
    X = s.node_coords()
    u = poly(X, N, 11)[..., None]
    dt = 0.05
    q = s.predictor(u, dt)
    qck = ck_predictor(u.reshape(-1), L, dt, [float(v) for v in s.ref.x], N)
    assert torch.allclose(q.reshape(N + 1, -1), qck, atol=1e-13)


@pytest.mark.parametrize("N", [2, 3])
def test_ck_minus_picard_is_order_dt_to_the_N_plus_1(N):
    """For general data the two predictors differ by O(dt^(N+1)) (both are order N+1 in time)."""
    mat = torch.tensor([[2.5, 20.0, 20.0]], dtype=torch.float64)
    s, L = _cell_ops(N, 3, Elastic(), mat)
    g = torch.Generator().manual_seed(5)
    u = torch.rand([1] + [N + 1] * 3 + [9], generator=g, dtype=torch.float64) - 0.5
    errs = []
    for dt in (2e-3, 1e-3, 5e-4):
        q = s.predictor(u, dt)
        qck = ck_predictor(u.reshape(-1), L, dt, [float(v) for v in s.ref.x], N)
        errs.append(float((q.reshape(N + 1, -1) - qck).abs().max()))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > N + 1 - 0.3, (errs, rates)


def test_ncp_predictor_matches_conservative_for_constant_speed():
    """dq/dt + a.grad q written as a flux or as a non-conservative product gives the same predictor."""
    a = [0.8, -0.5]
    g = Grid((3, 2), (0, 0), (1, 1), [('periodic', 'periodic')] * 2)
    s1 = ADERDG(Advection(a), g, 3)
    s2 = ADERDG(AdvectionNCP(a), g, 3)
    X = s1.node_coords()
    u = torch.sin(2 * math.pi * X[0]) * torch.cos(2 * math.pi * X[1])
    u = u[..., None]
    assert torch.allclose(s1.predictor(u, 0.01), s2.predictor(u, 0.01), atol=1e-14)


# ---- the scheme's Cauchy-Kowalevski predictor (linear PDEs, Sec. 2 and Sec. 3.3) -------------

@pytest.mark.parametrize("N", [2, 4])
def test_scheme_ck_predictor_equals_dense_ck_elastic(N):
    """Taylor recursion with the sum-factorised operator = the dense Kronecker-assembled expansion."""
    mat = torch.tensor([[2.7, 30.0, 25.0]], dtype=torch.float64)
    s, L = _cell_ops(N, 3, Elastic(), mat)
    g = torch.Generator().manual_seed(21)
    u = torch.rand([1] + [N + 1] * 3 + [9], generator=g, dtype=torch.float64) - 0.5
    dt = 0.004
    q = s.predictor_ck(u, dt)
    qck = ck_predictor(u.reshape(-1), L, dt, [float(v) for v in s.ref.x], N)
    assert torch.allclose(q.reshape(N + 1, -1), qck, atol=1e-13 * float(qck.abs().max()))


def test_scheme_ck_predictor_equals_dense_ck_flux_form():
    N = 3
    s, L = _cell_ops(N, 2, Advection([0.6, -0.3]), h=0.5)
    g = torch.Generator().manual_seed(22)
    u = torch.rand([1, N + 1, N + 1, 1], generator=g, dtype=torch.float64) - 0.5
    q = s.predictor_ck(u, 0.03)
    qck = ck_predictor(u.reshape(-1), L, 0.03, [float(v) for v in s.ref.x], N)
    assert torch.allclose(q.reshape(N + 1, -1), qck, atol=1e-14)


@pytest.mark.parametrize("pde_cls", [Advection, AdvectionNCP])
@pytest.mark.parametrize("dim,N", [(2, 3), (3, 2)])
def test_ck_predictor_exact_for_polynomial_data(pde_cls, dim, N):
    """Data of total degree <= N: the truncated Taylor series is the exact solution u0(x - a t)."""
    a = [0.7, -0.4, 0.25][:dim]
    g = Grid((2,) * dim, (0.0,) * dim, (1.0,) * dim, [('periodic', 'periodic')] * dim)
    s = ADERDG(pde_cls(a), g, N, predictor="ck")
    X = s.node_coords()
    u = poly(X, N, 9)[..., None]
    dt = 0.03
    q = s.predictor_ck(u, dt)
    for k in range(N + 1):
        t = float(s.ref.x[k]) * dt
        Xs = [X[d] - a[d] * t for d in range(dim)]
        assert torch.allclose(q[:, k, ..., 0], poly(Xs, N, 9), atol=1e-12)


@pytest.mark.parametrize("N", [1, 2])
def test_ck_point_source_error_is_order_dt_to_the_N_plus_1(N):
    """u^n = 0 with a point source: q at the time nodes against the exact solution of the cell's
    linear ODE du/dt = L u + g R(t), the Duhamel integral of the matrix exponential (24-point
    Gauss-Legendre in time); g is read off the Picard predictor's source term.  The error falls as
    dt^(N+1) (Taylor truncation plus the degree-N interpolant of the wavelet)."""
    from oracle.aderdg import PointSource, ricker
    from oracle.refelem import gauss_legendre
    mat = torch.tensor([[2.6, 28.0, 24.0]], dtype=torch.float64)
    s, L = _cell_ops(N, 3, Elastic(), mat)
    M = torch.tensor([1.0, -0.5, 0.25, 0.7, -0.3, 0.2], dtype=torch.float64)
    s.set_point_source(PointSource(cell=0, xi=(0.3, 0.6, 0.45), M=M, f0=2.0, t0=0.5))
    t = 0.4
    tt = torch.tensor([t], dtype=torch.float64)
    gvec = (s.source_nodes(tt)[0, 0] / ricker(tt, 2.0, 0.5)[0]).reshape(-1)
    gx, gw = gauss_legendre(24)
    u0 = torch.zeros([1] + [N + 1] * 3 + [9], dtype=torch.float64)
    errs = []
    for dt in (4e-3, 2e-3, 1e-3):
        q = s.predictor_ck(u0, dt, t).reshape(N + 1, -1)
        err = 0.0
        for k in range(N + 1):
            T_ = float(s.ref.x[k]) * dt
            ex = torch.zeros_like(gvec)
            for z, wz in zip([float(v) for v in gx], [float(v) for v in gw]):
                sig = z * T_
                ex = ex + wz * T_ * float(ricker(torch.tensor(t + sig, dtype=torch.float64), 2.0, 0.5)) * (
                    torch.linalg.matrix_exp((T_ - sig) * L) @ gvec)
            err = max(err, float((q[k] - ex).abs().max()))
        errs.append(err)
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > N + 1 - 0.3, (errs, rates)


# ---- continuous extension Runge-Kutta initial guess (Sec. 5) ----------------------------------

@pytest.mark.parametrize("dim,N", [(2, 4), (3, 5)])
def test_cerk_guess_exact_for_cubic_in_time_solutions(dim, N):
    """Data of total degree <= 3 under constant advection: the exact local solution is a cubic in
    time, which the uniform-order-3 continuous extension reproduces at every time node."""
    a = [0.7, -0.4, 0.25][:dim]
    g = Grid((2,) * dim, (0.0,) * dim, (1.0,) * dim, [('periodic', 'periodic')] * dim)
    s = ADERDG(Advection(a), g, N, initial_guess="cerk")
    X = s.node_coords()
    u = poly(X, 3, 13)[..., None]
    dt = 0.04
    q0 = s.cerk_guess(u, dt)
    for k in range(N + 1):
        t = float(s.ref.x[k]) * dt
        Xs = [X[d] - a[d] * t for d in range(dim)]
        assert torch.allclose(q0[:, k, ..., 0], poly(Xs, 3, 13), atol=1e-12)


def test_cerk_guess_error_is_order_dt_to_the_4():
    """General data: the guess at the time nodes against the exact local solution exp(tau dt L) u
    of the cell's linear ODE (dense Kronecker-assembled L): error ~ dt^4."""
    N = 3
    mat = torch.tensor([[2.6, 27.0, 22.0]], dtype=torch.float64)
    s, L = _cell_ops(N, 3, Elastic(), mat)
    g = torch.Generator().manual_seed(41)
    u = torch.rand([1] + [N + 1] * 3 + [9], generator=g, dtype=torch.float64) - 0.5
    errs = []
    for dt in (2e-3, 1e-3, 5e-4):
        q0 = s.cerk_guess(u, dt).reshape(N + 1, -1)
        ex = torch.stack([torch.linalg.matrix_exp(float(x) * dt * L) @ u.reshape(-1) for x in s.ref.x])
        errs.append(float((q0 - ex).abs().max()))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 4 - 0.3, (errs, rates)


@pytest.mark.parametrize("iters", [0, 1, 2])
def test_picard_from_the_cerk_guess_gains_one_order_per_iteration(iters):
    """Distance of the predictor started from the CERK guess to the converged fixed point of
    Eq. (5) after `iters` iterations: O(dt^(4 + iters)) (the iteration contracts by O(dt))."""
    N = 5
    mat = torch.tensor([[2.6, 27.0, 22.0]], dtype=torch.float64)
    s, L = _cell_ops(N, 3, Elastic(), mat)
    g = torch.Generator().manual_seed(43)
    u = torch.rand([1] + [N + 1] * 3 + [9], generator=g, dtype=torch.float64) - 0.5
    errs = []
    for dt in (4e-3, 2e-3, 1e-3):
        qs = dense_spacetime_solve(s.ref.K1, s.ref.w, s.ref.e0, L, u.reshape(-1), dt)
        q = s.predictor(u, dt, iters=iters, guess="cerk").reshape(N + 1, -1)
        errs.append(float((q - qs).abs().max()))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 4 + iters - 0.4, (errs, rates)


def test_converged_predictor_does_not_depend_on_the_guess():
    N = 3
    mat = torch.tensor([[2.6, 27.0, 22.0]], dtype=torch.float64)
    s, _ = _cell_ops(N, 3, Elastic(), mat)
    g = torch.Generator().manual_seed(47)
    u = torch.rand([1] + [N + 1] * 3 + [9], generator=g, dtype=torch.float64) - 0.5
    a = s.predictor(u, 2e-3, iters=40, guess="constant")
    b = s.predictor(u, 2e-3, iters=40, guess="cerk")
    assert torch.allclose(a, b, atol=1e-14)
