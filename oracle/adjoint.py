"""Adjoint of the linear-elastic ADER-DG step (oracle; test infrastructure only).

With a fixed dt the elastic step is affine in the state and in the moment tensor:
u^{n+1} = A(m) u^n + b^n(M, m).  The adjoint step maps lambda^{n+1} to
lambda^n = A(m)^T lambda^{n+1} (+ dJ/du^n) and accumulates the gradients
(lambda^{n+1})^T d(A u^n + b^n)/dm  per cell (rho, lambda, mu)  and  (lambda^{n+1})^T db^n/dM.
Here these vector-Jacobian products are taken by reverse-mode automatic differentiation of the
oracle's own forward step (a library primitive standing in for the hand derivation); the tests
pin them against finite differences, a dot-product identity and a densely assembled A.
"""
import torch

from .aderdg import PointSource


def step_vjp(solver, u_n, lam, dt, t=0.0):
    """(lambda^n without dJ/du^n, dJ/dmaterial [C,3], dJ/dM [6]) for one step."""
    mat0 = solver.mat
    src0 = solver.source
    mat = mat0.detach().clone().requires_grad_(True)
    solver.mat = mat
    inputs = [u_n.detach().clone().requires_grad_(True), mat]
    if src0 is not None:
        M = src0.M.detach().clone().requires_grad_(True)
        solver.source = PointSource(src0.cell, src0.xi, M, src0.f0, src0.t0, src0.vars)
        inputs.append(M)
    try:
        out = solver.step(inputs[0], torch.as_tensor(dt, dtype=torch.float64), t)
        grads = torch.autograd.grad(out, inputs, grad_outputs=lam, allow_unused=True)
    finally:
        solver.mat = mat0
        solver.source = src0
    gu = grads[0]
    gm = grads[1] if grads[1] is not None else torch.zeros_like(mat0)
    gM = grads[2] if len(grads) > 2 and grads[2] is not None else torch.zeros(6, dtype=torch.float64)
    return gu.detach(), gm.detach(), gM.detach()


def misfit(solver, u0, steps, dt, obs, t0=0.0):
    """J = 1/2 sum_k dt |v_rec(u^{k+1}) - obs[k]|^2 over the receivers, forward in time."""
    u = u0
    t = t0
    J = 0.0
    for k in range(steps):
        u = solver.step(u, torch.as_tensor(dt, dtype=torch.float64), t)
        t += dt
        r = solver.record(u) - obs[k]
        J = J + 0.5 * dt * (r * r).sum()
    return J
