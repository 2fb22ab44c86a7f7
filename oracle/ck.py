"""Brute-force Cauchy-Kowalevski predictor for a LINEAR PDE on one cell (oracle; test
infrastructure only).

For linear problems the paper evaluates the space-time predictor "directly by the
Cauchy-Kovalevsky algorithm" (Sec. 3.3): time derivatives are replaced by repeated applications
of the spatial operator, q(t^n + tau dt) = sum_{k<=N} (tau dt)^k / k! L^k u.  Here L is assembled
as a dense matrix from Kronecker products of the 1-D collocation derivative with the constant
coefficient matrices A_d of  dq/dt + sum_d A_d dq/dx_d = 0 (so L = -sum_d (1/h_d) D_d (x) A_d),
independently of the Picard code, and is also used to build the dense space-time system that the
converged Picard iteration must solve.
"""
import math
import torch


def spatial_operator(D1, A, h):
    """Dense L acting on flattened u[node (z,y,x order, x fastest), var]: shape [n^d nv, n^d nv].

    D1: [n, n] collocation derivative; A: list over directions of [nv, nv]; h: cell widths."""
    dim = len(A)
    n = D1.shape[0]
    nv = A[0].shape[0]
    eye = torch.eye(n, dtype=torch.float64)
    L = torch.zeros((n ** dim * nv, n ** dim * nv), dtype=torch.float64)
    for d in range(dim):
        # node axes in memory order (z, y, x): direction d sits at position dim-1-d
        op = None
        for pos in range(dim):
            f = D1 if pos == dim - 1 - d else eye
            op = f if op is None else torch.kron(op, f)
        L = L - torch.kron(op, A[d]) / h[d]
    return L


def ck_predictor(u, L, dt, tau, order):
    """q at the relative times ``tau`` (list in [0,1]): sum_{k<=order} (tau dt)^k / k! L^k u.
    ``u`` flattened [n^d nv].  Returns [len(tau), n^d nv]."""
    terms = [u]
    for k in range(1, order + 1):
        terms.append(L @ terms[-1])
    out = []
    for t in tau:
        s = torch.zeros_like(u)
        for k, v in enumerate(terms):
            s = s + (t * dt) ** k / math.factorial(k) * v
        out.append(s)
    return torch.stack(out)


def dense_spacetime_solve(K1, w, e0, L, u, dt):
    """Direct solution of the linear element-local space-time system
    (K1 (x) I - dt diag(w) (x) L) q = e0 (x) u  (Eq. (5) with R = L q)."""
    nt = K1.shape[0]
    m = u.shape[0]
    A = torch.kron(K1, torch.eye(m, dtype=torch.float64)) - dt * torch.kron(torch.diag(w), L)
    b = torch.kron(e0, u)
    return torch.linalg.solve(A, b).reshape(nt, m)
