"""Reference element on [0,1] (oracle; test infrastructure only).

The discrete solution of Sec. 3.3 is a tensor product of one-dimensional Lagrange polynomials
through Gauss-Legendre points (the paragraph after Eq. (5)).  Everything here is one-dimensional;
the d-dimensional operators are tensor products applied axis by axis.

Nodes come from Newton's method on the three-term Legendre recurrence, carried out in
``numpy.longdouble``; basis values and derivatives come from the Lagrange product formula
and its product-rule derivative.  No barycentric formulas, no eigen-solvers.
"""
import numpy as np
import torch

LD = np.longdouble


def gauss_legendre(n):
    """n-point Gauss-Legendre rule mapped to [0,1]: ascending nodes x and weights w, sum(w)=1.

    Newton's method on P_n(t) for t in [-1,1], with P_n and P_n' from the recurrence
    (k+1) P_{k+1} = (2k+1) t P_k - k P_{k-1} and P_n'(t) = n (t P_n - P_{n-1}) / (t^2 - 1);
    weights 2 / ((1 - t^2) P_n'(t)^2).  Then x = (t+1)/2 and w -> w/2.
    """
    t_all, w_all = [], []
    for i in range(n):
        t = LD(np.cos(np.pi * (i + 0.75) / (n + 0.5)))
        for _ in range(100):
            p_prev, p = LD(1), t
            for k in range(1, n):
                p_prev, p = p, ((2 * k + 1) * t * p - k * p_prev) / (k + 1)
            if n == 1:
                p_prev, p = LD(1), t
            dp = n * (t * p - p_prev) / (t * t - 1)
            step = p / dp
            t = t - step
            if abs(step) < LD(1e-30):
                break
        p_prev, p = LD(1), t
        for k in range(1, n):
            p_prev, p = p, ((2 * k + 1) * t * p - k * p_prev) / (k + 1)
        dp = n * (t * p - p_prev) / (t * t - 1)
        t_all.append(t)
        w_all.append(LD(2) / ((1 - t * t) * dp * dp))
    t_all = np.array(t_all, dtype=LD)
    w_all = np.array(w_all, dtype=LD)
    order = np.argsort(t_all)
    x = (t_all[order] + 1) / 2
    w = w_all[order] / 2
    return x, w


def lagrange_values(nodes, xi):
    """phi_m(xi) for every node m: product over k != m of (xi - x_k) / (x_m - x_k).

    ``nodes`` and ``xi`` are longdouble arrays; result [len(xi), len(nodes)].
    """
    n = len(nodes)
    out = np.ones((len(xi), n), dtype=LD)
    for m in range(n):
        for k in range(n):
            if k != m:
                out[:, m] *= (xi - nodes[k]) / (nodes[m] - nodes[k])
    return out


def lagrange_derivatives(nodes, xi):
    """phi_m'(xi) by the product rule: sum over l != m of 1/(x_m - x_l) times the product over
    k != m, l of (xi - x_k)/(x_m - x_k).  Result [len(xi), len(nodes)]."""
    n = len(nodes)
    out = np.zeros((len(xi), n), dtype=LD)
    for m in range(n):
        for l in range(n):
            if l == m:
                continue
            term = np.full(len(xi), LD(1) / (nodes[m] - nodes[l]), dtype=LD)
            for k in range(n):
                if k != m and k != l:
                    term *= (xi - nodes[k]) / (nodes[m] - nodes[k])
            out[:, m] += term
    return out


def _t(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), dtype=torch.float64)


class RefElement:
    """One-dimensional tables of the order-N scheme (n = N+1 Gauss-Legendre nodes on [0,1]).

    x, w   nodes and weights (sum w = 1)
    D      D[i, m] = phi_m'(x_i)         (collocation derivative, exact for degree <= N)
    e0, e1 phi_m(0), phi_m(1)            (extrapolation to the left / right end)
    K1     K1[k, l] = e1[k] e1[l] - w[l] D[l, k]
           Time part of the element-local space-time weak form, Eq. (5) of Sec. 3.3: the time
           derivative is integrated by parts, the value at the start of the interval is taken
           from the old solution (upwinding in time), quadrature at the same nodes.  The
           predictor solves  sum_l K1[k,l] q_l = e0[k] u + dt w[k] R(q)_k.
    ns     number of FV subcells per direction, 2N+1 (Sec. 3.5)
    P1     P1[s, m] = average of phi_m over subcell s  (DG -> subcell averages)
    R1     constrained least-squares left inverse of P1 preserving the cell mean
           (subcell averages -> DG); R1 P1 = I.
    """

    def __init__(self, order):
        self.N = order
        n = order + 1
        self.n = n
        x, w = gauss_legendre(n)
        self._xl, self._wl = x, w
        D = lagrange_derivatives(x, x)
        e0 = lagrange_values(x, np.array([LD(0)], dtype=LD))[0]
        e1 = lagrange_values(x, np.array([LD(1)], dtype=LD))[0]
        K1 = np.outer(e1, e1) - (w[None, :] * D.T)
        self.x, self.w, self.D = _t(x), _t(w), _t(D)
        self.e0, self.e1, self.K1 = _t(e0), _t(e1), _t(K1)
        # FV subcells, Sec. 3.5: (2N+1) subcells per direction.
        ns = 2 * order + 1
        self.ns = ns
        P1 = np.zeros((ns, n), dtype=LD)
        for s in range(ns):
            pts = (s + x) / ns  # same n-point rule on the subinterval, exact for degree <= 2N+1
            P1[s, :] = (w[:, None] * lagrange_values(x, pts)).sum(axis=0)
        self.P1 = _t(P1)
        # R1: minimise |P1 u - U|^2 subject to w.u = mean(U).  KKT system
        #   [2 P1^T P1  w] [u ]   [2 P1^T U   ]
        #   [w^T        0] [mu] = [1^T U / ns ]
        P1d = P1.astype(np.float64)
        wd = w.astype(np.float64)
        kkt = np.zeros((n + 1, n + 1))
        kkt[:n, :n] = 2 * P1d.T @ P1d
        kkt[:n, n] = wd
        kkt[n, :n] = wd
        rhs = np.zeros((n + 1, ns))
        rhs[:n, :] = 2 * P1d.T
        rhs[n, :] = 1.0 / ns
        self.R1 = _t(np.linalg.solve(kkt, rhs)[:n, :])

    def values_at(self, xi):
        """phi_m(xi) for points xi in [0,1]: float64 tensor [len(xi), n]."""
        xi = np.asarray(xi, dtype=LD).reshape(-1)
        return _t(lagrange_values(self._xl, xi))

    def derivatives_at(self, xi):
        xi = np.asarray(xi, dtype=LD).reshape(-1)
        return _t(lagrange_derivatives(self._xl, xi))
