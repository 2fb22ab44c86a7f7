"""ADER-DG time step (oracle; test infrastructure only).

Follows Sec. 3.3-3.4 of the paper in its order:

1. per cell, solve the element-local space-time weak form Eq. (5) for the predictor q_h by the
   fixed-point (discrete Picard) iteration, or, for linear PDEs, evaluate it by the
   Cauchy-Kowalevski procedure (Sec. 2 and Sec. 3.3);
2. per face, a numerical normal flux from both adjacent cells: Rusanov (Sec. 3.3, phase 2), with a
   path-conservative fluctuation for the non-conservative product B(Q).grad Q of Eq. (1);
3. per cell, the corrector Eq. (6) with a diagonal mass matrix;
plus the CFL condition Eq. (7), the point sources of Eq. (1) and receiver read-out.

Array layout (all float64):  state u[C, n, ..., n, nvar] with the D spatial node axes ordered
(z, y, x), i.e. flat node index a + n*(b + n*c) with x fastest; cell index i + nx*(j + ny*k).
The space-time predictor q[C, n_t, n, ..., n, nvar] puts time on axis 1.

Readings of the paper taken here (the paper is silent or garbled on these points):
* Gauss-Legendre nodes; reference cell [0,1]^d; predictor initial guess q^0 = u^n (constant in
  time); a fixed number of Picard iterations, N+1 by default, with no tolerance exit.
* Flux divergence in the predictor in strong (collocation) form.
* Time averages are taken node by node after the last iteration: qbar = sum_k w_k q_k,
  Fbar_d = sum_k w_k F_d(q_k), (B grad q)bar = sum_k w_k B(q_k) grad q_k.
* Face data extrapolate the nodal time-averaged polynomials (qbar and Fbar_d).
* Rusanov on time-averaged face states with ONE wave speed per face: the max over all face nodes
  and both sides of the max |eigenvalue|.
* Eq. (6) is printed with both signs flipped relative to integration by parts of Eq. (1); the
  standard form  int theta dq = int int grad theta . F - oint theta G  is used, in nodal
  strong form (so the non-conservative and source terms of Eq. (1), dropped from the paper's
  pared-down Eq. (4), are restored).
* Non-conservative faces: G = (FL + FR)/2 - s (qR - qL)/2, and the fluctuation of the straight
  segment path, Bbar_n (qR - qL) with Bbar_n = int_0^1 B_n(m_L + z (m_R - m_L)) dz by 3-point
  Gauss-Legendre, is split in halves:  left cell sees G + Bbar dq/2, right cell G - Bbar dq/2.
* Boundaries: periodic; reflecting wall (mirror state with the normal momentum negated, Euler);
  absorbing: zero exterior state for linear PDEs, transmissive copy for Euler; exterior material
  is the interior one.
* CFL: dt = CFL / (d (2N+1)) * min_d h_d / lambda_max with lambda_max over all cells, nodes and
  directions of the state at t^n.
* Continuous extension Runge-Kutta initial guess (Sec. 5 names it, gives no scheme): the
  classical four-stage Runge-Kutta method on the cell-local ODE dq/dt = R(q) with its natural
  continuous extension of uniform order 3, evaluated at the time nodes; the Picard iterations
  then start from it (their number is the scheme's ``picard_iters``).
* Cauchy-Kowalevski predictor (linear PDEs): the local solution's Taylor series in time about
  t^n, cut after degree N, with each time derivative replaced by the spatial operator applied to
  the previous one; a point source's time factor is replaced by its degree-N interpolant through
  the step's Gauss-Legendre time nodes (the samples the Picard predictor uses).  q_h is then
  evaluated at the time nodes and everything after the predictor is shared with the Picard form.
"""
import math
import torch

from .refelem import RefElement, gauss_legendre


def contract(X, M, axis):
    """Y[..., i, ...] = sum_m M[i, m] X[..., m, ...] along ``axis``."""
    Y = torch.tensordot(X, M, dims=([axis], [1]))
    return torch.movedim(Y, -1, axis)


def extrapolate(X, e, axis):
    """sum_m e[m] X[..., m, ...]: the value at one end of the interval; removes ``axis``."""
    return torch.tensordot(X, e, dims=([axis], [0]))


def ricker(t, f0, t0):
    """Ricker wavelet (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2)."""
    a = (math.pi * f0 * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * torch.exp(-a)


class Grid:
    """Uniform Cartesian grid of nx x ny (x nz) cells on [lo, hi] with per-face boundary kinds
    'periodic', 'wall' or 'absorbing' given as bc[d] = (kind_lo, kind_hi)."""

    def __init__(self, ncell, lo, hi, bc):
        self.ncell = tuple(int(v) for v in ncell)
        self.dim = len(self.ncell)
        self.lo = [float(v) for v in lo]
        self.hi = [float(v) for v in hi]
        self.bc = [tuple(b) for b in bc]
        self.h = [(self.hi[d] - self.lo[d]) / self.ncell[d] for d in range(self.dim)]
        self.C = 1
        for v in self.ncell:
            self.C *= v
        c = torch.arange(self.C)
        self.idx = []
        rem = c
        for d in range(self.dim):
            self.idx.append(rem % self.ncell[d])
            rem = rem // self.ncell[d]

    def cell_of(self, idx):
        c = torch.zeros_like(idx[0])
        stride = 1
        for d in range(self.dim):
            c = c + idx[d] * stride
            stride *= self.ncell[d]
        return c

    def neighbor(self, d, side):
        """Index of the neighbour across the face on ``side`` (+1 / -1) in direction d, or -1 if
        that face is a non-periodic domain boundary."""
        idx = [t.clone() for t in self.idx]
        j = idx[d] + side
        n = self.ncell[d]
        kind = self.bc[d][1 if side > 0 else 0]
        outside = (j < 0) | (j >= n)
        if kind == 'periodic':
            j = j % n
            outside = torch.zeros_like(outside)
        idx[d] = torch.where(outside, torch.zeros_like(j), j)
        nb = self.cell_of(idx)
        return torch.where(outside, torch.full_like(nb, -1), nb)

    def cell_center_and_lower(self):
        lower = [self.lo[d] + self.idx[d].double() * self.h[d] for d in range(self.dim)]
        return lower


class PointSource:
    """Moment-tensor point source of Eq. (1) (the delta_i terms): adds -M R(t) delta(x - x0) to the
    six stress components, R a Ricker moment-rate wavelet.  ``cell`` and ``xi`` (reference
    coordinates in [0,1]^3) locate x0."""

    def __init__(self, cell, xi, M, f0, t0, vars_=(3, 4, 5, 6, 7, 8)):
        self.cell = int(cell)
        self.xi = [float(v) for v in xi]
        self.M = M if torch.is_tensor(M) else torch.tensor(M, dtype=torch.float64)
        self.f0 = float(f0)
        self.t0 = float(t0)
        self.vars = list(vars_)


class ADERDG:
    """The ADER-DG scheme of order N on a Grid for one PDE (see module docstring)."""

    def __init__(self, pde, grid, order, cfl=0.9, picard_iters=0, material=None,
                 predictor="picard", initial_guess="constant"):
        assert pde.dim == grid.dim
        assert predictor in ("picard", "ck")
        assert initial_guess in ("constant", "cerk")
        self.initial_guess = initial_guess
        assert predictor == "picard" or getattr(pde, "linear", False), "CK needs a linear PDE"
        self.predictor_kind = predictor
        self.pde, self.grid = pde, grid
        self.D = grid.dim
        self.N = order
        self.ref = RefElement(order)
        self.n = self.ref.n
        self.nv = pde.nvar
        self.cfl = float(cfl)
        self.I = picard_iters if picard_iters and picard_iters > 0 else order + 1
        self.mat = material
        self.source = None
        self.receivers = None
        self.bary = None
        g3x, g3w = gauss_legendre(3)
        self.path_z = [float(v) for v in g3x]
        self.path_w = [float(v) for v in g3w]

    # ----- layout helpers ---------------------------------------------------------------
    def sax(self, d):
        """Axis of spatial direction d in a state array u[C, n..., nv]."""
        return 1 + (self.D - 1 - d)

    def qax(self, d):
        """Axis of spatial direction d in a space-time array q[C, nt, n..., nv]."""
        return 2 + (self.D - 1 - d)

    def node_coords(self):
        """Physical coordinates of every node: list over d of tensors [C, n, ..., n]."""
        lower = self.grid.cell_center_and_lower()
        out = []
        for d in range(self.D):
            shape = [1] * (self.D + 1)
            shape[self.sax(d)] = self.n
            xd = lower[d].reshape([-1] + [1] * self.D) + self.grid.h[d] * self.ref.x.reshape(shape)
            out.append(xd.expand([self.grid.C] + [self.n] * self.D))
        return out

    def tensor_basis(self, xi):
        """Phi_j(xi) = prod_d phi_{j_d}(xi_d) as a tensor [n, ..., n] in (z, y, x) order."""
        out = None
        for d in reversed(range(self.D)):
            v = self.ref.values_at([xi[d]])[0]
            out = v if out is None else torch.einsum('...,m->...m', out, v)
        return out

    def tensor_weights(self):
        return self.tensor_basis_weights()

    def tensor_basis_weights(self):
        out = None
        for d in reversed(range(self.D)):
            out = self.ref.w if out is None else torch.einsum('...,m->...m', out, self.ref.w)
        return out

    def set_point_source(self, src):
        self.source = src

    def set_receivers(self, cells, xis, vars_=(0, 1, 2)):
        """Receivers at reference coordinates ``xis`` in ``cells``: record the given variables."""
        self.receivers = (torch.as_tensor(cells), [self.tensor_basis(x) for x in xis], list(vars_))

    # ----- PDE pieces --------------------------------------------------------------------
    def max_speed(self, u):
        lam = None
        for d in range(self.D):
            mat = None
            if self.mat is not None:
                mat = self.mat.reshape([self.grid.C] + [1] * self.D + [self.mat.shape[-1]])
                mat = mat.expand([self.grid.C] + [self.n] * self.D + [self.mat.shape[-1]])
            s = self.pde.max_speed(u, d, mat)
            m = s.max()
            lam = m if lam is None else torch.maximum(lam, m)
        return lam

    def cfl_dt(self, u):
        """Eq. (7): dt = CFL_N / (d (2N+1)) * h / |lambda_max|."""
        lam = self.max_speed(u)
        return self.cfl / (self.D * (2 * self.N + 1)) * min(self.grid.h) / lam

    def ncp_term(self, q, axfun):
        """sum_d B_d (1/h_d) D_d q at every node: B_d(m) cell-constant (material), or B_d(q) of
        the node's own state (``pde.ncp_state``)."""
        out = 0.0
        for d in range(self.D):
            gq = contract(q, self.ref.D, axfun(d)) / self.grid.h[d]
            if getattr(self.pde, "ncp_state", False):
                out = out + self.pde.ncp(q, gq, d)
                continue
            B = self.pde.ncp_matrix(self.mat, d)  # [C, nv, nv]
            if B.dim() == 2:
                B = B.unsqueeze(0).expand(q.shape[0], -1, -1)
            out = out + torch.einsum('cij,c...j->c...i', B, gq)
        return out

    def source_nodes(self, t_nodes):
        """Point source values at the space-time nodes [C, nt, n.., nv]: node j of the source
        cell gets -M R(t_k) Phi_j(xi0) / (W_j h^d) (the delta function tested against the nodal
        basis with the diagonal Gauss-Legendre mass matrix)."""
        src = self.source
        S = torch.zeros([self.grid.C, len(t_nodes)] + [self.n] * self.D + [self.nv], dtype=torch.float64)
        phi = self.tensor_basis(src.xi)
        W = self.tensor_basis_weights()
        vol = 1.0
        for hd in self.grid.h:
            vol *= hd
        shape = phi / (W * vol)
        amp = ricker(t_nodes, src.f0, src.t0)  # [nt]
        for a, var in enumerate(src.vars):
            S[src.cell, ..., var] = -src.M[a] * amp.reshape([-1] + [1] * self.D) * shape
        return S

    def rhs(self, q, t_nodes):
        """R(q) = -div F(q) - B(q).grad q + point sources, at every space-time node."""
        R = torch.zeros_like(q)
        for d in range(self.D):
            if self.pde.has_flux:
                R = R - contract(self.pde.flux(q, d), self.ref.D, self.qax(d)) / self.grid.h[d]
        if self.pde.has_ncp:
            R = R - self.ncp_term(q, self.qax)
        if self.source is not None:
            R = R + self.source_nodes(t_nodes)
        return R

    # ----- 1. space-time predictor ----------------------------------------------------
    def cerk_guess(self, u, dt, t=0.0):
        """Initial guess of the Picard iteration by a continuous extension Runge-Kutta scheme
        (Sec. 5): the cell-local ODE dq/dt = R(q) (the predictor's right-hand side, no neighbour
        coupling) advanced over the step by the classical four-stage Runge-Kutta method, and its
        natural continuous extension (uniform order 3) evaluated at the time nodes:
            q(t + theta dt) = u + dt sum_i b_i(theta) k_i,
            b_1 = theta - 3 theta^2/2 + 2 theta^3/3,  b_2 = b_3 = theta^2 - 2 theta^3/3,
            b_4 = -theta^2/2 + 2 theta^3/3  (b_i(1) = 1/6, 1/3, 1/3, 1/6).
        Returns [C, nt, n.., nv]."""
        def R(q, tt):
            tn = torch.as_tensor([float(tt)], dtype=torch.float64)
            return self.rhs(q.unsqueeze(1), tn)[:, 0]
        h = float(dt)
        k1 = R(u, t)
        k2 = R(u + 0.5 * h * k1, t + 0.5 * h)
        k3 = R(u + 0.5 * h * k2, t + 0.5 * h)
        k4 = R(u + h * k3, t + h)
        out = []
        for th in self.ref.x.tolist():
            b1 = th - 1.5 * th ** 2 + 2.0 * th ** 3 / 3.0
            b2 = th ** 2 - 2.0 * th ** 3 / 3.0
            b4 = -0.5 * th ** 2 + 2.0 * th ** 3 / 3.0
            out.append(u + h * (b1 * k1 + b2 * (k2 + k3) + b4 * k4))
        return torch.stack(out, dim=1)

    def predictor(self, u, dt, t=0.0, iters=None, trace=None, guess=None):
        """Element-local space-time predictor, Eq. (5): solve
            sum_l K1[k,l] q_l = e0[k] u + dt w_k R(q)_k
        by the fixed-point iteration q^{r+1} = K1^{-1} (e0 u + dt W R(q^r)), from q^0 = u (constant
        in time) or from the continuous extension Runge-Kutta guess (``guess="cerk"``; default:
        the scheme's ``initial_guess``)."""
        ref = self.ref
        nt = self.n
        iters = self.I if iters is None else iters
        guess = self.initial_guess if guess is None else guess
        if guess == "cerk":
            q = self.cerk_guess(u, dt, t)
        else:
            q = u.unsqueeze(1).expand([u.shape[0], nt] + list(u.shape[1:])).clone()
        t_nodes = t + ref.x * dt
        wt = ref.w.reshape([1, nt] + [1] * (self.D + 1))
        e0 = ref.e0.reshape([1, nt] + [1] * (self.D + 1))
        for _ in range(iters):
            R = self.rhs(q, t_nodes)
            b = e0 * u.unsqueeze(1) + dt * wt * R
            bt = torch.movedim(b, 1, 0)
            sol = torch.linalg.solve(ref.K1, bt.reshape(nt, -1)).reshape(bt.shape)
            q_new = torch.movedim(sol, 0, 1)
            if trace is not None:
                trace.append(float((q_new - q).abs().max()))
            q = q_new
        return q

    # ----- 1'. Cauchy-Kowalevski predictor (linear PDEs) -------------------------------
    def linear_operator(self, a):
        """L a = -sum_d (1/h_d) (D_d F_d(a) + B_d D_d a) for a spatial array a[C, n.., nv]: the
        right-hand side of Eq. (1) without sources (linear PDE: F_d and B_d do not depend on a)."""
        out = torch.zeros_like(a)
        for d in range(self.D):
            if self.pde.has_flux:
                out = out - contract(self.pde.flux(a, d), self.ref.D, self.sax(d)) / self.grid.h[d]
        if self.pde.has_ncp:
            out = out - self.ncp_term(a, self.sax)
        return out

    def source_shape(self):
        """g[C, n.., nv]: the point source's spatial factor, -M_a Phi_j(xi0) / (W_j h^d) on the
        stress variables of the source cell, so that the source term is g R(t)."""
        src = self.source
        g = torch.zeros([self.grid.C] + [self.n] * self.D + [self.nv], dtype=torch.float64)
        phi = self.tensor_basis(src.xi)
        W = self.tensor_basis_weights()
        vol = 1.0
        for hd in self.grid.h:
            vol *= hd
        shape = phi / (W * vol)
        for a, var in enumerate(src.vars):
            g[src.cell, ..., var] = -src.M[a] * shape
        return g

    def source_taylor(self, t, dt):
        """Monomial coefficients s_k (k = 0..N, in tau = (time - t)/dt) of the degree-N polynomial
        through the Ricker values at the time nodes t + x_k dt (a Vandermonde solve)."""
        src = self.source
        V = self.ref.x.unsqueeze(1) ** torch.arange(self.n, dtype=torch.float64).unsqueeze(0)
        amp = ricker(t + self.ref.x * dt, src.f0, src.t0)
        return torch.linalg.solve(V, amp)

    def predictor_ck(self, u, dt, t=0.0):
        """Cauchy-Kowalevski predictor (Sec. 2, Sec. 3.3; linear PDEs).  With
        q(t + tau dt) = sum_{k<=N} a_k tau^k, du/dt = L u + g s(tau) gives
            a_0 = u,   a_{k+1} = dt / (k+1) (L a_k + g s_k),   k = 0..N-1
        (the k-th time derivative is dt^-k k! a_k).  Returns q at the time nodes, [C, nt, n.., nv],
        like the Picard predictor."""
        a = [u]
        if self.source is not None:
            s = self.source_taylor(t, dt)
            g = self.source_shape()
        for k in range(self.N):
            La = self.linear_operator(a[k])
            if self.source is not None:
                La = La + s[k] * g
            a.append(dt / (k + 1) * La)
        q = []
        for xt in self.ref.x:
            qt = a[self.N]
            for k in range(self.N - 1, -1, -1):  # Horner in tau
                qt = qt * xt + a[k]
            q.append(qt)
        return torch.stack(q, dim=1)

    # ----- time averages, volume term and face data ----------------------------------
    def time_average(self, X):
        w = self.ref.w.reshape([1, self.n] + [1] * (X.dim() - 2))
        return (w * X).sum(dim=1)

    def face_data(self, q, dt, t):
        """Time averages of q, F_d(q), B grad q and the sources, the volume update, and the face
        extrapolations (qbar, Fbar_d) on both ends of every direction."""
        ref, D = self.ref, self.D
        qbar = self.time_average(q)
        Fbar = [self.time_average(self.pde.flux(q, d)) if self.pde.has_flux else None for d in range(D)]
        vol = torch.zeros_like(qbar)
        for d in range(D):
            if Fbar[d] is not None:
                vol = vol - contract(Fbar[d], ref.D, self.sax(d)) / self.grid.h[d]
        if self.pde.has_ncp:
            vol = vol - self.time_average(self.ncp_term(q, self.qax))
        if self.source is not None:
            vol = vol + self.time_average(self.source_nodes(t + ref.x * dt))
        vol = dt * vol
        faces = []
        for d in range(D):
            ax = self.sax(d)
            qp = extrapolate(qbar, ref.e1, ax)
            qm = extrapolate(qbar, ref.e0, ax)
            if Fbar[d] is not None:
                Fp = extrapolate(Fbar[d], ref.e1, ax)
                Fm = extrapolate(Fbar[d], ref.e0, ax)
            else:
                Fp = torch.zeros_like(qp)
                Fm = torch.zeros_like(qm)
            faces.append((qp, qm, Fp, Fm))
        return qbar, Fbar, vol, faces

    # ----- 2. Riemann solver ------------------------------------------------------------
    def ghost(self, d, kind, q, F):
        if kind == 'wall':
            return self.pde.mirror(q, d), self.pde.mirror_flux(F, d)
        if kind == 'absorbing':
            if getattr(self.pde, 'linear', False):
                return torch.zeros_like(q), torch.zeros_like(F)
            return q.clone(), F.clone()
        raise ValueError(kind)

    def wave_speed(self, d, qL, qR, mL, mR):
        """One Rusanov speed per face: max over the face nodes and both sides."""
        if self.pde.has_flux and not getattr(self.pde, 'linear', False):
            sL = self.pde.max_speed(qL, d)
            sR = self.pde.max_speed(qR, d)
            s = torch.maximum(sL, sR)
            return s.reshape(s.shape[0], -1).amax(dim=1)
        sL = self.pde.max_speed(qL, d, mL)
        sR = self.pde.max_speed(qR, d, mR)
        if sL.dim() > 1:
            sL = sL.reshape(sL.shape[0], -1).amax(dim=1)
            sR = sR.reshape(sR.shape[0], -1).amax(dim=1)
        # ties take the left value (a definite subgradient for the adjoint)
        return torch.where(sL >= sR, sL, sR)

    def riemann(self, d, qL, qR, FL, FR, mL=None, mR=None):
        """Rusanov flux and halved path-conservative fluctuation on a batch of faces.
        Returns (Phi_L, Phi_R): what the left and right cell see on this face."""
        s = self.wave_speed(d, qL, qR, mL, mR)
        s = s.reshape([-1] + [1] * (qL.dim() - 1))
        dq = qR - qL
        G = 0.5 * (FL + FR) - 0.5 * s * dq
        if not self.pde.has_ncp:
            return G, G
        if getattr(self.pde, "ncp_state", False):
            # path-conservative fluctuation along the straight segment in state space, per face
            # node: int_0^1 B_n(qL + z (qR - qL)) dz dq by the 3-point rule
            fl = 0.0
            for z, wz in zip(self.path_z, self.path_w):
                fl = fl + wz * self.pde.ncp(qL + z * dq, dq, d)
            return G + 0.5 * fl, G - 0.5 * fl
        Bbar = 0.0
        for z, wz in zip(self.path_z, self.path_w):
            m = mL + z * (mR - mL) if mL is not None else None
            Bbar = Bbar + wz * self.pde.ncp_matrix(m, d)
        if Bbar.dim() == 2:
            Bbar = Bbar.unsqueeze(0).expand(qL.shape[0], -1, -1)
        half = 0.5 * torch.einsum('cij,c...j->c...i', Bbar, dq)
        return G + half, G - half

    def face_fluxes(self, faces):
        """For every cell and direction: Phi_L on its right face, Phi_R on its left face."""
        out = []
        mat = self.mat
        for d in range(self.D):
            qp, qm, Fp, Fm = faces[d]
            nbr = self.grid.neighbor(d, +1)
            nbl = self.grid.neighbor(d, -1)
            # right faces: this cell is L
            qR = qm[nbr.clamp(min=0)].clone()
            FR = Fm[nbr.clamp(min=0)].clone()
            mR = mat[nbr.clamp(min=0)].clone() if mat is not None else None
            bnd = nbr < 0
            if bnd.any():
                gq, gF = self.ghost(d, self.grid.bc[d][1], qp[bnd], Fp[bnd])
                qR[bnd], FR[bnd] = gq, gF
                if mat is not None:
                    mR[bnd] = mat[bnd]
            PhiL_right, _ = self.riemann(d, qp, qR, Fp, FR, mat, mR)
            # left faces: this cell is R
            qL = qp[nbl.clamp(min=0)].clone()
            FL = Fp[nbl.clamp(min=0)].clone()
            mL = mat[nbl.clamp(min=0)].clone() if mat is not None else None
            bnd = nbl < 0
            if bnd.any():
                gq, gF = self.ghost(d, self.grid.bc[d][0], qm[bnd], Fm[bnd])
                qL[bnd], FL[bnd] = gq, gF
                if mat is not None:
                    mL[bnd] = mat[bnd]
            _, PhiR_left = self.riemann(d, qL, qm, FL, Fm, mL, mat)
            out.append((PhiL_right, PhiR_left))
        return out

    # ----- 3. corrector -----------------------------------------------------------------
    def correct(self, u, vol, faces, fluxes, dt):
        """Eq. (6) in nodal strong form (diagonal mass matrix):
        u_j += vol_j - sum_d dt/h_d / w_{j_d} [ e1_{j_d} (Phi_L^+ - Fbar^+) - e0_{j_d} (Phi_R^- - Fbar^-) ]."""
        ref = self.ref
        out = u + vol
        for d in range(self.D):
            ax = self.sax(d)
            qp, qm, Fp, Fm = faces[d]
            PhiL, PhiR = fluxes[d]
            shape = [1] * (self.D + 2)
            shape[ax] = self.n
            c1 = (ref.e1 / ref.w).reshape(shape)
            c0 = (ref.e0 / ref.w).reshape(shape)
            out = out - dt / self.grid.h[d] * (c1 * (PhiL - Fp).unsqueeze(ax) - c0 * (PhiR - Fm).unsqueeze(ax))
        return out

    # ----- whole step -----------------------------------------------------------------
    def step(self, u, dt, t=0.0, details=False):
        if self.predictor_kind == "ck":
            q = self.predictor_ck(u, dt, t)
        else:
            q = self.predictor(u, dt, t)
        qbar, Fbar, vol, faces = self.face_data(q, dt, t)
        fluxes = self.face_fluxes(faces)
        u_new = self.correct(u, vol, faces, fluxes, dt)
        if details:
            return u_new, dict(q=q, qbar=qbar, Fbar=Fbar, vol=vol, faces=faces, fluxes=fluxes)
        return u_new

    def record(self, u):
        """Receiver values [nrec, len(vars)]: the nodal polynomial of the receiver's cell
        evaluated at the receiver's reference point."""
        cells, phis, vars_ = self.receivers
        out = []
        for c, phi in zip(cells.tolist(), phis):
            out.append(torch.stack([(u[c, ..., v] * phi).sum() for v in vars_]))
        return torch.stack(out)

    def run(self, u, steps, t=0.0, dt=None, t_end=None, seismo=None):
        """Advance ``steps`` steps (or until t_end); CFL step when dt is None."""
        k = 0
        while True:
            if steps is not None and k >= steps:
                break
            if t_end is not None and t >= t_end - 1e-14 * max(1.0, abs(t_end)):
                break
            dtk = self.cfl_dt(u) if dt is None else torch.as_tensor(float(dt), dtype=torch.float64)
            if t_end is not None:
                dtk = torch.minimum(dtk, torch.as_tensor(t_end - t, dtype=torch.float64))
            u = self.step(u, dtk, t)
            t = t + float(dtk)
            if seismo is not None:
                seismo.append(self.record(u))
            k += 1
        return u, t
