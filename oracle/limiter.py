"""A-posteriori finite-volume subcell limiter (oracle; test infrastructure only), Sec. 3.5.

After the unlimited ADER-DG step, each cell's candidate solution is checked a posteriori:

* physical admissibility: density and pressure positive (and finite) at every Gauss-Legendre node
  and every subcell average of the candidate;
* numerical admissibility: a relaxed discrete maximum principle (DMP) on the subcell averages.

Cells failing either check ("troubled") are recomputed from the old time level with a robust FV
scheme on 2N+1 subcells per direction: MUSCL-Hancock with minmod slopes and a Rusanov flux.

Readings of the paper taken here (silent or only cited points):
* Representation at t^n of each cell: its stored subcell averages if it was troubled in the
  previous step, else the subcell averages P(u^n) of its DG polynomial.
* DMP bounds per variable: min / max over the cell and its face neighbours (inside the domain) of
  those representations; a candidate subcell value passes if m - delta <= x <= M + delta with
  delta = max(1e-4, 1e-3 (M - m)).  Comparisons are written so that NaN fails.
* FV recompute: one MUSCL-Hancock step with the DG dt on the subcells of the troubled cell, with a
  halo of 2 subcells taken from the t^n representations of all neighbours; boundaries reflect the
  subcell grid (wall: normal momentum negated; absorbing: plain copy; periodic: wrap).
* Untroubled face neighbours of a troubled cell replace their DG numerical flux on the shared face
  by the FV subface fluxes integrated against their test functions, which keeps the scheme
  exactly conservative.
* The troubled cell's new DG polynomial is R(U_sub) (mean-preserving least squares); U_sub is kept
  as its representation for the next step.  Neither recompute nor cascade is iterated.
* First-order fallback (Table 1 names Godunov's scheme beside MUSCL-Hancock): if the
  MUSCL-Hancock result of any troubled cell is not physically admissible, the step's FV recompute
  is redone for every troubled cell with zero slopes (the first-order Godunov-type scheme with
  the Rusanov flux), so that each subface keeps one flux and the scheme stays conservative.
  Physical admissibility: finite, density and pressure above ``floor`` (0: positive).
"""
import torch

DELTA0 = 1e-4
EPS = 1e-3


class Limiter:
    def __init__(self, solver, delta0=DELTA0, eps=EPS, floor=0.0):
        self.s = solver
        self.floor = float(floor)
        self.last_fallback = False
        self.pde = solver.pde
        self.D = solver.D
        self.ref = solver.ref
        self.ns = self.ref.ns
        self.delta0 = delta0
        self.eps = eps

    # ---- projections ---------------------------------------------------------------------
    def _apply(self, X, M, D):
        for d in range(D):
            ax = 1 + (D - 1 - d)
            X = torch.movedim(torch.tensordot(X, M, dims=([ax], [1])), -1, ax)
        return X

    def project(self, u):
        """DG nodal values [C, n..., nv] -> subcell averages [C, ns..., nv] (P = P1 per axis)."""
        return self._apply(u, self.ref.P1, self.D)

    def reconstruct(self, U):
        """Subcell averages [C, ns..., nv] -> DG nodal values (R = R1 per axis)."""
        return self._apply(U, self.ref.R1, self.D)

    def initial_rep(self, u, U_sub=None, flags=None):
        """Representation at t^0: P(u^0), except for the cells in ``flags`` whose subcell averages
        ``U_sub`` are given (initial data that jumps inside a cell starts in the FV space, as at
        the start of a limited run); their DG state becomes R(U_sub).  Returns (u0, rep0)."""
        rep = self.project(u)
        if flags is None:
            return u, rep
        u = u.clone()
        rep[flags] = U_sub[flags]
        u[flags] = self.reconstruct(U_sub[flags])
        return u, rep

    # ---- detection -----------------------------------------------------------------------
    def admissible(self, q):
        """Density and pressure above the floor (positive for floor 0) and all values finite,
        over all axes but the first."""
        rho = q[..., 0]
        p = self.pde.pressure(q)
        ok = (rho > self.floor) & (p > self.floor) & torch.isfinite(q).all(dim=-1)
        return ok.reshape(ok.shape[0], -1).all(dim=1)

    def detect(self, u_star, rep):
        C = u_star.shape[0]
        nv = u_star.shape[-1]
        cand = self.project(u_star)
        flat = rep.reshape(C, -1, nv)
        mn = flat.amin(dim=1)
        mx = flat.amax(dim=1)
        lo, hi = mn.clone(), mx.clone()
        for d in range(self.D):
            for side in (-1, 1):
                nb = self.s.grid.neighbor(d, side)
                has = nb >= 0
                idx = nb.clamp(min=0)
                lo = torch.where(has[:, None], torch.minimum(lo, mn[idx]), lo)
                hi = torch.where(has[:, None], torch.maximum(hi, mx[idx]), hi)
        delta = torch.clamp(self.eps * (hi - lo), min=self.delta0)
        cf = cand.reshape(C, -1, nv)
        ok = ((cf >= (lo - delta)[:, None, :]) & (cf <= (hi + delta)[:, None, :])).all(dim=2).all(dim=1)
        ok = ok & self.admissible(u_star) & self.admissible(cand)
        return ~ok, cand

    # ---- global subcell grid -----------------------------------------------------------------
    def to_global(self, rep):
        """[C, ns(z), ns(y), ns(x), nv] -> global subcell array [Nz ns, Ny ns, Nx ns, nv]
        (axes in (z, y, x) order)."""
        g = self.s.grid
        D, ns = self.D, self.ns
        nc = list(reversed(g.ncell))  # (z, y, x)
        X = rep.reshape(nc + [ns] * D + [rep.shape[-1]])
        perm = []
        for k in range(D):
            perm += [k, D + k]
        X = X.permute(perm + [2 * D])
        return X.reshape([nc[k] * ns for k in range(D)] + [rep.shape[-1]])

    def from_global(self, G):
        g = self.s.grid
        D, ns = self.D, self.ns
        nc = list(reversed(g.ncell))
        X = G.reshape(sum([[nc[k], ns] for k in range(D)], []) + [G.shape[-1]])
        perm = [2 * k for k in range(D)] + [2 * k + 1 for k in range(D)]
        X = X.permute(perm + [2 * D])
        return X.reshape([g.C] + [ns] * D + [G.shape[-1]])

    def pad(self, G, w=2):
        """Pad the global subcell array by w subcells per side with the boundary conditions."""
        g = self.s.grid
        for d in range(self.D):
            ax = self.D - 1 - d
            kinds = g.bc[d]
            n = G.shape[ax]
            if kinds[0] == 'periodic':
                lo = G.narrow(ax, n - w, w)
                hi = G.narrow(ax, 0, w)
            else:
                lo = G.narrow(ax, 0, w).flip(ax)
                hi = G.narrow(ax, n - w, w).flip(ax)
                if kinds[0] == 'wall':
                    lo = self.pde.mirror(lo, d)
                if kinds[1] == 'wall':
                    hi = self.pde.mirror(hi, d)
            G = torch.cat([lo, G, hi], dim=ax)
        return G

    @staticmethod
    def minmod(a, b):
        return torch.where(a * b > 0, torch.sign(a) * torch.minimum(a.abs(), b.abs()),
                           torch.zeros_like(a))

    def fv_global(self, rep, dt, slopes=True):
        """One MUSCL-Hancock / Rusanov step on the whole subcell grid from the t^n representation.
        Returns the new subcell averages of every cell and, per direction, the time-averaged
        numerical flux through every subface (index i = flux between global subcells i-1 and i,
        i = 0..N_d ns, along that direction)."""
        g = self.s.grid
        D = self.D
        G = self.pad(self.to_global(rep), 2)
        dx = [g.h[d] / self.ns for d in range(D)]
        core = [slice(1, G.shape[k] - 1) for k in range(D)]  # the cells that get slopes: 1 halo layer
        sig = []
        for d in range(D):
            ax = D - 1 - d
            fwd = G.narrow(ax, 1, G.shape[ax] - 1) - G.narrow(ax, 0, G.shape[ax] - 1)
            a = fwd.narrow(ax, 0, fwd.shape[ax] - 1)   # U_i - U_{i-1} for i = 1..n-2
            b = fwd.narrow(ax, 1, fwd.shape[ax] - 1)   # U_{i+1} - U_i
            s = self.minmod(a, b) if slopes else torch.zeros_like(a)
            # restrict the other axes to the core
            idx = [slice(None)] * (D + 1)
            for k in range(D):
                if k != ax:
                    idx[k] = core[k]
            sig.append(s[tuple(idx)])
        U = G[tuple(core + [slice(None)])]
        # half-step evolution of the face-extrapolated values (same increment for all faces)
        inc = torch.zeros_like(U)
        for d in range(D):
            Up = U + 0.5 * sig[d]
            Um = U - 0.5 * sig[d]
            inc = inc - dt / (2 * dx[d]) * (self.pde.flux(Up, d) - self.pde.flux(Um, d))
        new = U.clone()
        fluxes = []
        for d in range(D):
            ax = D - 1 - d
            Up = U + 0.5 * sig[d] + inc    # right face value of each subcell
            Um = U - 0.5 * sig[d] + inc    # left face value
            L = Up.narrow(ax, 0, Up.shape[ax] - 1)
            R = Um.narrow(ax, 1, Um.shape[ax] - 1)
            s = torch.maximum(self.pde.max_speed(L, d), self.pde.max_speed(R, d))[..., None]
            f = 0.5 * (self.pde.flux(L, d) + self.pde.flux(R, d)) - 0.5 * s * (R - L)
            # f[i] is the flux between core cells i and i+1 along ax; core cell k <-> padded k+1
            upd = torch.zeros_like(U)
            n_ax = U.shape[ax]
            upd.narrow(ax, 1, n_ax - 2).add_(f.narrow(ax, 0, n_ax - 2) - f.narrow(ax, 1, n_ax - 2))
            new = new + dt / dx[d] * upd
            # fluxes through global subfaces 0..N ns of the interior, with the other axes interior
            idx = [slice(1, -1)] * D + [slice(None)]
            idx[ax] = slice(None)
            fluxes.append(f[tuple(idx)])
        inner = [slice(1, -1)] * D + [slice(None)]
        U_new = self.from_global(new[tuple(inner)])
        return U_new, fluxes

    # ---- neighbour fix -------------------------------------------------------------------
    def face_flux_nodes(self, fsub):
        """Subface fluxes over one cell face [.., ns^(D-1) (transverse, z/y/x order), nv] ->
        the equivalent nodal flux G_eff[j] = (1/W_j) sum_s f_s prod_e P1[s_e, j_e] / ns^(D-1)."""
        ref = self.ref
        X = fsub
        D1 = self.D - 1
        for k in range(D1):
            ax = 1 + k
            X = torch.movedim(torch.tensordot(X, ref.P1, dims=([ax], [0])), -1, ax)
            X = X / self.ns
            shape = [1] * X.dim()
            shape[ax] = ref.n
            X = X / ref.w.reshape(shape)
        return X

    def face_neighbours(self, mask):
        """Cells that share a face with a cell of ``mask`` (inside the domain)."""
        g = self.s.grid
        out = torch.zeros_like(mask)
        for d in range(self.D):
            for side in (1, -1):
                nb = g.neighbor(d, side)
                out |= (nb >= 0) & mask[nb.clamp(min=0)]
        return out

    @staticmethod
    def initial_status(flags, persist=2):
        """Hybrid status at t^0 (Sec. 3.5): the cells that start in the FV space along the
        initial discontinuity count as troubled at the initial time and take ``persist`` FV
        steps; the others start in DG (0)."""
        flags = torch.as_tensor(flags, dtype=torch.bool)
        return torch.where(flags, torch.full(flags.shape, persist, dtype=torch.long),
                           torch.zeros(flags.shape, dtype=torch.long))

    def step_hybrid(self, u, rep, status, dt, t=0.0, persist=2, layer=True):
        """One step of the hybrid ADER-DG / FV scheme (Sec. 3.5): cells stay FV for several steps
        after they were troubled, and their face neighbours form an interface layer that also
        computes with FV.  ``status``[C] holds the FV steps a cell still has to take (0: DG).
          known  = (status > 0) | (face neighbours of those, with ``layer``): the cells that
                   compute with FV in this step whatever their DG candidate;
          detected = troubled candidates outside ``known`` (a known cell is not checked);
          FV set = detected | (status > 0) | (face neighbours of those, with ``layer``);
          status_new = persist where detected, else max(status - 1, 0).
        With ``layer`` no result depends on the DG predictor of a cell with status > 0: its face
        neighbours are known FV cells, so its DG data reach only candidates that are neither
        checked nor kept.  With persist = 0 and layer = False this is ``step``.
        Returns (u_new, fv[C], rep_new, admissible, status_new)."""
        u_new, fv, rep_new, ok, detected = self.step(u, rep, dt, t, status=status, layer=layer,
                                                     return_detected=True)
        status_new = torch.where(detected, torch.full_like(status, persist),
                                 (status - 1).clamp(min=0))
        return u_new, fv, rep_new, ok, status_new

    def step(self, u, rep, dt, t=0.0, force=False, status=None, layer=False,
             return_detected=False):
        """One limited step.  Returns (u_new, troubled[C] bool, rep_new, admissible); the
        troubled set is recomputed with FV.  ``status`` / ``layer``: see ``step_hybrid``."""
        s = self.s
        g = s.grid
        D, ns = self.D, self.ns
        u_star, info = s.step(u, dt, t, details=True)
        troubled, cand = self.detect(u_star, rep)
        if status is not None:
            known = status > 0
            if layer:
                known = known | self.face_neighbours(known)
            troubled = troubled & ~known
        detected = troubled
        if force:
            troubled = torch.ones_like(troubled)
        if status is not None:
            troubled = troubled | (status > 0)
        if layer:
            troubled = troubled | self.face_neighbours(troubled)
        u_new = u_star.clone()
        rep_new = cand.clone()
        self.last_fallback = False
        if troubled.any():
            U_all, fluxes = self.fv_global(rep, dt)
            if not bool(self.admissible(U_all[troubled]).all()):
                # first-order fallback for every troubled cell of the step
                U_all, fluxes = self.fv_global(rep, dt, slopes=False)
                self.last_fallback = True
            u_new[troubled] = self.reconstruct(U_all[troubled])
            rep_new[troubled] = U_all[troubled]
            nc = list(reversed(g.ncell))
            for d in range(D):
                ax = D - 1 - d
                f = fluxes[d]  # global subface array, axis ax has N_d ns + 1 entries
                PhiL, PhiR = info['fluxes'][d]
                for side in (1, -1):
                    nb = g.neighbor(d, side)
                    fix = (~troubled) & (nb >= 0)
                    fix = fix & troubled[nb.clamp(min=0)]
                    if not fix.any():
                        continue
                    cells = torch.nonzero(fix).flatten()
                    # subface fluxes on the face of each fixed cell
                    idxs = []
                    for c in cells.tolist():
                        i_d = int(g.idx[d][c])
                        k = (i_d + 1) * ns if side > 0 else i_d * ns
                        if g.bc[d][0] == 'periodic':
                            k = k % (g.ncell[d] * ns)
                        sl = []
                        for e in range(D):
                            ie = int(g.idx[e][c])
                            sl.append(slice(ie * ns, (ie + 1) * ns))
                        sl[d] = k
                        idxs.append(f[tuple(reversed(sl))])
                    fsub = torch.stack(idxs)  # [m, ns^(D-1) transverse (z/y/x order), nv]
                    Geff = self.face_flux_nodes(fsub)
                    shape = [1] * (D + 2)
                    shape[1 + (D - 1 - d)] = s.n
                    if side > 0:   # the fixed cell is on the left of the face
                        corr = -dt / g.h[d] * (s.ref.e1 / s.ref.w).reshape(shape) * \
                            (Geff - PhiL[cells]).unsqueeze(1 + (D - 1 - d))
                    else:          # the fixed cell is on the right of the face
                        corr = dt / g.h[d] * (s.ref.e0 / s.ref.w).reshape(shape) * \
                            (Geff - PhiR[cells]).unsqueeze(1 + (D - 1 - d))
                    u_new[cells] = u_new[cells] + corr
            fixed = torch.zeros_like(troubled)
            for d in range(D):
                for side in (1, -1):
                    nb = g.neighbor(d, side)
                    fixed |= (~troubled) & (nb >= 0) & troubled[nb.clamp(min=0)]
            if fixed.any():
                rep_new[fixed] = self.project(u_new[fixed])
            admissible = self.admissible(rep_new[troubled])
        else:
            admissible = torch.ones(0, dtype=torch.bool)
        if return_detected:
            return u_new, troubled, rep_new, bool(admissible.all()), detected
        return u_new, troubled, rep_new, bool(admissible.all())
