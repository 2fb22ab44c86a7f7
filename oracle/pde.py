"""PDE terms of  dQ/dt + div F(Q) + B(Q).grad Q = S(Q) + sum of point sources  (Eq. (1), Sec. 2)
(oracle; test infrastructure only).

Each class supplies what the paper's user functions supply (Table 2): ``flux`` (F_d), the
non-conservative matrices B_d (``ncp_matrix``, cell-constant: they depend on the per-cell
material only), ``max_speed`` (the eigenvalue bound used by the CFL condition Eq. (7) and by the
Rusanov flux) and, for wall boundaries, the mirror maps.  Arrays carry the variables on the
last axis.
"""
import torch


class Advection:
    """Scalar linear advection dq/dt + div(a q) = 0 with a constant velocity a (test PDE)."""

    nvar = 1
    has_flux = True
    has_ncp = False
    nmat = 0

    def __init__(self, a):
        self.a = [float(v) for v in a]
        self.dim = len(self.a)

    def flux(self, q, d):
        return self.a[d] * q

    def max_speed(self, q, d, mat=None):
        return torch.full(q.shape[:-1], abs(self.a[d]), dtype=q.dtype)

    linear = True


class AdvectionNCP:
    """Scalar advection written as a non-conservative product, dq/dt + a . grad q = 0.

    Exercises the path-conservative face treatment with a closed form: for a_d > 0 the
    fluctuation to the left state must vanish and the one to the right state is a_d (qR - qL).
    """

    nvar = 1
    has_flux = False
    has_ncp = True
    nmat = 0

    def __init__(self, a):
        self.a = [float(v) for v in a]
        self.dim = len(self.a)

    def ncp_matrix(self, mat, d):
        shape = mat.shape[:-1] if mat is not None else ()
        return torch.full(tuple(shape) + (1, 1), self.a[d], dtype=torch.float64)

    def max_speed(self, q, d, mat=None):
        shape = mat.shape[:-1] if mat is not None else q.shape[:-1]
        return torch.full(tuple(shape), abs(self.a[d]), dtype=torch.float64)

    linear = True


class Euler:
    """Compressible Euler equations, Eq. (8) of Sec. 6.1: Q = (rho, j, E), F_d = (j_d,
    j j_d / rho + p e_d, (E + p) j_d / rho), ideal gas p = (gamma-1)(E - |j|^2 / (2 rho)) with
    gamma = 1.4 (the pressure equation of Sec. 6.1)."""

    has_flux = True
    has_ncp = False
    nmat = 0
    linear = False

    def __init__(self, dim, gamma=1.4):
        self.dim = dim
        self.nvar = dim + 2
        self.gamma = float(gamma)

    def pressure(self, q):
        rho = q[..., 0]
        j2 = sum(q[..., 1 + i] ** 2 for i in range(self.dim))
        return (self.gamma - 1.0) * (q[..., -1] - 0.5 * j2 / rho)

    def flux(self, q, d):
        rho = q[..., 0]
        E = q[..., -1]
        p = self.pressure(q)
        vd = q[..., 1 + d] / rho
        comps = [q[..., 1 + d]]
        for i in range(self.dim):
            c = q[..., 1 + i] * vd
            if i == d:
                c = c + p
            comps.append(c)
        comps.append((E + p) * vd)
        return torch.stack(comps, dim=-1)

    def sound_speed(self, q):
        """sqrt(gamma p / rho); a negative c^2 (a non-admissible state, which the limiter rejects)
        counts as 0 so that wave-speed estimates stay finite; NaN propagates."""
        c2 = self.gamma * self.pressure(q) / q[..., 0]
        return torch.sqrt(torch.where(c2 < 0, torch.zeros_like(c2), c2))

    def max_speed(self, q, d, mat=None):
        """|v_d| + c: the largest |eigenvalue| of dF_d/dQ (eigenvalues v_d - c, v_d, v_d + c)."""
        return torch.abs(q[..., 1 + d] / q[..., 0]) + self.sound_speed(q)

    def mirror(self, q, d):
        """Reflecting-wall ghost state: the momentum component normal to the wall changes sign."""
        s = torch.ones(self.nvar, dtype=q.dtype)
        s[1 + d] = -1.0
        return q * s

    def mirror_flux(self, F, d):
        """F_d of the mirrored state: every component except the normal momentum flux changes
        sign (mass, tangential momentum and energy fluxes are odd in v_d, j_d^2/rho + p is even)."""
        s = -torch.ones(self.nvar, dtype=F.dtype)
        s[1 + d] = 1.0
        return F * s


# Elastic stress components in the order (xx, yy, zz, xy, xz, yz) (Sec. 2.1), stored after the
# three velocity components.
SIGMA = {(0, 0): 3, (1, 1): 4, (2, 2): 5, (0, 1): 6, (1, 0): 6, (0, 2): 7, (2, 0): 7,
         (1, 2): 8, (2, 1): 8}


class Elastic:
    """Linear isotropic elastic waves, Sec. 2.1, in velocity-stress form Q = (v, sigma):

        dv_i/dt - (1/rho) sum_j d sigma_ij / dx_j = 0
        d sigma_ij/dt - lambda delta_ij div v - mu (dv_i/dx_j + dv_j/dx_i) = 0

    so every term is a non-conservative product B_d(m) dQ/dx_d with the per-cell material
    m = (rho, lambda, mu); F = 0.  Eigenvalues of B_n: 0 (x3), +-vs (x2 each), +-vp.
    """

    dim = 3
    nvar = 9
    has_flux = False
    has_ncp = True
    nmat = 3
    linear = True

    def ncp_matrix(self, mat, d):
        rho, lam, mu = mat[..., 0], mat[..., 1], mat[..., 2]
        B = torch.zeros(tuple(mat.shape[:-1]) + (9, 9), dtype=mat.dtype)
        # velocity rows: -(1/rho) d sigma_{i d} / dx_d
        for i in range(3):
            B[..., i, SIGMA[(i, d)]] = -1.0 / rho
        # normal stress rows: -lambda dv_d/dx_d, and -2 mu dv_d/dx_d for sigma_dd
        for i in range(3):
            B[..., SIGMA[(i, i)], d] = -lam - (2.0 * mu if i == d else 0.0)
        # shear stress rows sigma_ij (i<j): -mu (dv_j/dx_i + dv_i/dx_j)
        for (i, j) in ((0, 1), (0, 2), (1, 2)):
            if d == i:
                B[..., SIGMA[(i, j)], j] = -mu
            if d == j:
                B[..., SIGMA[(i, j)], i] = -mu
        return B

    def max_speed(self, q, d, mat=None):
        rho, lam, mu = mat[..., 0], mat[..., 1], mat[..., 2]
        return torch.sqrt((lam + 2.0 * mu) / rho)

    @staticmethod
    def energy_density(q, mat):
        """Kinetic plus strain energy 1/2 rho |v|^2 + 1/2 sigma : C^{-1} : sigma (isotropic
        compliance), per node."""
        rho, lam, mu = mat[..., 0], mat[..., 1], mat[..., 2]
        v = q[..., 0:3]
        sxx, syy, szz = q[..., 3], q[..., 4], q[..., 5]
        sxy, sxz, syz = q[..., 6], q[..., 7], q[..., 8]
        tr = sxx + syy + szz
        s2 = sxx ** 2 + syy ** 2 + szz ** 2 + 2 * (sxy ** 2 + sxz ** 2 + syz ** 2)
        strain = (s2 - lam / (3 * lam + 2 * mu) * tr ** 2) / (4 * mu)
        return 0.5 * rho * (v ** 2).sum(-1) + strain


class ShallowWater:
    """Shallow water equations with bathymetry, Eq. (9) of Sec. 2: Q = (h, hu, hv, b),
    F_x = (hu, hu u, hv u, 0), F_y = (hv, hu v, hv v, 0); the hydrostatic pressure and the
    bathymetry slope are the non-conservative product, g h d(b + h)/dx_d on the momentum of
    direction d (the bathymetry b is a state variable that the equations keep constant)."""

    has_flux = True
    has_ncp = True
    ncp_state = True     # B depends on the state (not on cell-constant material)
    nmat = 0
    linear = False

    def __init__(self, g=9.81):
        self.dim = 2
        self.nvar = 4
        self.g = float(g)

    def flux(self, q, d):
        ud = q[..., 1 + d] / q[..., 0]
        return torch.stack([q[..., 1 + d], q[..., 1] * ud, q[..., 2] * ud,
                            torch.zeros_like(ud)], dim=-1)

    def ncp(self, q, dq, d):
        """B_d(q) dq: g h (dq_h + dq_b) on the momentum of direction d, zero elsewhere."""
        out = torch.zeros_like(dq)
        out[..., 1 + d] = self.g * q[..., 0] * (dq[..., 0] + dq[..., 3])
        return out

    def max_speed(self, q, d, mat=None):
        """|u_d| + sqrt(g h): the largest |eigenvalue| of the direction-d system matrix."""
        h = q[..., 0]
        return torch.abs(q[..., 1 + d] / h) + torch.sqrt(self.g * h)

    def mirror(self, q, d):
        """Reflecting-wall ghost state: the normal momentum changes sign."""
        s = torch.ones(self.nvar, dtype=q.dtype)
        s[1 + d] = -1.0
        return q * s

    def mirror_flux(self, F, d):
        """F_d of the mirrored state: the normal momentum flux h u_d^2 is even in u_d, the others
        are odd."""
        s = -torch.ones(self.nvar, dtype=F.dtype)
        s[1 + d] = 1.0
        return F * s
