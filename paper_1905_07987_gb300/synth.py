"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 6.1 and 6.2).

This module holds no arithmetic of the ADER-DG method: it evaluates analytic initial data at
node coordinates the CALLER supplies, draws seeded material fields, sources, receivers and
ensemble sizes, and names the workload sizes.  The CUDA library and the test oracle both receive
its arrays as inputs, so that parity runs start from identical data.

Random numbers come from splitmix64 (Steele, Lea, Flood 2014): state += 0x9E3779B97F4A7C15;
z = state; z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) * 0x94D049BB133111EB;
z ^ (z >> 31), all modulo 2^64; a double in [0,1) is (z >> 11) * 2^-53.
"""
import math
import numpy as np

MASK = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed):
        self.state = int(seed) & MASK

    def next_u64(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        return z ^ (z >> 31)

    def uniform(self):
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


# ------------------------------------------------------------------------------------------
# Time-step factor.  Eq. (7) bounds dt by CFL_N / (d (2N+1)) * h / |lambda_max| with an
# order-dependent CFL_N < 1.  KAPPA[N] is the largest CFL_N for which the one-dimensional
# ADER-DG scheme of order N with the Rusanov (upwind) flux is von Neumann stable (amplification
# <= 1 + 1e-3 over all wavenumbers), rounded down; the workloads run at 0.9 of it, 0.9 being the
# safety factor the workload descriptions quote as "CFL 0.9".
KAPPA = {1: 1.0, 2: 0.85, 3: 0.72, 4: 0.62, 5: 0.55, 6: 0.49}
SAFETY = 0.9


def cfl_number(order, safety=SAFETY):
    return safety * KAPPA[order]


GAMMA = 1.4


def euler_conserved(rho, vel, p, gamma=GAMMA):
    """(rho, rho v, p/(gamma-1) + rho |v|^2 / 2) stacked on the last axis."""
    rho = np.asarray(rho, dtype=np.float64)
    comps = [rho]
    ke = np.zeros_like(rho)
    for v in vel:
        v = np.broadcast_to(np.asarray(v, dtype=np.float64), rho.shape)
        comps.append(rho * v)
        ke = ke + 0.5 * rho * v * v
    comps.append(np.broadcast_to(np.asarray(p, dtype=np.float64), rho.shape) / (gamma - 1.0) + ke)
    return np.stack(comps, axis=-1)


def node_coordinates(nodes, ncell, lo, hi):
    """Physical coordinates of every node of every cell for 1-D reference nodes ``nodes`` on
    [0,1]: list over d of arrays [C, n, ..., n] (node axes ordered (z, y, x), x fastest; cell
    index i + nx*(j + ny*k))."""
    nodes = np.asarray(nodes, dtype=np.float64)
    n = len(nodes)
    D = len(ncell)
    C = int(np.prod(ncell))
    c = np.arange(C)
    idx = []
    for d in range(D):
        idx.append(c % ncell[d])
        c = c // ncell[d]
    out = []
    for d in range(D):
        h = (hi[d] - lo[d]) / ncell[d]
        shape = [1] * (D + 1)
        shape[1 + (D - 1 - d)] = n
        x = lo[d] + h * idx[d].reshape([-1] + [1] * D) + h * nodes.reshape(shape)
        out.append(np.broadcast_to(x, [C] + [n] * D).copy())
    return out


def subcell_centres(ns, ncell, lo, hi):
    """Centres of the ns^d equal subcells of every cell (same layout as node_coordinates)."""
    return node_coordinates((np.arange(ns) + 0.5) / ns, ncell, lo, hi)


def discontinuous_cells(U_sub):
    """Cells whose sampled subcell values are not all equal (the initial data jumps inside them):
    bool [C].  U_sub: [C, ns, ..., ns, nvar]."""
    C = U_sub.shape[0]
    flat = U_sub.reshape(C, -1, U_sub.shape[-1])
    return (flat.max(axis=1) - flat.min(axis=1)).max(axis=1) > 0


def entropy_wave(X, t=0.0, amp=0.2):
    """Density wave rho = 1 + amp sin(2 pi (sum_d x_d - d t)) advected with v = (1,..,1), p = 1:
    an exact solution of the Euler equations (Sec. 6.1 workloads)."""
    D = len(X)
    s = sum(X) - D * t
    rho = 1.0 + amp * np.sin(2.0 * math.pi * s)
    return euler_conserved(rho, [1.0] * D, 1.0)


def explosion(X, r0=0.5, inside=(1.0, 1.0), outside=(0.125, 0.1)):
    """Spherical explosion (multi-dimensional Sod problem, Sec. 6.1): (rho, p) = inside for
    |x| < r0, else outside; zero velocity; centre at the origin."""
    D = len(X)
    r2 = sum(x * x for x in X)
    ins = r2 < r0 * r0
    rho = np.where(ins, inside[0], outside[0])
    p = np.where(ins, inside[1], outside[1])
    return euler_conserved(rho, [0.0] * D, p)


def constant_state(X, rho=1.0, vel=None, p=1.0):
    D = len(X)
    vel = vel if vel is not None else [0.3, -0.2, 0.1][:D]
    shape = X[0].shape
    return euler_conserved(np.full(shape, rho), vel, np.full(shape, p))


# ------------------------------------------------------------------------------------------
# Elastic workloads (Sec. 6.2): units km, s, g/cm^3 (so lambda, mu in GPa).
def swe_flow_over_bump(X, L=1.0):
    """Shallow water (h, hu, hv, b) on a periodic box of side L: a smooth periodic bathymetry with
    a moving, perturbed surface (every term of the system active).  X: node coordinates (x, y)."""
    x, y = X
    b = 0.1 + 0.05 * np.sin(2 * math.pi * x / L) * np.cos(2 * math.pi * y / L)
    h = 1.0 - b + 0.02 * np.cos(2 * math.pi * (x + 2 * y) / L)
    hu = 0.3 * h * (1 + 0.1 * np.sin(2 * math.pi * y / L))
    hv = -0.2 * h * (1 + 0.1 * np.cos(2 * math.pi * x / L))
    return np.stack([h, hu, hv, b], axis=-1)


def swe_lake_at_rest(X, L=1.0, level=1.0):
    """Shallow water at rest over the bathymetry of swe_flow_over_bump: h + b = level, no flow."""
    x, y = X
    b = 0.1 + 0.05 * np.sin(2 * math.pi * x / L) * np.cos(2 * math.pi * y / L)
    h = level - b
    return np.stack([h, 0.0 * h, 0.0 * h, b], axis=-1)


def smooth_field(ncell, seed, modes=8, min_wavelength_cells=8.0):
    """Seeded smooth field in [0,1] on the cell centres: sum of ``modes`` random Fourier modes
    with wavelengths >= ``min_wavelength_cells`` cells, affinely mapped to [0,1]."""
    rng = SplitMix64(seed)
    D = len(ncell)
    C = int(np.prod(ncell))
    c = np.arange(C)
    centre = []
    for d in range(D):
        centre.append((c % ncell[d] + 0.5) / ncell[d])
        c = c // ncell[d]
    f = np.zeros(C)
    nmin = min(ncell)
    kmax = max(1.0, nmin / min_wavelength_cells)
    for _ in range(modes):
        k = [(2.0 * rng.uniform() - 1.0) * kmax for _ in range(D)]
        phase = 2.0 * math.pi * rng.uniform()
        amp = 0.5 + rng.uniform()
        f += amp * np.cos(2.0 * math.pi * sum(k[d] * centre[d] for d in range(D)) + phase)
    lo, hi = f.min(), f.max()
    if hi - lo < 1e-300:
        return np.full(C, 0.5)
    return (f - lo) / (hi - lo)


def elastic_material(ncell, seed, rho_range=(2.5, 3.0), vp_range=(5.0, 7.0)):
    """Per-cell (rho, lambda, mu) with rho, vp from two seeded smooth fields and vs = vp / sqrt(3)
    (so lambda = mu = rho vs^2).  Returns float64 [C, 3]."""
    f1 = smooth_field(ncell, seed)
    f2 = smooth_field(ncell, seed ^ 0x5DEECE66D)
    rho = rho_range[0] + (rho_range[1] - rho_range[0]) * f1
    vp = vp_range[0] + (vp_range[1] - vp_range[0]) * f2
    vs = vp / math.sqrt(3.0)
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    return np.stack([rho, lam, mu], axis=-1)


def locate(x, ncell, lo, hi):
    """Cell index and reference coordinates of point x (half-open cells [x_k, x_k+1); the last
    cell also owns the upper domain face)."""
    idx, xi = [], []
    for d in range(len(ncell)):
        h = (hi[d] - lo[d]) / ncell[d]
        s = (x[d] - lo[d]) / h
        k = int(math.floor(s))
        k = min(max(k, 0), ncell[d] - 1)
        idx.append(k)
        xi.append(s - k)
    c = 0
    stride = 1
    for d in range(len(ncell)):
        c += idx[d] * stride
        stride *= ncell[d]
    return c, xi


def moment_tensor(seed=None):
    """Moment tensor (xx, yy, zz, xy, xz, yz); a fixed double-couple-like tensor, or a seeded one."""
    if seed is None:
        return np.array([0.0, 0.0, 0.0, 1.0, 0.0, 0.0])
    rng = SplitMix64(seed)
    return np.array([2.0 * rng.uniform() - 1.0 for _ in range(6)])


def receivers_top(ncell, lo, hi, nside=8):
    """nside x nside receivers on the top face z = hi[2] at ((i+1/2) L/nside, (j+1/2) L/nside)."""
    pts = []
    for j in range(nside):
        for i in range(nside):
            pts.append([lo[0] + (i + 0.5) * (hi[0] - lo[0]) / nside,
                        lo[1] + (j + 0.5) * (hi[1] - lo[1]) / nside, hi[2]])
    return np.array(pts)


def plane_wave_elastic(X, material, t=0.0, kind='p', direction=(1.0, 0.0, 0.0), L=1.0, amp=1.0):
    """Exact plane P or S wave in a homogeneous medium (rho, lambda, mu), periodic over length L
    along the coordinate axis ``direction``: v = amp a sin(2 pi (x_d - c t)/L) with polarisation
    a = n (P, c = vp) or a perpendicular to n (S, c = vs), and the stress that makes it a
    travelling solution of the velocity-stress system, sigma = -(1/c) [lambda (a.n) I +
    mu (a n^T + n a^T)] amp sin(.)."""
    rho, lam, mu = material
    n = np.asarray(direction, dtype=np.float64)
    d = int(np.argmax(np.abs(n)))
    if kind == 'p':
        a = n.copy()
        c = math.sqrt((lam + 2 * mu) / rho)
    else:
        a = np.zeros(3)
        a[(d + 1) % 3] = 1.0
        c = math.sqrt(mu / rho)
    phase = 2.0 * math.pi * (X[d] - c * t) / L
    s = amp * np.sin(phase)
    v = [a[i] * s for i in range(3)]
    # From d sigma/dt = E : grad v with v = a f(x_d - c t):  sigma = -(1/c) [lam (a.n) I + mu (a n^T + n a^T)] f
    an = float(a @ n)
    S = np.zeros((3, 3))
    for i in range(3):
        S[i, i] += lam * an
        for j in range(3):
            S[i, j] += mu * (a[i] * n[j] + n[i] * a[j])
    S = -S / c
    sig = [S[0, 0] * s, S[1, 1] * s, S[2, 2] * s, S[0, 1] * s, S[0, 2] * s, S[1, 2] * s]
    return np.stack(v + sig, axis=-1)


def ensemble_sides(nruns=16, seed=20190520, choices=(24, 32, 40, 48, 64)):
    rng = SplitMix64(seed)
    return [choices[rng.next_u64() % len(choices)] for _ in range(nruns)]


# ------------------------------------------------------------------------------------------
# Named workloads (sizes of the paper-shaped scenarios).
WORKLOADS = {
    'euler2d_p3_27': dict(pde='euler', dim=2, order=3, ncell=(27, 27), lo=(0.0, 0.0), hi=(1.0, 1.0),
                          bc='periodic', t_end=1.0, init='entropy_wave'),
    'euler3d_p4_81': dict(pde='euler', dim=3, order=4, ncell=(81, 81, 81), lo=(0.0,) * 3, hi=(1.0,) * 3,
                          bc='periodic', steps=50, init='entropy_wave'),
    'elastic3d_p5_81': dict(pde='elastic', dim=3, order=5, ncell=(81, 81, 81), lo=(0.0,) * 3,
                            hi=(40.5,) * 3, bc='absorbing', steps=300, init='zero', seed=1905),
    'explosion3d_p3_64': dict(pde='euler', dim=3, order=3, ncell=(64, 64, 64), lo=(-1.0,) * 3,
                              hi=(1.0,) * 3, bc='wall', steps=200, init='explosion', limiter=True),
}
