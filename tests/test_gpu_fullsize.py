"""Parity at the full sizes of the benchmark's workloads, in the launch configurations the
benchmark times, where the oracle cannot run the whole grid:

* the 64^3 order-3 spherical explosion with the a-posteriori limiter (Sec. 3.5): teacher-forced
  5x5x5 neighbourhoods of sampled cells (front cells, their fixed neighbours, wall and corner
  cells) at steps with thousands of troubled cells, and a 200-step run checked for
  conservation, positivity and the symmetry of the troubled set;
* the adjoint of the order-4 elastic step on 40^3 cells (Picard and Cauchy-Kowalevski forms, the
  latter also mixed-precision): the dot-product identity between the forward step and the
  adjoint step, and a central finite difference of the material gradient.

A cell's limited update depends on cells at most two cells away (its candidate and DMP bounds on
its face neighbours, the FV recompute of a face neighbour on that neighbour's 3^3 neighbourhood
of t^n representations), so the oracle on the 5x5x5 block around it (clipped at the walls)
reproduces it exactly."""
import numpy as np
import pytest
import torch

from oracle.aderdg import ADERDG, Grid
from oracle.limiter import Limiter
from oracle.pde import Euler
from paper_1905_07987_gb300 import ader, synth

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(autouse=True, scope="module")
def _build():
    from paper_1905_07987_gb300 import build
    build.build()


N_EXP, NC_EXP = 3, 64


def explosion_ctx(n=NC_EXP, N=N_EXP, limiter=1, precision="fp64"):
    x, w = ader.reference_nodes(N)
    X = synth.node_coordinates(x, (n,) * 3, (-1,) * 3, (1,) * 3)
    ns = 2 * N + 1
    Us = synth.explosion(synth.subcell_centres(ns, (n,) * 3, (-1,) * 3, (1,) * 3))
    fl = synth.discontinuous_cells(Us)
    cfg = ader.make_config("euler", 3, N, (n,) * 3, (-1,) * 3, (1,) * 3, "wall",
                           synth.cfl_number(N), limiter=limiter, precision=precision)
    ctx = ader.Context(cfg)
    ctx.set_state(torch.from_numpy(synth.explosion(X).reshape(-1).copy()).cuda())
    ctx.set_subcell_state(torch.from_numpy(Us.reshape(-1).copy()).cuda(),
                          torch.from_numpy(fl.astype(np.uint8)).cuda())
    return ctx, w


def dev_state(ctx):
    t = torch.empty(ctx.count, dtype=torch.float64, device="cuda")
    ctx.get_state(t)
    return t


def dev_rep(ctx, ns):
    t = torch.empty(ctx.cells * ns ** 3 * ctx.nvar, dtype=torch.float64, device="cuda")
    ctx.get_subcell_state(t)
    return t


def block_of(centre, n):
    """Cell ranges [lo, hi] per direction of the 5x5x5 block around `centre`, clipped at the
    walls, and the block's cell indices (x fastest)."""
    rng = [(max(0, c - 2), min(n - 1, c + 2)) for c in centre]
    idx = [i + n * (j + n * k)
           for k in range(rng[2][0], rng[2][1] + 1)
           for j in range(rng[1][0], rng[1][1] + 1)
           for i in range(rng[0][0], rng[0][1] + 1)]
    return rng, idx


def oracle_block(rng, n, N):
    h = 2.0 / n
    nc = tuple(b - a + 1 for a, b in rng)
    lo = tuple(-1.0 + h * a for a, _ in rng)
    hi = tuple(-1.0 + h * (b + 1) for _, b in rng)
    s = ADERDG(Euler(3), Grid(nc, lo, hi, [("wall", "wall")] * 3), N, cfl=synth.cfl_number(N))
    return s, Limiter(s)


def pick_samples(flags, n, rng):
    """Front cells (troubled), untroubled cells next to one (their face flux is fixed), cells on
    the walls and a corner, and random cells."""
    F = flags.reshape(n, n, n).astype(bool)  # [k][j][i]
    tr = np.argwhere(F)
    nb = np.zeros_like(F)
    for ax in range(3):
        for sh in (-1, 1):
            r = np.roll(F, sh, axis=ax)
            # no wrap-around at the walls
            sl = [slice(None)] * 3
            sl[ax] = 0 if sh == 1 else n - 1
            r[tuple(sl)] = False
            nb |= r
    fixed = np.argwhere(nb & ~F)
    out = [tuple(int(v) for v in tr[i][::-1]) for i in rng.choice(len(tr), 3, replace=False)]
    out += [tuple(int(v) for v in fixed[i][::-1]) for i in rng.choice(len(fixed), 3, replace=False)]
    out += [(0, 0, 0), (n - 1, n // 2, 0), (n // 2, n - 1, 5)]
    out += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(2)]
    return out


def check_step_on_samples(ctx, n, N, rng):
    """Teacher forcing: the GPU's state and representation at t^n go into the oracle on the
    block around each sampled cell; after one GPU step the sampled cell's FV flag, state and
    representation must equal the oracle's.  Returns the number of troubled cells."""
    ns = 2 * N + 1
    nn = (N + 1) ** 3
    u = dev_state(ctx).view(ctx.cells, nn, 5)
    rep = dev_rep(ctx, ns).view(ctx.cells, ns ** 3, 5)
    scale = u.abs().amax(dim=(0, 1)).cpu().numpy()
    ctx.step()
    dt = ctx.last_dt()
    flags = ctx.flags()
    u1 = dev_state(ctx).view(ctx.cells, nn, 5)
    rep1 = dev_rep(ctx, ns).view(ctx.cells, ns ** 3, 5)
    scale = np.maximum(scale, u1.abs().amax(dim=(0, 1)).cpu().numpy())
    samples = pick_samples(flags, n, rng)
    for centre in samples:
        br, idx = block_of(centre, n)
        s, lim = oracle_block(br, n, N)
        it = torch.tensor(idx, device="cuda")
        ub = u[it].cpu().reshape((len(idx),) + (N + 1,) * 3 + (5,))
        rb = rep[it].cpu().reshape((len(idx),) + (ns,) * 3 + (5,))
        un, tr, rn, ok = lim.step(ub, rb, torch.tensor(dt, dtype=torch.float64))
        cid = centre[0] + n * (centre[1] + n * centre[2])
        loc = (centre[0] - br[0][0]) + s.grid.ncell[0] * (
            (centre[1] - br[1][0]) + s.grid.ncell[1] * (centre[2] - br[2][0]))
        assert bool(flags[cid]) == bool(tr[loc]), centre
        got = u1[cid].cpu().numpy()
        ref = un[loc].reshape(nn, 5).numpy()
        assert (np.abs(got - ref).max(axis=0) <= TOL * scale).all(), (centre, np.abs(got - ref).max(axis=0) / scale)
        gr = rep1[cid].cpu().numpy()
        rr = rn[loc].reshape(ns ** 3, 5).numpy()
        assert (np.abs(gr - rr).max(axis=0) <= TOL * scale).all(), (centre, "rep")
    del u, rep, u1, rep1
    torch.cuda.empty_cache()
    return int(flags.sum())


def test_explosion_64_sampled_neighbourhoods_match_the_oracle():
    """64^3 cells, order 3, wall boundaries, limiter on (FP64): at a step with more than 5000
    troubled cells (multi-block compaction, the FV recompute over thousands of blocks) sampled
    cells equal the oracle on their neighbourhood."""
    ctx, _ = explosion_ctx()
    for _ in range(5):
        ctx.step()
    ctx.sync()
    assert ctx.troubled_count() >= 5000, ctx.troubled_count()
    ntr = check_step_on_samples(ctx, NC_EXP, N_EXP, np.random.default_rng(4))
    assert ntr >= 5000
    ctx.close()


def test_explosion_64_200_steps_conserve_and_stay_admissible():
    """200 steps of the 64^3 explosion (the workload's length): mass and energy conserved to
    round-off, density and pressure positive, the troubled set symmetric under the reflections and
    axis permutations of the cube up to cells that flip at round-off of a DMP bound; sampled
    neighbourhoods still equal the oracle at the last step."""
    ctx, w = explosion_ctx()
    W = torch.from_numpy(np.einsum("i,j,k->ijk", w, w, w).reshape(-1)).cuda()

    def totals():
        st = dev_state(ctx).view(ctx.cells, -1, 5)
        return (st * W[None, :, None]).sum(dim=(0, 1)).cpu().numpy()

    m0 = totals()
    for _ in range(199):
        ctx.step()
    ctx.sync()
    ntr = check_step_on_samples(ctx, NC_EXP, N_EXP, np.random.default_rng(9))
    ctx.sync()
    m1 = totals()
    assert abs(m1[0] - m0[0]) <= 1e-12 * abs(m0[0])
    assert abs(m1[4] - m0[4]) <= 1e-12 * abs(m0[4])
    st = dev_state(ctx).view(ctx.cells, -1, 5)
    rho = st[..., 0]
    p = 0.4 * (st[..., 4] - 0.5 * (st[..., 1:4] ** 2).sum(-1) / rho)
    assert float(rho.min()) > 0 and float(p.min()) > 0
    F = ctx.flags().reshape(NC_EXP, NC_EXP, NC_EXP).astype(bool)
    asym = 0
    for G in (F[::-1], F[:, ::-1], F[:, :, ::-1], F.transpose(0, 2, 1), F.transpose(2, 1, 0)):
        asym = max(asym, int((G != F).sum()))
    assert ntr > 0 and asym <= max(8, ntr // 200), (asym, ntr)
    ctx.close()


# (predictor, adjoint precision, dot-product tolerance, finite-difference tolerance).  The mixed
# CK adjoint (float-float base term, binary32 level corrections) is compared with the FP64 forward
# step: its binary32 parts leave ~1e-7 of |x| |y| on these random (not smooth) vectors.
ADJ40 = [("picard", "fp64", 1e-13, 1e-6), ("ck", "fp64", 1e-13, 1e-6), ("ck", "mixed", 1e-6, 1e-5)]


@pytest.mark.parametrize("predictor,precision,tol_dot,tol_fd", ADJ40)
def test_adjoint_40_dot_product_and_material_derivative(predictor, precision, tol_dot, tol_fd):
    """Order-4 elastic step on 40^3 cells (the adjoint's multi-block launch at size; the Picard
    adjoint's per-block slabs, the CK adjoint's one block per cell): <A x, y> = <x, A^T y> for
    the FP64 forward step at fixed dt and the adjoint step, and the material gradient of
    <A(m) x, y> against a central finite difference of the FP64 forward step along a random
    direction."""
    n, N = 40, 4
    L = 0.5 * n
    mat = synth.elastic_material((n,) * 3, seed=1905)
    cfg = ader.make_config("elastic", 3, N, (n,) * 3, (0, 0, 0), (L,) * 3, "absorbing",
                           synth.cfl_number(N), predictor=predictor)
    ctx = ader.Context(cfg)
    mat_d = torch.from_numpy(mat.reshape(-1).copy()).cuda()
    ctx.set_material(mat_d)
    actx = ctx
    if precision != "fp64":
        actx = ader.Context(ader.make_config("elastic", 3, N, (n,) * 3, (0, 0, 0), (L,) * 3,
                                             "absorbing", synth.cfl_number(N),
                                             predictor=predictor, precision=precision))
        actx.set_material(mat_d)
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(ctx.count, dtype=torch.float64, device="cuda", generator=g)
    y = torch.randn(ctx.count, dtype=torch.float64, device="cuda", generator=g)
    vp = np.sqrt((mat[:, 1] + 2 * mat[:, 2]) / mat[:, 0]).max()
    dt = 0.8 * synth.cfl_number(N) / (3 * (2 * N + 1)) * 0.5 / vp

    def forward(m_d):
        ctx.set_material(m_d)
        ctx.set_state(x)
        ctx.set_time(0.0)
        ctx.step(dt=dt)
        return dev_state(ctx)

    Ax = forward(mat_d)
    lam = y.clone()
    gm = torch.zeros(ctx.cells * 3, dtype=torch.float64, device="cuda")
    gM = torch.zeros(6, dtype=torch.float64, device="cuda")
    actx.adjoint_step(0.0, dt, x, lam, gm, gM)
    actx.sync()
    lhs = float(torch.dot(Ax, y))
    rhs = float(torch.dot(x, lam))
    # normalised by |A x| |y|: one wrong face or cell term out of 64 000 cells would show at
    # ~1e-5, rounding at ~1e-16
    assert abs(lhs - rhs) <= tol_dot * float(Ax.norm() * y.norm()), (lhs, rhs)
    # directional derivative of <A(m) x, y> along a random per-cell perturbation that keeps every
    # cell's P-wave speed (rho, lam, mu scaled together, and lam + 2 mu held fixed), so that no
    # face's max(vp_L, vp_R) switches sides between the two evaluations
    r = np.random.default_rng(2)
    a = r.standard_normal(ctx.cells)
    b = r.standard_normal(ctx.cells)
    dmn = a[:, None] * mat + b[:, None] * np.stack([0 * mat[:, 2], -2 * mat[:, 2], mat[:, 2]], 1)
    dm = torch.from_numpy(dmn.reshape(-1).copy()).cuda()
    eps = 1e-5
    jp = float(torch.dot(forward(mat_d + eps * dm), y))
    jm = float(torch.dot(forward(mat_d - eps * dm), y))
    fd = (jp - jm) / (2 * eps)
    an = float(torch.dot(gm, dm))
    assert abs(fd - an) <= tol_fd * abs(an), (fd, an)
    ctx.close()
    if actx is not ctx:
        actx.close()
