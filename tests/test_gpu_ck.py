"""GPU parity of the Cauchy-Kowalevski predictor of the 3-D elastic family (Sec. 2, Sec. 3.3: the
predictor of linear PDEs evaluated by the Cauchy-Kowalevski procedure) against the oracle's
Cauchy-Kowalevski step, through the C ABI."""
import numpy as np
import pytest
import torch

from cases import Case, rel_linf
from oracle.aderdg import ADERDG, Grid, PointSource
from oracle.pde import Elastic
from paper_1905_07987_gb300 import ader, synth

pytestmark = pytest.mark.gpu
TOL = 1e-12


def waves(X, L):
    """Four superposed plane waves (P along x; S along x, y and z): all nine components vary."""
    m = (2.7, 30.0, 25.0)
    return (synth.plane_wave_elastic(X, m, kind='p', L=L)
            + synth.plane_wave_elastic(X, m, kind='s', L=L / 2)
            + synth.plane_wave_elastic(X, m, kind='s', direction=(0.0, 1.0, 0.0), L=L / 3)
            + synth.plane_wave_elastic(X, m, kind='s', direction=(0.0, 0.0, 1.0), L=L / 2))


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 6])
def test_ck_elastic_step_with_source(order):
    """Absorbing boundaries, seeded material, point source, random state.  45 cells: the orders
    that put 16, 4 or 2 cells in one block (1-3) end on a ragged block."""
    ncell = (5, 3, 3)
    mat = synth.elastic_material(ncell, seed=order)
    c = Case("elastic", 3, order, ncell, hi=(2.5, 1.5, 1.5), bc="absorbing", material=mat,
             predictor="ck")
    rng = np.random.default_rng(100 + order)
    u0 = rng.standard_normal(c.shape)
    c.point_source((1.3, 0.7, 0.8), synth.moment_tensor(seed=7), 2.0, 0.5)
    c.set(u0)
    c.ctx.set_time(0.37)
    c.ctx.step()
    dt = c.ctx.last_dt()
    assert rel_linf(c.get(), c.oracle_step(u0, dt, 0.37)) <= TOL


def change_rel(got, ref, u0):
    """max over variables of max|got - ref| / max|ref - u0| (error relative to the step's change)."""
    nv = ref.shape[-1]
    g = got.reshape(-1, nv)
    r = ref.reshape(-1, nv)
    d = np.abs(r - u0.reshape(-1, nv)).max(axis=0)
    return float((np.abs(g - r).max(axis=0) / np.maximum(d, 1e-300)).max())


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 6])
def test_ck_mixed_step_with_source(order):
    """Mixed-precision form (float-float base term L u and a_1, binary32 higher Taylor terms)
    against the oracle's FP64 Cauchy-Kowalevski step: within 2e-6 of the step's change (binary32
    rounding, 6e-8, over sums of up to 18n + 24 terms)."""
    ncell = (5, 3, 3)
    mat = synth.elastic_material(ncell, seed=order)
    c = Case("elastic", 3, order, ncell, hi=(2.5, 1.5, 1.5), bc="absorbing", material=mat,
             predictor="ck", precision="mixed")
    rng = np.random.default_rng(200 + order)
    u0 = rng.standard_normal(c.shape)
    c.point_source((1.3, 0.7, 0.8), synth.moment_tensor(seed=7), 2.0, 0.5)
    c.set(u0)
    c.ctx.set_time(0.37)
    c.ctx.step()
    ref = c.oracle_step(u0, c.ctx.last_dt(), 0.37)
    assert change_rel(c.get(), ref, u0) < 2e-6


def test_ck_mixed_wide_magnitudes():
    """State values from 1e-40 to 1e3 and exact zeros: the float-float splits of the mixed form
    (integer-pipe bit operations, binary32 range) keep the step within the same bound."""
    ncell = (3, 3, 2)
    mat = synth.elastic_material(ncell, seed=9)
    c = Case("elastic", 3, 4, ncell, hi=(1.5, 1.5, 1.0), bc="absorbing", material=mat,
             predictor="ck", precision="mixed")
    rng = np.random.default_rng(31)
    u0 = rng.standard_normal(c.shape) * 10.0 ** rng.uniform(-40, 3, c.shape)
    u0[rng.random(c.shape) < 0.1] = 0.0
    c.set(u0)
    c.ctx.step()
    got = c.get()
    assert np.isfinite(got).all()
    ref = c.oracle_step(u0, c.ctx.last_dt())
    assert change_rel(got, ref, u0) < 2e-6


# Tensor-core form (TF32 split operands, FP32 accumulation): every contraction carries a relative
# error eps_tc <= 3 x 2^-22 (split truncations and the dropped lo x lo product) + 3n x 2^-24 (FP32
# accumulation of the three n-term products) ~ 2e-6 of sum_m |table_im| |x_m|; relative to the
# step's change this is multiplied by the cancellation ratio sum |D| |u| / |D u|, about 1.5 on
# random states and up to ~10 on the smooth waves of the full-size test.
TOL_TC_RANDOM = 2e-5
TOL_TC_SMOOTH = 5e-5


@pytest.mark.parametrize("order", [1, 3, 5])
def test_ck_tf32x3_step_with_source(order):
    """Every contraction on the tensor cores (ADER_PREC_MIXED_TF32X3) against the oracle's FP64
    Cauchy-Kowalevski step, random state, point source, absorbing boundaries; 45 cells on the
    persistent blocks (more blocks than cells at order 1 and 3 on 152 SMs)."""
    ncell = (5, 3, 3)
    mat = synth.elastic_material(ncell, seed=order)
    c = Case("elastic", 3, order, ncell, hi=(2.5, 1.5, 1.5), bc="absorbing", material=mat,
             predictor="ck", precision="tf32x3")
    rng = np.random.default_rng(300 + order)
    u0 = rng.standard_normal(c.shape)
    c.point_source((1.3, 0.7, 0.8), synth.moment_tensor(seed=7), 2.0, 0.5)
    c.set(u0)
    c.ctx.set_time(0.37)
    c.ctx.step()
    c.ctx.sync()
    ref = c.oracle_step(u0, c.ctx.last_dt(), 0.37)
    err = change_rel(c.get(), ref, u0)
    print("tf32x3 order %d: error / step change %.3e" % (order, err))
    assert err < TOL_TC_RANDOM


def test_ck_tf32x3_many_cells_and_steps_track_fp64():
    """12^3 cells (each persistent block loops over several cells, the next cell's state
    prefetched by TMA), 6 steps with a source: the state stays within a small multiple of the
    one-step bound of the FP64 Cauchy-Kowalevski run."""
    ncell = (12, 12, 12)
    L = 6.0
    mat = synth.elastic_material(ncell, seed=4)
    out = {}
    for prec in ("fp64", "tf32x3"):
        c = Case("elastic", 3, 5, ncell, hi=(L,) * 3, bc="absorbing", material=mat,
                 predictor="ck", precision=prec)
        x, _ = ader.reference_nodes(5)
        u0 = waves(c.X, L)
        c.point_source((L / 2,) * 3, synth.moment_tensor(seed=3), 2.0, 0.5)
        c.set(u0)
        c.ctx.set_time(0.45)
        c.ctx.run(6)
        out[prec] = c.get()
        c.ctx.close()
    d = np.abs(out["tf32x3"] - out["fp64"]).max()
    scale = np.abs(out["fp64"] - u0).max()
    print("tf32x3 6 steps: |diff| / |change| %.3e" % (d / scale))
    assert d <= 6 * TOL_TC_SMOOTH * scale


def test_ck_tf32x3_is_rejected_where_it_is_not_built():
    for kw in (dict(pde="elastic", order=4, predictor="ck"), dict(pde="elastic", order=5, predictor="picard"),
               dict(pde="euler", order=3, predictor="picard")):
        cfg = ader.make_config(kw["pde"], 3, kw["order"], (2, 2, 2), (0,) * 3, (1,) * 3,
                               "absorbing" if kw["pde"] == "elastic" else "periodic",
                               synth.cfl_number(kw["order"]), predictor=kw["predictor"],
                               precision="tf32x3")
        with pytest.raises(ader.AderError) as e:
            ader.Context(cfg)
        assert e.value.status == ader.EUNSUPPORTED, kw


def test_ck_periodic_multistep_and_receivers():
    ncell = (4, 3, 3)
    mat = synth.elastic_material(ncell, seed=12)
    c = Case("elastic", 3, 4, ncell, hi=(2.0, 1.5, 1.5), bc="periodic", material=mat,
             predictor="ck")
    u0 = waves(c.X, 1.5)
    pts = synth.receivers_top(ncell, c.lo, c.hi, nside=3)
    seismo = c.receivers(pts, 8)
    c.point_source((0.9, 0.8, 0.7), synth.moment_tensor(seed=3), 2.0, 0.5)
    c.set(u0)
    c.ctx.set_time(0.4)
    u = torch.from_numpy(u0)
    t = 0.4
    rec = []
    for _ in range(6):
        dt = float(c.oracle.cfl_dt(u))
        u = c.oracle.step(u, torch.tensor(dt, dtype=torch.float64), t)
        t += dt
        rec.append(c.oracle.record(u).numpy())
    c.ctx.run(6)
    assert rel_linf(c.get(), u.numpy()) <= 10 * TOL
    got = seismo[:6].cpu().numpy()
    ref = np.stack(rec)
    assert np.abs(got - ref).max() <= 10 * TOL * np.abs(ref).max()


@pytest.mark.parametrize("order", [2, 4])
def test_ck_and_picard_steps_agree_on_polynomial_data(order):
    """Homogeneous material and data of total degree <= N: both predictors give the exact local
    solution, so the CUDA Cauchy-Kowalevski and Picard steps agree (a check that does not go
    through the oracle)."""
    ncell = (3, 2, 2)
    mat = np.tile(np.array([2.6, 28.0, 24.0]), (12, 1))
    out = {}
    for kind in ("picard", "ck"):
        c = Case("elastic", 3, order, ncell, hi=(1.5, 1.0, 1.0), bc="absorbing", material=mat,
                 predictor=kind)
        X = c.X
        rng = np.random.default_rng(5)
        u0 = np.zeros(c.shape)
        for v in range(9):
            cf = rng.standard_normal(4)
            u0[..., v] = (cf[0] + cf[1] * X[0] + cf[2] * X[1] * X[2] ** (order - 2)
                          + cf[3] * X[2] ** order)
        c.set(u0)
        c.ctx.step(dt=2e-3)
        out[kind] = c.get()
    assert rel_linf(out["ck"], out["picard"]) <= 1e-11


def test_ck_is_rejected_where_it_is_not_built():
    # the adjoint of the CK step is built for orders 1-5 (the forward CK predictor for 1-6)
    cfg = ader.make_config("elastic", 3, 6, (2, 2, 2), (0,) * 3, (1,) * 3, "absorbing",
                           synth.cfl_number(6), predictor="ck")
    c = ader.Context(cfg)
    c.set_material(torch.from_numpy(synth.elastic_material((2, 2, 2), seed=1).reshape(-1).copy()).cuda())
    u = torch.zeros(c.count, dtype=torch.float64, device="cuda")
    lam = torch.zeros_like(u)
    gm = torch.zeros(8 * 3, dtype=torch.float64, device="cuda")
    gM = torch.zeros(6, dtype=torch.float64, device="cuda")
    for static in (False, True):
        with pytest.raises(ader.AderError) as e:
            c.adjoint_step(0.0, 1e-3, u, lam, gm, gM, static=static)
        assert e.value.status == ader.EUNSUPPORTED
    c.close()
    euler = ader.make_config("euler", 3, 3, (2, 2, 2), (0,) * 3, (1,) * 3, "periodic",
                             synth.cfl_number(3), predictor="ck")
    with pytest.raises(ader.AderError) as e:
        ader.Context(euler)
    assert e.value.status == ader.EUNSUPPORTED


@pytest.mark.parametrize("precision", ["fp64", "mixed", "tf32x3"])
def test_ck_full_size_sampled_cells_elastic_81(precision):
    """81^3 cells at order 5 (FP64 and mixed form), the benchmark's elastic workload (seeded material, absorbing
    boundaries, Ricker moment-tensor source at the centre) with a smooth wave state, in the launch
    configuration the benchmark times.  Sampled cells (the source cell, a face neighbour of it,
    corners of the interior and random ones) are checked against the oracle's Cauchy-Kowalevski
    step on their 3x3x3 neighbourhood (a cell's update depends only on itself and its face
    neighbours)."""
    N, n, h = 5, 81, 0.5
    L = n * h
    x, _ = ader.reference_nodes(N)
    matn = synth.elastic_material((n,) * 3, seed=1905)
    M = synth.moment_tensor()
    cfg = ader.make_config("elastic", 3, N, (n,) * 3, (0,) * 3, (L,) * 3, "absorbing",
                           synth.cfl_number(N), predictor="ck", precision=precision)
    ctx = ader.Context(cfg)
    ctx.set_material(torch.from_numpy(matn.reshape(-1).copy()).cuda())
    ctx.set_point_source((L / 2,) * 3, M, 2.0, 0.5)
    slab_cache = {}

    def slab(k):  # the state of the cells of layer k, [n*n, 6, 6, 6, 9]
        if k not in slab_cache:
            X = synth.node_coordinates(x, (n, n, 1), (0.0, 0.0, k * h), (L, L, (k + 1) * h))
            slab_cache[k] = waves(X, L)
        return slab_cache[k]

    per = n * n * 216 * 9
    u = torch.empty(ctx.count, dtype=torch.float64, device="cuda")
    for k in range(n):
        u[k * per:(k + 1) * per].copy_(torch.from_numpy(slab(k).reshape(-1)))
        if k > 2:
            slab_cache.pop(k - 3, None)
    ctx.set_state(u)
    del u
    slab_cache.clear()
    ctx.set_time(0.45)
    ctx.step()
    dt = ctx.last_dt()
    got = torch.empty(ctx.count, dtype=torch.float64, device="cuda")
    ctx.get_state(got)
    torch.cuda.synchronize()
    got = got.view(n ** 3, -1)
    sc, sxi = synth.locate((L / 2,) * 3, (n,) * 3, (0.0,) * 3, (L,) * 3)
    si, sj, sk = sc % n, (sc // n) % n, sc // (n * n)
    rng = np.random.default_rng(0)
    samples = [(si, sj, sk), (si + 1, sj, sk), (1, 1, 1), (79, 79, 79), (40, 7, 63)]
    samples += [tuple(int(v) for v in rng.integers(1, 80, 3)) for _ in range(3)]
    for (i, j, k) in samples:
        idx, loc = [], []
        for dk in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    idx.append((i + di) + n * ((j + dj) + n * (k + dk)))
                    loc.append(slab(k + dk)[(i + di) + n * (j + dj)])
        sub = ADERDG(Elastic(), Grid((3, 3, 3), ((i - 1) * h, (j - 1) * h, (k - 1) * h),
                                     ((i + 2) * h, (j + 2) * h, (k + 2) * h),
                                     [("periodic", "periodic")] * 3), N,
                     cfl=synth.cfl_number(N), material=torch.from_numpy(matn[idx]), predictor="ck")
        if sc in idx:
            sub.set_point_source(PointSource(idx.index(sc), sxi, torch.tensor(M), 2.0, 0.5))
        out = sub.step(torch.from_numpy(np.stack(loc)), torch.tensor(dt, dtype=torch.float64),
                       0.45).numpy()
        centre = i + n * (j + n * k)
        g = got[centre].cpu().numpy().reshape(out[13].shape)
        if precision == "fp64":
            assert rel_linf(g, out[13]) <= TOL, (i, j, k)
        elif precision == "mixed":
            assert change_rel(g, out[13], loc[13]) < 2e-6, (i, j, k)
        else:
            # the TF32 error of a face value is relative to the data of the cell it comes from:
            # next to the source cell the scale is that cell's (much larger) change, so the error
            # is measured against the largest change in the 3x3x3 neighbourhood
            nv = out.shape[-1]
            chg = np.abs(out - np.stack(loc)).reshape(-1, nv).max(axis=0)
            err = float((np.abs(g - out[13]).reshape(-1, nv).max(axis=0) / np.maximum(chg, 1e-300)).max())
            print("tf32x3 81^3 cell %s: error / neighbourhood step change %.3e" % ((i, j, k), err))
            assert err < TOL_TC_SMOOTH, (i, j, k)
    ctx.close()


@pytest.mark.parametrize("predictor", ["picard", "ck"])
def test_elastic_nonfinite_state_is_reported(predictor):
    """A NaN in the elastic state reaches the new state through the update u^n + dt (...), where
    the corrector latches it (the CFL kernel reads only the material): ADER_ENONFINITE at the next
    ader_sync, with the CFL dt and with a fixed dt; a clean state afterwards steps normally."""
    ncell = (4, 3, 4)
    mat = synth.elastic_material(ncell, seed=3)
    c = Case("elastic", 3, 3, ncell, lo=(0.0,) * 3, hi=tuple(0.5 * n for n in ncell),
             bc="absorbing", material=mat, predictor=predictor)
    u0 = waves(c.X, 2.0)
    bad = u0.copy()
    bad[5, 1, 2, 0, 4] = np.nan
    for dt in (0.0, 1e-3):
        c.set(bad)
        c.ctx.step(dt)
        with pytest.raises(ader.AderError) as e:
            c.ctx.sync()
        assert e.value.status == ader.ENONFINITE, dt
    c.set(u0)
    c.ctx.step()
    c.ctx.sync()
