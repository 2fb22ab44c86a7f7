"""Benchmark: ADER-DG DOF-updates/s of the GB300 library on the 3-D Euler entropy-wave workload
(81^3 cells, order 4, 5 variables: 332 M degrees of freedom), one JSON line on stdout.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--prec fp64]

A step is one ADER-DG time step of the whole grid (CFL reduction, predictor, Riemann solver,
corrector).  ``value`` is device-timed with CUDA events on the library's stream, the state
resident in HBM; ``e2e`` is the same metric through the C ABI with host buffers (host-to-device
copy of the state, the step, device-to-host copy of the new state, every step).  For N > 1 each
rank advances its own replica (the method needs no exchange between independent grids);
``value`` sums all ranks.  ``--impl reference`` times the CPU oracle on a bounded sample of the
same workload on this machine's cores.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "euler3d_p4_81": dict(pde="euler", dim=3, order=4, ncell=(81, 81, 81), lo=(0.0,) * 3,
                          hi=(1.0,) * 3, bc="periodic"),
    # smaller grid of the same scheme, used for single-kernel profiles (state 0.32 GB > L2)
    "euler3d_p4_40": dict(pde="euler", dim=3, order=4, ncell=(40, 40, 40), lo=(0.0,) * 3,
                          hi=(1.0,) * 3, bc="periodic"),
    "euler2d_p3_27": dict(pde="euler", dim=2, order=3, ncell=(27, 27), lo=(0.0,) * 2,
                          hi=(1.0,) * 2, bc="periodic"),
}
FP64_SMS, FP64_FMA_PER_CLK, SM_MAX_MHZ = 152, 2, 2070.0
# DRAM bytes (read + write) per cell of the predictor kernels, from one ncu capture of the same
# kernels on 40^3 cells, scaled to a launch by the number of cells (the traffic is per cell:
# state in, next state and face records out; the mixed form also writes the face wave speeds).
# FP64: k_predictor<Euler<3>,3,4> on 64 000 cells, read 331.102464 MB, write 1031.607040 MB;
# mixed (the kernel with the continuous extension Runge-Kutta stages, captured with that guess):
# read 320.445184 MB, write 1103.791872 MB.
TRAFFIC_PER_CELL = {"fp64": (331.102464e6 + 1031.607040e6) / 64000,
                    "mixed": (320.445184e6 + 1103.791872e6) / 64000}
FP64_PEAK = FP64_SMS * FP64_FMA_PER_CLK * 2 * SM_MAX_MHZ * 1e6  # FLOP/s


def predictor_flops_per_cell(pde, D, N, iters):
    """Algorithmic FP64 flops of the fused predictor kernel for one cell (FMA = 2 flops,
    add / multiply / divide = 1): per Picard iteration the nodal fluxes (aux 2D+5, D flux vectors
    of D+4) at the space-time nodes, the D derivative contractions and the time solve; then the
    epilogue (fluxes, time averages, volume term, face extrapolations)."""
    n = N + 1
    NST = n ** (D + 1)
    NV = D + 2
    NL = n ** D * NV
    NF = n ** (D - 1)
    cF = (2 * D + 5) + D * (D + 4)           # aux (1/rho, p) + D flux vectors per node
    it = cF * NST + D * NST * NV * (2 * n + 2) + NL * n * (2 * n + 2)
    epi = (cF * NST + (D + 1) * NL * 2 * n + D * NL * (6 * n + 5) + 2 * NL
           + 2 * D * NF * NV * 2 * n * 2)
    return iters * it + epi


def cerk_flops_per_cell(D, N):
    """Algorithmic FP64 flops of the continuous extension Runge-Kutta guess of an Euler cell:
    four stages, each the nodal fluxes and the D derivative contractions at one time level plus
    the stage state (one FMA per line), and the dense output (4 FMA per line and time node)."""
    n = N + 1
    NS = n ** D
    NV = D + 2
    NL = NS * NV
    cF = (2 * D + 5) + D * (D + 4)
    stage = cF * NS + D * NS * NV * (2 * n + 2) + 2 * NL
    return 4 * stage + NL * n * 8


def sample_clocks(stop_after_s):
    """nvidia-smi clock / throttle samples every 200 ms (started before the timed region)."""
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        return subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                text=True)
    except OSError:
        return None


def parse_clocks(proc, gpu_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            if int(f[0]) != gpu_index:
                continue
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
            "samples": len(sm)}


def build_initial(ader, synth, wl):
    x, _ = ader.reference_nodes(wl["order"])
    X = synth.node_coordinates(x, wl["ncell"], wl["lo"], wl["hi"])
    u = synth.entropy_wave(X)
    return u.reshape(-1)


def oracle_sample(wl, budget_s):
    """Time the CPU oracle on a bounded sample of the workload: a 6^3 (2-D: 12^2) periodic
    block of cells of the same size and order; returns (DOF-updates/s, description, threads)."""
    import torch

    from oracle.aderdg import ADERDG, Grid
    from oracle.pde import Euler
    from paper_1905_07987_gb300 import synth
    D, N = wl["dim"], wl["order"]
    m = 6 if D == 3 else 12
    h = (wl["hi"][0] - wl["lo"][0]) / wl["ncell"][0]
    g = Grid((m,) * D, (0.0,) * D, (m * h,) * D, [("periodic", "periodic")] * D)
    s = ADERDG(Euler(D), g, N, cfl=synth.cfl_number(N))
    X = s.node_coords()
    u = torch.from_numpy(synth.entropy_wave([x.numpy() for x in X]))
    s.step(u, s.cfl_dt(u))  # warm-up
    steps, t0 = 0, time.perf_counter()
    while True:
        u = s.step(u, s.cfl_dt(u))
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= 100000:
            break
    dofs = g.C * (N + 1) ** D * (D + 2)
    desc = "%d^%d periodic cells of the same h and order, %d oracle steps in %.1f s" % (m, D, steps, el)
    return dofs * steps / el, desc, torch.get_num_threads(), el / steps


FP32_PEAK = FP64_SMS * 128 * 2 * SM_MAX_MHZ * 1e6  # FLOP/s


def model_flops_per_cell(D, N, nv, iters, cF=30):
    """Algorithmic flops per cell and step of the predictor in the sum-factorised model (the
    contractions the method must do, no padding): I [2 (d+1) nv n^(d+2) + cF n^(d+1)] for the
    Picard iterations plus the epilogue 2 (2d+1) nv n^(d+1) + 12 d nv n^d, cF ~ 30 flops per
    space-time node for the flux.  785 k flop for the Euler order-4 cell."""
    n = N + 1
    it = 2 * (D + 1) * nv * n ** (D + 2) + cF * n ** (D + 1)
    epi = 2 * (2 * D + 1) * nv * n ** (D + 1) + 12 * D * nv * n ** D
    return iters * it + epi


def measure_fma_peaks(stream):
    """FP64 and binary32 FMA throughput of this GPU measured now (libpeaks.so: 8 independent FMA
    chains per thread, 8 blocks of 256 threads per SM, CUDA events on the bench stream); returns
    {"fp64": TFLOP/s, "fp32": TFLOP/s, ...} or None if the library is missing."""
    import ctypes
    import torch
    path = os.path.join(ROOT, "paper_1905_07987_gb300", "peaks", "libpeaks.so")
    if not os.path.exists(path):
        return None
    L = ctypes.CDLL(path)
    L.peaks_fma_launch.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_void_p]
    L.peaks_fma_launch.restype = ctypes.c_int
    L.peaks_fma_flops.argtypes = [ctypes.c_int, ctypes.c_int]
    L.peaks_fma_flops.restype = ctypes.c_double
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = sms * 8
    out = {"method": "8 independent FMA chains per thread, %d blocks x 256 threads, best of 3 "
                     "CUDA-event timed launches" % blocks}
    sink = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    for name, fp64, iters in (("fp64", 1, 4000), ("fp32", 0, 60000)):
        with torch.cuda.stream(stream):
            L.peaks_fma_launch(fp64, sink.data_ptr(), blocks, 200, stream.cuda_stream)  # warm-up
            best = None
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if L.peaks_fma_launch(fp64, sink.data_ptr(), blocks, iters, stream.cuda_stream) != 0:
                    return None
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
        out[name] = L.peaks_fma_flops(blocks, iters) / (best * 1e-3) / 1e12
        out[name + "_ms"] = best
    return out


def density_error(ctx, wl, t, nodes, weights):
    """(L2, Linf) error of the density against the exact entropy wave at time t, evaluated at the
    Gauss-Legendre nodes (L2 with the nodal quadrature) on the GPU with plain torch ops."""
    import torch
    D, N = wl["dim"], wl["order"]
    n = N + 1
    st = torch.empty(ctx.count, dtype=torch.float64, device="cuda")
    ctx.get_state(st)
    torch.cuda.synchronize()
    rho = st.view(ctx.cells, n ** D, D + 2)[:, :, 0]
    nc = wl["ncell"]
    lo, hi = wl["lo"], wl["hi"]
    c = torch.arange(ctx.cells, device="cuda")
    xi = torch.tensor(nodes, device="cuda", dtype=torch.float64)
    w = torch.tensor(weights, device="cuda", dtype=torch.float64)
    j = torch.arange(n ** D, device="cuda")
    s = torch.zeros(ctx.cells, n ** D, dtype=torch.float64, device="cuda")
    W = torch.ones(n ** D, dtype=torch.float64, device="cuda")
    rem_c, rem_j = c, j
    vol = 1.0
    for d in range(D):
        h = (hi[d] - lo[d]) / nc[d]
        vol *= h
        ic = rem_c % nc[d]
        rem_c = rem_c // nc[d]
        a = rem_j % n
        rem_j = rem_j // n
        s = s + (lo[d] + h * (ic[:, None].double() + xi[a][None, :]))
        W = W * w[a]
    ex = 1.0 + 0.2 * torch.sin(2 * math.pi * (s - D * t))
    err = rho - ex
    l2 = math.sqrt(float((err * err * W[None, :]).sum()) * vol)
    return l2, float(err.abs().max())


def density_l2_quadrature(ctx, wl, t, nodes, device="cuda"):
    """L2 error of the density against the exact entropy wave at time t with (N+2)-point
    Gauss-Legendre quadrature per cell and dimension (the nodal values interpolated there with
    the Lagrange basis of the solution nodes), on the GPU with plain torch ops.  Quadrature off
    the solution nodes avoids their superconvergence, so refinement shows the order N+1 of the
    scheme."""
    import torch
    D, N = wl["dim"], wl["order"]
    n, q = N + 1, N + 2
    xg, wg = np.polynomial.legendre.leggauss(q)
    xq, wq = (xg + 1.0) / 2.0, wg / 2.0
    V = np.ones((q, n))
    for a in range(n):
        for b in range(n):
            if b != a:
                V[:, a] *= (xq - nodes[b]) / (nodes[a] - nodes[b])
    st = torch.empty(ctx.count, dtype=torch.float64, device=device)
    ctx.get_state(st)
    if device == "cuda":
        torch.cuda.synchronize()
    nc, lo, hi = wl["ncell"], wl["lo"], wl["hi"]
    # node index j = a_0 + n a_1 + ...; cell index c = i_0 + nc_0 i_1 + ... (x fastest)
    rho = st.view(ctx.cells, n ** D, D + 2)[:, :, 0].reshape((ctx.cells,) + (n,) * D)
    Vt = torch.tensor(V, device=device)
    for ax in range(1, D + 1):
        rho = torch.movedim(torch.tensordot(rho, Vt, dims=([ax], [1])), -1, ax)
    c = torch.arange(ctx.cells, device=device)
    s = torch.zeros((ctx.cells,) + (q,) * D, dtype=torch.float64, device=device)
    W = torch.ones((q,) * D, dtype=torch.float64, device=device)
    xqt = torch.tensor(xq, device=device)
    wqt = torch.tensor(wq, device=device)
    vol = 1.0
    for d in range(D):
        h = (hi[d] - lo[d]) / nc[d]
        vol *= h
        ic = (c // math.prod(nc[:d])) % nc[d]
        shape = [1] * D
        shape[D - 1 - d] = q  # dimension d is tensor axis D-1-d (x is the last axis)
        s = s + (lo[d] + h * (ic.double().view((-1,) + (1,) * D) + xqt.view(shape)))
        W = W * wqt.view(shape)
    ex = 1.0 + 0.2 * torch.sin(2 * math.pi * (s - D * t))
    err = rho - ex
    return math.sqrt(float((err * err * W).sum()) * vol)


# Forms of the headline workload: (precision, initial guess of the Picard predictor, iterations;
# 0 = N+1).  The continuous extension Runge-Kutta guess (Sec. 5) is followed by max(1, N-3)
# iterations (order 4: one).
FORMS = {"fp64": ("fp64", "constant", 0), "mixed": ("mixed", "constant", 0),
         "mixed_cerk": ("mixed", "cerk", 1), "fp64_cerk": ("fp64", "cerk", 1)}


def run_form(ader, synth, wl, form, args, stream, u0_dev, err_steps):
    """Warm up, time K steps with CUDA events (plus per-phase events), then run untimed to
    err_steps steps in total and measure the density error against the exact solution."""
    import torch
    D, N = wl["dim"], wl["order"]
    prec, guess, iters = FORMS[form]
    cfg = ader.make_config(wl["pde"], D, N, wl["ncell"], wl["lo"], wl["hi"], wl["bc"],
                           synth.cfl_number(N), precision=prec, initial_guess=guess,
                           picard_iters=iters)
    ctx = ader.Context(cfg, stream=stream.cuda_stream)
    ctx.set_state(u0_dev)
    ctx.set_time(0.0)
    for _ in range(args.warmup):
        ctx.step()
    ctx.sync()
    clk = sample_clocks(0)
    time.sleep(0.3)
    ctx.enable_timing(True)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_total = e0.elapsed_time(e1)
    clocks = parse_clocks(clk, torch.cuda.current_device())
    phases, nrec = ctx.phase_times()
    ctx.enable_timing(False)
    ctx.sync()
    done = args.warmup + args.steps
    err = None
    if err_steps and err_steps > done:
        ctx.run(err_steps - done)
    if err_steps:
        x, w = ader.reference_nodes(N)
        t = ctx.time()
        l2, linf = density_error(ctx, wl, t, x, w)
        err = {"steps": max(done, err_steps), "t": t, "l2_rho": l2, "linf_rho": linf,
               "l2_rho_quadrature": density_l2_quadrature(ctx, wl, t, x)}
    return ctx, ms_total, phases, nrec, clocks, err


def _dev_state(ctx):
    import torch
    t = torch.empty(ctx.count, dtype=torch.float64, device="cuda")
    ctx.get_state(t)
    torch.cuda.synchronize()
    return t


def extra_euler2d(ader, synth, stream):
    """2-D entropy wave, order 3, 27^2 periodic cells, to t = 1 (CFL steps), replayed as CUDA
    graphs of 2 steps; DOF-updates/s and the density error against the exact solution."""
    import torch
    N, nc = 3, (27, 27)
    cfg = ader.make_config("euler", 2, N, nc, (0, 0), (1, 1), "periodic", synth.cfl_number(N))
    ctx = ader.Context(cfg, stream=stream.cuda_stream)
    x, w = ader.reference_nodes(N)
    u0 = torch.from_numpy(synth.entropy_wave(synth.node_coordinates(x, nc, (0, 0), (1, 1))).reshape(-1).copy()).cuda()
    torch.cuda.synchronize()
    ctx.set_state(u0)
    ctx.run_graph(2, 4, t_end=1.0)  # warm-up and capture
    ctx.sync()
    ctx.set_state(u0)
    ctx.set_time(0.0)
    steps = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    while True:
        ctx.run_graph(2, 64, t_end=1.0)
        steps += 128
        if ctx.time() >= 1.0 - 1e-14:
            break
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    wl = dict(dim=2, order=N, ncell=nc, lo=(0, 0), hi=(1, 1))
    l2, linf = density_error(ctx, wl, ctx.time(), x, w)
    dofs = 729 * 16 * 4
    ctx.close()
    return {"workload": "euler2d_p3_27 (entropy wave to t = 1)", "steps_launched": steps,
            "value": dofs * steps / (ms * 1e-3), "unit": "DOF-updates/s (incl. no-op steps after t_end)",
            "ms_total": ms, "l2_rho_vs_exact": l2, "linf_rho_vs_exact": linf, "dtype": "f64"}


def extra_elastic(ader, synth, stream, steps=2, warmup=1, n=81):
    """3-D elastic, order 5, 81^3 cells (h = 0.5 km), seeded material, moment-tensor Ricker source
    at the centre, 64 receivers on the top face: FP64 and mixed predictor; mixed vs FP64 state."""
    import torch
    N = 5
    L = 0.5 * n
    mat = torch.from_numpy(synth.elastic_material((n,) * 3, seed=1905).reshape(-1).copy()).cuda()
    out = {"workload": "elastic3d_p5_%d" % n, "dofs": n ** 3 * 216 * 9}
    finals = {}
    for form in ("fp64", "mixed", "ck", "ck_mixed", "ck_tf32x3"):
        prec = {"mixed": "mixed", "ck_mixed": "mixed", "ck_tf32x3": "tf32x3"}.get(form, "fp64")
        cfg = ader.make_config("elastic", 3, N, (n,) * 3, (0, 0, 0), (L,) * 3, "absorbing",
                               synth.cfl_number(N), precision=prec,
                               predictor="ck" if form.startswith("ck") else "picard")
        ctx = ader.Context(cfg, stream=stream.cuda_stream)
        ctx.set_material(mat)
        ctx.set_point_source((L / 2,) * 3, synth.moment_tensor(), 2.0, 0.5)
        seismo = torch.zeros(steps + warmup + 1, 64, 3, dtype=torch.float64, device="cuda")
        ctx.set_receivers(synth.receivers_top((n,) * 3, (0, 0, 0), (L,) * 3), seismo, steps + warmup + 1)
        ctx.set_state(torch.zeros(ctx.count, dtype=torch.float64, device="cuda"))
        ctx.set_time(0.45)  # near the wavelet peak so the source is active
        for _ in range(warmup):
            ctx.step()
        ctx.sync()
        ctx.enable_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ph, nr = ctx.phase_times()
        ctx.enable_timing(False)
        finals[form] = _dev_state(ctx)
        out[form] = {"ms_per_step": ms / steps, "value": out["dofs"] * steps / (ms * 1e-3),
                     "predictor_ms": ph["predictor"] / max(nr, 1),
                     "riemann_ms": ph["riemann"] / max(nr, 1),
                     "corrector_ms": ph["corrector"] / max(nr, 1)}
        ctx.close()
        del seismo
    d = (finals["mixed"] - finals["fp64"]).abs().max().item()
    scale = max(finals["fp64"].abs().max().item(), 1e-300)
    out["mixed_vs_fp64_rel_linf"] = d / scale
    out["mixed_speedup"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    # Cauchy-Kowalevski predictor: FP64-pipe roofline of its algorithmic flops per cell, N+1
    # applications of the spatial operator (18n+24 FMA per node: six derivatives along each
    # direction, eight rows of B_d), the Taylor update (9 MUL + 9 FMA per node, N times) and the
    # face extrapolation (6 n^2 9 dot products of length n)
    nn, NS = N + 1, (N + 1) ** 3
    flops_cell = (N + 1) * NS * 2 * (18 * nn + 24) + N * NS * 27 + 6 * nn * nn * 9 * 2 * nn
    ck = out["ck"]
    ck["predictor_tflops"] = flops_cell * n ** 3 / (ck["predictor_ms"] * 1e-3) / 1e12
    ck["predictor_flops_per_cell"] = flops_cell
    ck["predictor_frac_of_fp64_peak"] = ck["predictor_tflops"] * 1e12 / FP64_PEAK
    # mixed form: the same algorithmic (FP64-equivalent) flops against the FP32 pipe
    ckm = out["ck_mixed"]
    ckm["predictor_tflops"] = flops_cell * n ** 3 / (ckm["predictor_ms"] * 1e-3) / 1e12
    ckm["predictor_frac_of_fp32_peak"] = ckm["predictor_tflops"] * 1e12 / FP32_PEAK
    out["ck_speedup_vs_fp64_picard"] = out["fp64"]["ms_per_step"] / ck["ms_per_step"]
    out["ck_speedup_vs_mixed_picard"] = out["mixed"]["ms_per_step"] / ck["ms_per_step"]
    out["ck_mixed_speedup_vs_fp64_ck"] = ck["ms_per_step"] / ckm["ms_per_step"]
    out["ck_mixed_vs_fp64_ck_rel_linf"] = ((finals["ck_mixed"] - finals["ck"]).abs().max().item()
                                           / max(finals["ck"].abs().max().item(), 1e-300))
    # tensor-core form: the same algorithmic flops as tensor-pipe work (TF32 split operands)
    ckt = out["ck_tf32x3"]
    ckt["predictor_tflops"] = flops_cell * n ** 3 / (ckt["predictor_ms"] * 1e-3) / 1e12
    ckt["speedup_vs_ck_mixed"] = ckm["ms_per_step"] / ckt["ms_per_step"]
    ckt["predictor_speedup_vs_ck_mixed"] = ckm["predictor_ms"] / ckt["predictor_ms"]
    out["ck_tf32x3_vs_fp64_ck_rel_linf"] = ((finals["ck_tf32x3"] - finals["ck"]).abs().max().item()
                                            / max(finals["ck"].abs().max().item(), 1e-300))
    # the two predictors differ by their O(dt^(N+1)) truncation (a difference, not an error)
    out["ck_vs_picard_fp64_rel_linf"] = (finals["ck"] - finals["fp64"]).abs().max().item() / scale
    return out


def extra_cerk(ader, synth, stream, steps=2, warmup=1, err_steps=20):
    """81^3 order-4 Euler entropy wave in FP64: the Picard predictor from the constant guess with
    N+1 = 5 iterations against the continuous extension Runge-Kutta guess (order 4 in dt) with
    max(0, N-3) = 1 iteration; ms per step, predictor ms, and the density error against the
    exact solution after err_steps CFL steps for both."""
    import torch
    wl = WORKLOADS["euler3d_p4_81"]
    D, N = wl["dim"], wl["order"]
    u0 = torch.from_numpy(build_initial(ader, synth, wl)).to("cuda")
    dofs = math.prod(wl["ncell"]) * (N + 1) ** D * (D + 2)
    out = {"workload": "euler3d_p4_81, FP64, Picard from the constant guess (5 iterations) vs the "
                       "CERK guess (1 iteration)", "dofs": dofs}
    for name, guess, iters in (("constant_5", "constant", 0), ("cerk_1", "cerk", 1)):
        cfg = ader.make_config(wl["pde"], D, N, wl["ncell"], wl["lo"], wl["hi"], wl["bc"],
                               synth.cfl_number(N), picard_iters=iters, initial_guess=guess)
        ctx = ader.Context(cfg, stream=stream.cuda_stream)
        ctx.set_state(u0)
        ctx.set_time(0.0)
        for _ in range(warmup):
            ctx.step()
        ctx.sync()
        ctx.enable_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ph, nr = ctx.phase_times()
        ctx.enable_timing(False)
        ctx.run(err_steps - warmup - steps)
        x, w = ader.reference_nodes(N)
        l2, linf = density_error(ctx, wl, ctx.time(), x, w)
        out[name] = {"ms_per_step": ms / steps, "value": dofs * steps / (ms * 1e-3),
                     "predictor_ms": ph["predictor"] / max(nr, 1), "l2_rho": l2,
                     "steps_for_error": err_steps}
        ctx.close()
    cells = math.prod(wl["ncell"])
    for name, iters, extra in (("constant_5", N + 1, 0), ("cerk_1", 1, cerk_flops_per_cell(D, N))):
        fl = (predictor_flops_per_cell(wl["pde"], D, N, iters) + extra) * cells
        tf = fl / (out[name]["predictor_ms"] * 1e-3) / 1e12
        out[name]["predictor_tflops"] = tf
        out[name]["predictor_frac_of_fp64_peak"] = tf * 1e12 / FP64_PEAK
    out["cerk_speedup"] = out["constant_5"]["ms_per_step"] / out["cerk_1"]["ms_per_step"]
    out["cerk_over_constant_l2_error"] = out["cerk_1"]["l2_rho"] / out["constant_5"]["l2_rho"]
    return out


def extra_convergence(ader, synth, stream, res, sides=(27, 54)):
    """The 3-D order-4 entropy wave on coarser grids of the same domain, run with the same
    forms to the time the 81^3 forms reached after their error steps (the last step clipped to
    it); L2 density errors (quadrature off the nodes) at 27^3 / 54^3 / 81^3 and the observed
    orders between them (the scheme's is N+1 = 5)."""
    import torch
    base = WORKLOADS["euler3d_p4_81"]
    D, N = base["dim"], base["order"]
    x, _ = ader.reference_nodes(N)
    out = {"workload": "euler3d_p4 entropy wave at %s cells per side" % "/".join(
        str(v) for v in tuple(sides) + (base["ncell"][0],))}
    for form in ("fp64", "mixed_cerk"):
        if form not in res or not res[form]["err"]:
            continue
        T = res[form]["err"]["t"]
        errs, steps = [], []
        prec, guess, iters = FORMS[form]
        for n in sides:
            wl = dict(base, ncell=(n,) * 3)
            cfg = ader.make_config(wl["pde"], D, N, wl["ncell"], wl["lo"], wl["hi"], wl["bc"],
                                   synth.cfl_number(N), precision=prec, initial_guess=guess,
                                   picard_iters=iters)
            ctx = ader.Context(cfg, stream=stream.cuda_stream)
            ctx.set_state(torch.from_numpy(build_initial(ader, synth, wl)).to("cuda"))
            ctx.set_time(0.0)
            ctx.step(t_end=T)
            k = 1
            rest = max(0, int(math.ceil((T - ctx.time()) / ctx.last_dt())) + 1)
            while rest > 0 and ctx.time() < T * (1 - 1e-14):
                ctx.run(rest, t_end=T)
                k += rest
                rest = 1
            ctx.sync()
            errs.append(density_l2_quadrature(ctx, wl, ctx.time(), x))
            steps.append(k)
            ctx.close()
            torch.cuda.empty_cache()
        errs.append(res[form]["err"]["l2_rho_quadrature"])
        steps.append(res[form]["err"]["steps"])
        hs = list(sides) + [base["ncell"][0]]
        orders = [math.log(errs[i] / errs[i + 1]) / math.log(hs[i + 1] / hs[i])
                  for i in range(len(hs) - 1)]
        out[form] = {"t": T, "cells_per_side": hs, "steps": steps, "l2_rho": errs,
                     "observed_order": orders}
    if "fp64" in out and "mixed_cerk" in out:
        out["mixed_cerk_over_fp64"] = [m / f for m, f in zip(out["mixed_cerk"]["l2_rho"],
                                                              out["fp64"]["l2_rho"])]
    return out


def _adjoint_gradient_40(ader, synth, stream, n, N, steps, k, predictor, precision="fp64"):
    """One misfit gradient through ader_misfit_gradient (see extra_adjoint) with the given
    predictor; returns the timing record."""
    import torch
    L = 0.5 * n
    cells = n ** 3
    dofs = cells * (N + 1) ** 3 * 9
    mat = torch.from_numpy(synth.elastic_material((n,) * 3, seed=1905).reshape(-1).copy()).cuda()
    cfg = ader.make_config("elastic", 3, N, (n,) * 3, (0, 0, 0), (L,) * 3, "absorbing",
                           synth.cfl_number(N), predictor=predictor, precision=precision)
    ctx = ader.Context(cfg, stream=stream.cuda_stream)
    ctx.set_material(mat)
    # three cells below the centre of the top face, so that the receivers record signal and the
    # adjoint field meets the forward field within the steps of the gradient
    ctx.set_point_source((L / 2, L / 2, L - 1.25), synth.moment_tensor(), 2.0, 0.5)
    seismo = torch.zeros(steps + 2, 64, 3, dtype=torch.float64, device="cuda")
    ctx.set_receivers(synth.receivers_top((n,) * 3, (0, 0, 0), (L,) * 3), seismo, steps + 2)
    u0 = torch.zeros(ctx.count, dtype=torch.float64, device="cuda")
    ctx.set_state(u0)
    ctx.set_time(0.45)
    ctx.step()  # dt from the CFL condition of the material
    dt = ctx.last_dt()
    obs = torch.from_numpy(1e-3 * np.random.default_rng(3).standard_normal(steps * 64 * 3)).cuda()
    gm = torch.zeros(cells * 3, dtype=torch.float64, device="cuda")
    gM = torch.zeros(6, dtype=torch.float64, device="cuda")
    ctx.misfit_gradient(u0, 0.45, dt, 2, 2, obs, gm, gM)  # warm-up (allocates the work buffers)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.set_state(u0)
    ctx.set_time(0.45)
    e0.record(stream)
    ctx.run(steps, dt=dt)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1)
    gm.zero_()
    gM.zero_()
    e0.record(stream)
    J = ctx.misfit_gradient(u0, 0.45, dt, steps, k, obs, gm, gM)
    e1.record(stream)
    torch.cuda.synchronize()
    tot = e0.elapsed_time(e1)
    # one adjoint step alone (forward face data, Riemann adjoint, cell adjoint)
    lam = torch.from_numpy(np.random.default_rng(4).standard_normal(ctx.count)).cuda()
    u1 = torch.from_numpy(np.random.default_rng(5).standard_normal(ctx.count)).cuda()
    ctx.adjoint_step(0.45, dt, u1, lam, gm, gM)
    e0.record(stream)
    for _ in range(3):
        ctx.adjoint_step(0.45, dt, u1, lam, gm, gM)
    e1.record(stream)
    torch.cuda.synchronize()
    adj = e0.elapsed_time(e1) / 3
    ok = bool(torch.isfinite(gm).all().item() and torch.isfinite(gM).all().item())
    # the gradient itself (the timed call's), for the comparison between forms
    gm.zero_()
    gM.zero_()
    ctx.misfit_gradient(u0, 0.45, dt, steps, k, obs, gm, gM)
    grads = (gm.cpu().numpy().copy(), gM.cpu().numpy().copy())
    ctx.close()
    del seismo
    return {"forward_ms_per_step": fwd / steps, "adjoint_step_ms": adj, "gradient_ms": tot,
            "gradient_over_forward": tot / fwd, "value": dofs * steps / (tot * 1e-3), "J": J,
            "finite": ok, "_grads": grads}


def extra_adjoint(ader, synth, stream, n=40, N=4, steps=12, k=4,
                  forms=("picard", "ck", "ck_mixed")):
    """Adjoint of the linear-elastic step through the C ABI (ader_misfit_gradient): order N, n^3
    cells (h = 0.5 km), seeded material, moment-tensor Ricker source at the centre, 64 receivers
    on the top face, a seeded misfit over `steps` steps with a checkpoint every k steps.  Reports
    the whole gradient (forward sweep, recomputation of each segment, adjoint sweep, gradients with
    respect to per-cell rho, lambda, mu and the moment tensor) against the same number of forward
    steps, with the Picard predictor and with the Cauchy-Kowalevski predictor (its own adjoint),
    FP64, and with the mixed Cauchy-Kowalevski forward step and mixed-precision adjoint; the
    gradients of the mixed form against the FP64 CK form."""
    dofs = n ** 3 * (N + 1) ** 3 * 9
    out = {"workload": "adjoint_elastic3d_p%d_%d" % (N, n), "dofs": dofs, "steps": steps,
           "k_ckpt": k, "unit": "DOF-updates/s (gradient: forward, recomputation and adjoint, "
           "each step counted once)", "dtype": "f64"}
    spec = {"picard": ("picard", "fp64"), "ck": ("ck", "fp64"), "ck_mixed": ("ck", "mixed")}
    for form in forms:
        out[form] = _adjoint_gradient_40(ader, synth, stream, n, N, steps, k, *spec[form])
    if "ck" in out and "ck_mixed" in out:
        # the mixed form (mixed forward, mixed-precision adjoint) against the FP64 CK form
        (gmm, gMm), (gmf, gMf) = out["ck_mixed"]["_grads"], out["ck"]["_grads"]
        m = out["ck_mixed"]
        m["J_rel_diff_to_fp64_ck"] = abs(m["J"] - out["ck"]["J"]) / abs(out["ck"]["J"])
        m["grad_mat_rel_diff_to_fp64_ck"] = float(np.abs(gmm - gmf).max() / np.abs(gmf).max())
        m["grad_M_rel_diff_to_fp64_ck"] = float(np.abs(gMm - gMf).max() / np.abs(gMf).max())
    for form in forms:
        del out[form]["_grads"]
    out["value"] = out[forms[-1]]["value"]
    if "picard" in out:
        for form in forms[1:]:
            out[form]["gradient_speedup_over_picard"] = (out["picard"]["gradient_ms"]
                                                         / out[form]["gradient_ms"])
            out[form]["adjoint_step_speedup_over_picard"] = (out["picard"]["adjoint_step_ms"]
                                                             / out[form]["adjoint_step_ms"])
    return out


def extra_explosion(ader, synth, stream, steps=200, warmup=3, n=64):
    """3-D spherical explosion, order 3, n^3 cells (default 64^3) on [-1,1]^3, wall boundaries,
    a-posteriori subcell limiter (7^3 subcells), the workload's 200 steps from t = 0 timed in
    full (after `warmup` steps on the same data, then a reset): FP64 and mixed predictor, the
    FP64 form with the hybrid ADER-DG / FV status (troubled cells stay FV two more steps, an FV
    interface layer), and the FP64 and mixed forms with the continuous extension Runge-Kutta guess
    and one Picard iteration (Sec. 5).  Per form: ms per step over the 200 steps, FV cells, conservation of mass
    and energy over the run, the minimum density and pressure at the end, and the symmetry of the
    last step's FV set under the reflections and axis permutations of the cube."""
    import torch
    N = 3
    x, w = ader.reference_nodes(N)
    X = synth.node_coordinates(x, (n,) * 3, (-1,) * 3, (1,) * 3)
    Us = synth.explosion(synth.subcell_centres(2 * N + 1, (n,) * 3, (-1,) * 3, (1,) * 3))
    fl = torch.from_numpy(synth.discontinuous_cells(Us).astype(np.uint8)).cuda()
    Us_d = torch.from_numpy(Us.reshape(-1).copy()).cuda()
    u0_d = torch.from_numpy(synth.explosion(X).reshape(-1).copy()).cuda()
    W = torch.from_numpy(np.einsum("i,j,k->ijk", w, w, w).reshape(-1)).cuda()
    dofs = n ** 3 * 64 * 5
    out = {"workload": f"explosion3d_p3_{n} (limiter on, {steps} steps from t = 0)", "dofs": dofs}
    # forms: (name, precision, limiter mode, initial guess, Picard iterations; 0 = N+1)
    for form, prec, limiter, guess, iters in (("fp64", "fp64", 1, "constant", 0),
                                              ("mixed", "mixed", 1, "constant", 0),
                                              ("fp64_hybrid", "fp64", 3, "constant", 0),
                                              ("fp64_cerk", "fp64", 1, "cerk", 1),
                                              ("mixed_cerk", "mixed", 1, "cerk", 1)):
        cfg = ader.make_config("euler", 3, N, (n,) * 3, (-1,) * 3, (1,) * 3, "wall", synth.cfl_number(N),
                               limiter=limiter, precision=prec, initial_guess=guess,
                               picard_iters=iters)
        ctx = ader.Context(cfg, stream=stream.cuda_stream)

        def reset():
            ctx.set_state(u0_d)
            ctx.set_subcell_state(Us_d, fl)
            ctx.set_time(0.0)

        def totals():
            st = _dev_state(ctx).view(ctx.cells, -1, 5)
            return (st * W[None, :, None]).sum(dim=(0, 1))

        reset()
        for _ in range(warmup):
            ctx.step()
        ctx.sync()
        reset()
        m0 = totals()
        torch.cuda.synchronize()
        ctx.enable_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ph, nr = ctx.phase_times()
        ctx.enable_timing(False)
        ctx.sync()
        m1 = totals()
        st = _dev_state(ctx).view(ctx.cells, -1, 5)
        rho = st[..., 0]
        p = 0.4 * (st[..., 4] - 0.5 * (st[..., 1:4] ** 2).sum(-1) / rho)
        F = ctx.flags().reshape(n, n, n).astype(bool)
        asym = max(int((G != F).sum()) for G in (F[::-1], F[:, ::-1], F[:, :, ::-1],
                                                F.transpose(0, 2, 1), F.transpose(2, 1, 0)))
        nfv = ctx.troubled_count()
        key = "fv_cells_last_step" if limiter == 3 else "troubled_cells_last_step"
        out[form] = {"ms_per_step": ms / steps, "value": dofs * steps / (ms * 1e-3),
                     key: nfv, "fv_fraction": nfv / n ** 3,
                     "t_end": ctx.time(),
                     "phase_ms_per_step": {k: v / max(nr, 1) for k, v in ph.items()},
                     "mass_rel_drift": abs(float(m1[0] - m0[0])) / abs(float(m0[0])),
                     "energy_rel_drift": abs(float(m1[4] - m0[4])) / abs(float(m0[4])),
                     "min_rho": float(rho.min()), "min_p": float(p.min()),
                     "fv_set_max_asymmetric_cells": asym, "steps_timed": steps}
        if limiter == 3:
            out[form]["fv_set_note"] = ("the hybrid FV set: troubled cells, cells still counting "
                                        "their FV steps, and their face neighbours")
        del st, rho, p
        ctx.close()
    out["mixed_speedup"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    out["hybrid_speedup"] = out["fp64"]["ms_per_step"] / out["fp64_hybrid"]["ms_per_step"]
    for form in ("fp64_cerk", "mixed_cerk"):
        out[form]["speedup_over_fp64"] = out["fp64"]["ms_per_step"] / out[form]["ms_per_step"]
    return out


def _ensemble(ader, synth, stream, sides, predictor):
    """The 16-run ensemble (mixed precision) with its materials, sources and zero states; the
    fixed dt of all runs."""
    import torch
    cfgs = [ader.make_config("elastic", 3, 4, (s,) * 3, (0, 0, 0), (0.5 * s,) * 3, "absorbing",
                             synth.cfl_number(4), precision="mixed", predictor=predictor)
            for s in sides]
    ens = ader.Ensemble(cfgs, stream=stream.cuda_stream)
    dts = []
    for i, (s, r) in enumerate(zip(sides, ens.runs)):
        mat = synth.elastic_material((s,) * 3, seed=100 + i)
        r.set_material(torch.from_numpy(mat.reshape(-1).copy()).cuda())
        r.set_point_source((0.25 * s,) * 3, synth.moment_tensor(seed=200 + i), 2.0, 0.5)
        r.set_state(torch.zeros(r.count, dtype=torch.float64, device="cuda"))
        r.set_time(0.45)
        vpmax = float(np.sqrt((mat[:, 1] + 2 * mat[:, 2]) / mat[:, 0]).max())
        dts.append(synth.cfl_number(4) / (3 * 9) * 0.5 / vpmax)
    return ens, min(dts)  # one fixed dt for the ensemble (as for the adjoint runs)


def _time_shapes(ens, dt, stream, shapes_in):
    import torch
    shapes = {}
    for name, shape in shapes_in:
        ens.set_launch(*shape)
        ens.step(4, dt=dt)
        ens.sync()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        ens.step(4, dt=dt)
        f1.record(stream)
        torch.cuda.synchronize()
        ens.sync()
        shapes[name] = f0.elapsed_time(f1) / 4
    return shapes


def swe_model_flops_per_cell(N, D=2, nv=4, iters=None, cF=21):
    """Algorithmic flops per cell and step of the shallow-water predictor in the sum-factorised
    model: per Picard iteration the D derivative contractions of the nv flux components, the
    derivative of the surface h + b for the non-conservative product g h d(h + b)/dx_d, the time
    solve, and cF ~ 21 flops per space-time node for the fluxes and the product; then the same
    epilogue as the Euler model.  38.1 k flop for the order-3 cell (N + 1 iterations)."""
    n = N + 1
    I = iters or n
    it = (2 * D * nv + 2 * D + 2 * nv) * n ** (D + 2) + cF * n ** (D + 1)
    epi = 2 * (2 * D + 1) * nv * n ** (D + 1) + 12 * D * nv * n ** D
    return I * it + epi


def extra_swe(ader, synth, stream, n=1024, N=3, steps=5, warmup=2):
    """Shallow water equations with bathymetry (Eq. (9)), FP64, order 3 (the order of the paper's
    oscillating lake), n^2 periodic cells on the unit square: a flow over a smooth bump (every term
    active) timed per phase, the mass drift, and the lake at rest over the same bathymetry at full
    size (surface and momentum after the steps: round-off)."""
    import torch
    x, w = ader.reference_nodes(N)
    nc, lo, hi = (n, n), (0.0, 0.0), (1.0, 1.0)
    X = synth.node_coordinates(x, nc, lo, hi)
    npc = (N + 1) ** 2
    dofs = n * n * npc * 4
    W = torch.from_numpy(np.outer(w, w).reshape(-1)).cuda() / (n * n)
    cfg = ader.make_config("swe", 2, N, nc, lo, hi, "periodic", synth.cfl_number(N))
    ctx = ader.Context(cfg, stream=stream.cuda_stream)
    out = {"workload": "swe2d_p3_%d (flow over a periodic bump, FP64)" % n, "dofs": dofs}

    def mass():
        u = _dev_state(ctx).view(n * n, npc, 4)
        return float((u[:, :, 0] * W).sum())

    u0 = torch.from_numpy(np.ascontiguousarray(synth.swe_flow_over_bump(X)).reshape(-1)).cuda()
    ctx.set_state(u0)
    ctx.set_time(0.0)
    m0 = mass()
    for _ in range(warmup):
        ctx.step()
    ctx.sync()
    ctx.enable_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ph, nr = ctx.phase_times()
    ctx.enable_timing(False)
    ctx.sync()
    pred = ph["predictor"] / max(nr, 1)
    fl = swe_model_flops_per_cell(N) * n * n
    peak = (_PEAKS[0] or {}).get("fp64")
    out["fp64"] = {"ms_per_step": ms, "value": dofs / (ms * 1e-3),
                   "phase_ms_per_step": {k: v / max(nr, 1) for k, v in ph.items()},
                   "predictor_model_flops_per_cell": swe_model_flops_per_cell(N),
                   "predictor_tflops": fl / (pred * 1e-3) / 1e12,
                   "predictor_frac_of_fp64_peak": fl / (pred * 1e-3) / (peak * 1e12 if peak else FP64_PEAK),
                   "fp64_peak_source": "measured in this run (libpeaks)" if peak else "derived",
                   "mass_rel_drift": abs(mass() - m0) / abs(m0), "steps": warmup + steps}
    lake = torch.from_numpy(np.ascontiguousarray(synth.swe_lake_at_rest(X)).reshape(-1)).cuda()
    ctx.set_state(lake)
    ctx.set_time(0.0)
    for _ in range(steps):
        ctx.step()
    ctx.sync()
    u = _dev_state(ctx).view(-1, 4)
    out["lake_at_rest"] = {"steps": steps,
                           "max_surface_deviation": float((u[:, 0] + u[:, 3] - 1.0).abs().max()),
                           "max_momentum": float(u[:, 1:3].abs().max())}
    ctx.close()
    return out


def extra_ensemble(ader, synth, stream, steps=4):
    """16 elastic order-4 runs, cube sides drawn by seed from {24,32,40,48,64}, each with its own
    seeded material and source, mixed predictor, advanced by one CUDA graph per step block; the
    autotuner picks between one persistent launch per phase for all runs, one cooperative launch
    for whole steps and per-run kernels on forked streams.  The same runs with the mixed
    Cauchy-Kowalevski predictor beside it (persistent launch per phase, or per-run kernels)."""
    import torch
    sides = synth.ensemble_sides(16)
    ens, dt = _ensemble(ader, synth, stream, sides, "picard")
    # the launch shapes the autotuner chooses between, each timed here too
    shapes = _time_shapes(ens, dt, stream, (("per_run_4_branches", (4, 4, 1)),
                                            ("persistent_per_phase", (0, 4, 2)),
                                            ("fused_cooperative", (-1, 4, 2))))
    best = ens.autotune(dt)
    ens.step(2, dt=dt)
    ens.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ens.step(steps, dt=dt)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ens.sync()
    dofs = sum(s ** 3 for s in sides) * 125 * 9
    ens.close()
    ens, dt_ck = _ensemble(ader, synth, stream, sides, "ck")
    ck_shapes = _time_shapes(ens, dt_ck, stream, (("per_run_4_branches", (4, 4, 1)),
                                                  ("persistent_per_phase", (0, 4, 1))))
    ens.close()
    ck_ms = min(ck_shapes.values())
    return {"workload": "ensemble16_elastic_p4", "sides": sides, "dofs": dofs,
            "ms_per_step": ms / steps, "value": dofs * steps / (ms * 1e-3), "unit": "DOF-updates/s",
            "dtype": "f32+f64", "autotuned": {"branches": best[0], "steps_per_graph": best[1],
                                              "persistent_blocks_per_sm": best[2],
                                              "ms_per_step_at_tuning": best[3]},
            "launch": {0: "persistent launches shared by all runs, one per phase",
                       -1: "one cooperative persistent launch for whole steps"}.get(
                           best[0], "per-run kernels on %d forked streams" % best[0]),
            "ms_per_step_by_launch_shape": shapes,
            "ck_mixed": {"predictor": "Cauchy-Kowalevski, mixed", "ms_per_step": ck_ms,
                         "value": dofs / (ck_ms * 1e-3),
                         "ms_per_step_by_launch_shape": ck_shapes}}


def _ensemble_gradient(ader, synth, stream, sides, steps, k, predictor):
    import torch
    cfgs = [ader.make_config("elastic", 3, 4, (s,) * 3, (0, 0, 0), (0.5 * s,) * 3, "absorbing",
                             synth.cfl_number(4), precision="mixed", predictor=predictor)
            for s in sides]
    ens = ader.Ensemble(cfgs, stream=stream.cuda_stream)
    keep, dts = [], []
    for i, (s, r) in enumerate(zip(sides, ens.runs)):
        L = 0.5 * s
        mat = synth.elastic_material((s,) * 3, seed=100 + i)
        r.set_material(torch.from_numpy(mat.reshape(-1).copy()).cuda())
        r.set_point_source((0.5 * L, 0.5 * L, L - 1.25), synth.moment_tensor(seed=200 + i), 2.0, 0.5)
        sm = torch.zeros(steps + 2, 64, 3, dtype=torch.float64, device="cuda")
        r.set_receivers(synth.receivers_top((s,) * 3, (0, 0, 0), (L,) * 3), sm, steps + 2)
        keep.append(sm)
        vpmax = float(np.sqrt((mat[:, 1] + 2 * mat[:, 2]) / mat[:, 0]).max())
        dts.append(synth.cfl_number(4) / (3 * 9) * 0.5 / vpmax)
    dt = min(dts)
    u0 = [torch.zeros(r.count, dtype=torch.float64, device="cuda") for r in ens.runs]
    rng = np.random.default_rng(3)
    obs = [torch.from_numpy(1e-4 * rng.standard_normal(steps * 64 * 3)).cuda() for _ in sides]
    gm = [torch.zeros(r.cells * 3, dtype=torch.float64, device="cuda") for r in ens.runs]
    gM = [torch.zeros(6, dtype=torch.float64, device="cuda") for r in ens.runs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = ens.misfit_gradient(u0, 0.45, dt, steps, k, obs, gm, gM)
    el = time.perf_counter() - t0
    ok = all(bool(torch.isfinite(g).all()) for g in gm + gM)
    dofs = sum(s ** 3 for s in sides) * 125 * 9
    ens.close()
    del keep
    torch.cuda.empty_cache()
    return {"steps": steps, "k_ckpt": k, "gradient_s": el, "s_per_gradient_step": el / steps,
            "value": dofs * steps / el, "J_sum": float(sum(J)), "finite": ok}


def extra_ensemble_adjoint(ader, synth, stream, steps=20, k=5, picard_steps=1):
    """Batched adjoint of the 16-run ensemble (the ensemble workload's draw of cube sides, order 4,
    mixed forward, each run with its seeded material, source and 64 top-face receivers): the
    misfit gradient of every run with respect to per-cell rho, lambda, mu and the moment tensor
    through ader_ensemble_misfit_gradient.  The source sits three cells below the top-face centre
    so that the receivers record signal.  Bounded samples: `steps` steps with a checkpoint every
    `k` with the Cauchy-Kowalevski predictor and its adjoint, and `picard_steps` with the Picard
    predictor and its adjoint (the full 300-step workload is timed with --adjoint-steps 300)."""
    sides = synth.ensemble_sides(16)
    dofs = sum(s ** 3 for s in sides) * 125 * 9
    out = {"workload": "ensemble16_adjoint_p4 (batched misfit gradient)", "sides": sides,
           "dofs": dofs, "unit": "DOF-updates/s (gradient: forward, recomputation and adjoint, "
           "each step counted once; host wall clock around the synchronising call)",
           "forward": "mixed",
           "adjoint": {"ck": "mixed precision (float-float base term, binary32 corrections, FP64 "
                             "adjoint state and gradient sums)", "picard": "f64"}}
    out["ck"] = _ensemble_gradient(ader, synth, stream, sides, steps, k, "ck")
    if picard_steps:
        out["picard"] = _ensemble_gradient(ader, synth, stream, sides, picard_steps, 1, "picard")
        out["ck_speedup_per_step"] = (out["picard"]["s_per_gradient_step"]
                                      / out["ck"]["s_per_gradient_step"])
    out["value"] = out["ck"]["value"]
    out["finite"] = out["ck"]["finite"]
    out["full_workload_estimate_s"] = out["ck"]["s_per_gradient_step"] * 300
    return out


_WORLD = [1]
_PEAKS = [None]  # the FMA throughputs measured by this run (rank 0)


def barrier():
    if _WORLD[0] > 1:
        import torch
        torch.distributed.barrier()


def max_over_ranks(x):
    """Largest value over the ranks (the timing rule: the slowest rank sets the time)."""
    if _WORLD[0] > 1:
        import torch
        dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())
    return x


def replica_value(world, dofs_per_rank, steps, ms_total):
    """Whole-job DOF-updates/s of `world` independent replicas (weak scaling): the units all
    ranks processed over the slowest rank's time."""
    return world * dofs_per_rank * steps / (ms_total * 1e-3)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="euler3d_p4_81", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="mixed_cerk", choices=sorted(FORMS),
                    help="form reported as the headline value")
    ap.add_argument("--forms", default="fp64,mixed,mixed_cerk", help="forms to time (comma list)")
    ap.add_argument("--err-steps", type=int, default=50,
                    help="steps after which the error against the exact solution is measured")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--extras", default="",
                    help="comma list of the other workloads to run (default: all of them)")
    ap.add_argument("--elastic-n", type=int, default=81,
                    help="cells per side of the elastic workload (81; smaller for profiling)")
    ap.add_argument("--swe-n", type=int, default=1024,
                    help="cells per side of the shallow-water workload (1024; smaller for profiling)")
    ap.add_argument("--adjoint-forms", default="picard,ck,ck_mixed",
                    help="forms of the 40^3 adjoint workload (picard, ck, ck_mixed)")
    ap.add_argument("--adjoint-steps", type=int, default=20,
                    help="steps of the ensemble gradient sample (300: the full workload, "
                         "checkpoint every 20)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads (2-D Euler, elastic, explosion, ensemble)")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    D, N = wl["dim"], wl["order"]
    cells = int(np.prod(wl["ncell"]))
    dofs = cells * (N + 1) ** D * (D + 2)
    metric = "ADER-DG DOF-updates/s on 1 GB300 (FP64 vs mixed @ stated err); % roofline"
    config = {"workload": args.workload, "pde": wl["pde"], "dim": D, "order": N,
              "cells": list(wl["ncell"]), "dofs": dofs, "init": "entropy wave (analytic)",
              "cfl": "0.9 x order-%d stability limit" % N,
              "l2": "inputs larger than L2 (state %.2f GB)" % (dofs * 8 / 1e9),
              "precision": FORMS[args.prec][0], "form": args.prec,
              "initial_guess": FORMS[args.prec][1],
              "picard_iters": FORMS[args.prec][2] or N + 1}

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    _WORLD[0] = world

    if args.impl == "reference":
        if rank != 0:
            return
        config["precision"] = "fp64 (the CPU oracle computes in binary64)"
        v, desc, cores, per_step = oracle_sample(wl, min(args.cpu_budget, 20.0))
        line = {"impl": "reference", "metric": metric, "value": v, "unit": "DOF-updates/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": dofs / v * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": {"value": v, "unit": "DOF-updates/s", "cores": cores,
                                 "kind": "oracle", "sample": desc},
                "e2e": {"value": v, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    from paper_1905_07987_gb300 import ader, synth

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    u0 = build_initial(ader, synth, wl)
    u0_dev = torch.from_numpy(u0).to("cuda")
    torch.cuda.synchronize()

    peaks = measure_fma_peaks(stream) if world == 1 or rank == 0 else None
    _PEAKS[0] = peaks
    forms = [f for f in args.forms.split(",") if f]
    if args.prec not in forms:
        forms.append(args.prec)
    res = {}
    head_ctx = None
    for prec in forms:
        ctx, ms_total, phases, nrec, clocks, err = run_form(ader, synth, wl, prec, args, stream,
                                                            u0_dev, args.err_steps)
        ms_total = max_over_ranks(ms_total)
        res[prec] = dict(value=replica_value(world, dofs, args.steps, ms_total),
                         ms_per_step=ms_total / args.steps, phases=phases, nrec=nrec,
                         clocks=clocks, err=err)
        if prec == args.prec:
            head_ctx = ctx
        else:
            ctx.close()
    head = res[args.prec]

    # ---- end-to-end through the C ABI with host buffers --------------------------------------
    e2e = None
    if not args.no_e2e:
        # every step: the step's input state from pinned host memory to the device, one step, the
        # new state back to pinned host memory, through ader_step_host_batch (the copies of the
        # neighbouring steps' states overlap each step); the plain loop of set_state / step /
        # get_state beside it
        ctx = head_ctx
        h_in = [torch.from_numpy(u0).pin_memory() for _ in range(2)]
        h_out = [torch.empty(dofs, dtype=torch.float64).pin_memory() for _ in range(2)]
        ins = [h_in[i % 2] for i in range(args.steps)]
        outs = [h_out[i % 2] for i in range(args.steps)]
        ctx.step_host_batch(ins[:1], outs[:1])  # staging buffers and copy streams
        # the host links are shared with the other GPUs' jobs on the machine: the batch and the
        # plain loop alternate three times and each reports its median (every sample kept)
        t_batch, t_loop = [], []
        for _ in range(3):
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.step_host_batch(ins, outs)
            torch.cuda.synchronize()
            t_batch.append(max_over_ranks(time.perf_counter() - t0))
            t0 = time.perf_counter()
            for _ in range(args.steps):
                ctx.set_state(h_in[0])
                ctx.step()
                ctx.get_state(h_out[0])
            torch.cuda.synchronize()
            t_loop.append(max_over_ranks(time.perf_counter() - t0))
        el, el_loop = statistics.median(t_batch), statistics.median(t_loop)
        e2e = {"value": world * dofs * args.steps / el, "unit": "DOF-updates/s",
               "h2d_bytes_per_step": dofs * 8, "d2h_bytes_per_step": dofs * 8,
               "call": "ader_step_host_batch (copies of neighbouring steps overlap each step)",
               "sequential_loop_value": world * dofs * args.steps / el_loop,
               "samples": "median of 3 alternating runs of each; ms per step: batch %s, loop %s"
                          % ([round(1e3 * t / args.steps, 1) for t in t_batch],
                             [round(1e3 * t / args.steps, 1) for t in t_loop])}
    head_ctx.close()

    # ---- roofline of the dominant kernel (the predictor) of each form --------------------------
    # algorithmic flops per cell in the sum-factorised model (the unit of the roofline) and in the
    # kernel's own operation count (the flux evaluation counted operation by operation)
    def form_flops(form):
        """(model flops, kernel-count flops) per cell of the form's predictor; the CERK
        guess adds three single-time-level evaluations of the flux and its derivatives (1/n of
        an iteration each) and the dense output (4 FMA per line and time node)."""
        _, guess, iters = FORMS[form]
        I = iters or N + 1
        n = N + 1
        nv = D + 2
        m = model_flops_per_cell(D, N, nv, I)
        k = predictor_flops_per_cell(wl["pde"], D, N, I)
        if guess == "cerk":
            it = 2 * (D + 1) * nv * n ** (D + 2) + 30 * n ** (D + 1)
            m += 3 * it / n + 8 * n ** D * nv * n
            k += cerk_flops_per_cell(D, N)
        return m * cells, k * cells

    def roofline(form):
        r = res[form]
        prec = FORMS[form][0]
        flops_model, flops_kernel = form_flops(form)
        nrec = max(r["nrec"], 1)
        pred_ms = r["phases"]["predictor"] / nrec
        achieved = flops_model / (pred_ms * 1e-3) / 1e12
        key = "fp64" if prec == "fp64" else "fp32"
        derived = (FP64_PEAK if prec == "fp64" else FP32_PEAK) / 1e12
        if peaks and peaks.get(key):
            peak, src = peaks[key], "measured in this run (%s FMA throughput, libpeaks)" % key.upper()
        else:
            peak, src = derived, "derived: 152 SMs x %d FMA/clk x 2 flop x 2070 MHz" % (
                2 if prec == "fp64" else 128)
        kname = "k_predictor (FP64)" if prec == "fp64" else \
            "k_predictor_mixed (binary32 Picard iterations and flux remainders; float-float base terms, time averages and contractions; FP64 face wave speeds)"
        if FORMS[form][1] == "cerk":
            kname += ", continuous extension Runge-Kutta guess + %d iteration(s)" % FORMS[form][2]
        return {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": TRAFFIC_PER_CELL.get(prec, 0) * cells if TRAFFIC_PER_CELL.get(prec) else None,
                "peak_source": src, "flops_per_cell": flops_model / cells,
                "flops_model": "sum-factorised model I [2(d+1) nv n^(d+2) + 30 n^(d+1)] + 2(2d+1) nv n^(d+1) + 12 d nv n^d",
                "kernel_count_flops_per_cell": flops_kernel / cells,
                "frac_kernel_count": flops_kernel / (pred_ms * 1e-3) / 1e12 / peak,
                "frac_of_derived_peak": achieved / derived, "derived_peak": derived,
                "ms_per_launch": pred_ms,
                "phase_ms_per_step": {k: v / nrec for k, v in r["phases"].items()}}

    roof = roofline(args.prec)
    roof_forms = {k: roofline(k) for k in res}
    forms_out = {}
    for k, r in res.items():
        forms_out[k] = {"value": r["value"], "ms_per_step": r["ms_per_step"],
                        "predictor_ms": r["phases"]["predictor"] / max(r["nrec"], 1), "err": r["err"]}
    if "fp64" in res and res["fp64"]["err"]:
        for k, r in res.items():
            if k != "fp64" and r["err"]:
                forms_out[k]["l2_error_over_fp64"] = r["err"]["l2_rho"] / res["fp64"]["err"]["l2_rho"]
                forms_out[k]["speedup_over_fp64"] = r["value"] / res["fp64"]["value"]
    launches_per_step = 1 + 1 + 1 + D + 1 + 1
    # the FP64 form of the same workload (the scheme's reference arithmetic), with its error
    fp64_entry = None
    if "fp64" in res:
        r = res["fp64"]
        fp64_entry = {"value": r["value"], "unit": "DOF-updates/s", "ms_per_step": r["ms_per_step"],
                      "dtype": "f64", "err_vs_exact": r["err"], "roofline": roof_forms["fp64"]}
    line = {"metric": metric, "value": head["value"], "unit": "DOF-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if FORMS[args.prec][0] == "fp64" else "f32+f64",
            "data": "synthetic", "config": config, "roofline": roof, "roofline_forms": roof_forms,
            "forms": forms_out, "fp64": fp64_entry, "err_vs_exact": head["err"],
            "measured_peaks": peaks,
            "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "clocks": head["clocks"]}
    if not args.no_extra and world == 1:
        extra = {}
        for name, fn in (("euler3d_p4_convergence", extra_convergence),
                         ("euler2d_p3_27", extra_euler2d), ("explosion3d_p3_64", extra_explosion),
                         ("elastic3d_p5_81", extra_elastic), ("ensemble16_elastic_p4", extra_ensemble),
                         ("adjoint_elastic3d_p4_40", extra_adjoint), ("euler3d_p4_81_cerk", extra_cerk),
                         ("ensemble16_adjoint_p4", extra_ensemble_adjoint),
                         ("swe2d_p3_1024", extra_swe)):
            if args.extras and name not in args.extras.split(","):
                continue
            try:
                if fn is extra_convergence:
                    extra[name] = fn(ader, synth, stream, res)
                elif fn is extra_ensemble_adjoint:
                    ks = 20 if args.adjoint_steps >= 100 else 5
                    extra[name] = fn(ader, synth, stream, steps=args.adjoint_steps, k=ks,
                                     picard_steps=0 if args.adjoint_steps >= 100 else 1)
                elif fn is extra_adjoint:
                    extra[name] = fn(ader, synth, stream,
                                     forms=tuple(f for f in args.adjoint_forms.split(",") if f))
                elif fn is extra_elastic:
                    extra[name] = fn(ader, synth, stream, n=args.elastic_n)
                elif fn is extra_swe:
                    extra[name] = fn(ader, synth, stream, n=args.swe_n)
                else:
                    extra[name] = fn(ader, synth, stream)
            except Exception as exc:  # report, keep the headline line
                extra[name] = {"error": "%s: %s" % (type(exc).__name__, exc)}
            torch.cuda.empty_cache()
        line["workloads"] = extra
    if world == 1 and rank == 0:
        v, desc, cores, _ = oracle_sample(wl, args.cpu_budget)
        line["cpu_baseline"] = {"value": v, "unit": "DOF-updates/s", "cores": cores,
                                "kind": "oracle", "sample": desc}
        import torch as _t
        nt = _t.get_num_threads()
        _t.set_num_threads(1)
        v1, desc1, _, _ = oracle_sample(wl, max(2.0, args.cpu_budget / 2))
        _t.set_num_threads(nt)
        line["cpu_baseline"]["one_thread"] = {"value": v1, "cores": 1, "sample": desc1}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
