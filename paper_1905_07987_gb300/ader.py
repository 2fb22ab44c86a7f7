"""ctypes binding of the C ABI in include/ader.h (argument marshalling only).

Every step of the method runs in the CUDA kernels of libader.so; this module only converts
arguments.  Tensors passed with ``on_device`` are torch CUDA tensors (their ``data_ptr()`` goes
to the library, on the context's stream); host data may be numpy arrays or CPU tensors.
The library is loaded on first use; if it is missing the call raises (there is no fallback).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libader.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ENONFINITE, EADMISSIBLE, ETIMEOUT, EUNSUPPORTED = range(9)
PDE = {"advection": 0, "euler": 1, "elastic": 2, "swe": 3}
BC = {"periodic": 0, "wall": 1, "absorbing": 2}
PREC = {"fp64": 0, "mixed": 1, "tf32x3": 3}
PREDICTOR = {"picard": 0, "ck": 1}
GUESS = {"constant": 0, "cerk": 1}


class AderError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, status_string(status), status))


class Config(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("order", ctypes.c_int),
        ("pde", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("bc", (ctypes.c_int * 2) * 3),
        ("cfl", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("adv", ctypes.c_double * 3),
        ("picard_iters", ctypes.c_int),
        ("limiter", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("predictor", ctypes.c_int),
        ("initial_guess", ctypes.c_int),
        ("grav", ctypes.c_double),
        ("adm_floor", ctypes.c_double),
    ]


_lib = None

_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_L = ctypes.c_int64
_SIGS = {
    "ader_status_string": ([_I], ctypes.c_char_p),
    "ader_reference_nodes": ([_I, _P, _P], _I),
    "ader_reference_tables": ([_I, _P, _P, _P], _I),
    "ader_create": ([ctypes.POINTER(Config), _P, ctypes.POINTER(_P)], _I),
    "ader_destroy": ([_P], None),
    "ader_sizes": ([_P, ctypes.POINTER(_L), ctypes.POINTER(_L), ctypes.POINTER(_I)], _I),
    "ader_set_state": ([_P, _P, _L, _I], _I),
    "ader_get_state": ([_P, _P, _L, _I], _I),
    "ader_step_host_batch": ([_P, _I, _P, _P, _D, _D], _I),
    "ader_set_material": ([_P, _P, _I], _I),
    "ader_set_point_source": ([_P, _P, _P, _D, _D], _I),
    "ader_set_receivers": ([_P, _I, _P, _P, _L], _I),
    "ader_set_time": ([_P, _D], _I),
    "ader_get_time": ([_P, ctypes.POINTER(_D)], _I),
    "ader_step": ([_P, _D, _D], _I),
    "ader_run": ([_P, _I, _D, _D], _I),
    "ader_last_dt": ([_P, ctypes.POINTER(_D)], _I),
    "ader_get_flags": ([_P, _P, _I], _I),
    "ader_troubled_count": ([_P, ctypes.POINTER(_L)], _I),
    "ader_sync": ([_P], _I),
    "ader_run_graph": ([_P, _I, _I, _D, _D], _I),
    "ader_set_subcell_state": ([_P, _P, _P, _I], _I),
    "ader_get_subcell_state": ([_P, _P, _I], _I),
    "ader_adjoint_step": ([_P, _D, _D, _P, _P, _P, _P, _P], _I),
    "ader_receivers_adjoint": ([_P, _P, _D, _P], _I),
    "ader_adjoint_step_static": ([_P, _D, _D, _P, _P, _P, _P, _P], _I),
    "ader_misfit_gradient": ([_P, _P, _D, _D, _I, _I, _P, ctypes.POINTER(_D), _P, _P], _I),
    "ader_ensemble_create": ([ctypes.POINTER(Config), _I, _P, ctypes.POINTER(_P)], _I),
    "ader_ensemble_destroy": ([_P], None),
    "ader_ensemble_run": ([_P, _I], _P),
    "ader_ensemble_step": ([_P, _I, _D, _D], _I),
    "ader_ensemble_sync": ([_P], _I),
    "ader_ensemble_set_launch": ([_P, _I, _I, _I], _I),
    "ader_ensemble_autotune": ([_P, _D, _P, ctypes.POINTER(_D)], _I),
    "ader_ensemble_set_wait_limit": ([_P, _L], _I),
    "ader_ensemble_misfit_gradient": ([_P, _P, _D, _D, _I, _I, _P, _P, _P, _P, _L], _I),
    "ader_enable_timing": ([_P, _I], _I),
    "ader_phase_times": ([_P, _P, ctypes.POINTER(_I)], _I),
}

PHASES = ("cfl", "dt", "predictor", "riemann", "corrector", "limiter", "receivers")


def lib():
    """Load libader.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libader.so not found at %s: build it first "
                               "(python -c 'import __graft_entry__ as g; g.build()')" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def status_string(s):
    try:
        return lib().ader_status_string(int(s)).decode()
    except Exception:  # noqa: BLE001 - only used inside error messages
        return "status"


def check(status, what):
    if status != OK:
        raise AderError(status, what)


def reference_nodes(order):
    x = np.zeros(order + 1)
    w = np.zeros(order + 1)
    check(lib().ader_reference_nodes(order, x.ctypes.data, w.ctypes.data), "ader_reference_nodes")
    return x, w


def reference_tables(order):
    """(D, Kw, Vi) of the library, each [n, n] (see ader_reference_tables)."""
    n = order + 1
    D, Kw, Vi = (np.zeros((n, n)) for _ in range(3))
    check(lib().ader_reference_tables(order, D.ctypes.data, Kw.ctypes.data, Vi.ctypes.data),
          "ader_reference_tables")
    return D, Kw, Vi


def _ptr(a, dtype=np.float64):
    """(pointer, on_device, keepalive, element count) of a numpy array or torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            if a.dtype != {np.float64: torch.float64, np.uint8: torch.uint8}[dtype]:
                raise ValueError("tensor must be %s" % np.dtype(dtype).name)
            return a.data_ptr(), 1 if a.is_cuda else 0, a, a.numel()
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, 0, arr, arr.size


def make_config(pde, dim, order, ncell, lo, hi, bc, cfl, gamma=1.4, adv=(0.0, 0.0, 0.0),
                picard_iters=0, limiter=False, precision="fp64", predictor="picard",
                initial_guess="constant", grav=9.81, adm_floor=0.0):
    c = Config()
    c.dim = dim
    c.order = order
    c.pde = PDE[pde] if isinstance(pde, str) else int(pde)
    for d in range(3):
        c.n[d] = int(ncell[d]) if d < dim else 1
        c.lo[d] = float(lo[d]) if d < dim else 0.0
        c.hi[d] = float(hi[d]) if d < dim else 1.0
    if isinstance(bc, str):
        bc = [(bc, bc)] * dim
    for d in range(3):
        for s in range(2):
            k = bc[d][s] if d < dim else "periodic"
            c.bc[d][s] = BC[k] if isinstance(k, str) else int(k)
    c.cfl = float(cfl)
    c.gamma = float(gamma)
    for d in range(3):
        c.adv[d] = float(adv[d]) if d < len(adv) else 0.0
    c.picard_iters = int(picard_iters)
    c.limiter = int(limiter)
    c.precision = PREC[precision] if isinstance(precision, str) else int(precision)
    c.predictor = PREDICTOR[predictor] if isinstance(predictor, str) else int(predictor)
    c.initial_guess = GUESS[initial_guess] if isinstance(initial_guess, str) else int(initial_guess)
    c.grav = float(grav)
    c.adm_floor = float(adm_floor)
    return c


def _default_stream():
    try:
        import torch
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
    except ImportError:  # pragma: no cover
        return 0


class Context:
    """Owns one ader_ctx.  Methods map one-to-one to the C ABI."""

    def __init__(self, config, stream=None, handle=None):
        L = lib()
        if stream is None:
            stream = _default_stream()
        self.config = config
        self._stream = stream
        self._owned = handle is None
        if handle is None:
            h = _P()
            check(L.ader_create(ctypes.byref(config), _P(stream), ctypes.byref(h)), "ader_create")
        else:
            h = _P(handle)
        self._h = h
        cells, nodes, nvar = _L(), _L(), _I()
        check(L.ader_sizes(h, ctypes.byref(cells), ctypes.byref(nodes), ctypes.byref(nvar)), "ader_sizes")
        self.cells, self.nodes, self.nvar = cells.value, nodes.value, nvar.value
        self.count = self.cells * self.nodes * self.nvar

    def close(self):
        if getattr(self, "_h", None):
            if self._owned:
                lib().ader_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def set_state(self, q):
        p, dev, keep, n = _ptr(q)
        check(lib().ader_set_state(self._h, p, n, dev), "ader_set_state")

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.count)
        p, dev, keep, n = _ptr(out)
        if isinstance(out, np.ndarray) and keep is not out:
            raise ValueError("output array must be contiguous float64")
        check(lib().ader_get_state(self._h, p, n, dev), "ader_get_state")
        return out

    def step_host_batch(self, h_in, h_out, dt=0.0, t_end=0.0):
        """One step of each of the host states h_in[i] (host tensors or arrays, pinned memory
        for overlapped copies) into h_out[i]; see ader_step_host_batch."""
        n = len(h_in)
        if len(h_out) != n:
            raise ValueError("h_in and h_out differ in length")
        ins, outs, keep = (ctypes.c_void_p * n)(), (ctypes.c_void_p * n)(), []
        for i in range(n):
            for a, dst in ((h_in[i], ins), (h_out[i], outs)):
                p, dev, k, cnt = _ptr(a)
                if dev or cnt != self.count:
                    raise ValueError("host state of %d doubles expected" % self.count)
                if a is h_out[i] and isinstance(a, np.ndarray) and k is not a:
                    raise ValueError("output array must be contiguous float64")
                dst[i] = p
                keep.append(k)
        check(lib().ader_step_host_batch(self._h, n, ins, outs, float(dt), float(t_end)),
              "ader_step_host_batch")

    def set_material(self, mat):
        p, dev, keep, n = _ptr(mat)
        if n != 3 * self.cells:
            raise ValueError("material must hold 3 values per cell")
        check(lib().ader_set_material(self._h, p, dev), "ader_set_material")

    def set_point_source(self, x0, M, f0, t0):
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        M = np.ascontiguousarray(M, dtype=np.float64)
        check(lib().ader_set_point_source(self._h, x0.ctypes.data, M.ctypes.data, float(f0), float(t0)),
              "ader_set_point_source")

    def set_receivers(self, xyz, seismo, max_steps):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        p, dev, keep, n = _ptr(seismo)
        if not dev:
            raise ValueError("seismogram buffer must be device memory")
        if n < int(max_steps) * len(xyz) * 3:
            raise ValueError("seismogram buffer smaller than max_steps x nrec x 3")
        self._seismo = seismo
        check(lib().ader_set_receivers(self._h, len(xyz), xyz.ctypes.data, p, int(max_steps)),
              "ader_set_receivers")

    def set_subcell_state(self, U_sub, flags):
        """Cells with flags != 0 start in the FV space with subcell averages U_sub."""
        p, dev, keep, n = _ptr(U_sub)
        fp, fdev, fkeep, fn = _ptr(flags, np.uint8)
        if fn != self.cells or fdev != dev:
            raise ValueError("flags must hold one byte per cell, on the same side as U_sub")
        check(lib().ader_set_subcell_state(self._h, p, fp, dev), "ader_set_subcell_state")

    def get_subcell_state(self, out):
        p, dev, keep, n = _ptr(out)
        check(lib().ader_get_subcell_state(self._h, p, dev), "ader_get_subcell_state")
        return out

    def adjoint_step(self, t_n, dt, u_n, lam, grad_mat, grad_M, dJdu=None, static=False):
        """lam <- A^T lam (+ dJdu) for the step from t_n with fixed dt at forward state u_n;
        accumulates grad_mat [cells,3] and grad_M [6].  All CUDA float64 tensors.  static=True
        calls the allocation-free variant (work memory in the library's fixed device array)."""
        ptrs = []
        for a in (u_n, lam, grad_mat, grad_M) + ((dJdu,) if dJdu is not None else ()):
            p, dev, keep, n = _ptr(a)
            if not dev:
                raise ValueError("adjoint buffers must be device tensors")
            ptrs.append(p)
        if lam.numel() != self.count or u_n.numel() != self.count or grad_mat.numel() != 3 * self.cells \
                or grad_M.numel() != 6 or (dJdu is not None and dJdu.numel() != self.count):
            raise ValueError("adjoint buffer sizes")
        dj = ptrs[4] if dJdu is not None else None
        fn = lib().ader_adjoint_step_static if static else lib().ader_adjoint_step
        check(fn(self._h, float(t_n), float(dt), ptrs[0], ptrs[1], dj, ptrs[2], ptrs[3]),
              "ader_adjoint_step_static" if static else "ader_adjoint_step")

    def receivers_adjoint(self, res, scale, dJdu):
        p, dev, keep, n = _ptr(res)
        q, dev2, keep2, n2 = _ptr(dJdu)
        if not (dev and dev2) or n2 != self.count:
            raise ValueError("receiver adjoint buffers must be device tensors of the right size")
        check(lib().ader_receivers_adjoint(self._h, p, float(scale), q), "ader_receivers_adjoint")

    def misfit_gradient(self, u0, t0, dt, steps, k_ckpt, obs, grad_mat=None, grad_M=None):
        """(J, grad_mat, grad_M) of the receiver misfit (device tensors in and out)."""
        J = _D()
        pu = _ptr(u0)
        po = _ptr(obs)
        gm = _ptr(grad_mat)[0] if grad_mat is not None else None
        gM = _ptr(grad_M)[0] if grad_M is not None else None
        check(lib().ader_misfit_gradient(self._h, pu[0], float(t0), float(dt), int(steps), int(k_ckpt),
                                         po[0], ctypes.byref(J), gm, gM), "ader_misfit_gradient")
        return J.value

    def set_time(self, t):
        check(lib().ader_set_time(self._h, float(t)), "ader_set_time")

    def time(self):
        t = _D()
        check(lib().ader_get_time(self._h, ctypes.byref(t)), "ader_get_time")
        return t.value

    def step(self, dt=0.0, t_end=0.0):
        check(lib().ader_step(self._h, float(dt), float(t_end)), "ader_step")

    def run(self, steps, dt=0.0, t_end=0.0):
        check(lib().ader_run(self._h, int(steps), float(dt), float(t_end)), "ader_run")

    def run_graph(self, steps, replays, dt=0.0, t_end=0.0):
        check(lib().ader_run_graph(self._h, int(steps), int(replays), float(dt), float(t_end)),
              "ader_run_graph")

    def last_dt(self):
        v = _D()
        check(lib().ader_last_dt(self._h, ctypes.byref(v)), "ader_last_dt")
        return v.value

    def flags(self):
        out = np.zeros(self.cells, dtype=np.uint8)
        check(lib().ader_get_flags(self._h, out.ctypes.data, 0), "ader_get_flags")
        return out

    def troubled_count(self):
        v = _L()
        check(lib().ader_troubled_count(self._h, ctypes.byref(v)), "ader_troubled_count")
        return v.value

    def enable_timing(self, on=True):
        check(lib().ader_enable_timing(self._h, 1 if on else 0), "ader_enable_timing")

    def phase_times(self):
        """(dict phase -> summed ms, recorded steps); synchronises and clears the record."""
        ms = np.zeros(7)
        n = _I()
        check(lib().ader_phase_times(self._h, ms.ctypes.data, ctypes.byref(n)), "ader_phase_times")
        return dict(zip(PHASES, ms.tolist())), n.value

    def sync(self):
        check(lib().ader_sync(self._h), "ader_sync")


class Ensemble:
    """Several independent runs advanced together (one CUDA graph launch per steps_per_graph
    steps).  ``runs[i]`` are non-owning Context views of the member contexts."""

    def __init__(self, configs, stream=None):
        L = lib()
        if stream is None:
            stream = _default_stream()
        arr = (Config * len(configs))(*configs)
        h = _P()
        check(L.ader_ensemble_create(arr, len(configs), _P(stream), ctypes.byref(h)), "ader_ensemble_create")
        self._h = h
        self.runs = [Context(cfg, stream=stream, handle=L.ader_ensemble_run(h, i))
                     for i, cfg in enumerate(configs)]

    def step(self, steps, dt=0.0, t_end=0.0):
        check(lib().ader_ensemble_step(self._h, int(steps), float(dt), float(t_end)), "ader_ensemble_step")

    def sync(self):
        check(lib().ader_ensemble_sync(self._h), "ader_ensemble_sync")

    def set_launch(self, branches, steps_per_graph, blocks_per_sm=1):
        """branches >= 1: per-run kernels on that many forked streams; 0: one persistent launch per
        phase for all runs with blocks_per_sm predictor blocks per SM; -1: one cooperative
        persistent launch for all steps of a graph (grid-wide barriers between the phases)."""
        check(lib().ader_ensemble_set_launch(self._h, int(branches), int(steps_per_graph),
                                             int(blocks_per_sm)), "ader_ensemble_set_launch")

    def misfit_gradient(self, u0, t0, dt, steps, k_ckpt, obs, grad_mat=None, grad_M=None,
                        mem_budget=0):
        """Per-run misfit J (list) and gradients for every run (lists of device tensors; grad
        lists may be None)."""
        n = len(self.runs)

        def arr(ts):
            a = (ctypes.c_void_p * n)()
            for i, t in enumerate(ts):
                p, dev, keep, _ = _ptr(t)
                if not dev:
                    raise ValueError("ensemble gradient buffers must be device tensors")
                a[i] = p
            return a
        J = (ctypes.c_double * n)()
        gm = arr(grad_mat) if grad_mat is not None else None
        gM = arr(grad_M) if grad_M is not None else None
        check(lib().ader_ensemble_misfit_gradient(self._h, arr(u0), float(t0), float(dt), int(steps),
                                                  int(k_ckpt), arr(obs), J, gm, gM,
                                                  int(mem_budget)), "ader_ensemble_misfit_gradient")
        return list(J)

    def set_wait_limit(self, polls):
        """Polls of a grid-barrier wait of the fused launch before it gives up (0: at once)."""
        check(lib().ader_ensemble_set_wait_limit(self._h, int(polls)), "ader_ensemble_set_wait_limit")

    def autotune(self, dt):
        """(branches, steps_per_graph, blocks_per_sm, ms_per_step) of the fastest launch shape."""
        best = np.zeros(3, dtype=np.int32)
        ms = _D()
        check(lib().ader_ensemble_autotune(self._h, float(dt), best.ctypes.data, ctypes.byref(ms)),
              "ader_ensemble_autotune")
        return int(best[0]), int(best[1]), int(best[2]), ms.value

    def close(self):
        if getattr(self, "_h", None):
            for r in self.runs:
                r.close()
            lib().ader_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
