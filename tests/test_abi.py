"""CPU checks of the C-ABI library: it loads, exports every function include/ader.h declares,
and its host-side reference tables agree with a library Gauss-Legendre rule (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1905_07987_gb300 import ader

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ader_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(ader.LIB_PATH):
        from paper_1905_07987_gb300 import build
        build.build()
    return ader.lib()


def test_library_exports_every_declared_symbol(lib):
    names = declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("order", range(1, 7))
def test_reference_nodes_match_library_rule(lib, order):
    x, w = ader.reference_nodes(order)
    xr, wr = np.polynomial.legendre.leggauss(order + 1)
    assert np.allclose(x, (xr + 1) / 2, atol=2e-16 * 4, rtol=0)
    assert np.allclose(w, wr / 2, atol=1e-15, rtol=0)


def test_status_strings(lib):
    for s in range(9):
        assert ader.status_string(s)
    assert ader.status_string(0) == "ok"


def test_invalid_arguments_are_rejected_without_a_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.ader_create(None, None, ctypes.byref(h)) == ader.EINVAL
    cfg = ader.make_config("euler", 2, 9, (4, 4), (0, 0), (1, 1), "periodic", 0.5)
    assert lib.ader_create(ctypes.byref(cfg), None, ctypes.byref(h)) == ader.EUNSUPPORTED
    cfg = ader.make_config("elastic", 2, 3, (4, 4), (0, 0), (1, 1), "periodic", 0.5)
    assert lib.ader_create(ctypes.byref(cfg), None, ctypes.byref(h)) == ader.EUNSUPPORTED
    cfg = ader.make_config("euler", 2, 3, (4, 4), (0, 0), (1, 1), [("periodic", "wall")] * 2, 0.5)
    assert lib.ader_create(ctypes.byref(cfg), None, ctypes.byref(h)) == ader.EINVAL
    # the Cauchy-Kowalevski predictor: linear elastic family only; unknown predictor ids
    cfg = ader.make_config("euler", 3, 3, (4, 4, 4), (0,) * 3, (1,) * 3, "periodic", 0.5, predictor="ck")
    assert lib.ader_create(ctypes.byref(cfg), None, ctypes.byref(h)) == ader.EUNSUPPORTED
    cfg = ader.make_config("elastic", 3, 3, (4, 4, 4), (0,) * 3, (1,) * 3, "absorbing", 0.5, predictor=7)
    assert lib.ader_create(ctypes.byref(cfg), None, ctypes.byref(h)) == ader.EINVAL
    # the continuous extension Runge-Kutta guess: the Picard predictor only; unknown guess ids
    for prec in ("fp64", "mixed"):
        cfg = ader.make_config("elastic", 3, 3, (4, 4, 4), (0,) * 3, (1,) * 3, "absorbing", 0.5,
                               predictor="ck", initial_guess="cerk", precision=prec)
        assert lib.ader_create(ctypes.byref(cfg), None, ctypes.byref(h)) == ader.EUNSUPPORTED
    # the tensor-core form: the elastic Cauchy-Kowalevski predictor at orders 1, 3, 5 only; the
    # value 2 of ader_prec is not built
    for pde, order, pred in (("euler", 3, "picard"), ("elastic", 4, "ck"), ("elastic", 5, "picard")):
        cfg = ader.make_config(pde, 3, order, (4, 4, 4), (0,) * 3, (1,) * 3,
                               "periodic" if pde == "euler" else "absorbing", 0.5, predictor=pred,
                               precision="tf32x3")
        assert lib.ader_create(ctypes.byref(cfg), None, ctypes.byref(h)) == ader.EUNSUPPORTED
    cfg = ader.make_config("elastic", 3, 5, (4, 4, 4), (0,) * 3, (1,) * 3, "absorbing", 0.5,
                           predictor="ck", precision=2)
    assert lib.ader_create(ctypes.byref(cfg), None, ctypes.byref(h)) == ader.EUNSUPPORTED
    cfg = ader.make_config("euler", 3, 3, (4, 4, 4), (0,) * 3, (1,) * 3, "periodic", 0.5, initial_guess=5)
    assert lib.ader_create(ctypes.byref(cfg), None, ctypes.byref(h)) == ader.EINVAL
    cfg = ader.make_config("euler", 3, 3, (4, 4, 4), (0,) * 3, (1,) * 3, "periodic", 0.5, limiter=4)
    assert lib.ader_create(ctypes.byref(cfg), None, ctypes.byref(h)) == ader.EINVAL
    cfg = ader.make_config("elastic", 3, 3, (4, 4, 4), (0,) * 3, (1,) * 3, "absorbing", 0.5, limiter=3)
    assert lib.ader_create(ctypes.byref(cfg), None, ctypes.byref(h)) == ader.EUNSUPPORTED
    assert lib.ader_step(None, 0.0, 0.0) == ader.EINVAL
    lib.ader_destroy(None)


@pytest.mark.parametrize("order", range(1, 7))
def test_reference_tables_match_the_oracle(lib, order):
    """The library's host tables (its own node and table derivations) against the oracle's: the
    collocation derivative D and the predictor's time solve K1^{-1} W to round-off, and the
    Lagrange-to-monomial table Vi of the Cauchy-Kowalevski source term against a 50-digit inverse
    of the Vandermonde matrix of the same nodes."""
    mpmath = pytest.importorskip("mpmath")
    from oracle.refelem import RefElement
    D, Kw, Vi = ader.reference_tables(order)
    ref = RefElement(order)
    Do = ref.D.numpy()
    assert np.abs(D - Do).max() <= 1e-13 * np.abs(Do).max()
    Kwo = np.linalg.solve(ref.K1.numpy(), np.diag(ref.w.numpy()))
    assert np.abs(Kw - Kwo).max() <= 1e-13 * np.abs(Kwo).max()
    x, _ = ader.reference_nodes(order)
    n = order + 1
    mpmath.mp.dps = 50
    V = mpmath.matrix([[mpmath.mpf(float(xt)) ** k for k in range(n)] for xt in x])
    Vinv = V ** -1
    ex = np.array([[float(Vinv[k, t]) for t in range(n)] for k in range(n)])
    assert np.abs(Vi - ex).max() <= 1e-14 * np.abs(ex).max()


def test_reference_tables_reject_orders_outside_the_kernels(lib):
    n = 8
    buf = np.zeros(n * n)
    for order in (0, 7):
        assert lib.ader_reference_tables(order, buf.ctypes.data, None, None) == ader.EINVAL
