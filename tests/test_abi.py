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
    assert lib.ader_step(None, 0.0, 0.0) == ader.EINVAL
    lib.ader_destroy(None)
