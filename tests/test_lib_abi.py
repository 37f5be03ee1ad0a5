"""CPU checks of the C-ABI boundary: the library builds, loads and exports every function
include/sbp.h declares; argument validation rejects bad input before any device work."""
import ctypes as C
import shutil

import numpy as np
import pytest

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not __import__("os").path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def L():
    from paper_2003_12811_gb300 import build
    build.build()
    from paper_2003_12811_gb300 import binding
    return binding.lib()


def test_exports_every_declared_symbol(L):
    from paper_2003_12811_gb300 import binding
    names = binding.header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def _desc(order=4, n=20, kinds=(1, 1, 1, 1), precision=0, beta=0.0):
    from paper_2003_12811_gb300 import binding as B
    x1, x2 = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n))
    x1, x2 = np.ascontiguousarray(x1), np.ascontiguousarray(x2)
    blocks = (B.BlockDesc * 1)()
    blocks[0].n1 = blocks[0].n2 = n
    blocks[0].x1 = x1.ctypes.data_as(C.POINTER(C.c_double))
    blocks[0].x2 = x2.ctypes.data_as(C.POINTER(C.c_double))
    for f, k in enumerate(kinds):
        blocks[0].faces[f].kind = k
    return B.GridDesc(order, precision, 1, blocks, beta), (x1, x2, blocks)


@pytest.mark.parametrize("kw,code", [
    (dict(order=3), -1),
    (dict(order=6, n=20), -1),          # too few nodes for order 6
    (dict(precision=7), -1),
    (dict(kinds=(5, 1, 1, 1)), -1),
    (dict(beta=0.5), -1),
    (dict(kinds=(2, 1, 1, 1)), -3),      # interface pointing at itself
])
def test_validation_before_device_work(L, kw, code):
    desc, keep = _desc(**kw)
    h = C.c_void_p()
    rc = L.sbp_grid_create(C.byref(desc), C.byref(h))
    assert rc == code and not h.value
    assert len(L.sbp_last_error(None)) > 0


def test_null_handle_calls_are_rejected(L):
    assert L.sbp_step(None, 1, 0.1, None) == -1
    assert L.sbp_destroy(None) == 0
    E = C.c_double()
    assert L.sbp_energy(None, 0.1, C.byref(E)) == -1
