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


@pytest.mark.parametrize("prec", ("fp32", "fp64"))
def test_footprint_covers_every_device_buffer(L, prec):
    """sbp_grid_footprint (host arithmetic only) is at least the sum of the buffers the handle
    allocates: per block 17 field planes in the working precision (u 2 x 2, c 10, 1/(rho J), r 2),
    7 FP64 metric planes, the closure matrices of D_xx^FC along both directions
    (2 x NCLOS x NCLOSJ x 3 words per boundary line) and, per interface face, a 7-word trace per
    face node; an interface adds exactly its two traces."""
    import re
    import os
    from paper_2003_12811_gb300.binding import footprint_bytes
    import workloads as W
    es = 4 if prec == "fp32" else 8
    tab = open(os.path.join(os.path.dirname(__file__), "..", "paper_2003_12811_gb300", "csrc", "sbp_tables.inc")).read()
    d = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define SBP6_(\w+) (-?\d+)", tab)}
    P = W.config3(n1=401, n2=201, order=6)
    need = 0
    for blk in P.blocks:
        pitch = (blk.N1 + 31) // 32 * 32
        plane = blk.N2 * pitch
        need += 17 * plane * es + 7 * plane * 8
        need += 2 * d["NCLOS"] * d["NCLOSJ"] * 3 * (blk.N1 + blk.N2) * es
        need += sum(7 * (blk.N2 if f < 2 else blk.N1) * es for f, face in enumerate(blk.faces) if face.kind == "interface")
    fp = footprint_bytes(P, prec)
    assert need <= fp <= 1.05 * need + (1 << 20), (need, fp)


def test_sbp3_validation_before_device_work(L):
    """sbp3_create rejects bad arguments before any CUDA call (so this runs without a GPU)."""
    n = 27
    X = np.zeros(3 * n * n * n)
    kinds = (C.c_int * 6)(*([1] * 6))
    h = C.c_void_p()
    P = C.POINTER(C.c_double)
    xp = X.ctypes.data_as(P)
    assert L.sbp3_create(5, 0, n, n, n, xp, kinds, 1.0, C.byref(h)) == -1          # order
    assert L.sbp3_create(6, 3, n, n, n, xp, kinds, 1.0, C.byref(h)) == -1          # precision
    assert L.sbp3_create(6, 0, 26, n, n, xp, kinds, 1.0, C.byref(h)) == -1         # too few nodes
    assert L.sbp3_create(6, 0, n, n, n, None, kinds, 1.0, C.byref(h)) == -1        # no coordinates
    bad = (C.c_int * 6)(*([1] * 5 + [2]))
    assert L.sbp3_create(6, 0, n, n, n, xp, bad, 1.0, C.byref(h)) == -1            # face kind
    assert L.sbp3_create(6, 0, n, n, n, xp, kinds, 0.0, C.byref(h)) == -1          # beta
    # a plane of 2^27 elements or more is rejected before X is read (X here is far too short)
    assert L.sbp3_create(6, 1, 1 << 17, 1024, n, xp, kinds, 1.0, C.byref(h)) == -1
    assert b"2^27" in L.sbp3_last_error(None)
    X[5] = np.nan
    assert L.sbp3_create(6, 0, n, n, n, xp, kinds, 1.0, C.byref(h)) == -1          # non-finite X
    assert b"non-finite" in L.sbp3_last_error(None)
    out = C.c_longlong()
    assert L.sbp3_footprint(6, 1, 256, 256, 256, C.byref(out)) == 0
    # 64 FP32 fields + 3 FP64 coordinate fields per node, and per x1 line the order-6 closure
    # matrices: 2 sides x 9 rows x 12 columns x 6 coefficients
    assert out.value == 256 ** 3 * (64 * 4 + 3 * 8) + 256 ** 2 * 2 * 9 * 12 * 6 * 4
    assert L.sbp3_footprint(5, 1, 256, 256, 256, C.byref(out)) == -1
    # every call rejects a NULL handle before any device work
    d = np.zeros(3 * 27 ** 3)
    dp = d.ctypes.data_as(P)
    assert L.sbp3_set_material(None, 0, 1, dp, dp) == -1
    assert L.sbp3_set_state(None, dp, dp) == -1
    assert L.sbp3_get_state(None, dp, dp) == -1
    assert L.sbp3_apply(None, dp, dp) == -1
    assert L.sbp3_step(None, 1, 1e-3, None) == -1
    assert L.sbp3_set_tuning(None, 0) == -1
    assert L.sbp3_autotune(None, None, None) == -1
    assert L.sbp3_profile(None, 1) == -1
    assert L.sbp3_destroy(None) == -1
    assert L.sbp3_get_info(None, None, None, None) == -1
