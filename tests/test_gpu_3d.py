"""Parity of the 3-D CUDA operator (include/sbp3.h) with the FP64 3-D oracle, element by element.

Bars are relative to the size of one term of the operator's sums, t = max(w) max|c| max(1/h)^2
max|u|: an acceleration is a sum of ~250 such terms that cancel down to the result, so rounding
errors scale with t, not with the result.  FP64: 1e-12 t (the two sides add the same terms in
different orders).  FP32: u and the coefficients are rounded to FP32 (relative 6e-8) and the
sums accumulate in FP32: 1e-5 t.
"""
import numpy as np
import pytest

from workloads import box3d as B
from oracle.scheme3d import Oracle3D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


MIXED = ("traction", "displacement", "displacement", "traction", "displacement", "traction")


def _term_scale(O, u):
    return O.w.max() * np.abs(O.c).max() * max(1.0 / op.h for op in O.op) ** 2 * np.abs(u).max()


@pytest.mark.parametrize("order,N", [(2, (9, 7, 8)), (4, (21, 18, 19)), (6, (30, 28, 27)), (6, (45, 33, 29))])
@pytest.mark.parametrize("faces", [MIXED, ("traction",) * 6, ("displacement",) * 6])
def test_apply_fp64(order, N, faces):
    from paper_2003_12811_gb300 import Solver3D
    b = B.random_block3(N=N, order=order, faces=faces)
    O = Oracle3D(b)
    u = B.random_state3(b, seed=5)
    ref = O.accel(u)
    S = Solver3D.from_block(b, "fp64")
    got = S.apply(u)
    S.close()
    assert np.abs(got - ref).max() < 1e-12 * _term_scale(O, u)


@pytest.mark.parametrize("order,N", [(6, (30, 28, 27)), (6, (64, 29, 31)), (4, (37, 18, 21)), (2, (9, 7, 8)),
                                     (2, (5, 6, 5))])
@pytest.mark.parametrize("smooth", [True, False])
def test_apply_fp32(order, N, smooth):
    from paper_2003_12811_gb300 import Solver3D
    b = B.random_block3(N=N, order=order, faces=MIXED)
    O = Oracle3D(b)
    u = B.smooth_state3(b, seed=6) if smooth else B.random_state3(b, seed=6)
    ref = O.accel(u)
    S = Solver3D.from_block(b, "fp32")
    got = S.apply(u)
    S.close()
    assert np.abs(got - ref).max() < 1e-5 * _term_scale(O, u)


def test_material_in_chunks_equals_whole():
    """Setting the material plane chunk by plane chunk gives the same device coefficients as one
    call (the apply results are bitwise equal)."""
    from paper_2003_12811_gb300 import Solver3D
    from paper_2003_12811_gb300.binding import _pair45
    b = B.random_block3(N=(30, 28, 27), order=6, faces=MIXED)
    u = B.random_state3(b, seed=7)
    A = Solver3D.from_block(b, "fp32")
    ra = A.apply(u)
    A.close()
    S = Solver3D(b.X, b.faces, 6, "fp32")
    P = _pair45(b.C)
    for k0, k1 in ((0, 5), (5, 6), (6, 20), (20, 27)):
        S.sbp3_set_material(k0, k1 - k0, b.rho[k0:k1], P[:, k0:k1])
    rb = S.apply(u)
    S.close()
    assert np.array_equal(ra, rb)


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-11), ("fp32", 5e-5)])
def test_leapfrog_against_oracle(prec, bar):
    from paper_2003_12811_gb300 import Solver3D
    b = B.random_block3(N=(30, 28, 27), order=6, faces=MIXED)
    O = Oracle3D(b)
    dt = O.suggest_dt(0.8)
    u0 = B.smooth_state3(b, seed=1)
    u1 = u0 + dt * B.smooth_state3(b, seed=2)
    if prec == "fp32":
        u0 = u0.astype(np.float32).astype(np.float64)
        u1 = u1.astype(np.float32).astype(np.float64)
    S = Solver3D.from_block(b, prec)
    S.set_state(u0, u1)
    S.step(60, dt)
    gp, gc = S.state()
    S.close()
    rp, rc = O.leapfrog(u0, u1, dt, 60)
    err = np.sqrt(np.sum((gc - rc) ** 2) / np.sum(rc ** 2))
    assert err < bar, err
    # the previous level is the level before the last step, exactly
    assert np.sqrt(np.sum((gp - rp) ** 2) / np.sum(rp ** 2)) < bar


def test_state_roundtrip_and_errors():
    from paper_2003_12811_gb300 import Solver3D, SbpError
    b = B.random_block3(N=(28, 27, 27), order=6, faces=MIXED)
    S = Solver3D(b.X, b.faces, 6, "fp64")
    u0, u1 = B.random_state3(b, 1), B.random_state3(b, 2)
    with pytest.raises(SbpError) as e:
        S.step(1, 1e-3)                          # no material yet
    assert e.value.code == -8
    S.set_state(u0, u1)
    a, c = S.state()
    assert np.array_equal(a, u0) and np.array_equal(c, u1)
    with pytest.raises(SbpError) as e:
        S.apply(u0)
    assert e.value.code == -8
    S.close()
    # a mirrored coordinate makes J < 0 at every node: the material call reports it
    X = b.X.copy()
    X[0] = -X[0]
    S = Solver3D(X, b.faces, 6, "fp64")
    from paper_2003_12811_gb300.binding import _pair45
    with pytest.raises(SbpError) as e:
        S.sbp3_set_material(0, 27, b.rho, _pair45(b.C))
    assert e.value.code == -2
    S.close()


def test_fullsize_sampled_parity():
    """The bench workload (256^3 nodes, order 6) in FP32 (the configuration the bench times) and in
    FP64: the accelerations at sampled nodes -- interior, next to the displacement faces x1 = 0
    and x2 = 1, under the traction top face x3 = 1, and at the corner of three faces -- against
    the oracle on a 27^3 crop around each sample ('open' cut faces, the whole block's spacing)."""
    from paper_2003_12811_gb300 import Solver3D
    N = (256, 256, 256)
    faces = ("displacement",) * 5 + ("traction",)
    g1, g2, g3 = B.ref_grid3(*N)
    u = np.array([np.sin(2.1 * g1 + 0.3) * np.cos(1.7 * g2) * np.sin(1.3 * g3 + 0.5),
                  np.cos(1.1 * g1) * np.sin(2.3 * g2 + 0.2) * np.cos(0.9 * g3),
                  np.sin(1.5 * g1 + 0.7) * np.sin(1.2 * g2) * np.cos(2.0 * g3 + 0.1)])
    del g1, g2, g3
    samples = [((100, 117, 140), (113, 130, 153)),     # (crop lo, node)
               ((0, 60, 90), (2, 73, 103)),
               ((70, 229, 30), (83, 254, 43)),
               ((140, 40, 229), (153, 53, 255)),
               ((0, 229, 229), (0, 255, 255))]
    got = {}
    for prec in ("fp32", "fp64"):
        X = B.block3_coords(N)
        S = Solver3D(X, faces, 6, prec)
        del X
        for k0 in range(0, 256, 64):
            rho, P = B.material3_planes(N, k0=k0, k1=k0 + 64)
            S.sbp3_set_material(k0, 64, rho, P)
        a = S.apply(u)
        S.close()
        got[prec] = np.array([a[:, n3, n2, n1] for _, (n1, n2, n3) in samples])
        del a
    for s_i, (lo, node) in enumerate(samples):
        hi = tuple(l + 27 for l in lo)
        c = B.random_block3_crop(N, lo, hi, order=6, faces=faces)
        sub = u[:, lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        O = Oracle3D(c)
        ac = O.accel(sub)
        i1, i2, i3 = (node[0] - lo[0], node[1] - lo[1], node[2] - lo[2])
        ref = ac[:, i3, i2, i1]
        t = _term_scale(O, sub)
        assert np.abs(got["fp32"][s_i] - ref).max() < 1e-5 * t, (node, got["fp32"][s_i], ref)
        assert np.abs(got["fp64"][s_i] - ref).max() < 1e-12 * t, (node, got["fp64"][s_i], ref)


def test_tuning_variants_bitwise_equal():
    """Every launch shape of the interior kernel computes bitwise the same step; the autotuner picks
    one of them and leaves the state alone."""
    from paper_2003_12811_gb300 import Solver3D
    b = B.random_block3(N=(40, 37, 33), order=6, faces=MIXED)
    u0 = B.smooth_state3(b, seed=1)
    u1 = u0 + 1e-3 * B.smooth_state3(b, seed=2)
    outs = []
    for v in range(4):
        S = Solver3D.from_block(b, "fp32")
        S.set_state(u0, u1)
        S.sbp3_set_tuning(v)
        S.step(3, 2e-3)
        outs.append(S.state())
        S.close()
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])
    S = Solver3D.from_block(b, "fp32")
    S.set_state(u0, u1)
    v, ms = S.sbp3_autotune()
    assert 0 <= v < 4 and all(m > 0 for m in ms)
    a, c = S.state()
    S.close()
    assert np.array_equal(c, u1.astype(np.float32).astype(np.float64))
