"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle on the same seeded inputs.

Bars: FP64 -- relative max-norm <= 1e-12 (operator applications and time stepping);
FP32 -- relative max-norm <= 2e-5 for one operator application on random fields and relative
L2 <= 1e-4 after time stepping smooth fields (the FP32 rounding of the O(h^-2) stencil terms,
each ~1e-7 of its size, summed over a few dozen terms, against results of order h^0)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.scheme import Oracle

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _solver(P, prec="fp64"):
    from paper_2003_12811_gb300 import Solver
    return Solver(P, prec)


def relmax(a, b):
    return max(np.abs(x - y).max() for x, y in zip(a, b)) / max(np.abs(y).max() for y in b)


def rell2(a, b):
    return math.sqrt(sum(np.sum((x - y) ** 2) for x, y in zip(a, b)) / sum(np.sum(y ** 2) for y in b))


SIZES = {2: (23, 21), 4: (40, 33), 6: (45, 37)}
CASES = [
    (("robin",) * 4, False, False),
    (("displacement",) * 4, False, False),
    (("robin", "displacement", "displacement", "robin"), True, False),
    (("displacement", "robin", "robin", "displacement"), True, True),
]


@pytest.mark.parametrize("order", (2, 4, 6))
@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec", ("fp64", "fp32"))
def test_apply_random_problem(order, case, prec):
    """One application of DD(c) + SATs (Sec. 4.6, 5, 6) on a random field, random material."""
    kinds, two, rev = CASES[case]
    P = W.random_problem(kinds=kinds, n=SIZES[order], order=order, two_blocks=two, reversed_interface=rev)
    O = Oracle(P)
    u = W.random_state(P)
    ref = O.unpack(O.A @ O.pack(u))
    S = _solver(P, prec)
    S.set_state(u, u, 0.0)
    got = S.apply()
    S.close()
    tol = FP64_TOL if prec == "fp64" else 2e-5
    assert relmax(got, ref) < tol


@pytest.mark.parametrize("order", (2, 4, 6))
def test_apply_with_data_mms(order):
    """Boundary data (traction, displacement), interface and body force at time t."""
    N = {2: 21, 4: 26, 6: 33}[order]
    P = W.mms_problem(N, order, kinds=("robin", "displacement", "robin", "displacement"), two_blocks=True)
    O = Oracle(P)
    u = [P.exact(b, 0.3) for b in P.blocks]
    ref = O.unpack(O.apply(O.pack(u), 0.37))
    S = _solver(P)
    S.set_state(u, u, 0.0)
    got = S.apply(with_data=True, t=0.37)
    S.close()
    assert relmax(got, ref) < FP64_TOL


def _run_both(P, nsteps, cfl, prec, init="exact"):
    O = Oracle(P)
    dt = O.suggest_dt(cfl)
    if init == "exact":
        up = [P.exact(b, -dt) for b in P.blocks]
        uc = [P.exact(b, 0.0) for b in P.blocks]
    else:
        uc = W.smooth_state(P)
        up = [u.copy() for u in uc]
    S = _solver(P, prec)
    S.set_state(up, uc, 0.0)
    S.step(nsteps, dt)
    gp, gc = S.state()
    S.close()
    rp, rc, _ = O.leapfrog(O.pack(up), O.pack(uc), 0.0, dt, nsteps)
    return gc, O.unpack(rc), gp, O.unpack(rp)


def test_config1_full_fp64():
    """Config 1: 101^2 Cartesian block, order 4, MMS with displacement SATs, 200 steps."""
    P = W.config1(N=101, order=4)
    gc, rc, gp, rp = _run_both(P, 200, 0.25, "fp64")
    assert relmax(gc, rc) < FP64_TOL
    assert relmax(gp, rp) < FP64_TOL


def test_config1_fp32():
    P = W.config1(N=101, order=4)
    gc, rc, _, _ = _run_both(P, 200, 0.25, "fp32")
    assert rell2(gc, rc) < 1e-4


@pytest.mark.parametrize("prec,tol", (("fp64", FP64_TOL), ("fp32", 1e-4)))
def test_config2_reduced(prec, tol):
    """Config 2 geometry and material on 2x2 blocks of 41^2, order 6, MMS, 100 steps."""
    P = W.config2(n=41, order=6)
    gc, rc, _, _ = _run_both(P, 100, 0.25, prec)
    err = relmax(gc, rc) if prec == "fp64" else rell2(gc, rc)
    assert err < tol


@pytest.mark.parametrize("prec,tol", (("fp64", FP64_TOL), ("fp32", 1e-4)))
def test_config2_three_by_two_blocks(prec, tol):
    """Config 2 geometry on 3 x 2 blocks of 28^2 (order 6): 7 interfaces, 14 interface sides,
    more than one launch of interface traces per step; MMS, 60 steps."""
    P = W.config2(n=28, order=6, nbx=3, nby=2)
    assert sum(f.kind == "interface" for b in P.blocks for f in b.faces) == 14
    gc, rc, _, _ = _run_both(P, 60, 0.25, prec)
    err = relmax(gc, rc) if prec == "fp64" else rell2(gc, rc)
    assert err < tol


@pytest.mark.parametrize("prec,tol", (("fp64", FP64_TOL), ("fp32", 1e-4)))
def test_config3_reduced_with_source(prec, tol):
    """Config 3 topography, tilted VTI, Robin + traction-free top, interface, Ricker point
    source, order 6, on 2 blocks of 101 x 51, 150 steps from rest."""
    P = W.config3(n1=101, n2=51, order=6)
    O = Oracle(P)
    dt = O.suggest_dt(0.3)
    z = [np.zeros((2, b.N2, b.N1)) for b in P.blocks]
    S = _solver(P, prec)
    S.set_state(z, z, 0.0)
    S.step(150, dt)
    _, gc = S.state()
    S.close()
    _, rc, _ = O.leapfrog(O.pack(z), O.pack(z), 0.0, dt, 150)
    rc = O.unpack(rc)
    err = relmax(gc, rc) if prec == "fp64" else rell2(gc, rc)
    assert err < tol


@pytest.mark.parametrize("order", (4, 6))
def test_energy_matches_and_is_conserved(order):
    P = W.random_problem(kinds=("robin", "displacement", "displacement", "robin"), n=SIZES[order],
                         order=order, two_blocks=True)
    O = Oracle(P)
    dt = O.suggest_dt(0.3)
    u0 = W.smooth_state(P)
    S = _solver(P)
    S.set_state(u0, u0, 0.0)
    E = []
    for _ in range(20):
        S.step(10, dt)
        E.append(S.energy(dt))
    gp, gc = S.state()
    S.close()
    assert abs(O.energy_leapfrog(O.pack(gp), O.pack(gc), dt) - E[-1]) < 1e-12 * abs(E[-1])
    E = np.array(E)
    assert np.abs(E - E[0]).max() < 1e-12 * E[0]


@pytest.mark.parametrize("prec,tol", (("fp64", 1e-10), ("fp32", 1e-5)))
def test_suggest_dt(prec, tol):
    P = W.config2(n=41, order=6)
    O = Oracle(P)
    S = _solver(P, prec)
    got = S.suggest_dt(0.5)
    S.close()
    assert abs(got - O.suggest_dt(0.5)) < tol * got


@pytest.mark.parametrize("order", (2, 4, 6))
def test_minimum_sizes(order):
    """Smallest legal blocks: closures of both ends touch, interior region a single tile."""
    n = {2: 5, 4: 18, 6: 27}[order]
    P = W.random_problem(kinds=("displacement", "robin", "robin", "displacement"), n=(n, n), order=order)
    O = Oracle(P)
    u = W.random_state(P)
    ref = O.unpack(O.A @ O.pack(u))
    S = _solver(P)
    S.set_state(u, u, 0.0)
    got = S.apply()
    S.close()
    assert relmax(got, ref) < FP64_TOL


def test_errors_are_reported():
    from paper_2003_12811_gb300 import SbpError
    P = W.random_problem(n=(20, 19), order=4)
    P.blocks[0].X = P.blocks[0].X[:, :, ::-1].copy()     # mirrored grid: J < 0
    with pytest.raises(SbpError) as e:
        _solver(P)
    assert e.value.code == -2
    P = W.random_problem(n=(20, 19), order=4, two_blocks=True)
    P.blocks[1] = W.random_problem(n=(20, 23), order=4).blocks[0]
    P.blocks[1].faces[0] = W.Face("interface", nbr=(0, 1, False))
    with pytest.raises(SbpError) as e:
        _solver(P)
    assert e.value.code == -3


@pytest.mark.parametrize("prec", ("fp64", "fp32"))
def test_l2_diff_is_the_schemes_norm(prec):
    """sbp_l2_diff: the l2 error of Table 1 (sqrt(sum e^T (J H) e)) against the oracle's l2_error of
    the same field, and the reference norm against the oracle's J H quadrature."""
    from paper_2003_12811_gb300.binding import FIELD_CUR
    P = W.mms_problem(33, 6, kinds=("robin", "displacement", "robin", "displacement"), two_blocks=True)
    O = Oracle(P)
    u = [P.exact(b, 0.2) + 1e-3 * np.sin(3 * b.X[0] + 2 * b.X[1]) for b in P.blocks]
    if prec == "fp32":
        u = [np.asarray(x, np.float32).astype(np.float64) for x in u]
    S = _solver(P, prec)
    S.set_state(u, u, 0.0)
    e2, r2 = S.sbp_l2_diff(FIELD_CUR, [P.exact(b, 0.2) for b in P.blocks])
    S.close()
    eo = O.l2_error(O.pack(u), 0.2)
    assert math.sqrt(e2) == pytest.approx(eo, rel=1e-11)
    ex = O.pack([P.exact(b, 0.2) for b in P.blocks])
    assert r2 == pytest.approx(float(np.dot(ex, np.concatenate([np.tile(bo.J * bo.Hvec, 2) for bo in O.bops]) * ex)),
                               rel=1e-12)
