"""Parity at the full size of the 2 x 2-block curvilinear workload (4 blocks of 801 x 801, order 6,
rotated anisotropic stiffness, welded interfaces, traction data on the outer faces, manufactured
body force): the GPU result at sampled nodes against the FP64 oracle evaluated on a window around
each node, in FP64 (the parity bar) and FP32.

A window spans every block the node's neighbourhood reaches (the four-block junction keeps all
four), keeps the real faces and interfaces it touches, and is cropped farther from the node than
the domain of dependence of the compared quantity (an application reaches at most 12 nodes: the
widest closure row of D_xx^FC; a step one application), so it reproduces the full-grid value."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.scheme import Oracle

pytestmark = pytest.mark.gpu

N, NB = 801, 2
NSTEPS = 10
SAMPLES = [
    (0, 800, 800), (3, 0, 0), (1, 0, 800), (2, 800, 0),        # the four-block junction
    (0, 800, 400), (1, 0, 400), (0, 400, 800), (2, 400, 0),    # interfaces, both sides
    (1, 400, 800), (3, 400, 0), (2, 800, 400), (3, 0, 400),
    (0, 795, 300), (1, 4, 500), (2, 300, 5),                   # closure depth next to interfaces
    (0, 0, 400), (1, 800, 300), (0, 300, 0), (3, 500, 800),    # traction faces
    (0, 0, 0), (1, 800, 0), (2, 0, 800), (3, 800, 800),        # outer corners
    (0, 800, 0), (1, 0, 0), (0, 0, 800), (2, 0, 0),            # interface meets an outer face
    (0, 400, 400), (3, 300, 600),                              # interior
]
# tolerances relative to the window's largest value: FP64 -- the parity bar; FP32 -- per
# application the rounding of the O(h^-2)-weighted stencil terms (~1e-7 of each, a few dozen
# terms); after NSTEPS steps of the smooth manufactured solution, the FP32 rounding of every level
# carried through NSTEPS applications
TOL_APPLY = {"fp64": 1e-12, "fp32": 2e-5}
TOL_STEPS = {"fp64": 1e-12, "fp32": 1e-4}


def window(b, i1, i2, R):
    """{block: (i1_lo, i1_hi, i2_lo, i2_hi)} of every block within R nodes of node (i1, i2) of
    block b (blocks b = by * NB + bx share their interface nodes)."""
    bx, by = b % NB, b // NB
    g1, g2 = bx * (N - 1) + i1, by * (N - 1) + i2
    win = {}
    for cy in range(NB):
        for cx in range(NB):
            lo1, hi1 = max(0, g1 - R - cx * (N - 1)), min(N, g1 + R + 1 - cx * (N - 1))
            lo2, hi2 = max(0, g2 - R - cy * (N - 1)), min(N, g2 + R + 1 - cy * (N - 1))
            if lo1 < hi1 and lo2 < hi2:
                win[cy * NB + cx] = (lo1, hi1, lo2, hi2)
    # the oracle needs at least 27 nodes per direction (order 6) in every kept block
    for k, (lo1, hi1, lo2, hi2) in list(win.items()):
        if hi1 - lo1 < 27 or hi2 - lo2 < 27:
            lo1, hi1 = (lo1, max(hi1, lo1 + 27)) if lo1 == 0 else (min(lo1, hi1 - 27), hi1)
            lo2, hi2 = (lo2, max(hi2, lo2 + 27)) if lo2 == 0 else (min(lo2, hi2 - 27), hi2)
            win[k] = (lo1, hi1, lo2, hi2)
    return win


def crop(fields, win):
    return [fields[b][:, lo2:hi2, lo1:hi1] for b, (lo1, hi1, lo2, hi2) in sorted(win.items())]


def local(win, b, i1, i2):
    lo1, _, lo2, _ = win[b]
    return sorted(win).index(b), i1 - lo1, i2 - lo2


@pytest.fixture(scope="module")
def problem():
    import __graft_entry__
    __graft_entry__.build()
    return W.config2(n=N)


@pytest.fixture(scope="module", params=("fp64", "fp32"))
def solver(request, problem):
    from paper_2003_12811_gb300 import Solver
    S = Solver(problem, request.param)
    yield S, request.param
    S.close()


def test_window_helper_covers_the_junction():
    win = window(0, 800, 800, 30)
    assert sorted(win) == [0, 1, 2, 3]
    assert win[0] == (770, 801, 770, 801) and win[3] == (0, 31, 0, 31)


def test_operator_with_data_at_full_size(problem, solver):
    """One application with the traction data and the body force at time t, on a random field."""
    S, prec = solver
    P = problem
    u = W.random_state(P, seed=11)
    t = 0.123
    S.set_state(u, u, 0.0)
    r = S.apply(with_data=True, t=t)
    for (b, i1, i2) in SAMPLES:
        win = window(b, i1, i2, 26)
        O = Oracle(W.config2(n=N, window=win))
        ref = O.unpack(O.apply(O.pack(crop(u, win)), t))
        k, j1, j2 = local(win, b, i1, i2)
        scale = max(np.abs(ref[k]).max(), 1e-30)
        err = np.abs(r[b][:, i2, i1] - ref[k][:, j2, j1]).max() / scale
        assert err < TOL_APPLY[prec], ((b, i1, i2), err)


def test_steps_at_full_size(problem, solver):
    """NSTEPS leapfrog steps of the manufactured solution with its data, from t = 0."""
    S, prec = solver
    P = problem
    dt = S.suggest_dt(0.25)
    up = [P.exact(b, -dt) for b in P.blocks]
    uc = [P.exact(b, 0.0) for b in P.blocks]
    S.set_state(up, uc, 0.0)
    S.step(NSTEPS, dt)
    _, cur = S.state()
    R = 12 * (NSTEPS + 1) + 4
    for (b, i1, i2) in SAMPLES[::2] + [(3, 0, 0)]:
        win = window(b, i1, i2, R)
        Pw = W.config2(n=N, window=win)
        O = Oracle(Pw)
        _, un, _ = O.leapfrog(O.pack(crop(up, win)), O.pack(crop(uc, win)), 0.0, dt, NSTEPS)
        ref = O.unpack(un)
        k, j1, j2 = local(win, b, i1, i2)
        scale = np.abs(ref[k]).max()
        err = np.abs(cur[b][:, i2, i1] - ref[k][:, j2, j1]).max() / scale
        assert err < TOL_STEPS[prec], ((b, i1, i2), err)
        assert math.isfinite(err)
