"""Parity at the full topography workload (2 x 4001x2001, order 6; FP32 in the launch
configuration bench.py times, and FP64 at the parity bar) (column-marching interior, tiled strips with in-kernel SATs on the
auxiliary stream, sources): the GPU result at sampled nodes against the oracle evaluated on a
window around each node.  The operator (and a few leapfrog steps) at a node only reads nodes
within its stencil, so a window whose cropped edges are farther than that domain of dependence
reproduces the full-grid value; windows keep the real faces, the interface (both blocks) and the
point source when they reach them."""
import numpy as np
import pytest

import workloads as W
from oracle.scheme import Oracle

pytestmark = pytest.mark.gpu

N1, N2 = 4001, 2001
SAMPLES = [
    (0, 2000, 1000), (1, 1234, 777),                       # interior
    (1, 3000, 2000), (1, 3000, 1995),                      # traction-free surface, closure depth
    (1, 0, 2000), (1, 4000, 2000), (0, 0, 0), (0, 4000, 0),  # corners
    (0, 0, 1000), (1, 4000, 1000), (0, 2000, 0), (0, 5, 3),  # Robin sides and bottom
    (0, 1500, 2000), (1, 1500, 0), (0, 2500, 1996), (1, 2500, 3),   # interface, both sides
    (0, 0, 2000), (1, 4000, 0),                            # interface meets a side
    (1, 2000, 1999), (1, 2001, 2000),                      # at the point source
]


# tolerance relative to the window's largest value: FP32 -- the rounding of the O(h^-2)-weighted
# stencil terms (~1e-7 of each) summed over a few dozen terms; FP64 -- the parity bar
TOL = {"fp32": 2e-5, "fp64": 1e-12}


@pytest.fixture(scope="module")
def problem():
    import __graft_entry__
    __graft_entry__.build()
    P = W.config3()
    return P, W.smooth_state(P, seed=3, amplitude=1e-3)


@pytest.fixture(scope="module", params=("fp32", "fp64"))
def full(request, problem):
    from paper_2003_12811_gb300 import Solver
    P, u = problem
    S = Solver(P, request.param)
    dt = S.suggest_dt(0.3)
    yield P, S, u, dt, request.param
    S.close()


def _window(b, i1, i2, R):
    lo1, hi1 = max(0, i1 - R), min(N1, i1 + R + 1)
    win = {b: (lo1, hi1, max(0, i2 - R), min(N2, i2 + R + 1))}
    if b == 0 and i2 + R >= N2 - 1:
        win[1] = (lo1, hi1, 0, min(N2, R + 1))
    if b == 1 and i2 - R <= 0:
        win[0] = (lo1, hi1, max(0, N2 - R - 1), N2)
    return win


def _crop(fields, win):
    return [fields[b][:, lo2:hi2, lo1:hi1] for b, (lo1, hi1, lo2, hi2) in sorted(win.items())]


def _local(win, b, i1, i2):
    lo1, _, lo2, _ = win[b]
    return sorted(win).index(b), i1 - lo1, i2 - lo2


def test_operator_at_full_size(full):
    """One application on a random field (FP32 rounding of the stencil terms ~1e-7 of their size;
    a smooth field would cancel those terms and measure only that cancellation)."""
    P, S, _, dt, prec = full
    u = W.random_state(P, seed=4)
    t = 0.11                                   # inside the Ricker pulse
    S.set_state(u, u, 0.0)
    r = S.apply(with_data=True, t=t)
    for (b, i1, i2) in SAMPLES:
        win = _window(b, i1, i2, 26)       # >= 27 nodes per direction (order-6 minimum)
        O = Oracle(W.config3(window=win))
        ref = O.unpack(O.apply(O.pack(_crop(u, win)), t))
        k, j1, j2 = _local(win, b, i1, i2)
        scale = max(np.abs(ref[k]).max(), 1e-30)
        err = np.abs(r[b][:, i2, i1] - ref[k][:, j2, j1]).max() / scale
        assert err < TOL[prec], ((b, i1, i2), err)


def test_steps_at_full_size(full):
    """Three leapfrog steps of a smooth field with the source on."""
    P, S, u, dt, prec = full
    nsteps = 3
    S.set_state(u, u, 0.0)
    S.step(nsteps, dt)
    _, cur = S.state()
    for (b, i1, i2) in SAMPLES[::2] + [(1, 2000, 1999)]:
        win = _window(b, i1, i2, 12 * (nsteps + 1) + 4)
        O = Oracle(W.config3(window=win))
        u0 = O.pack(_crop(u, win))
        _, un, _ = O.leapfrog(u0, u0, 0.0, dt, nsteps)
        ref = O.unpack(un)
        k, j1, j2 = _local(win, b, i1, i2)
        scale = np.abs(ref[k]).max()
        err = np.abs(cur[b][:, i2, i1] - ref[k][:, j2, j1]).max() / scale
        assert err < TOL[prec], ((b, i1, i2), err)
