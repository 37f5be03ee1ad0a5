"""FP32 leapfrog over many small steps: the FP32 path keeps the increment d^n = u^n - u^{n-1} as a
field of its own (d^{n+1} = d^n + dt^2 w r, u^{n+1} = u^n + d^{n+1}), so the acceleration term
dt^2 w r -- of the size of half an ulp of u^n when dt is small against h -- is added to a number of
the size of d^n and keeps its digits.  The two-level form 2 u^n - u^{n-1} + dt^2 w r rounds it
against u^n instead; its rounding errors then act as velocity errors and grow like N^(3/2) eps
(a few 1e-3 relative after 1500 steps here).  In increment form the error stays at the level of
single-step rounding: the bar is 2e-5 relative L2 against the FP64 oracle."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.scheme import Oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _rell2(a, b):
    return math.sqrt(sum(np.sum((x - y) ** 2) for x, y in zip(a, b)) / sum(np.sum(y ** 2) for y in b))


@pytest.mark.parametrize("nsteps", (1500,))
def test_fp32_small_steps_config2_geometry(nsteps):
    """Config 2 geometry, material and manufactured data on 2 x 2 blocks of 41^2 (order 6), at a
    tenth of the CFL step (the ratio dt / h of config 2 at full size), against the oracle."""
    from paper_2003_12811_gb300 import Solver
    P = W.config2(n=41, order=6)
    O = Oracle(P)
    dt = O.suggest_dt(0.25) / 10
    up = [P.exact(b, -dt) for b in P.blocks]
    uc = [P.exact(b, 0.0) for b in P.blocks]
    S = Solver(P, "fp32")
    S.set_state(up, uc, 0.0)
    S.step(nsteps, dt)
    _, gc = S.state()
    S.close()
    _, rc, _ = O.leapfrog(O.pack(up), O.pack(uc), 0.0, dt, nsteps)
    err = _rell2(gc, O.unpack(rc))
    assert err < 2e-5, err


def test_increment_survives_device_state_and_rk4():
    """The increment is re-formed whenever the two levels are written by something other than a
    leapfrog step: after sbp_set_state_device and after RK4 steps, leapfrog steps continue exactly
    as from sbp_set_state with the same (FP32-representable) levels."""
    import torch
    from paper_2003_12811_gb300 import Solver
    P = W.random_problem(kinds=("robin", "displacement", "robin", "displacement"), n=(45, 37), order=6,
                         two_blocks=True)
    u0 = [np.asarray(x, dtype=np.float32).astype(np.float64) for x in W.smooth_state(P, seed=3, amplitude=0.1)]
    u1 = [np.asarray(x, dtype=np.float32).astype(np.float64) for x in W.smooth_state(P, seed=4, amplitude=0.1)]
    A = Solver(P, "fp32")
    dt = A.suggest_dt(0.3)
    A.set_state(u0, u1, 0.0)
    A.step(9, dt)
    ref = A.state()
    A.close()
    # RK4 steps first, then the same levels set through the device path
    B = Solver(P, "fp32")
    z = [np.zeros((2, b.N2, b.N1)) for b in P.blocks]
    B.sbp_set_state_rk4(z, u1, 0.0)
    B.sbp_step_rk4(2, dt, torch.cuda.current_stream().cuda_stream)
    pitch = lambda n1: (n1 + 3) // 4 * 4
    dev = []
    for b, blk in enumerate(P.blocks):
        pp = torch.zeros((2, blk.N2, pitch(blk.N1)), dtype=torch.float32, device="cuda")
        pc = torch.zeros_like(pp)
        pp[:, :, :blk.N1] = torch.from_numpy(u0[b]).float()
        pc[:, :, :blk.N1] = torch.from_numpy(u1[b]).float()
        dev.append((pp, pc))
    torch.cuda.synchronize()
    sh = torch.cuda.current_stream().cuda_stream
    for b, blk in enumerate(P.blocks):
        B.sbp_set_state_device(b, dev[b][0].data_ptr(), dev[b][1].data_ptr(), pitch(blk.N1), 0.0, sh)
    B.sbp_step(9, dt, sh)
    got = B.state()
    B.close()
    for x, y in zip(got[0] + got[1], ref[0] + ref[1]):
        assert np.array_equal(x, y)
