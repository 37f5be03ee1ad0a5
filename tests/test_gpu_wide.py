"""GPU parity of the wide-stencil variant (sbp_grid_desc.stencil = SBP_STENCIL_WIDE: the flux and
divergence passes with the narrow scheme's SATs) against the oracle's wide operator: single
applications on random problems, leapfrog and RK4 runs with boundary data, body force, interfaces
and point sources, and the discrete energy."""
import dataclasses
import math

import numpy as np
import pytest

import workloads as W
from oracle.scheme import Oracle

pytestmark = pytest.mark.gpu

SIZES = {2: (23, 21), 4: (40, 33), 6: (45, 37)}
CASES = [
    (("robin",) * 4, False, False),
    (("displacement",) * 4, False, False),
    (("robin", "displacement", "displacement", "robin"), True, False),
    (("displacement", "robin", "robin", "displacement"), True, True),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _wide(P):
    return dataclasses.replace(P, stencil="wide")


def _relmax(a, b):
    return max(np.abs(x - y).max() for x, y in zip(a, b)) / max(np.abs(y).max() for y in b)


@pytest.mark.parametrize("order", (2, 4, 6))
@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec", ("fp64", "fp32"))
def test_wide_apply_random_problem(order, case, prec):
    from paper_2003_12811_gb300 import Solver
    kinds, two, rev = CASES[case]
    P = _wide(W.random_problem(kinds=kinds, n=SIZES[order], order=order, two_blocks=two, reversed_interface=rev))
    O = Oracle(P)
    u = W.random_state(P)
    ref = O.unpack(O.A @ O.pack(u))
    S = Solver(P, prec)
    S.set_state(u, u, 0.0)
    got = S.apply()
    S.close()
    assert _relmax(got, ref) < (1e-12 if prec == "fp64" else 2e-5)


@pytest.mark.parametrize("order", (2, 4, 6))
def test_wide_leapfrog_with_data_and_sources(order):
    from paper_2003_12811_gb300 import Solver
    N = {2: 21, 4: 26, 6: 33}[order]
    P = _wide(W.mms_problem(N, order, kinds=("robin", "displacement", "robin", "displacement"), two_blocks=True))
    P.sources = [W.PointSource(block=0, x_ref=(0.45, 0.6), direction=(0.6, -0.8), amplitude=0.3, alpha_p=3.0, t0=0.2),
                 W.PointSource(block=1, x_ref=(0.5, 1.0), direction=(0.0, 1.0), amplitude=0.2, alpha_p=4.0, t0=0.1)]
    O = Oracle(P)
    dt = O.suggest_dt(0.3)
    up = [P.exact(b, -dt) for b in P.blocks]
    uc = [P.exact(b, 0.0) for b in P.blocks]
    _, ref, _ = O.leapfrog(O.pack(up), O.pack(uc), 0.0, dt, 60)
    S = Solver(P, "fp64")
    S.set_state(up, uc, 0.0)
    S.step(60, dt)
    _, got = S.state()
    S.close()
    assert _relmax(got, O.unpack(ref)) < 1e-12


def test_wide_rk4_matches_oracle():
    from paper_2003_12811_gb300 import Solver
    P = _wide(W.mms_problem(26, 4, kinds=("robin", "displacement", "robin", "displacement"), two_blocks=True))
    O = Oracle(P)
    dt = O.suggest_dt(0.4)
    u0 = [P.exact(b, 0.0) for b in P.blocks]
    v0 = [np.stack([-W.MMS_W[L] * np.cos(W.MMS_K[L, 0] * b.X[0] + W.MMS_K[L, 1] * b.X[1]) for L in range(2)])
          for b in P.blocks]
    ur, vr, _ = O.rk4(O.pack(u0), O.pack(v0), 0.0, dt, 20)
    S = Solver(P, "fp64")
    S.sbp_set_state_rk4(u0, v0, 0.0)
    S.sbp_step_rk4(20, dt)
    ug, vg = S.state_rk4()
    S.close()
    assert _relmax(ug, O.unpack(ur)) < 1e-12 and _relmax(vg, O.unpack(vr)) < 1e-12


def test_wide_energy_matches_oracle_and_is_conserved():
    from paper_2003_12811_gb300 import Solver
    P = _wide(W.random_problem(kinds=("robin", "displacement", "displacement", "robin"), n=SIZES[4], order=4,
                               two_blocks=True))
    for b in P.blocks:
        for f in b.faces:
            f.g = None
    O = Oracle(P)
    dt = O.suggest_dt(0.3)
    u0 = W.smooth_state(P, seed=4, amplitude=0.1)
    S = Solver(P, "fp64")
    S.set_state(u0, u0, 0.0)
    E = []
    for _ in range(5):
        S.step(10, dt)
        E.append(S.energy(dt))
    up, uc = S.state()
    S.close()
    Eo = O.energy_leapfrog(O.pack(up), O.pack(uc), dt)
    assert abs(E[-1] - Eo) <= 1e-12 * abs(Eo)
    assert max(abs(e - E[0]) for e in E) <= 1e-11 * abs(E[0])


def test_wide_rejected_where_only_the_narrow_scheme_is_built():
    from paper_2003_12811_gb300 import Batch, SbpError, Solver
    P = _wide(W.shot_problem(61, 3))
    S = Solver(P, "fp32")
    B = Batch(6, 2)
    with pytest.raises(SbpError) as e:
        B.sbp_batch_add(S, 10, 1e-3)
    assert e.value.code == -1
    B.close()
    S.sbp_set_receivers([(0, 5, 60)])
    with pytest.raises(SbpError) as e:
        S.sbp_misfit_gradient(4, 1e-3, np.zeros((4, 1, 2)))
    assert e.value.code == -8
    S.close()
