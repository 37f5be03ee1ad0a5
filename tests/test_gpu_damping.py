"""The velocity-dependent terms on the GPU against the oracle: the dissipative Robin term (remark of
Sec. 5.1; leapfrog with the centred velocity, a 2 x 2 solve per face node) and the super-grid layer
dissipation (Sec. 7.3; leapfrog with the backward velocity), in leapfrog and RK4, for the narrow
and the wide operator; and the energy the Robin damping removes per step."""
import dataclasses
import math

import numpy as np
import pytest

import workloads as W
from oracle.scheme import Oracle

pytestmark = pytest.mark.gpu

NS = {2: (23, 21), 4: (40, 33), 6: (45, 37)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _problem(order, stencil="narrow", seed=3):
    P = W.random_problem(kinds=("robin", "displacement", "robin", "robin"), n=NS[order], order=order,
                         two_blocks=True, seed=seed)
    rng = np.random.default_rng(seed)
    for b in P.blocks:
        h1, h2 = b.spacing
        for f, face in enumerate(b.faces):
            if face.kind == "robin":
                nf = b.N2 if f < 2 else b.N1
                a, c = 0.5 + rng.random(nf), 0.5 + rng.random(nf)
                face.V = np.stack([a, 0.4 * np.sqrt(a * c) * (2 * rng.random(nf) - 1), c])
        x1, x2 = W.ref_grid(b.N1, b.N2)
        b.sponge = (0.5 * b.rho * 3.0 * h1 * h2 / (32 * min(h1, h2))) * np.clip((x1 - 0.6) / 0.4, 0, 1) ** 2
    P.sources = [W.PointSource(block=1, x_ref=(0.5, 0.5), direction=(0.6, 0.8), amplitude=0.5, alpha_p=3.0, t0=0.2)]
    return dataclasses.replace(P, stencil=stencil)


def _relmax(a, b):
    return max(np.abs(x - y).max() for x, y in zip(a, b)) / max(np.abs(y).max() for y in b)


def _rell2(a, b):
    return math.sqrt(sum(np.sum((x - y) ** 2) for x, y in zip(a, b)) / sum(np.sum(y ** 2) for y in b))


@pytest.mark.parametrize("order", (2, 4, 6))
@pytest.mark.parametrize("stencil", ("narrow", "wide"))
def test_damped_leapfrog_matches_oracle(order, stencil):
    from paper_2003_12811_gb300 import Solver
    P = _problem(order, stencil)
    O = Oracle(P)
    dt = O.suggest_dt(0.3)
    up = W.smooth_state(P, seed=5, amplitude=0.1)
    uc = [a + dt * b for a, b in zip(up, W.smooth_state(P, seed=6, amplitude=0.1))]
    _, ref, _ = O.leapfrog(O.pack(up), O.pack(uc), 0.0, dt, 40)
    ref = O.unpack(ref)
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-4)):
        S = Solver(P, prec)
        S.set_state(up, uc, 0.0)
        S.step(40, dt)
        _, got = S.state()
        S.close()
        err = _relmax(got, ref) if prec == "fp64" else _rell2(got, ref)
        assert err < tol, (prec, err)


@pytest.mark.parametrize("order", (2, 6))
def test_damped_rk4_matches_oracle(order):
    from paper_2003_12811_gb300 import Solver
    P = _problem(order)
    O = Oracle(P)
    dt = O.suggest_dt(0.4)
    u0 = W.smooth_state(P, seed=5, amplitude=0.1)
    v0 = W.smooth_state(P, seed=6, amplitude=0.1)
    ur, vr, _ = O.rk4(O.pack(u0), O.pack(v0), 0.0, dt, 20)
    S = Solver(P, "fp64")
    S.sbp_set_state_rk4(u0, v0, 0.0)
    S.sbp_step_rk4(20, dt)
    ug, vg = S.state_rk4()
    S.close()
    assert _relmax(ug, O.unpack(ur)) < 1e-12 and _relmax(vg, O.unpack(vr)) < 1e-12


def test_robin_damping_removes_the_predicted_energy():
    """GPU leapfrog with Robin damping only (homogeneous data): each step's energy loss (sbp_energy)
    equals |u^{n+1} - u^{n-1}|^2 / (4 dt) in the oracle's damping norm H Bv."""
    from paper_2003_12811_gb300 import Solver
    P = _problem(4)
    P.sources = []
    for b in P.blocks:
        b.sponge = None
    O = Oracle(P)
    dt = O.suggest_dt(0.3)
    HB = O.Bv.multiply(O.hvec[:, None]).tocsr()
    up = W.smooth_state(P, seed=5, amplitude=0.1)
    uc = [a + dt * b for a, b in zip(up, W.smooth_state(P, seed=6, amplitude=0.1))]
    S = Solver(P, "fp64")
    S.set_state(up, uc, 0.0)
    E_prev = S.energy(dt)
    prev = O.pack(up)
    for n in range(10):
        S.step(1, dt)
        E = S.energy(dt)
        a, b = S.state()
        d = O.pack(b) - prev
        loss = float(d @ (HB @ d)) / (4 * dt)
        assert abs((E_prev - E) - loss) <= 1e-10 * abs(E_prev), (n, E_prev - E, loss)
        prev = O.pack(a)
        E_prev = E
    S.close()
