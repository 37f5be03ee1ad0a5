"""The persistent tile-queue step (sbp_batch_*): shots of different sizes and step counts served
together must give each shot's result as if it were served alone (bitwise: the per-node arithmetic
does not depend on the mix or on the work schedule), equal the plain sbp_step path within FP32
rounding, and match the FP64 oracle within the FP32 tolerance; admission checks."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.scheme import Oracle

pytestmark = pytest.mark.gpu

SIDES = (61, 97, 53, 128)
STEPS = (40, 26, 55, 12)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _relmax(a, b):
    return max(np.abs(x - y).max() for x, y in zip(a, b)) / max(np.abs(y).max() for y in b)


def _rell2(a, b):
    return math.sqrt(sum(np.sum((x - y) ** 2) for x, y in zip(a, b)) / sum(np.sum(y ** 2) for y in b))


def _serve(indices, ksteps=4, rows=0):
    """Run the shots `indices` together in one batch; returns {index: (u, dt)}."""
    import torch
    from paper_2003_12811_gb300 import Batch, Solver
    B = Batch(6, 8)
    if rows:
        B.sbp_batch_set_rows(rows)
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    solvers, slots, dts = {}, {}, {}
    for i in indices:
        P = W.shot_problem(SIDES[i], 900 + i, f_peak=8.0)
        S = Solver(P, "fp32")
        dts[i] = S.suggest_dt(0.3)
        z = [np.zeros((2, b.N2, b.N1)) for b in P.blocks]
        S.set_state(z, z, 0.0)
        solvers[i] = S
        slots[i] = B.sbp_batch_add(S, STEPS[i], dts[i])
    out = {}
    while slots:
        B.sbp_batch_step(ksteps, sh)
        rem = B.sbp_batch_poll(sh)
        for i, s in list(slots.items()):
            if rem[s] == 0:
                B.sbp_batch_remove(s, sh)
                _, u = solvers[i].state()
                assert solvers[i].sbp_get_time() == pytest.approx(STEPS[i] * dts[i], rel=1e-12)
                out[i] = (u, dts[i])
                solvers[i].close()
                del slots[i]
    B.close()
    return out


def test_mix_equals_alone_bitwise_and_equals_plain_steps():
    from paper_2003_12811_gb300 import Solver
    mix = _serve(range(len(SIDES)))
    for i in range(len(SIDES)):
        alone = _serve([i], ksteps=7, rows=32)        # another tick length and tile shape
        assert all(np.array_equal(a, b) for a, b in zip(mix[i][0], alone[i][0])), i
        P = W.shot_problem(SIDES[i], 900 + i, f_peak=8.0)
        S = Solver(P, "fp32")
        z = [np.zeros((2, b.N2, b.N1)) for b in P.blocks]
        S.set_state(z, z, 0.0)
        S.step(STEPS[i], mix[i][1])
        _, u = S.state()
        S.close()
        assert _relmax(mix[i][0], u) < 1e-5, (i, _relmax(mix[i][0], u))


def test_served_shot_matches_the_oracle():
    res = _serve([0, 2])
    for i in (0, 2):
        P = W.shot_problem(SIDES[i], 900 + i, f_peak=8.0)
        O = Oracle(P)
        z = O.pack([np.zeros((2, b.N2, b.N1)) for b in P.blocks])
        _, u, _ = O.leapfrog(z, z, 0.0, res[i][1], STEPS[i])
        ref = O.unpack(u)
        assert _rell2(res[i][0], ref) < 1e-4, (i, _rell2(res[i][0], ref))
        assert _relmax(res[i][0], ref) < 1e-3, (i, _relmax(res[i][0], ref))


def test_admission_checks():
    from paper_2003_12811_gb300 import Batch, SbpError, Solver
    B = Batch(6, 1)
    P = W.shot_problem(61, 5)
    S64 = Solver(P, "fp64")
    with pytest.raises(SbpError) as e:
        B.sbp_batch_add(S64, 10, 1e-3)
    assert e.value.code == -1
    S64.close()
    Q = W.random_problem(kinds=("robin",) * 4, n=(45, 37), order=6, two_blocks=True)
    SQ = Solver(Q, "fp32")
    with pytest.raises(SbpError) as e:
        B.sbp_batch_add(SQ, 10, 1e-3)
    assert e.value.code == -1
    SQ.close()
    S1, S2 = Solver(P, "fp32"), Solver(P, "fp32")
    z = [np.zeros((2, b.N2, b.N1)) for b in P.blocks]
    S1.set_state(z, z, 0.0)
    S2.set_state(z, z, 0.0)
    B.sbp_batch_add(S1, 4, 1e-3)
    with pytest.raises(SbpError) as e:
        B.sbp_batch_add(S2, 4, 1e-3)                 # batch full
    assert e.value.code == -8
    B.close()
    S1.close()
    S2.close()


def test_batch_engine_serves_requests():
    """The batch serving engine on a few requests arriving together and later: every result equals
    the shot served alone."""
    from paper_2003_12811_gb300.serve import BatchServingEngine, GpuBatchBackend, Request
    probs = [W.shot_problem(s, 900 + i, f_peak=8.0) for i, s in enumerate(SIDES)]
    reqs = [Request(rid=i, arrival=0.02 * i, problem=p, nsteps=n) for i, (p, n) in enumerate(zip(probs, STEPS))]
    be = GpuBatchBackend(max_shots=4)
    eng = BatchServingEngine(1 << 40, backend=be, tick_steps=8, max_active=4)
    res = eng.run(reqs)
    be.close()
    alone = {}
    for i in range(len(SIDES)):
        alone.update(_serve([i]))
    for r in res:
        assert all(np.array_equal(a, b) for a, b in zip(r.fields, alone[r.rid][0])), r.rid
