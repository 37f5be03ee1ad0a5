"""Error reporting of device-side failures (no GPU fault is provoked).

A bounded wait that runs out inside a kernel sets a bit in the handle's error word; the next call
that checks the word returns SBP_E_TIMEOUT and clears it.  The probe waits on an mbarrier that
nothing arrives at and issues no copy, so nothing is left in flight when it gives up."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

SBP_E_INVALID_ARG, SBP_E_TIMEOUT = -1, -6


@pytest.fixture(scope="module")
def solver():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_12811_gb300 import Solver
    P = W.random_problem(kinds=("robin", "displacement", "robin", "displacement"), n=(40, 33), order=4)
    S = Solver(P, "fp32")
    u = W.random_state(P)
    S.set_state(u, u, 0.0)
    yield P, S
    S.close()


def test_timeout_is_reported_once_and_cleared(solver):
    from paper_2003_12811_gb300 import SbpError
    P, S = solver
    ref = S.apply()
    S.sbp_check()                                   # nothing recorded so far
    S.sbp_debug_wait_probe(256)
    with pytest.raises(SbpError) as e:
        S.sbp_check()
    assert e.value.code == SBP_E_TIMEOUT
    S.sbp_check()                                   # the report cleared the word
    got = S.apply()                                 # the context and the handle stay usable
    assert max(np.abs(a - b).max() for a, b in zip(got, ref)) == 0.0


def test_timeout_reported_by_the_next_checking_call(solver):
    from paper_2003_12811_gb300 import SbpError
    P, S = solver
    S.sbp_debug_wait_probe(64)
    with pytest.raises(SbpError) as e:
        S.apply()                                   # sbp_apply checks the word after its kernels
    assert e.value.code == SBP_E_TIMEOUT
    S.apply()


@pytest.mark.parametrize("polls", (0, -3, (1 << 20) + 1))
def test_probe_rejects_bad_poll_counts(solver, polls):
    from paper_2003_12811_gb300 import SbpError
    P, S = solver
    with pytest.raises(SbpError) as e:
        S.sbp_debug_wait_probe(polls)
    assert e.value.code == SBP_E_INVALID_ARG
