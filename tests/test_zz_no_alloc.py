"""sbp_apply_noalloc: the operator application for callers that cannot allocate device memory.

It must give the same result as sbp_apply (the allocating path) on the same handle, on two calls
in a row (the fixed scratch array is shared and reused between calls).  This file is collected
last on purpose."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _pitched(fields, pitch, dtype):
    """Pack per-block (2, n2, n1) arrays into the library layout (2 planes of n2 x pitch per block)."""
    out = []
    for u in fields:
        p = np.zeros((2, u.shape[1], pitch(u.shape[2])), dtype=dtype)
        p[:, :, :u.shape[2]] = u
        out.append(p.ravel())
    return np.concatenate(out)


def _unpitched(flat, shapes, pitch):
    out, off = [], 0
    for (n2, n1) in shapes:
        P = pitch(n1)
        a = flat[off:off + 2 * n2 * P].reshape(2, n2, P)[:, :, :n1]
        out.append(np.array(a, dtype=np.float64))
        off += 2 * n2 * P
    return out


@pytest.mark.parametrize("prec,tol", (("fp64", 1e-12), ("fp32", 2e-5)))
def test_apply_noalloc_matches_apply_twice(prec, tol):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_12811_gb300 import Solver

    P = W.random_problem(kinds=("robin", "displacement", "displacement", "robin"), n=(45, 37), order=6,
                         two_blocks=True)
    S = Solver(P, prec)
    pitch = lambda n1: (n1 + 31) // 32 * 32
    dtype = np.float64 if prec == "fp64" else np.float32
    shapes = [(b.N2, b.N1) for b in P.blocks]
    rng = np.random.default_rng(7)
    for call in range(2):
        u = [rng.standard_normal((2, n2, n1)) for (n2, n1) in shapes]
        S.set_state(u, u, 0.0)
        ref = S.apply()
        u_dev = torch.from_numpy(_pitched(u, pitch, dtype)).cuda()
        r_dev = torch.full_like(u_dev, float("nan"))
        torch.cuda.synchronize()
        S.sbp_apply_noalloc(u_dev.data_ptr(), r_dev.data_ptr(), False, 0.0, torch.cuda.current_stream().cuda_stream)
        got = _unpitched(r_dev.cpu().numpy(), shapes, pitch)
        err = max(np.abs(g - r).max() for g, r in zip(got, ref)) / max(np.abs(r).max() for r in ref)
        assert err < tol, (call, err)
    S.close()
