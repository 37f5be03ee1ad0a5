"""sbp_apply_noalloc: the operator application for callers that cannot allocate device memory
(code held to a fixed memory pool that it may not grow, or a real-time loop that may not pay for
cudaMalloc's implicit synchronisation).

It must give the same result as sbp_apply (the allocating path) on the same handle, on two calls
in a row (the fixed scratch array is shared and reused between calls), and match the FP64 oracle:
without data, and with boundary data, body force and a point source at a time t > 0.  This file is
collected last on purpose."""
import numpy as np
import pytest

import workloads as W
from oracle.scheme import Oracle

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


def _relmax(a, b):
    return max(np.abs(x - y).max() for x, y in zip(a, b)) / max(np.abs(y).max() for y in b)


def _problem(with_data):
    if not with_data:
        return W.random_problem(kinds=("robin", "displacement", "displacement", "robin"), n=(45, 37), order=6,
                                two_blocks=True)
    # traction and displacement data, an interface, the manufactured body force and a Ricker point force
    P = W.mms_problem(33, 6, kinds=("robin", "displacement", "robin", "displacement"), two_blocks=True)
    P.sources.append(W.PointSource(block=1, x_ref=(0.37, 0.58), direction=(0.6, -0.8), amplitude=0.5,
                                   alpha_p=3.0, t0=0.3))
    return P


@pytest.mark.parametrize("with_data", (False, True))
@pytest.mark.parametrize("prec,tol", (("fp64", 1e-12), ("fp32", 2e-5)))
def test_apply_noalloc_matches_apply_and_oracle_twice(prec, tol, with_data):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_12811_gb300 import Solver

    P = _problem(with_data)
    O = Oracle(P)
    S = Solver(P, prec)
    pitch = lambda n1: (n1 + 31) // 32 * 32
    dtype = np.float64 if prec == "fp64" else np.float32
    shapes = [(b.N2, b.N1) for b in P.blocks]
    rng = np.random.default_rng(7)
    for call in range(2):
        t = 0.21 + 0.07 * call if with_data else 0.0
        if with_data:
            # a rough field (the FP32 bar assumes stencil terms that do not cancel), plus the data terms
            u = [P.exact(b, t) + 0.5 * rng.standard_normal((2, n2, n1)) for b, (n2, n1) in zip(P.blocks, shapes)]
        else:
            u = [rng.standard_normal((2, n2, n1)) for (n2, n1) in shapes]
        S.set_state(u, u, 0.0)
        ref = S.apply(with_data=with_data, t=t)
        u_dev = torch.from_numpy(_pitched(u, pitch, dtype)).cuda()
        r_dev = torch.full_like(u_dev, float("nan"))
        torch.cuda.synchronize()
        S.sbp_apply_noalloc(u_dev.data_ptr(), r_dev.data_ptr(), with_data, t, torch.cuda.current_stream().cuda_stream)
        got = _unpitched(r_dev.cpu().numpy(), shapes, pitch)
        # the same operator as the allocating path ...
        assert _relmax(got, ref) < tol, (call, _relmax(got, ref))
        # ... and as the oracle (FP32: the u planes are rounded to FP32 on both GPU paths)
        u_in = [np.asarray(x, dtype=dtype).astype(np.float64) for x in u]
        oref = O.unpack(O.apply(O.pack(u_in), t) if with_data else O.A @ O.pack(u_in))
        assert _relmax(got, oref) < tol, (call, _relmax(got, oref))
    S.close()
