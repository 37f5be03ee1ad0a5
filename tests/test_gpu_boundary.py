"""The C-ABI boundary beyond host arrays: the Voigt stiffness layout of sbp_set_material, and state
kept in caller-owned device buffers (torch tensors) through sbp_set_state_device /
sbp_get_field_device -- stream-ordered copies that must give bitwise the results of the host-array
path, with pointer, alignment and pitch checks."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

SBP_E_INVALID_ARG = -1


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _voigt_planes(Cfull):
    """Voigt planes C11 C12 C13 C22 C23 C33 of a tensor with minor symmetry (index 3 = (1,2))."""
    rep = {0: (0, 0), 1: (1, 1), 2: (0, 1)}
    ent = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))
    return np.stack([Cfull[rep[a] + rep[b]] for a, b in ent])


@pytest.mark.parametrize("prec", ("fp64", "fp32"))
def test_voigt_layout_equals_pair_layout(prec):
    from paper_2003_12811_gb300 import Solver
    from paper_2003_12811_gb300.binding import C_VOIGT6
    from paper_2003_12811_gb300.binding import C_PAIR10, pair10
    P, _ = W.config5(n=41, blob=True)            # tilted VTI stiffness: minor symmetry holds
    u = W.random_state(P, seed=2)
    S1, S2 = Solver(P, prec), Solver(P, prec)
    for b, blk in enumerate(P.blocks):
        V = _voigt_planes(blk.C)
        # the pair layout of the same Voigt entries (the rotated tensor's mirror entries agree
        # only to rounding, so both handles get the material from the one set of Voigt planes)
        full = np.zeros((3, 3) + V.shape[1:])
        for k, (i, j) in enumerate(((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))):
            full[i, j] = full[j, i] = V[k]
        S1.sbp_set_material(b, blk.rho, pair10(W.voigt_to_tensor(full)), C_PAIR10)
        S2.sbp_set_material(b, blk.rho, V, C_VOIGT6)
    for S in (S1, S2):
        S.set_state(u, u, 0.0)
    r1, r2 = S1.apply(), S2.apply()
    S1.close()
    S2.close()
    assert all(np.array_equal(a, b) for a, b in zip(r1, r2))


@pytest.mark.parametrize("prec", ("fp64", "fp32"))
def test_bad_layout_is_rejected(prec):
    from paper_2003_12811_gb300 import Solver, SbpError
    P, _ = W.config5(n=41)
    S = Solver(P, prec)
    blk = P.blocks[0]
    with pytest.raises(SbpError) as e:
        S.sbp_set_material(0, blk.rho, np.zeros((10, blk.N2, blk.N1)), 7)
    assert e.value.code == SBP_E_INVALID_ARG
    S.close()


def _to_device(fields, pitch, dtype):
    import torch
    out = []
    for u in fields:
        t = torch.zeros((2, u.shape[1], pitch), dtype=dtype, device="cuda")
        t[:, :, :u.shape[2]] = torch.from_numpy(u).to(dtype)
        out.append(t)
    return out


@pytest.mark.parametrize("prec", ("fp64", "fp32"))
def test_device_state_steps_bitwise_equal_to_host_path(prec):
    """State in torch tensors (a pitch of the caller's choosing), stepped through the C-ABI on a
    torch stream, read back into torch tensors: bitwise the host-array path's result."""
    import torch
    from paper_2003_12811_gb300 import Solver
    from paper_2003_12811_gb300.binding import FIELD_CUR, FIELD_PREV
    P = W.random_problem(kinds=("robin", "displacement", "robin", "displacement"), n=(45, 37), order=6,
                         two_blocks=True)
    P.sources.append(W.PointSource(block=1, x_ref=(0.4, 0.6), direction=(0.0, -1.0), amplitude=1.0,
                                   alpha_p=3.0, t0=0.2))
    tdt = torch.float64 if prec == "fp64" else torch.float32
    align = 2 if prec == "fp64" else 4                 # elements per 16 bytes
    u0 = W.smooth_state(P, seed=3, amplitude=0.1)
    u1 = W.smooth_state(P, seed=4, amplitude=0.1)
    # the host path rounds the FP64 host arrays to the handle precision; feed the device path the
    # same rounded values
    u0 = [np.asarray(x, dtype=np.float32).astype(np.float64) if prec == "fp32" else x for x in u0]
    u1 = [np.asarray(x, dtype=np.float32).astype(np.float64) if prec == "fp32" else x for x in u1]
    H = Solver(P, prec)
    dt = H.suggest_dt(0.3)
    H.set_state(u0, u1, 0.05)
    H.step(17, dt)
    ref_prev, ref_cur = H.state()
    H.close()

    D = Solver(P, prec)
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    pitches = [((blk.N1 + 11 + align - 1) // align) * align for blk in P.blocks]
    dprev = _to_device(u0, pitches[0], tdt)[:1] + _to_device(u0[1:], pitches[1], tdt)
    dcur = _to_device(u1, pitches[0], tdt)[:1] + _to_device(u1[1:], pitches[1], tdt)
    torch.cuda.synchronize()
    for b in range(len(P.blocks)):
        D.sbp_set_state_device(b, dprev[b].data_ptr(), dcur[b].data_ptr(), pitches[b], 0.05, sh)
    D.sbp_step(17, dt, sh)
    outs = []
    for b, blk in enumerate(P.blocks):
        op = torch.full((2, blk.N2, pitches[b]), float("nan"), dtype=tdt, device="cuda")
        oc = torch.full_like(op, float("nan"))
        D.sbp_get_field_device(b, FIELD_PREV, op.data_ptr(), pitches[b], sh)
        D.sbp_get_field_device(b, FIELD_CUR, oc.data_ptr(), pitches[b], sh)
        outs.append((op, oc))
    stream.synchronize()
    D.close()
    for b, blk in enumerate(P.blocks):
        op, oc = outs[b]
        assert np.array_equal(op[:, :, :blk.N1].double().cpu().numpy(), ref_prev[b])
        assert np.array_equal(oc[:, :, :blk.N1].double().cpu().numpy(), ref_cur[b])


@pytest.mark.parametrize("prec", ("fp64", "fp32"))
def test_device_state_rejects_bad_buffers(prec):
    import torch
    from paper_2003_12811_gb300 import Solver, SbpError
    from paper_2003_12811_gb300.binding import FIELD_CUR
    P = W.random_problem(kinds=("robin",) * 4, n=(45, 37), order=6)
    S = Solver(P, prec)
    blk = P.blocks[0]
    tdt = torch.float64 if prec == "fp64" else torch.float32
    es = 8 if prec == "fp64" else 4
    good = ((blk.N1 + 15) // 16) * 16
    buf = torch.zeros(2 * blk.N2 * good + 64, dtype=tdt, device="cuda")
    p0 = buf.data_ptr()
    host = torch.zeros(2 * blk.N2 * good, dtype=tdt)
    bad = [
        (p0 + es, good),                   # not 16-byte aligned
        (p0, blk.N1 - 1),                  # pitch below n1
        (p0, good + 1),                    # row pitch not a multiple of 16 bytes
        (host.data_ptr(), good),           # host memory
        (0, good),                         # null
    ]
    for ptr, pitch in bad:
        with pytest.raises(SbpError) as e:
            S.sbp_set_state_device(0, ptr, p0, pitch, 0.0)
        assert e.value.code == SBP_E_INVALID_ARG, (ptr - p0, pitch)
        with pytest.raises(SbpError) as e:
            S.sbp_get_field_device(0, FIELD_CUR, ptr, pitch)
        assert e.value.code == SBP_E_INVALID_ARG, (ptr - p0, pitch)
    S.sbp_set_state_device(0, p0, p0, good, 0.0)
    S.sbp_check()
    S.close()
