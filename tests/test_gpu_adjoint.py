"""Misfit gradient on the GPU (sbp_set_receivers, sbp_record, sbp_misfit_gradient) against the
oracle's explicit-transpose adjoint: receiver traces, misfit, dPhi/drho at every node and dPhi/dC at
sampled nodes (corners, face nodes of every kind, interface nodes on both sides, closure depths,
interior); checkpoint-interval invariance; the state left behind."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as AD
from oracle.scheme import Oracle

pytestmark = pytest.mark.gpu

SIZES = {2: (13, 11), 4: (21, 19), 6: (29, 27)}
NSTEPS = 40


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _setup(order, seed=5, nsteps=NSTEPS):
    n = SIZES[order]
    kinds = ("displacement", "robin", "robin", "displacement")
    src = [W.PointSource(block=0, x_ref=(0.45, 0.55), direction=(0.3, -1.0), amplitude=1.0, alpha_p=3.0, t0=0.3)]
    P = W.random_problem(kinds=kinds, n=n, order=order, seed=seed, two_blocks=True)
    P.sources = src
    Q = W.random_problem(kinds=kinds, n=n, order=order, seed=seed + 1, two_blocks=True)
    Q.sources = src
    dt = Oracle(P).suggest_dt(0.5)
    u0 = W.smooth_state(P, seed=1, amplitude=0.1)
    rec = [(b, i1, i2) for b in (0, 1) for i1 in range(1, n[0], 3) for i2 in range(2, n[1], 4)]
    rec = sorted(set(rec) | {(0, 0, 0), (1, n[0] - 1, n[1] - 1)})
    oq = Oracle(Q)
    lv, _ = AD.forward(oq, u0, u0, 0.0, dt, nsteps)
    obs = AD.traces(oq, lv, rec)
    return P, u0, dt, rec, obs


def _params(order):
    n1, n2 = SIZES[order]
    out = []
    for P in range(10):
        out += [(0, P, 0, 0), (1, P, n1 - 1, n2 - 1)]                    # corners
    out += [(0, 4, n1 - 1, 3), (1, 9, 0, 5), (0, 3, n1 - 1, n2 // 2), (1, 1, 0, n2 // 2)]   # interface, both sides
    out += [(0, 2, 3, n2 - 1), (1, 5, n1 // 2, 0), (0, 7, 0, n2 // 2), (1, 8, n1 - 1, 4)]  # displacement / Robin faces
    out += [(0, 5, 2, 1), (1, 6, 4, n2 - 3), (0, 0, n1 // 2, 5)]         # closure depths
    out += [(1, 7, n1 // 2, n2 // 2), (0, 9, n1 // 2 + 1, n2 // 2)]     # interior
    return out


def _solver(P, prec, u0, rec):
    from paper_2003_12811_gb300 import Solver
    S = Solver(P, prec)
    S.set_state(u0, u0, 0.0)
    S.sbp_set_receivers(rec)
    return S


@pytest.mark.parametrize("order", (2, 4, 6))
def test_record_matches_oracle(order):
    P, u0, dt, rec, _ = _setup(order)
    S = _solver(P, "fp64", u0, rec)
    tr = S.sbp_record(NSTEPS, dt)
    S.close()
    orc = Oracle(P)
    lv, _ = AD.forward(orc, u0, u0, 0.0, dt, NSTEPS)
    ref = AD.traces(orc, lv, rec)
    assert np.max(np.abs(tr - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("order", (2, 4, 6))
def test_gradient_matches_oracle_fp64(order):
    P, u0, dt, rec, obs = _setup(order)
    params = _params(order)
    ref = AD.gradient(P, u0, u0, 0.0, dt, NSTEPS, rec, obs, params)
    S = _solver(P, "fp64", u0, rec)
    phi, gr, gc = S.sbp_misfit_gradient(NSTEPS, dt, obs, checkpoint_every=7)
    S.close()
    assert phi == pytest.approx(ref["misfit"], rel=1e-12)
    for b in range(2):
        scale = np.max(np.abs(ref["grad_rho"][b]))
        assert np.max(np.abs(gr[b] - ref["grad_rho"][b])) <= 1e-12 * scale, b
    got = np.array([gc[b][Pp, i2, i1] for (b, Pp, i1, i2) in params])
    scale = np.max(np.abs(ref["grad_C"]))
    err = np.abs(got - ref["grad_C"])
    assert np.all(err <= 1e-12 * scale), [(params[k], got[k], ref["grad_C"][k]) for k in np.argsort(-err)[:5]]


@pytest.mark.parametrize("order", (4, 6))
def test_gradient_fp32_close_to_oracle(order):
    P, u0, dt, rec, obs = _setup(order)
    params = _params(order)
    ref = AD.gradient(P, u0, u0, 0.0, dt, NSTEPS, rec, obs, params)
    S = _solver(P, "fp32", u0, rec)
    phi, gr, gc = S.sbp_misfit_gradient(NSTEPS, dt, obs)
    S.close()
    assert phi == pytest.approx(ref["misfit"], rel=1e-4)
    for b in range(2):
        scale = np.max(np.abs(ref["grad_rho"][b]))
        e = np.max(np.abs(gr[b] - ref["grad_rho"][b])) / scale
        assert e <= 2e-3, (b, e)
    got = np.array([gc[b][Pp, i2, i1] for (b, Pp, i1, i2) in params])
    e = np.max(np.abs(got - ref["grad_C"])) / np.max(np.abs(ref["grad_C"]))
    assert e <= 2e-3, e


@pytest.mark.parametrize("prec,tol", (("fp64", 1e-12), ("fp32", 1e-5)))
def test_checkpoint_interval_invariance_and_final_state(prec, tol):
    """The recomputed levels are bitwise those of the forward pass, so the checkpoint interval only
    changes how the gradient terms are grouped into per-segment sums (rounding); a repeated call is
    bitwise identical; the state left behind is the one sbp_step leaves."""
    P, u0, dt, rec, obs = _setup(6)
    res = []
    for K in (1, 6, 0, NSTEPS, 6):
        S = _solver(P, prec, u0, rec)
        res.append(S.sbp_misfit_gradient(NSTEPS, dt, obs, checkpoint_every=K))
        st = S.state()
        S.close()
        A = _solver(P, prec, u0, rec)
        A.step(NSTEPS, dt)
        ref = A.state()
        A.close()
        for x, y in zip(st[0] + st[1], ref[0] + ref[1]):
            assert np.array_equal(x, y)
    for phi, gr, gc in res[1:]:
        assert phi == res[0][0]                      # the misfit does not depend on the segments
        for b in range(2):
            for got, want in ((gr[b], res[0][1][b]), (gc[b], res[0][2][b])):
                assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    for x, y in zip(res[1][1] + res[1][2], res[4][1] + res[4][2]):   # same interval twice: bitwise
        assert np.array_equal(x, y)


def test_gradient_rejects_displacement_data():
    from paper_2003_12811_gb300 import Solver
    from paper_2003_12811_gb300.binding import SbpError
    P = W.mms_problem(20, 4)
    S = Solver(P, "fp64")
    z = [np.zeros((2, b.N2, b.N1)) for b in P.blocks]
    S.set_state(z, z, 0.0)
    S.sbp_set_receivers([(0, 3, 3)])
    with pytest.raises(SbpError):
        S.sbp_misfit_gradient(4, 1e-3, np.zeros((4, 1, 2)))
    with pytest.raises(SbpError):
        S.sbp_set_receivers([(0, 3, 3), (0, 3, 3)])
    S.close()


def test_misfit_gradient_workload_small():
    """The misfit-gradient workload at n = 41: observations from the model with the inclusion,
    gradient at the background model, checked against the oracle at sampled nodes."""
    Pb, rec = W.config5(n=41, nrec=8, blob=False)
    Pt, _ = W.config5(n=41, nrec=8, blob=True)
    z = [np.zeros((2, 41, 41))]
    nsteps = 60
    dt = Oracle(Pb).suggest_dt(0.5)
    ot = Oracle(Pt)
    lv, _ = AD.forward(ot, z, z, 0.0, dt, nsteps)
    obs = AD.traces(ot, lv, rec)
    params = [(0, 0, 20, 40), (0, 9, 20, 30), (0, 5, 0, 0), (0, 2, 40, 20), (0, 7, 20, 38)]
    ref = AD.gradient(Pb, z, z, 0.0, dt, nsteps, rec, obs, params)
    S = _solver(Pb, "fp64", z, rec)
    phi, gr, gc = S.sbp_misfit_gradient(nsteps, dt, obs)
    S.close()
    assert ref["misfit"] > 0 and phi == pytest.approx(ref["misfit"], rel=1e-12)
    # 60 steps; the density term sums psi_n . (u_{n+1} - 2 u_n + u_{n-1}), a second difference in
    # time that cancels about two digits of the FP64 levels (measured: 2.4e-12 of the largest entry)
    scale = np.max(np.abs(ref["grad_rho"][0]))
    assert np.max(np.abs(gr[0] - ref["grad_rho"][0])) <= 1e-11 * scale
    got = np.array([gc[0][Pp, i2, i1] for (_, Pp, i1, i2) in params])
    # the scale is the largest of five sampled entries, not of the field (measured: 4.1e-12 of it)
    assert np.max(np.abs(got - ref["grad_C"])) <= 1e-11 * np.max(np.abs(ref["grad_C"]))


def test_autograd_bridge_and_gpu_central_differences():
    """torch.autograd through sbp_misfit_gradient returns the library's gradient, and that gradient
    agrees with central differences of the GPU misfit itself (FP64)."""
    import torch
    from paper_2003_12811_gb300.autograd import misfit, pair_planes
    P, u0, dt, rec, obs = _setup(4, nsteps=30)
    S = _solver(P, "fp64", u0, rec)
    rho = [torch.tensor(b.rho, dtype=torch.float64, requires_grad=True) for b in P.blocks]
    C = [pair_planes(torch.tensor(b.C, dtype=torch.float64)).clone().requires_grad_(True) for b in P.blocks]
    phi = misfit(S, rho, C, u0, u0, 0.0, 30, dt, obs)
    phi.backward()
    S.set_state(u0, u0, 0.0)
    phi2, gr, gc = S.sbp_misfit_gradient(30, dt, obs)
    assert float(phi) == phi2
    for b in range(2):
        assert np.array_equal(rho[b].grad.numpy(), gr[b]) and np.array_equal(C[b].grad.numpy(), gc[b])

    def phi_at(rr, cc):
        with torch.no_grad():
            return float(misfit(S, rr, cc, u0, u0, 0.0, 30, dt, obs))

    for (b, i1, i2) in [(0, 3, 4), (1, 0, 7), (0, 20, 18)]:
        eps = 1e-6
        rp = [r.detach().clone() for r in rho]
        rm = [r.detach().clone() for r in rho]
        rp[b][i2, i1] += eps
        rm[b][i2, i1] -= eps
        Cd = [c.detach() for c in C]
        fd = (phi_at(rp, Cd) - phi_at(rm, Cd)) / (2 * eps)
        assert abs(fd - gr[b][i2, i1]) <= 1e-5 * abs(fd) + 100 * np.finfo(float).eps * phi2 / eps
    for (b, Pp, i1, i2) in [(0, 0, 5, 5), (1, 9, 20, 3), (0, 4, 0, 0)]:
        eps = 1e-5
        cp = [c.detach().clone() for c in C]
        cm = [c.detach().clone() for c in C]
        cp[b][Pp, i2, i1] += eps
        cm[b][Pp, i2, i1] -= eps
        Rd = [r.detach() for r in rho]
        fd = (phi_at(Rd, cp) - phi_at(Rd, cm)) / (2 * eps)
        assert abs(fd - gc[b][Pp, i2, i1]) <= 1e-5 * abs(fd) + 100 * np.finfo(float).eps * phi2 / eps
    S.close()


def test_voigt_gradient_matches_oracle_fp64():
    """sbp_misfit_gradient with the Voigt layout: dPhi/dC for the six Voigt entries at sampled
    nodes against the oracle's Voigt gradient (the derivative along the Voigt unit tensors)."""
    from paper_2003_12811_gb300.binding import C_VOIGT6
    order = 4
    P, u0, dt, rec, obs = _setup(order)
    n1, n2 = SIZES[order]
    nodes = [(0, 0, 0), (1, n1 - 1, n2 - 1), (0, n1 - 1, 3), (1, 0, 5), (0, 2, 1), (1, n1 // 2, n2 // 2)]
    params = [(b, ("voigt", V), i1, i2) for (b, i1, i2) in nodes for V in range(6)]
    ref = AD.gradient(P, u0, u0, 0.0, dt, NSTEPS, rec, obs, params)
    S = _solver(P, "fp64", u0, rec)
    phi, gr, gc = S.sbp_misfit_gradient(NSTEPS, dt, obs, checkpoint_every=9, layout=C_VOIGT6)
    S.close()
    assert phi == pytest.approx(ref["misfit"], rel=1e-12)
    assert gc[0].shape == (6, n2, n1)
    got = np.array([gc[b][V, i2, i1] for (b, (_, V), i1, i2) in params])
    scale = np.max(np.abs(ref["grad_C"]))
    assert np.all(np.abs(got - ref["grad_C"]) <= 1e-12 * scale)
