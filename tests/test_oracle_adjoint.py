"""Pins of the oracle's discrete adjoint and misfit gradient (Sec. 5.2 remark on adjoint reuse,
Theorems 3 and 5) against finite differences of the misfit, the self-adjoint form of the adjoint
recursion, and the zero-residual case."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as AD
from oracle.scheme import Oracle

SIZES = {2: (12, 11), 4: (20, 19), 6: (28, 27)}
NSTEPS = 40


def _setup(order, seed=5):
    """Two curvilinear blocks with an interface, displacement/Robin faces, a point source, a
    smooth initial state, receivers on a coarse lattice of both blocks, and observations made by a
    second random material."""
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
    oq = Oracle(Q)
    lv, _ = AD.forward(oq, u0, u0, 0.0, dt, NSTEPS)
    obs = AD.traces(oq, lv, rec)
    return P, u0, dt, rec, obs


@pytest.mark.parametrize("order", (2, 4, 6))
def test_gradient_matches_central_differences(order):
    P, u0, dt, rec, obs = _setup(order)
    n1, n2 = SIZES[order]
    # corner, interface (both sides), displacement-face node, closure-depth node, interior node
    cparams = [(0, 0, 0, 0), (0, 4, n1 - 1, 3), (1, 9, 0, 5), (0, 2, 3, n2 - 1), (0, 5, 2, 1), (1, 7, 5, 5)]
    rparams = [(0, 0, 0), (0, n1 - 1, 4), (1, 6, 6), (0, 3, n2 - 1)]
    G = AD.gradient(P, u0, u0, 0.0, dt, NSTEPS, rec, obs, cparams)
    phi = G["misfit"]
    assert phi > 0

    def fd(kind, b, i1, i2, eps):
        fp = AD.misfit_of(AD.perturbed(P, b, kind, i1, i2, eps), u0, u0, 0.0, dt, NSTEPS, rec, obs)
        fm = AD.misfit_of(AD.perturbed(P, b, kind, i1, i2, -eps), u0, u0, 0.0, dt, NSTEPS, rec, obs)
        return (fp - fm) / (2 * eps)

    # central differences: truncation O(eps^2) is far below the rounding floor ~ eps_mach * Phi / eps
    for k, (b, Pp, i1, i2) in enumerate(cparams):
        eps = 1e-5
        f = fd(Pp, b, i1, i2, eps)
        floor = 100 * np.finfo(float).eps * phi / eps
        assert abs(G["grad_C"][k] - f) <= 1e-5 * abs(f) + floor, (b, Pp, i1, i2, G["grad_C"][k], f)
    for (b, i1, i2) in rparams:
        eps = 1e-6
        f = fd("rho", b, i1, i2, eps)
        floor = 100 * np.finfo(float).eps * phi / eps
        g = G["grad_rho"][b][i2, i1]
        assert abs(g - f) <= 1e-5 * abs(f) + floor, (b, i1, i2, g, f)


@pytest.mark.parametrize("order", (4, 6))
def test_adjoint_recursion_has_self_adjoint_form(order):
    """psi_n = H^-1 diag(w) lambda_n obeys the forward leapfrog recursion run backwards with the
    untransposed operator (the consequence of H A_glob being symmetric)."""
    P, u0, dt, rec, obs = _setup(order)
    orc = Oracle(P)
    levels, _ = AD.forward(orc, u0, u0, 0.0, dt, NSTEPS)
    lams = AD.adjoint(orc, levels, rec, obs, dt)
    N = NSTEPS
    dofs = AD.receiver_dofs(orc, rec)
    res = AD.traces(orc, levels, rec) - obs
    scale = orc.wvec / orc.hvec
    psi = [None] + [scale * l for l in lams] + [np.zeros(orc.ndof)]
    for j in range(N, 1, -1):
        src = np.zeros(orc.ndof)
        np.add.at(src, dofs.ravel(), dt * res[j - 2].ravel())
        nxt = 2 * psi[j] - psi[j + 1] + dt * dt * orc.wvec * (orc.A @ psi[j]) + scale * src
        assert np.max(np.abs(nxt - psi[j - 1])) <= 1e-11 * np.max(np.abs(psi[j - 1])), j


def test_zero_residual_gives_zero_gradient():
    P, u0, dt, rec, _ = _setup(4)
    orc = Oracle(P)
    lv, _ = AD.forward(orc, u0, u0, 0.0, dt, 10)
    own = AD.traces(orc, lv, rec)
    G = AD.gradient(P, u0, u0, 0.0, dt, 10, rec, own, [(0, 0, 3, 3)])
    assert G["misfit"] == 0.0
    assert all(np.all(g == 0) for g in G["grad_rho"]) and np.all(G["grad_C"] == 0)


def test_gradient_rejects_displacement_data():
    P = W.mms_problem(20, 4)
    with pytest.raises(ValueError):
        AD.check_gradient_problem(P)


def test_voigt_unit_reproduces_the_voigt_tensor():
    """Sum_V c_V voigt_unit(V) is the tensor that workloads.voigt_to_tensor builds from the same
    symmetric Voigt matrix (an independent construction of C_IJKL from Voigt entries)."""
    rng = np.random.default_rng(3)
    a = rng.standard_normal((3, 3))
    cv = a + a.T
    m = sum(cv[AD.VOIGT_ENTRIES[V]] * AD.voigt_unit(V) for V in range(6))
    T1 = W.pair10_to_tensor(m[:, :, None, None])[..., 0, 0]
    T2 = W.voigt_to_tensor(cv.reshape(3, 3, 1, 1))[..., 0, 0]
    assert np.array_equal(T1, T2)


def test_voigt_gradient_matches_central_differences_and_pair_sum():
    """dPhi/dC_V for the six Voigt entries at a few nodes: central differences of the misfit under
    Voigt perturbations, and the sum of the pair-entry gradients each Voigt entry sets."""
    order = 4
    P, u0, dt, rec, obs = _setup(order)
    n1, n2 = SIZES[order]
    nodes = [(0, 0, 0), (1, 0, 5), (0, 5, 2), (1, 7, 5)]
    vparams = [(b, ("voigt", V), i1, i2) for (b, i1, i2) in nodes for V in range(6)]
    pparams = [(b, Pp, i1, i2) for (b, i1, i2) in nodes for Pp in range(10)]
    G = AD.gradient(P, u0, u0, 0.0, dt, NSTEPS, rec, obs, vparams + pparams)
    gv, gp = G["grad_C"][:len(vparams)], G["grad_C"][len(vparams):].reshape(len(nodes), 10)
    phi = G["misfit"]
    to_voigt = (0, 2, 2, 1, 5, 5, 4, 5, 4, 3)
    for k, (b, (_, V), i1, i2) in enumerate(vparams):
        eps = 1e-5
        fp = AD.misfit_of(AD.perturbed(P, b, ("voigt", V), i1, i2, eps), u0, u0, 0.0, dt, NSTEPS, rec, obs)
        fm = AD.misfit_of(AD.perturbed(P, b, ("voigt", V), i1, i2, -eps), u0, u0, 0.0, dt, NSTEPS, rec, obs)
        f = (fp - fm) / (2 * eps)
        floor = 100 * np.finfo(float).eps * phi / eps
        assert abs(gv[k] - f) <= 1e-5 * abs(f) + floor, (b, V, i1, i2, gv[k], f)
        node = k // 6
        s = sum(gp[node, e] for e in range(10) if to_voigt[e] == V)
        assert abs(gv[k] - s) <= 1e-10 * max(1e-300, np.abs(gp[node]).max()), (V, gv[k], s)
