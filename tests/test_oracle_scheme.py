"""Pins of the oracle's multi-block SBP-SAT scheme (Sec. 3.3, 4.3-4.7, 5, 6, 7) against
identities, closed forms, invariants, printed numbers and convergence rates."""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle.scheme import Oracle, BlockOps, delta_1d, ricker

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ORDERS = (2, 4, 6)
NSMALL = {2: (12, 11), 4: (20, 19), 6: (28, 27)}


def _cartesian_block(N1, N2, C, rho=None, kinds=("robin",) * 4, affine=None):
    x1, x2 = W.ref_grid(N1, N2)
    X = np.stack([x1, x2])
    if affine is not None:
        A, b0 = affine
        X = np.einsum("Ii,i...->I...", A, X) + np.asarray(b0).reshape(2, 1, 1)
    if C.ndim == 4:
        C = C.reshape(2, 2, 2, 2, 1, 1) * np.ones((1, 1, 1, 1, N2, N1))
    rho = np.ones((N2, N1)) if rho is None else rho
    return W.Block(X=X, rho=rho, C=C, faces=[W.Face(k) for k in kinds])


ISO = W.voigt_to_tensor(np.array([[3.0, 1.0, 0.0], [1.0, 3.0, 0.0], [0.0, 0.0, 1.0]]))  # lambda = mu = 1
ANISO = W.voigt_to_tensor(np.array([[4.0, 1.0, 0.2], [1.0, 3.0, 0.1], [0.2, 0.1, 1.0]]))


# ---------------------------------------------------------------- metric (Sec. 3.3)
def test_metric_identity_map():
    bo = BlockOps(_cartesian_block(20, 18, ISO), 4)
    assert np.allclose(bo.J, 1, atol=1e-13)
    assert np.allclose(bo.F[0][0], 1, atol=1e-12) and np.allclose(bo.F[0][1], 0, atol=1e-12)
    for f, fc in enumerate(bo.faces):
        assert np.allclose(fc["Jhat"], 1, atol=1e-12)
        m = f // 2
        assert np.allclose(fc["n"][m], -1 if f % 2 == 0 else 1, atol=1e-12)
        assert np.allclose(fc["n"][1 - m], 0, atol=1e-12)


@pytest.mark.parametrize("order", ORDERS)
def test_metric_affine_exact(order):
    A = np.array([[2.0, 0.5], [-0.3, 1.5]])
    N1, N2 = NSMALL[order]
    bo = BlockOps(_cartesian_block(N1, N2, ISO, affine=(A, [1.0, -2.0])), order)
    # G[i][I] = dX_I/dx_i = A[I][i]; J = det A; F_Ii = dx_i/dX_I = (A^-1)_iI
    assert np.allclose(bo.J, np.linalg.det(A), rtol=1e-12)
    Ainv = np.linalg.inv(A)
    for I in range(2):
        for i in range(2):
            assert np.allclose(bo.F[I][i], Ainv[i, I], rtol=1e-11, atol=1e-12)
    # Jhat on face x1 = const is |a_2| = |A[:,1]|
    assert np.allclose(bo.faces[0]["Jhat"], np.hypot(A[0, 1], A[1, 1]), rtol=1e-12)


@pytest.mark.parametrize("order", ORDERS)
def test_nanson_holds_identically(order):
    P = W.random_problem(n=NSMALL[order], order=order)
    bo = BlockOps(P.blocks[0], order)
    for f, fc in enumerate(bo.faces):
        m, idx = f // 2, fc["idx"]
        nu = -1 if f % 2 == 0 else 1
        for I in range(2):
            assert np.allclose(fc["Jhat"] * fc["n"][I], bo.J[idx] * bo.F[I][m][idx] * nu, rtol=1e-12, atol=1e-13)
        assert np.allclose(fc["n"][0] ** 2 + fc["n"][1] ** 2, 1, atol=1e-12)


def test_transformed_stiffness_symmetry_and_isotropic_form():
    """c_ijkl = c_klij (eq. C_symmetry); isotropic case equals the closed form of Sec. 3.2.3."""
    P = W.random_problem(n=(20, 19), order=4)
    blk = P.blocks[0]
    blk.C = ISO.reshape(2, 2, 2, 2, 1, 1) * np.ones((1, 1, 1, 1, blk.N2, blk.N1))
    bo = BlockOps(blk, 4)
    c, F, J = bo.c, bo.F, bo.J
    for i in range(2):
        for j in range(2):
            for k in range(2):
                for l in range(2):
                    assert np.allclose(c[i, j, k, l], c[k, l, i, j], rtol=1e-13)
                    # J [ lam F_ji F_lk + mu (F_Ki dJl F_Kk + F_li F_jk) ] with lam = mu = 1
                    ref = J * (F[j][i] * F[l][k] + ((F[0][i] * F[0][k] + F[1][i] * F[1][k]) if j == l else 0)
                               + F[l][i] * F[j][k])
                    assert np.allclose(c[i, j, k, l], ref, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- operator (Sec. 4.6-4.7)
@pytest.mark.parametrize("order", ORDERS)
def test_integration_by_parts_identity(order):
    """eq. ibp_discr_operator_clean: H DD_ik(c) - sum_f P_f nu_i c D_k = -(D_i^T H c D_k + W),
    a symmetric negative semidefinite matrix."""
    P = W.random_problem(n=NSMALL[order], order=order)
    bo = BlockOps(P.blocks[0], order)
    K = bo.elastic_operator()
    Hd = sp.diags(bo.Hvec)
    S = np.zeros((2 * bo.N, 2 * bo.N))
    for J in range(2):
        for L in range(2):
            blockJL = (Hd @ K[J][L]).toarray()
            for f in range(4):
                blockJL -= (bo.faces[f]["P"] @ bo.traction_rows(f)[J][L]).toarray()
            S[J * bo.N:(J + 1) * bo.N, L * bo.N:(L + 1) * bo.N] = blockJL
    scale = np.abs(S).max()
    assert np.abs(S - S.T).max() < 1e-13 * scale
    assert np.linalg.eigvalsh(0.5 * (S + S.T)).max() < 1e-12 * scale


@pytest.mark.parametrize("order", ORDERS)
def test_linear_displacement_annihilated(order):
    """Constant C on an affine grid: the operator maps any linear field to zero (all rows)."""
    A = np.array([[1.2, 0.2], [0.1, 0.9]])
    N1, N2 = NSMALL[order]
    bo = BlockOps(_cartesian_block(N1, N2, ANISO, affine=(A, [0.0, 0.0])), order)
    K = bo.elastic_operator()
    X = bo.blk.X
    u = [0.3 * X[0] - 1.1 * X[1] + 2.0, 0.7 * X[0] + 0.4 * X[1] - 1.0]
    for J in range(2):
        r = K[J][0] @ u[0].ravel() + K[J][1] @ u[1].ravel()
        assert np.abs(r).max() < 1e-9


@pytest.mark.parametrize("order", ORDERS)
def test_one_dimensional_reduction(order):
    """Cartesian grid, C constant, u = u(x1): r_j = D_xx^FC(c_1j1l) u_l on every x1 line."""
    N1, N2 = NSMALL[order]
    bo = BlockOps(_cartesian_block(N1, N2, ANISO), order)
    K = bo.elastic_operator()
    x = np.linspace(0, 1, N1)
    prof = [np.sin(3 * x) + x ** 2, np.cos(2 * x)]
    u = [np.tile(p, (N2, 1)) for p in prof]
    op1 = bo.op[0]
    for J in range(2):
        r = (K[J][0] @ u[0].ravel() + K[J][1] @ u[1].ravel()).reshape(N2, N1)
        ref = sum(op1.Dxx_fc(ANISO[0, J, 0, L] * np.ones(N1)) @ prof[L] for L in range(2))
        assert np.allclose(r, ref[None, :], rtol=1e-11, atol=1e-9)


# ---------------------------------------------------------------- full scheme (Sec. 5-7)
CASES = [
    (("robin",) * 4, False, False),
    (("displacement",) * 4, False, False),
    (("robin", "displacement", "displacement", "robin"), True, False),
    (("displacement", "robin", "robin", "displacement"), True, True),
]


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("case", range(len(CASES)))
def test_self_adjoint_and_negative_semidefinite(order, case):
    """Sec. 7.2: A = calH D^tot symmetric to machine precision and negative semidefinite
    (Theorems 2-5).  The paper prints 1.6e-16 / 3.6e-16 / 2.1e-16 for the symmetry deviation."""
    kinds, two, rev = CASES[case]
    P = W.random_problem(kinds=kinds, n=NSMALL[order], order=order, two_blocks=two, reversed_interface=rev)
    A = Oracle(P).symmetric_matrix().toarray()
    scale = np.abs(A).max()
    assert np.abs(A - A.T).max() / scale < 1e-14
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).max() < 1e-12 * scale


@pytest.mark.parametrize("order", ORDERS)
def test_traction_only_rigid_modes(order):
    """Pure traction (U = 0): rigid translations are in the null space (lambda_max = 0)."""
    P = W.random_problem(kinds=("robin",) * 4, n=NSMALL[order], order=order)
    for f in P.blocks[0].faces:
        f.U = None
    O = Oracle(P)
    for J in range(2):
        u = np.zeros(O.ndof)
        u[O._sl(0, J)] = 1.0
        assert np.abs(O.A @ u).max() < 1e-9 * np.abs(O.A).max()


@pytest.mark.parametrize("order", (4, 6))
def test_leapfrog_energy_conserved(order):
    """Homogeneous conditions: the leapfrog energy E^{n+1/2} is constant to roundoff."""
    P = W.random_problem(kinds=("robin", "displacement", "displacement", "robin"),
                         n=NSMALL[order], order=order, two_blocks=True)
    O = Oracle(P)
    dt = O.suggest_dt(0.3)
    u_prev = u = O.pack(W.smooth_state(P))
    Es = []
    for n in range(200):
        up2, u2, _ = O.leapfrog(u_prev, u, 0.0, dt, 1, homogeneous=True)
        Es.append(O.energy_leapfrog(u, u2, dt))
        u_prev, u = up2, u2
    Es = np.array(Es)
    assert Es.min() > 0
    assert np.abs(Es - Es[0]).max() / Es[0] < 1e-12


def test_interface_orientation_invariance():
    """Rotating block 1 by 180 degrees (reversed interface) leaves the scheme unchanged."""
    P = W.random_problem(kinds=("robin", "displacement", "displacement", "robin"), n=(20, 19), order=4,
                         two_blocks=True)
    O1 = Oracle(P)
    b1 = P.blocks[1]
    rot = lambda a: a[..., ::-1, ::-1].copy()
    swap = {0: 1, 1: 0, 2: 3, 3: 2}
    faces = [None] * 4
    for f, face in enumerate(b1.faces):
        nf = swap[f]
        Uq = None if face.U is None else face.U[:, ::-1].copy()
        faces[nf] = W.Face(face.kind, U=Uq)
    faces[1] = W.Face("interface", nbr=(0, 1, True))
    P2 = W.Problem("rot", 4, [P.blocks[0], W.Block(X=rot(b1.X), rho=rot(b1.rho), C=rot(b1.C), faces=faces)])
    P2.blocks[0].faces[1] = W.Face("interface", nbr=(1, 1, True))
    O2 = Oracle(P2)
    u = W.random_state(P)
    r1 = O1.unpack(O1.A @ O1.pack(u))
    r2 = O2.unpack(O2.A @ O2.pack([u[0], rot(u[1])]))
    scale = np.abs(r1[1]).max()
    assert np.abs(r1[0] - r2[0]).max() < 1e-11 * scale
    assert np.abs(r1[1] - rot(r2[1])).max() < 1e-11 * scale


@pytest.mark.slow
@pytest.mark.parametrize("order,floor", [(2, 1.8), (4, 2.9), (6, 3.7)])
def test_mms_convergence_rates(order, floor):
    """Sec. 7.1: manufactured solution and material of the paper, traction + displacement
    boundaries and an interface, RK4; observed rates reach at least min(q_b + 2, 2q) with
    q_b = q - 1 (the rule of thumb the paper quotes: 2, 3, 4), minus a small margin."""
    Ns = (21, 31, 41) if order < 6 else (31, 41, 51)
    errs = []
    for N in Ns:
        P = W.mms_problem(N, order, kinds=("robin", "displacement", "robin", "displacement"), two_blocks=True)
        O = Oracle(P)
        T = 0.5
        dt = O.suggest_dt(0.25)
        n = int(math.ceil(T / dt))
        dt = T / n
        u0 = O.pack([P.exact(b, 0.0) for b in P.blocks])
        v0 = O.pack([np.stack([-W.MMS_W[L] * np.cos(W.MMS_K[L, 0] * b.X[0] + W.MMS_K[L, 1] * b.X[1])
                               for L in range(2)]) for b in P.blocks])
        u, v, t = O.rk4(u0, v0, 0.0, dt, n)
        errs.append(O.l2_error(u, t))
    rate = math.log(errs[0] / errs[-1]) / math.log((Ns[-1] - 1) / (Ns[0] - 1))
    assert rate > floor, (errs, rate)


def test_leapfrog_mms_second_order_in_time():
    """Leapfrog with the MMS data converges (error falls with h at fixed CFL)."""
    errs = []
    for N in (21, 41):
        P = W.mms_problem(N, 4, kinds=("displacement",) * 4)
        O = Oracle(P)
        T = 0.25
        dt = O.suggest_dt(0.2)
        n = int(math.ceil(T / dt))
        dt = T / n
        up = O.pack([P.exact(b, -dt) for b in P.blocks])
        u = O.pack([P.exact(b, 0.0) for b in P.blocks])
        up, u, t = O.leapfrog(up, u, 0.0, dt, n)
        errs.append(O.l2_error(u, t))
    assert errs[1] < errs[0] / 3


# ---------------------------------------------------------------- CFL (Sec. 7), sources (Sec. 7.4)
def test_christoffel_isotropic_closed_form():
    """lambda = mu = rho = 1 on the unit square: v_max = sqrt(lambda + 2 mu) = sqrt(3)."""
    O = Oracle(W.Problem("iso", 4, [_cartesian_block(20, 20, ISO)]))
    v = O.vmax_nodes()[0]
    assert np.allclose(v, math.sqrt(3), rtol=1e-10)
    assert math.isclose(O.suggest_dt(0.5), 0.5 / 19 / math.sqrt(3), rel_tol=1e-10)


def test_christoffel_anisotropic_brute_force():
    A = np.array([[1.3, 0.2], [-0.1, 0.8]])
    O = Oracle(W.Problem("an", 4, [_cartesian_block(20, 19, ANISO, rho=2 * np.ones((19, 20)), affine=(A, [0, 0]))]))
    bo = O.bops[0]
    n = 0
    best = 0.0
    for th in np.linspace(0, np.pi, 20001):
        xi = (math.cos(th), math.sin(th))
        G = np.array([[sum(xi[i] * bo.c[i, j, k, l][n] * xi[k] for i in range(2) for k in range(2))
                       for l in range(2)] for j in range(2)])
        best = max(best, np.linalg.eigvalsh(0.5 * (G + G.T)).max())
    assert math.isclose(O.vmax_nodes()[0][n], math.sqrt(best / (bo.rho[n] * bo.J[n])), rel_tol=1e-8)


def test_ricker_alpha_m_matches_paper():
    gold = json.load(open(os.path.join(GOLD, "paper_numbers.json")))
    ap = 4.0
    t = np.linspace(-4, 4, 1 << 16)
    w = np.array([ricker(tt, ap, 0.0) for tt in t])
    spec = np.abs(np.fft.rfft(w))
    fr = np.fft.rfftfreq(len(t), t[1] - t[0])
    ipk = np.argmax(spec)
    assert abs(fr[ipk] - ap) < 0.01
    above = np.nonzero(spec[ipk:] < 0.05 * spec[ipk])[0][0] + ipk
    # linear interpolation of the 5% crossing
    f0, f1, s0, s1 = fr[above - 1], fr[above], spec[above - 1], spec[above]
    am = f0 + (0.05 * spec[ipk] - s0) * (f1 - f0) / (s1 - s0)
    assert abs(am / ap - gold["ricker_alpha_M_over_alpha_P"]["value"]) < 0.005
    assert abs(am - gold["ricker_alpha_M_for_4Hz"]["value"]) < 0.01


@pytest.mark.parametrize("q", (1, 2, 3))
def test_discrete_delta_moments(q):
    N, h = 41, 1.0 / 40
    for x0 in (0.0, 0.013, 0.5, 0.77, 1.0):
        nodes, w = delta_1d(N, h, x0, q)
        assert len(nodes) == 2 * q and nodes.min() >= 0 and nodes.max() < N
        for p in range(2 * q):
            assert math.isclose(np.sum(w * (nodes * h) ** p), x0 ** p, rel_tol=1e-10, abs_tol=1e-12)


def test_point_source_integrates_polynomials():
    """sum_nodes H_n phi_n (J f)_n = amp * W(t) * phi(X0) for low-degree phi (reading 8)."""
    blk = _cartesian_block(30, 28, ISO)
    src = W.PointSource(block=0, x_ref=(0.41, 1.0), direction=(0.0, -1.0), amplitude=2.0, alpha_p=3.0, t0=0.2)
    O = Oracle(W.Problem("src", 6, [blk], sources=[src]))
    t = 0.17
    d = O.data(t)
    bo = O.bops[0]
    x1, x2 = blk.X[0].ravel(), blk.X[1].ravel()
    for phi in (lambda a, b: 1 + 0 * a, lambda a, b: a * b ** 2 + a ** 3):
        got = np.sum(bo.Hvec * phi(x1, x2) * d[bo.N:2 * bo.N])
        assert math.isclose(got, -2.0 * ricker(t, 3.0, 0.2) * phi(0.41, 1.0), rel_tol=1e-10)
