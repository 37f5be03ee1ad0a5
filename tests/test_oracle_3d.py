"""Pins of the 3-D oracle (oracle/scheme3d.py) against facts the paper and the mathematics fix,
none of which reuses the 3-D oracle's own formulas:

* a plane motion of an extruded block is the 2-D scheme (the independently pinned 2-D oracle)
  on every x3-slice, with the displacement penalty's dimension factor d = 3 against d = 2;
* relabelling the reference axes cyclically (an even permutation, so J keeps its sign) moves
  the result along with the grid: every direction-specific index of the operator is exercised;
* diag(H) A is symmetric and negative semi-definite (Theorem 1 and 3 for d = 3);
* rigid translations (any grid) and rigid rotations (affine grid, constant C) are in the kernel
  of the operator with traction faces;
* the volume operator is exact for quadratic displacements on an affine grid with constant C
  (orders 4 and 6: their boundary closures differentiate quadratics exactly), and away from the
  closures it converges to the continuous operator at the interior order 2q;
* leapfrog conserves the discrete energy of the scheme.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from workloads import box3d as B
from oracle.scheme import Oracle
from oracle.scheme3d import Oracle3D


def _cyc(x):
    """Reference-axis relabelling (x1, x2, x3) -> (x2, x3, x1) of a (..., N3, N2, N1) array."""
    n = x.ndim
    return x.transpose(tuple(range(n - 3)) + (n - 1, n - 3, n - 2))


def test_pair45_roundtrip():
    rho, C = B.random_material3((5, 4, 3))
    assert np.array_equal(B.tensor_from_pair45(B.pair45(C)), C)
    M = C.reshape(9, 9, -1)
    assert np.allclose(M, M.transpose(1, 0, 2), rtol=0, atol=0)


@pytest.mark.parametrize("order,n,n3", [(4, (20, 19), 18), (6, (28, 27), 27)])
def test_plane_motion_reduces_to_2d(order, n, n3):
    """u = (u1(x1, x2), u2(x1, x2), 0) on a curvilinear 2-D block extruded along X3 = L3 x3,
    in a medium whose x3 = const plane is a mirror plane: the in-plane accelerations at every
    x3-slice equal the 2-D scheme's with penalty factor beta_2D = beta_3D * 3 / 2, and the
    out-of-plane acceleration vanishes away from the x3 faces (whose traction SAT sees C_33ab)."""
    P = W.random_problem(kinds=("robin", "displacement", "displacement", "robin"), n=n, order=order)
    for f in P.blocks[0].faces:
        f.U = None
    beta3 = 1.0
    P.beta = beta3 * 3 / 2
    O2 = Oracle(P)
    b3 = B.extrude_block(P.blocks[0], n3)
    b3.order, b3.beta = order, beta3
    b3.faces = ("traction", "displacement", "displacement", "traction", "traction", "traction")
    O3 = Oracle3D(b3)
    u2 = W.smooth_state(P)[0]
    u3 = np.zeros((3, n3) + u2.shape[1:])
    u3[0], u3[1] = u2[0][None], u2[1][None]
    a3 = O3.accel(u3)
    a2 = O2.unpack(O2.wvec * (O2.A @ O2.pack([u2])))[0]
    scale = np.abs(a2).max()
    assert np.abs(a3[:2] - a2[:, None]).max() < 1e-12 * scale
    assert np.abs(a3[2, 1:-1]).max() < 1e-12 * scale
    assert np.abs(a3[2, [0, -1]]).max() > 1e-3 * scale          # the x3 faces do act on u3


def test_plane_motion_wrong_dimension_factor_fails():
    """The same comparison with beta_2D = beta_3D (the penalty's d left at 2) does not match:
    the reduction test above is sensitive to the dimension factor."""
    P = W.random_problem(kinds=("displacement", "robin", "robin", "robin"), n=(20, 19), order=4)
    for f in P.blocks[0].faces:
        f.U = None
    P.beta = 1.0
    O2 = Oracle(P)
    b3 = B.extrude_block(P.blocks[0], 18)
    b3.order, b3.beta = 4, 1.0
    b3.faces = ("displacement", "traction", "traction", "traction", "traction", "traction")
    O3 = Oracle3D(b3)
    u2 = W.smooth_state(P)[0]
    u3 = np.zeros((3, 18) + u2.shape[1:])
    u3[0], u3[1] = u2[0][None], u2[1][None]
    a3 = O3.accel(u3)
    a2 = O2.unpack(O2.wvec * (O2.A @ O2.pack([u2])))[0]
    assert np.abs(a3[:2] - a2[:, None]).max() > 1e-3 * np.abs(a2).max()


def test_cyclic_relabel():
    b = B.random_block3(N=(19, 18, 20), order=4)
    O = Oracle3D(b)
    u = B.smooth_state3(b)
    a = O.accel(u)
    faces = [None] * 6
    newdir = {0: 2, 1: 0, 2: 1}
    for f in range(6):
        faces[2 * newdir[f // 2] + f % 2] = b.faces[f]
    bp = B.Block3D(X=_cyc(b.X), rho=_cyc(b.rho), C=_cyc(b.C), faces=tuple(faces), order=4)
    ap = Oracle3D(bp).accel(_cyc(u))
    assert np.abs(ap - _cyc(a)).max() < 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("faces", [("traction",) * 6,
                                   ("displacement", "traction", "displacement", "traction", "traction",
                                    "displacement"),
                                   ("displacement",) * 6])
def test_symmetric_negative_semidefinite(faces):
    b = B.random_block3(N=(7, 6, 8), order=2, faces=faces)
    O = Oracle3D(b)
    HA = (sp.diags(O.hvec) @ O.A).toarray()
    assert np.abs(HA - HA.T).max() < 1e-13 * np.abs(HA).max()
    ev = np.linalg.eigvalsh(0.5 * (HA + HA.T))
    assert ev.max() < 1e-10 * np.abs(ev).max()
    if "displacement" in faces:
        assert ev.max() < -1e-8 * np.abs(ev).max()               # no rigid motion survives


def test_symmetric_order4_and_6():
    for order, N in ((4, (19, 18, 20)), (6, (27, 28, 27))):
        b = B.random_block3(N=N, order=order)
        O = Oracle3D(b)
        HA = sp.diags(O.hvec) @ O.A
        d = (HA - HA.T).tocsr()
        assert abs(d).max() < 1e-13 * abs(HA).max()


def test_rigid_motions_in_kernel():
    # translations: any curvilinear grid and variable material
    b = B.random_block3(N=(19, 18, 20), order=4, faces=("traction",) * 6)
    O = Oracle3D(b)
    scale = abs(O.A).max()
    for l in range(3):
        u = np.zeros((3,) + b.rho.shape)
        u[l] = 1.0
        assert np.abs(O.A @ O.pack(u)).max() < 1e-11 * scale
    # rotations: affine grid, constant stiffness
    N = (19, 18, 20)
    g = np.array(B.ref_grid3(*N))
    Aff = np.array([[1.0, 0.1, 0.05], [0.2, 1.3, 0.0], [0.1, -0.1, 0.8]])
    X = np.einsum("Ii,i...->I...", Aff, g)
    rho, C = B.random_material3(N)
    C = np.broadcast_to(C[..., 2:3, 2:3, 2:3], C.shape).copy()
    ba = B.Block3D(X=X, rho=rho, C=C, faces=("traction",) * 6, order=4)
    Oa = Oracle3D(ba)
    for axis in range(3):
        om = np.zeros(3)
        om[axis] = 1.0
        u = np.cross(om[:, None], X.reshape(3, -1), axis=0).reshape(X.shape)
        assert np.abs(Oa.A @ Oa.pack(u)).max() < 1e-10 * abs(Oa.A).max()


@pytest.mark.parametrize("order,N", [(4, (19, 18, 20)), (6, (28, 27, 29))])
def test_volume_operator_exact_for_quadratics(order, N):
    """Affine grid, constant C: sum_ik DD_ik(c_ijkl) u_l = J C_IjKl d_I d_K u_l at every node for
    u_l = X^T Q_l X / 2 (so d_I d_K u_l = Q_l[I, K])."""
    g = np.array(B.ref_grid3(*N))
    Aff = np.array([[1.0, 0.1, 0.05], [0.2, 1.3, 0.0], [0.1, -0.1, 0.8]])
    X = np.einsum("Ii,i...->I...", Aff, g)
    rho, C = B.random_material3(N)
    C = np.broadcast_to(C[..., 3:4, 3:4, 3:4], C.shape).copy()
    O = Oracle3D(B.Block3D(X=X, rho=np.ones_like(rho), C=C, faces=("traction",) * 6, order=order))
    K = O.volume_operator()
    Q = np.random.default_rng(1).standard_normal((3, 3, 3))
    Q = Q + Q.transpose(0, 2, 1)
    u = np.array([0.5 * np.einsum("I...,IK,K...->...", X, Q[l], X) for l in range(3)])
    got = np.array([sum(K[j][l] @ u[l].ravel() for l in range(3)) for j in range(3)])
    c0 = C[..., 0, 0, 0]
    exact = np.array([O.J * np.einsum("IKl,lIK->", c0[:, j], Q) for j in range(3)])
    assert np.abs(got - exact).max() < 1e-10 * np.abs(exact).max()


def test_leapfrog_conserves_energy():
    b = B.random_block3(N=(19, 18, 20), order=4)
    O = Oracle3D(b)
    dt = O.suggest_dt(0.9)
    u0 = B.smooth_state3(b, seed=1)
    u1 = u0 + dt * B.smooth_state3(b, seed=2)
    E0 = O.energy(u0, u1, dt)
    a, c = O.leapfrog(u0, u1, dt, 40)
    E1 = O.energy(a, c, dt)
    assert E0 > 0
    assert abs(E1 - E0) < 1e-11 * E0


def test_crop_window_matches_whole_block_at_its_centre():
    """The oracle on a crop with 'open' cut faces and the whole block's spacing gives the whole
    block's accelerations wherever the stencils (and the metric rows they read) stay inside the
    crop: here the crop's central node.  This is what the full-size sampled parity relies on."""
    N = (40, 38, 41)
    b = B.random_block3(N=N, order=6)
    u = B.smooth_state3(b)
    a = Oracle3D(b).accel(u)
    for lo in ((6, 5, 7), (0, 11, 14), (13, 0, 14)):
        hi = tuple(l + 27 for l in lo)
        c = B.crop_block3(b, lo, hi)
        sub = u[:, lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        ac = Oracle3D(c).accel(sub)
        for node in ((13, 13, 13), (2, 13, 13) if lo[0] == 0 else (13, 13, 13), (13, 1, 13) if lo[1] == 0 else (13, 13, 13)):
            i1, i2, i3 = node
            got = ac[:, i3, i2, i1]
            ref = a[:, lo[2] + i3, lo[1] + i2, lo[0] + i1]
            assert np.abs(got - ref).max() < 1e-10 * np.abs(a).max()
        cc = B.random_block3_crop(N, lo, hi, order=6, faces=b.faces)
        assert np.array_equal(cc.X, c.X) and np.allclose(cc.C, c.C, rtol=1e-15, atol=0) and cc.faces == c.faces


@pytest.mark.parametrize("order,ns,margin,rate", [(2, (12, 23), 2, 1.9), (4, (19, 37), 7, 3.3)])
def test_volume_operator_interior_convergence(order, ns, margin, rate):
    """Affine grid, constant C, u_l = sin(k . X + phi_l): away from the closure rows the volume
    operator converges to the continuous J C_IjKl d_I d_K u_l = -J C_IjKl k_I k_K u_l at the
    interior order 2q (Sec. 4: order 2q in the interior)."""
    def max_err(n):
        N = (n, n, n)
        g = np.array(B.ref_grid3(*N))
        Aff = np.array([[1.0, 0.1, 0.05], [0.2, 1.3, 0.0], [0.1, -0.1, 0.8]])
        X = np.einsum("Ii,i...->I...", Aff, g)
        rho, C = B.random_material3(N)
        C = np.broadcast_to(C[..., 3:4, 3:4, 3:4], C.shape).copy()
        O = Oracle3D(B.Block3D(X=X, rho=np.ones_like(rho), C=C, faces=("traction",) * 6, order=order))
        K = O.volume_operator()
        kv = np.array([1.3, -0.7, 0.9])
        u = np.array([np.sin(np.einsum("I,I...->...", kv, X) + ph) for ph in (0.3, 1.1, -0.4)])
        got = np.array([sum(K[j][l] @ u[l].ravel() for l in range(3)) for j in range(3)])
        c0 = C[..., 0, 0, 0]
        exact = -O.J * np.einsum("IjKl,I,K,l...->j...", c0, kv, kv, u).reshape(3, -1)
        e = np.abs(got - exact).reshape(3, n, n, n)
        m = margin
        return e[:, m:n - m, m:n - m, m:n - m].max()
    e1, e2 = max_err(ns[0]), max_err(ns[1])
    assert np.log(e1 / e2) / np.log((ns[1] - 1) / (ns[0] - 1)) > rate
