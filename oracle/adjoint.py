"""Discrete adjoint of the leapfrog-stepped SBP-SAT scheme and the misfit gradient -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper proves the semi-discrete operator self-adjoint (Theorems 3 and 5) and remarks that an
adjoint solver can therefore reuse the forward solver (Sec. 5.2).  This module is the plain
definition of what such an adjoint must compute, written WITHOUT using self-adjointness: every
transpose is an explicit sparse transpose of the assembled matrix.

Time stepping (as ``Oracle.leapfrog``): the initial levels are u_0 (previous) and u_1 (current, time
t0); step n = 1..N computes
    u_{n+1} = 2 u_n - u_{n-1} + dt^2 (M u_n + s_n),   M = diag(w) A_glob,  s_n = diag(w) data(t_n),
with t_n = t0 + (n-1) dt and w = 1/(rho J).

Misfit (readings: receivers sit on grid nodes, both components are observed, and the time sum is
the rectangle rule over the N computed levels):
    Phi = 1/2 dt sum_{k=1..N} sum_r sum_J (u_{k+1}[J, x_r] - d[k-1, r, J])^2.

Adjoint (Lagrange multipliers lambda_n of the N step equations):
    lambda_N     = dPhi/du_{N+1}
    lambda_{j-1} = 2 lambda_j - lambda_{j+1} + dt^2 M^T lambda_j + dPhi/du_j,   j = N, ..., 2
    dPhi/dtheta  = sum_{n=1..N} dt^2 lambda_n^T (dM/dtheta u_n + ds_n/dtheta).

Parameters theta: the density rho at a node, and the ten independent entries of the stiffness in
pair form (the upper triangle of M[2I+J][2K+L] = C_IJKL, the layout ``sbp_set_material`` takes) at a
node.  A_glob is affine in C (linear in C except for the Robin J^ U terms), so
dA/dC_P(x) = A(E_{P,x}) - A(0) exactly, where E_{P,x} is the stiffness that is zero except for a unit
in pair entry P (both of its symmetric copies) at node x.  The data s_n do not depend on C as long
as no displacement face carries boundary data (point sources, forcing and Robin data are
independent of C); ``check_gradient_problem`` enforces that.  For rho, dw/drho = -w/rho, so
d(M u_n + s_n)/drho_x = -(M u_n + s_n)_x / rho_x at the two components of node x.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence, Tuple

import numpy as np

import workloads as W
from .scheme import Oracle


def check_gradient_problem(problem: W.Problem):
    for b in problem.blocks:
        for f in b.faces:
            if f.kind == "displacement" and f.g is not None:
                raise ValueError("misfit gradients need displacement faces without boundary data")


def receiver_dofs(oracle: Oracle, receivers: Sequence[Tuple[int, int, int]]):
    """Global dof indices (nrec, 2) of receivers given as (block, i1, i2)."""
    out = np.zeros((len(receivers), 2), dtype=np.int64)
    for r, (b, i1, i2) in enumerate(receivers):
        bo = oracle.bops[b]
        node = i2 * bo.N1 + i1
        for J in range(2):
            out[r, J] = oracle.offsets[b] + J * bo.N + node
    return out


def forward(oracle: Oracle, u_prev, u_cur, t0: float, dt: float, nsteps: int):
    """All levels u_0 .. u_{N+1} (packed vectors) and the step times t_1 .. t_N."""
    levels = [oracle.pack(u_prev), oracle.pack(u_cur)]
    times = []
    t = t0
    for n in range(nsteps):
        times.append(t)
        u_prev_v, u_v = levels[-2], levels[-1]
        levels.append(2 * u_v - u_prev_v + dt * dt * oracle.accel(u_v, t))
        t = t + dt
    return levels, times


def traces(oracle: Oracle, levels, receivers):
    """Recorded displacement d[k-1, r, J] = u_{k+1}[J, x_r], k = 1..N."""
    dofs = receiver_dofs(oracle, receivers)
    return np.stack([lv[dofs] for lv in levels[2:]])


def misfit(rec, observed, dt: float) -> float:
    r = np.asarray(rec) - np.asarray(observed)
    return 0.5 * dt * float(np.sum(r * r))


def adjoint(oracle: Oracle, levels, receivers, observed, dt: float):
    """lambda_1 .. lambda_N (list index n-1) by the explicit-transpose recursion."""
    dofs = receiver_dofs(oracle, receivers)
    N = len(levels) - 2
    res = traces(oracle, levels, receivers) - np.asarray(observed)
    MT = (oracle.A.T @ _diag_sparse(oracle.wvec)).tocsr()       # (diag(w) A)^T = A^T diag(w)

    def dphi(j):                                                # dPhi/du_j, j = 2..N+1
        g = np.zeros(oracle.ndof)
        np.add.at(g, dofs.ravel(), dt * res[j - 2].ravel())
        return g

    lam = [None] * (N + 2)                                      # lam[n], n = 1..N (+ zeros at N+1)
    lam[N + 1] = np.zeros(oracle.ndof)
    lam[N] = dphi(N + 1)
    for j in range(N, 1, -1):
        nxt = lam[j + 1]
        lam[j - 1] = 2 * lam[j] - nxt + dt * dt * (MT @ lam[j]) + dphi(j)
    return lam[1:N + 1]


def _diag_sparse(v):
    import scipy.sparse as sp
    return sp.diags(np.asarray(v, dtype=float))


def grad_rho(oracle: Oracle, levels, times, lams, dt: float):
    """dPhi/drho at every node, per block (N2, N1)."""
    acc = np.zeros(oracle.ndof)
    for n, lam in enumerate(lams, start=1):
        acc += dt * dt * lam * oracle.accel(levels[n], times[n - 1])
    out = []
    for b, bo in enumerate(oracle.bops):
        sl0, sl1 = oracle._sl(b, 0), oracle._sl(b, 1)
        g = -(acc[sl0] + acc[sl1]) / bo.rho
        out.append(g.reshape(bo.N2, bo.N1))
    return out


def pair_unit(P: int) -> np.ndarray:
    """4x4 pair matrix with ones at entry P of the packed upper triangle and at its mirror."""
    m = np.zeros((4, 4))
    idx = 0
    for p in range(4):
        for q in range(p, 4):
            if idx == P:
                m[p, q] = m[q, p] = 1.0
            idx += 1
    return m


# Voigt parametrisation (stiffness with minor symmetry): index 0 = (1,1), 1 = (2,2), 2 = (1,2) = (2,1)
# of a pair of tensor indices, entries in the order 11 12 13 22 23 33 of the symmetric 3x3 matrix
VOIGT_OF_PAIR = (0, 2, 2, 1)          # pair p = 2I+J -> Voigt index of (I, J)
VOIGT_ENTRIES = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def voigt_unit(V: int) -> np.ndarray:
    """4x4 pair matrix of the tensor whose Voigt matrix has a one at entry V (and its mirror):
    C_IJKL = 1 where the Voigt indices of (I,J) and (K,L) are the two indices of entry V."""
    a, b = VOIGT_ENTRIES[V]
    m = np.zeros((4, 4))
    for p in range(4):
        for q in range(4):
            if sorted((VOIGT_OF_PAIR[p], VOIGT_OF_PAIR[q])) == [a, b]:
                m[p, q] = 1.0
    return m


def _with_stiffness(problem: W.Problem, stiff: List[np.ndarray]) -> W.Problem:
    blocks = [dataclasses.replace(b, C=C) for b, C in zip(problem.blocks, stiff)]
    return dataclasses.replace(problem, blocks=blocks, sources=[], time_basis=[])


def _unit_matrix(P) -> np.ndarray:
    """Pair matrix of a stiffness parameter: P an int (pair entry) or ("voigt", V) (Voigt entry)."""
    if isinstance(P, tuple) and P[0] == "voigt":
        return voigt_unit(int(P[1]))
    return pair_unit(int(P))


def stiffness_derivative(problem: W.Problem, block: int, P, i1: int, i2: int, A0=None):
    """dA_glob/dC_P(x) = A(E) - A(0) (A_glob is affine in C); A0 = A(0) may be passed in.
    P: pair entry (int) or ("voigt", V)."""
    zero = [np.zeros_like(b.C) for b in problem.blocks]
    unit = [z.copy() for z in zero]
    unit[block][..., i2, i1] = W.pair10_to_tensor(_unit_matrix(P)[:, :, None, None])[..., 0, 0]
    A1 = Oracle(_with_stiffness(problem, unit)).A
    if A0 is None:
        A0 = Oracle(_with_stiffness(problem, zero)).A
    return (A1 - A0).tocsr()


def grad_stiffness(oracle: Oracle, levels, lams, dt: float, params):
    """dPhi/dC_P(x) for params given as (block, P, i1, i2), P a pair entry or ("voigt", V)."""
    U = np.stack(levels[1:len(lams) + 1], axis=1)              # u_1 .. u_N as columns
    WL = np.stack(lams, axis=1) * oracle.wvec[:, None]          # diag(w) lambda_n
    A0 = Oracle(_with_stiffness(oracle.problem, [np.zeros_like(b.C) for b in oracle.problem.blocks])).A
    out = []
    for (b, P, i1, i2) in params:
        dA = stiffness_derivative(oracle.problem, b, P, i1, i2, A0)
        out.append(dt * dt * float(np.sum(WL * (dA @ U))))
    return np.array(out)


def gradient(problem: W.Problem, u_prev, u_cur, t0, dt, nsteps, receivers, observed, stiff_params=()):
    """Misfit, its rho gradient at every node, its stiffness gradient at ``stiff_params``."""
    check_gradient_problem(problem)
    orc = Oracle(problem)
    levels, times = forward(orc, u_prev, u_cur, t0, dt, nsteps)
    rec = traces(orc, levels, receivers)
    phi = misfit(rec, observed, dt)
    lams = adjoint(orc, levels, receivers, observed, dt)
    g_rho = grad_rho(orc, levels, times, lams, dt)
    g_c = grad_stiffness(orc, levels, lams, dt, stiff_params) if len(stiff_params) else np.zeros(0)
    return dict(misfit=phi, traces=rec, grad_rho=g_rho, grad_C=g_c, levels=levels, lams=lams, oracle=orc)


def misfit_of(problem: W.Problem, u_prev, u_cur, t0, dt, nsteps, receivers, observed) -> float:
    """Phi alone (for finite-difference checks)."""
    orc = Oracle(problem)
    levels, _ = forward(orc, u_prev, u_cur, t0, dt, nsteps)
    return misfit(traces(orc, levels, receivers), observed, dt)


def perturbed(problem: W.Problem, block: int, kind, i1: int, i2: int, eps: float) -> W.Problem:
    """Copy of problem with rho (kind == 'rho'), pair entry P (kind == P) or Voigt entry V
    (kind == ("voigt", V)) at one node moved by eps."""
    blocks = list(problem.blocks)
    b = blocks[block]
    if kind == "rho":
        rho = b.rho.copy()
        rho[i2, i1] += eps
        blocks[block] = dataclasses.replace(b, rho=rho)
    else:
        C = b.C.copy()
        C[..., i2, i1] += eps * W.pair10_to_tensor(_unit_matrix(kind)[:, :, None, None])[..., 0, 0]
        blocks[block] = dataclasses.replace(b, C=C)
    return dataclasses.replace(problem, blocks=blocks)
