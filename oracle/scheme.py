"""Multi-dimensional SBP-SAT scheme for the 2-D anisotropic elastic wave equation -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Everything is an explicit sparse matrix over a block's nodes (x1 fastest, index i2*N1 + i1),
built from the 1-D operators by Kronecker products:
  D_1 = I (x) D_x1, D_2 = D_x2 (x) I, H = H_x2 (x) H_x1                    (Sec. 4.3)
Per block the scheme is  rho u_J'' = J^-1 [ DD_ik(c_iJkL) u_L + J SAT_J ] + f_J  (Sec. 5, eq.
semidiscrete_general with DD^Omega = J^-1 DD_ik(c), Theorem 1), so the oracle assembles the
global matrix A_glob with  (J * accel * rho) = A_glob u + data(t),  i.e.
  u'' = diag(1/(rho J)) (A_glob u + data(t)).
The paper's symmetric matrix (Sec. 7.2) is diag(H) A_glob.
"""
from __future__ import annotations

import math
from typing import List

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from .sbp1d import SBP1D

D_DIM = 2


def _diag(v):
    return sp.diags(np.asarray(v, dtype=float).ravel())


class BlockOps:
    """Operators, metric and transformed material of one block."""

    def __init__(self, blk: W.Block, order: int, stencil: str = "narrow"):
        self.blk = blk
        self.stencil = stencil
        self.N1, self.N2 = blk.N1, blk.N2
        self.N = self.N1 * self.N2
        h1, h2 = blk.spacing
        self.op = [SBP1D(order, self.N1, h1), SBP1D(order, self.N2, h2)]
        I1, I2 = sp.identity(self.N1, format="csr"), sp.identity(self.N2, format="csr")
        self.I1, self.I2 = I1, I2
        # reference first derivatives D_i (Sec. 4.3)
        self.Dr = [sp.kron(I2, self.op[0].D, format="csr"), sp.kron(self.op[1].D, I1, format="csr")]
        self.Hvec = np.kron(self.op[1].H, self.op[0].H)
        self.Hinv = _diag(1.0 / self.Hvec)
        # ---- numerical metric (Sec. 3.3): G[i][I] = D_i X_I approximates dX_I/dx_i = (F^-1)_iI
        X = [blk.X[0].ravel(), blk.X[1].ravel()]
        G = [[self.Dr[i] @ X[I] for I in range(2)] for i in range(2)]
        J = G[0][0] * G[1][1] - G[0][1] * G[1][0]            # J = det[(F^-1)_iI]
        if np.any(J <= 0):
            raise ValueError("non-positive Jacobian")
        self.G, self.J = G, J
        # F_Ii = (G^-1)_Ii
        self.F = [[G[1][1] / J, -G[0][1] / J], [-G[1][0] / J, G[0][0] / J]]
        # ---- transformed density and stiffness (eq. transf_density_stiffness)
        C = blk.C.reshape(2, 2, 2, 2, -1)
        F = self.F
        self.c = np.zeros((2, 2, 2, 2, self.N))
        for i in range(2):
            for j in range(2):
                for k in range(2):
                    for l in range(2):
                        s = 0.0
                        for I in range(2):
                            for K in range(2):
                                s = s + F[I][i] * C[I, j, K, l] * F[K][k]
                        self.c[i, j, k, l] = J * s
        self.rho = blk.rho.ravel()
        self.w = 1.0 / (self.rho * J)                         # 1/(rho J)
        # ---- faces (Sec. 3.2.2, 4.3)
        self.faces = []
        for f in range(4):
            m, side = f // 2, f % 2
            t = 1 - m
            nu = -1.0 if side == 0 else 1.0
            if f == 0:
                idx = np.arange(self.N2) * self.N1
            elif f == 1:
                idx = np.arange(self.N2) * self.N1 + self.N1 - 1
            elif f == 2:
                idx = np.arange(self.N1)
            else:
                idx = (self.N2 - 1) * self.N1 + np.arange(self.N1)
            Hf = self.op[t].H                                 # face quadrature H_{d omega_m}
            Jhat = np.sqrt(G[t][0][idx] ** 2 + G[t][1][idx] ** 2)     # |a_t| (eq. surfj_app_2d)
            n = [J[idx] * F[I][m][idx] * nu / Jhat for I in range(2)]  # Nanson
            P = sp.csr_matrix((Hf, (idx, idx)), shape=(self.N, self.N))   # e_f H_f e_f^T
            self.faces.append(dict(m=m, t=t, nu=nu, idx=idx, Hf=Hf, Jhat=Jhat, n=n, P=P,
                                   h1=self.op[m].H[0]))

    # ------------------------------------------------------------------ operator pieces
    def narrow(self, i, b):
        """D_ii^FC(b): the 1-D fully compatible operator on every grid line of direction i (Sec. 4.4)."""
        op = self.op[i]
        if i == 0:
            kr = lambda A: sp.kron(self.I2, A, format="csr")
        else:
            kr = lambda A: sp.kron(A, self.I1, format="csr")
        Bm = _diag(b)
        Dk, Hk, Bd, Hinv = kr(op.D), kr(op.Hm), kr(op.Bd), kr(op.Hinv)
        R = sp.csr_matrix((self.N, self.N))
        for alpha, c_alpha, Delta, hc, Avg in op.r_terms:
            Dl, Al = kr(Delta), kr(Avg)
            hcl = np.kron(np.ones(self.N2), hc) if i == 0 else np.kron(hc, np.ones(self.N1))
            R = R + (c_alpha / op.h ** 2) * (Dl.T @ _diag(hcl * (Al @ b)) @ Dl)
        return Hinv @ (-Dk.T @ Hk @ Bm @ Dk - R + Bd @ Bm @ Dk)

    def DD(self, i, k, b):
        """DD_ik(b) of eq. def_cd: narrow when i == k, D_i b D_k otherwise.  The wide-stencil variant
        (the comparison of Sec. 7.1) uses D_i b D_k for i == k as well."""
        if i == k and self.stencil == "narrow":
            return self.narrow(i, b)
        return self.Dr[i] @ _diag(b) @ self.Dr[k]

    def elastic_operator(self):
        """2x2 blocks K[j][l] = sum_{i,k} DD_ik(c_ijkl) (Sec. 4.6)."""
        K = [[None, None], [None, None]]
        for j in range(2):
            for l in range(2):
                acc = sp.csr_matrix((self.N, self.N))
                for i in range(2):
                    for k in range(2):
                        acc = acc + self.DD(i, k, self.c[i, j, k, l])
                K[j][l] = acc.tocsr()
        return K

    def traction_rows(self, f):
        """T[J][L]: N x N matrix whose face rows give J^ e_f^T T_JL = nu_i c_iJkL D_k (using eq. n-C_conversion)."""
        fc = self.faces[f]
        m, nu = fc["m"], fc["nu"]
        T = [[None, None], [None, None]]
        for J in range(2):
            for L in range(2):
                acc = sp.csr_matrix((self.N, self.N))
                for k in range(2):
                    acc = acc + _diag(nu * self.c[m, J, k, L]) @ self.Dr[k]
                T[J][L] = acc.tocsr()
        return T

    def traction_transpose(self, f):
        """Tt[J][L] = sum_k D_k^T diag(nu c_mLkJ): applied to P_f w gives (T_LJ)^T e_f J^ H_f w."""
        fc = self.faces[f]
        m, nu = fc["m"], fc["nu"]
        Tt = [[None, None], [None, None]]
        for J in range(2):
            for L in range(2):
                acc = sp.csr_matrix((self.N, self.N))
                for k in range(2):
                    acc = acc + self.Dr[k].T @ _diag(nu * self.c[m, L, k, J])
                Tt[J][L] = acc.tocsr()
        return Tt


def lagrange_weights(xs, x0):
    """Lagrange interpolation weights l_i(x0) on nodes xs."""
    w = np.ones(len(xs))
    for i in range(len(xs)):
        for j in range(len(xs)):
            if j != i:
                w[i] *= (x0 - xs[j]) / (xs[i] - xs[j])
    return w


def delta_1d(N, h, x0, q):
    """Discrete delta weights (reading of the Sec. 7.4 point source): the 2q nodes nearest x0
    (start = clamp(floor(x0/h) - q + 1, 0, N - 2q)), weights = Lagrange weights, so that
    sum_i w_i p(x_i) = p(x0) for polynomials of degree <= 2q - 1."""
    xi = x0 / h
    start = int(math.floor(xi)) - q + 1
    start = max(0, min(start, N - 2 * q))
    nodes = np.arange(start, start + 2 * q)
    return nodes, lagrange_weights(nodes * h, x0)


def ricker(t, alpha_p, t0):
    """W(t) = (1 - 2 pi^2 a^2 (t - t0)^2) exp(-pi^2 a^2 (t - t0)^2) (Sec. 7.4)."""
    s = (math.pi * alpha_p * (t - t0)) ** 2
    return (1 - 2 * s) * math.exp(-s)


class Oracle:
    """The full semidiscrete scheme of a multi-block problem (Sec. 5-6) plus time stepping."""

    def __init__(self, problem: W.Problem):
        self.problem = problem
        self.order = problem.order
        self.beta = problem.beta
        self.bops: List[BlockOps] = [BlockOps(b, problem.order, getattr(problem, "stencil", "narrow")) for b in problem.blocks]
        self.offsets = []
        off = 0
        for bo in self.bops:
            self.offsets.append(off)
            off += 2 * bo.N
        self.ndof = off
        self._assemble()

    # ------------------------------------------------------------------ layout helpers
    def pack(self, fields):
        return np.concatenate([np.asarray(u, dtype=float).reshape(2, -1).ravel() for u in fields])

    def unpack(self, vec):
        out = []
        for bo, off in zip(self.bops, self.offsets):
            out.append(vec[off:off + 2 * bo.N].reshape(2, bo.N2, bo.N1))
        return out

    def _sl(self, b, j):
        off = self.offsets[b] + j * self.bops[b].N
        return slice(off, off + self.bops[b].N)

    # ------------------------------------------------------------------ assembly
    def _assemble(self):
        nb = len(self.bops)
        # block matrix over (block, component)
        M = [[None] * (2 * nb) for _ in range(2 * nb)]

        def add(bu, J, bv, L, A):
            r, c = 2 * bu + J, 2 * bv + L
            M[r][c] = A if M[r][c] is None else (M[r][c] + A)

        basis = self.problem.time_basis
        K = len(basis)
        self.data_coef = np.zeros((K, self.ndof))    # harmonic data vectors
        d = D_DIM
        beta = self.beta
        for b, bo in enumerate(self.bops):
            Kop = bo.elastic_operator()
            for J in range(2):
                for L in range(2):
                    add(b, J, b, L, Kop[J][L])
            blk = bo.blk
            for f, face in enumerate(blk.faces):
                fc = bo.faces[f]
                m, P, idx = fc["m"], fc["P"], fc["idx"]
                if face.kind == "open":
                    continue
                if face.kind == "robin":
                    # J SAT_J = -H^-1 P_f ( nu_i c_iJkL D_k u_L + J^ U_JL u_L - J^ g_J )   (eq. sat_traction)
                    T = bo.traction_rows(f)
                    for J in range(2):
                        for L in range(2):
                            A = T[J][L]
                            if face.U is not None:
                                Uc = face.U[[0, 1, 2][J + L]] if (J, L) != (1, 0) else face.U[1]
                                Ufull = np.zeros(bo.N)
                                Ufull[idx] = fc["Jhat"] * Uc
                                A = A + _diag(Ufull)
                            add(b, J, b, L, -(bo.Hinv @ P @ A))
                        if face.g is not None:
                            for k in range(K):
                                gvec = np.zeros(bo.N)
                                gvec[idx] = fc["Jhat"] * face.g[J, k]
                                self.data_coef[k, self._sl(b, J)] += bo.Hinv @ (P @ gvec)
                elif face.kind == "displacement":
                    # J SAT_J = H^-1 sum_L (T_LJ - Z_LJ)^T e_f J^ H_f (u_L - g_L)       (eq. dirichlet_ansatz)
                    # with J^ Z_JL = beta d / h1 * nu_i c_iJkL nu_k = beta d / h1 * c_mJmL
                    Tt = bo.traction_transpose(f)
                    for J in range(2):
                        for L in range(2):
                            JZ = beta * d / fc["h1"] * bo.c[m, J, m, L]
                            A = bo.Hinv @ (Tt[J][L] @ P - P @ _diag(JZ))
                            add(b, J, b, L, A)
                            if face.g is not None:
                                for k in range(K):
                                    gvec = np.zeros(bo.N)
                                    gvec[idx] = face.g[L, k]
                                    self.data_coef[k, self._sl(b, J)] -= A @ gvec
                elif face.kind == "interface":
                    nbk, nf, rev = face.nbr
                    bv = self.bops[nbk]
                    fv = bv.faces[nf]
                    if len(fv["idx"]) != len(idx):
                        raise ValueError("non-conforming interface")
                    vidx = fv["idx"][::-1] if rev else fv["idx"]
                    # S maps neighbour node values onto this face's nodes (u's ordering)
                    S = sp.csr_matrix((np.ones(len(idx)), (idx, vidx)), shape=(bo.N, bv.N))
                    Tt = bo.traction_transpose(f)
                    Tu = bo.traction_rows(f)
                    Tv = bv.traction_rows(nf)
                    mv = fv["m"]
                    for J in range(2):
                        for L in range(2):
                            # J^ Z_JL = beta d/4 ( nu c nu^u / h1^u + nu c nu^v / h1^v )  (eq. after scheme_interface)
                            JZ = beta * d / 4 * (bo.c[m, J, m, L] / fc["h1"] + S @ bv.c[mv, J, mv, L] / fv["h1"])
                            Apen = bo.Hinv @ (-P @ _diag(JZ) + 0.5 * Tt[J][L] @ P)
                            # acts on the jump u_L - v_L
                            add(b, J, b, L, Apen)
                            add(b, J, nbk, L, -(Apen @ S))
                            # -1/2 H^-1 P ( J^ T^u u + J^ T^v v )
                            add(b, J, b, L, -0.5 * (bo.Hinv @ P @ Tu[J][L]))
                            add(b, J, nbk, L, -0.5 * (bo.Hinv @ P @ (S @ Tv[J][L])))
                else:
                    raise ValueError(face.kind)
            # body force: J f_J
            if blk.forcing is not None:
                for J in range(2):
                    for k in range(K):
                        self.data_coef[k, self._sl(b, J)] += bo.J * blk.forcing[J, k].ravel()
        for r in range(2 * nb):
            for c in range(2 * nb):
                if M[r][c] is None:
                    M[r][c] = sp.csr_matrix((self.bops[r // 2].N, self.bops[c // 2].N))
        self.A = sp.bmat(M, format="csr")
        self._assemble_damping()
        self.wvec = np.concatenate([np.concatenate([bo.w, bo.w]) for bo in self.bops])
        self.hvec = np.concatenate([np.concatenate([bo.Hvec, bo.Hvec]) for bo in self.bops])
        self.mass = np.concatenate([np.concatenate([bo.rho * bo.J * bo.Hvec] * 2) for bo in self.bops])
        # point sources: J f_J = dir_J * amp * W(t) * w1 w2 / H  (discrete delta, reading 8)
        self.src = []
        q = self.order // 2
        for s in self.problem.sources:
            bo = self.bops[s.block]
            n1, w1 = delta_1d(bo.N1, bo.op[0].h, s.x_ref[0], q)
            n2, w2 = delta_1d(bo.N2, bo.op[1].h, s.x_ref[1], q)
            vec = np.zeros((2, bo.N))
            for a, ia in enumerate(n1):
                for c_, ib in enumerate(n2):
                    node = ib * bo.N1 + ia
                    for J in range(2):
                        vec[J, node] += s.direction[J] * s.amplitude * w1[a] * w2[c_] / bo.Hvec[node]
            full = np.zeros(self.ndof)
            full[self.offsets[s.block]:self.offsets[s.block] + 2 * bo.N] = vec.ravel()
            self.src.append((full, s))

    def _assemble_damping(self):
        """Velocity-dependent terms, J-scaled as rho J u'' = A u - (Bv + Bs) u' + data:
        * Bv, the dissipative Robin term (remark of Sec. 5.1: T u + U u + V u' = g on a Robin face),
          from the SAT of eq. sat_traction with U replaced by V u': H^-1 P_f J^ V;
        * Bs, the super-grid layer dissipation (Sec. 7.3: E zero outside the layers, H E symmetric
          negative semidefinite inside; reading: fourth-order undivided-difference dissipation
          J E = -H^-1 sum_i Dt_i^T diag(s) Dt_i per component, Dt_i the undivided second difference
          along direction i at the nodes 1 .. N-2 of every grid line, s >= 0 the layer profile)."""
        nb = len(self.bops)
        Mv = [[None] * (2 * nb) for _ in range(2 * nb)]
        Ms = [[None] * (2 * nb) for _ in range(2 * nb)]
        for b, bo in enumerate(self.bops):
            blk = bo.blk
            for f, face in enumerate(blk.faces):
                if face.kind != "robin" or face.V is None:
                    continue
                fc = bo.faces[f]
                idx, P = fc["idx"], fc["P"]
                for J in range(2):
                    for L in range(2):
                        Vc = face.V[[0, 1, 2][J + L]] if (J, L) != (1, 0) else face.V[1]
                        Vfull = np.zeros(bo.N)
                        Vfull[idx] = fc["Jhat"] * Vc
                        A = bo.Hinv @ P @ _diag(Vfull)
                        r, c = 2 * b + J, 2 * b + L
                        Mv[r][c] = A if Mv[r][c] is None else Mv[r][c] + A
            if blk.sponge is not None:
                sfield = blk.sponge.ravel()
                K = sp.csr_matrix((bo.N, bo.N))
                for i in range(2):
                    N = bo.N1 if i == 0 else bo.N2
                    Dt = sp.diags([np.ones(N - 2), -2 * np.ones(N - 2), np.ones(N - 2)], [0, 1, 2], shape=(N - 2, N))
                    if i == 0:
                        Dl = sp.kron(bo.I2, Dt, format="csr")
                        cen = np.kron(np.arange(bo.N2) * bo.N1, np.ones(N - 2, dtype=int)) + np.tile(np.arange(1, N - 1), bo.N2)
                    else:
                        Dl = sp.kron(Dt, bo.I1, format="csr")
                        cen = np.kron(np.arange(1, N - 1) * bo.N1, np.ones(bo.N1, dtype=int)) + np.tile(np.arange(bo.N1), N - 2)
                    K = K + Dl.T @ _diag(sfield[cen]) @ Dl
                Bs = (bo.Hinv @ K).tocsr()
                for J in range(2):
                    Ms[2 * b + J][2 * b + J] = Bs
        for M in (Mv, Ms):
            for r in range(2 * nb):
                for c in range(2 * nb):
                    if M[r][c] is None:
                        M[r][c] = sp.csr_matrix((self.bops[r // 2].N, self.bops[c // 2].N))
        self.Bv = sp.bmat(Mv, format="csr")
        self.Bs = sp.bmat(Ms, format="csr")
        self.damped = self.Bv.nnz > 0 or self.Bs.nnz > 0

    # ------------------------------------------------------------------ semidiscrete scheme
    def data(self, t):
        out = self.data_coef.T @ W.eval_time_basis(self.problem.time_basis, t) if len(self.problem.time_basis) else np.zeros(self.ndof)
        for vec, s in self.src:
            out = out + vec * ricker(t, s.alpha_p, s.t0)
        return out

    def apply(self, u, t=None):
        """A_glob u (+ data(t) when t is given): the J-scaled operator plus SATs and sources."""
        r = self.A @ u
        if t is not None:
            r = r + self.data(t)
        return r

    def accel(self, u, t):
        return self.wvec * self.apply(u, t)

    def leapfrog(self, u_prev, u, t, dt, nsteps, homogeneous=False):
        """u^{n+1} = 2 u^n - u^{n-1} + dt^2 accel(u^n, t_n).  With velocity-dependent terms: the
        dissipative Robin term with the centred velocity (u^{n+1} - u^{n-1}) / (2 dt) (it acts on the
        two components of single face nodes, so the step solves a 2 x 2 system per face node), the
        layer dissipation with the backward velocity (u^n - u^{n-1}) / dt (explicit):
          (I + dt/2 W Bv) u^{n+1} = 2 u^n - u^{n-1} + dt^2 W (A u^n + data - Bs (u^n - u^{n-1}) / dt)
                                    + dt/2 W Bv u^{n-1}."""
        if self.damped:
            Mv = (sp.identity(self.ndof, format="csr") + 0.5 * dt * _diag(self.wvec) @ self.Bv).tocsc()
            lu = spla.splu(Mv)
        for n in range(nsteps):
            a = self.wvec * (self.A @ u) if homogeneous else self.accel(u, t)
            if not self.damped:
                u_prev, u = u, 2 * u - u_prev + dt * dt * a
            else:
                rhs = 2 * u - u_prev + dt * dt * a - dt * self.wvec * (self.Bs @ (u - u_prev)) \
                    + 0.5 * dt * self.wvec * (self.Bv @ u_prev)
                u_prev, u = u, lu.solve(rhs)
            t = t + dt
        return u_prev, u, t

    def rk4(self, u, v, t, dt, nsteps):
        """Classical RK4 on (u, v) (Sec. 7.1); v' = W (A u - (Bv + Bs) v + data)."""
        B = self.Bv + self.Bs

        def acc(uu, vv, tt):
            a = self.accel(uu, tt)
            return a - self.wvec * (B @ vv) if self.damped else a

        for n in range(nsteps):
            k1u, k1v = v, acc(u, v, t)
            k2u = v + 0.5 * dt * k1v
            k2v = acc(u + 0.5 * dt * k1u, k2u, t + 0.5 * dt)
            k3u = v + 0.5 * dt * k2v
            k3v = acc(u + 0.5 * dt * k2u, k3u, t + 0.5 * dt)
            k4u = v + dt * k3v
            k4v = acc(u + dt * k3u, k4u, t + dt)
            u = u + dt / 6 * (k1u + 2 * k2u + 2 * k3u + k4u)
            v = v + dt / 6 * (k1v + 2 * k2v + 2 * k3v + k4v)
            t = t + dt
        return u, v, t

    # ------------------------------------------------------------------ invariants
    def symmetric_matrix(self):
        """The paper's A = calH D^tot (Sec. 7.2) = diag(H) A_glob."""
        return (_diag(self.hvec) @ self.A).tocsr()

    def energy_leapfrog(self, u, u_next, dt):
        """E^{n+1/2} = 1/2 |u^{n+1} - u^n|^2_{rho J H} / dt^2 - 1/2 (u^{n+1})^T (H A_glob) u^n."""
        du = (u_next - u) / dt
        return 0.5 * np.dot(du, self.mass * du) - 0.5 * np.dot(u_next, self.hvec * (self.A @ u))

    def energy_semidiscrete(self, u, v):
        """E = 1/2 v^T rho J H v - 1/2 u^T (H A_glob) u (Sec. 7.2)."""
        return 0.5 * np.dot(v, self.mass * v) - 0.5 * np.dot(u, self.hvec * (self.A @ u))

    def l2_error(self, u, t):
        """sqrt(sum_blocks sum_J e_J^T (J H) e_J) against the exact solution (reading 9)."""
        s = 0.0
        for b, (bo, ub) in enumerate(zip(self.bops, self.unpack(u))):
            ex = self.problem.exact(bo.blk, t)
            e = (ub - ex).reshape(2, -1)
            s += np.sum(bo.J * bo.Hvec * (e[0] ** 2 + e[1] ** 2))
        return math.sqrt(s)

    # ------------------------------------------------------------------ time step (Sec. 7, a3)
    def vmax_nodes(self, nsample=720):
        """Largest quasi-P speed per node in the reference domain: max over directions xi of
        sqrt(lambda_max(xi_i c_ijkl xi_k) / (J rho)); sampled at nsample angles in [0, pi),
        refined by golden-section search around the best sample (reading 11)."""
        out = []
        for bo in self.bops:
            c = bo.c
            rj = bo.rho * bo.J

            def lam(th):
                x1, x2 = math.cos(th), math.sin(th)
                xs = (x1, x2)
                G = np.zeros((2, 2, bo.N))
                for j in range(2):
                    for l in range(2):
                        G[j, l] = sum(xs[i] * c[i, j, k, l] * xs[k] for i in range(2) for k in range(2))
                a, b_, d = G[0, 0], 0.5 * (G[0, 1] + G[1, 0]), G[1, 1]
                return 0.5 * (a + d) + np.sqrt(0.25 * (a - d) ** 2 + b_ * b_)

            ths = np.arange(nsample) * math.pi / nsample
            vals = np.stack([lam(t) for t in ths])
            best = np.argmax(vals, axis=0)
            lo = ths[best] - math.pi / nsample
            hi = ths[best] + math.pi / nsample
            gr = (math.sqrt(5) - 1) / 2
            # vectorised golden-section over nodes
            a_, b_ = lo.copy(), hi.copy()
            c_ = b_ - gr * (b_ - a_)
            d_ = a_ + gr * (b_ - a_)

            def lam_vec(th):
                x1, x2 = np.cos(th), np.sin(th)
                xs = (x1, x2)
                G = np.zeros((2, 2, bo.N))
                for j in range(2):
                    for l in range(2):
                        G[j, l] = sum(xs[i] * c[i, j, k, l] * xs[k] for i in range(2) for k in range(2))
                a, bb, d = G[0, 0], 0.5 * (G[0, 1] + G[1, 0]), G[1, 1]
                return 0.5 * (a + d) + np.sqrt(0.25 * (a - d) ** 2 + bb * bb)

            fc_, fd_ = lam_vec(c_), lam_vec(d_)
            for _ in range(40):
                left = fc_ > fd_
                b_ = np.where(left, d_, b_)
                a_ = np.where(left, a_, c_)
                nc = b_ - gr * (b_ - a_)
                nd = a_ + gr * (b_ - a_)
                fc_new, fd_new = lam_vec(nc), lam_vec(nd)
                c_, d_, fc_, fd_ = nc, nd, fc_new, fd_new
            lmax = np.maximum(np.maximum(fc_, fd_), vals.max(axis=0))
            out.append(np.sqrt(lmax / rj))
        return out

    def suggest_dt(self, cfl):
        """dt = CFL * min over nodes of h / v_max, h = min(h1, h2) of the block (Sec. 7)."""
        best = math.inf
        for bo, v in zip(self.bops, self.vmax_nodes()):
            h = min(bo.op[0].h, bo.op[1].h)
            best = min(best, float(np.min(h / v)))
        return cfl * best
