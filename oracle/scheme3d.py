"""The SBP-SAT elastic operator of Sec. 4.3-4.7 and the boundary SATs of Sec. 5 in three
dimensions, on one curvilinear block -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper states the scheme for d dimensions; this module writes it out for d = 3 with the
same explicit sparse matrices as the 2-D oracle (``oracle.scheme``), node index
(i3 * N2 + i2) * N1 + i1:
  D_1 = I (x) I (x) D_x1,  D_2 = I (x) D_x2 (x) I,  D_3 = D_x3 (x) I (x) I,
  H = H_x3 (x) H_x2 (x) H_x1,  H_face(m) = product of the other two H's     (Sec. 4.3)
Metric (Sec. 3.3): G_iI = D_i X_I, J = det G, F = G^-1 (F_Ii), c_ijkl = J F_Ii C_IjKl F_Kk;
the surface factor of a face x_m = const is |a_p x a_q| with a_i = (G_i1, G_i2, G_i3) and
p, q the other two directions (eq. surfj_app_3d), and the outward normal is
n_I = J F_Im nu / |a_p x a_q| (nu = -1 on x_m = 0, +1 on x_m = 1).
Volume operator (Sec. 4.6): K_jl = sum_ik DD_ik(c_ijkl), DD_ii = D_xx^FC along direction i (the
narrow operator of Sec. 4.4), DD_ik = D_i c D_k for i != k.
Faces: 'traction' -- the Robin SAT of eq. sat_traction with U = 0, g = 0:
  J SAT_J = -H^-1 P_f nu c_mJkL D_k u_L;
'displacement' -- eq. dirichlet_ansatz with g = 0 and the penalty of Theorem 3 for d = 3:
  J SAT_J = H^-1 sum_L (T_LJ - Z_LJ)^T e_f J^ H_f u_L,  J^ Z_JL = beta d / h1 c_mJmL,
with P_f = e_f H_f e_f^T and h1 the first weight of H_x along the face normal.
Semidiscrete: rho J u'' = A u, so u'' = diag(1 / (rho J)) A u.  The symmetric form is diag(H) A.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .sbp1d import SBP1D

D_DIM = 3


def _diag(v):
    return sp.diags(np.asarray(v, dtype=float).ravel())


class Oracle3D:
    """Explicit sparse operator of one 3-D block (workloads.box3d.Block3D)."""

    def __init__(self, blk):
        self.blk = blk
        self.order = blk.order
        N1, N2, N3 = blk.N
        self.Ns = (N1, N2, N3)
        self.N = N1 * N2 * N3
        hs = blk.h if getattr(blk, "h", None) is not None else tuple(1.0 / (n - 1) for n in self.Ns)
        self.op = [SBP1D(blk.order, n, h) for n, h in zip(self.Ns, hs)]
        self.I = [sp.identity(n, format="csr") for n in self.Ns]
        self.Dr = [self.kr(i, self.op[i].D) for i in range(3)]
        self.Hvec = np.kron(self.op[2].H, np.kron(self.op[1].H, self.op[0].H))
        self.Hinv = _diag(1.0 / self.Hvec)
        # ---- metric (Sec. 3.3)
        X = [blk.X[I].ravel() for I in range(3)]
        G = np.empty((self.N, 3, 3))
        for i in range(3):
            for I in range(3):
                G[:, i, I] = self.Dr[i] @ X[I]
        J = np.linalg.det(G)
        if np.any(J <= 0):
            raise ValueError("non-positive Jacobian")
        self.G, self.J = G, J
        self.F = np.linalg.inv(G)                  # F[n, I, i] = (G^-1)_Ii
        Cn = blk.C.reshape(3, 3, 3, 3, self.N)
        # c_ijkl = J F_Ii C_IjKl F_Kk
        self.c = np.einsum("n,nIi,IjKln,nKk->ijkln", J, self.F, Cn, self.F)
        self.rho = blk.rho.ravel()
        self.w = 1.0 / (self.rho * J)
        # ---- faces
        i1, i2, i3 = np.meshgrid(np.arange(N1), np.arange(N2), np.arange(N3), indexing="ij")
        node = (i3 * N2 + i2) * N1 + i1
        self.faces = []
        for f in range(6):
            m, side = f // 2, f % 2
            nu = -1.0 if side == 0 else 1.0
            sl = [slice(None)] * 3
            sl[m] = 0 if side == 0 else self.Ns[m] - 1
            idx = node[tuple(sl)].ravel()
            p, q = [t for t in range(3) if t != m]
            Hf = np.ones(self.N)
            for t in (p, q):
                Hf = Hf * self.kvec(t, self.op[t].H)
            Hf = Hf[idx]
            cr = np.cross(G[idx, p, :], G[idx, q, :])
            Jhat = np.linalg.norm(cr, axis=1)
            n = J[idx][:, None] * self.F[idx, :, m] * nu / Jhat[:, None]
            P = sp.csr_matrix((Hf, (idx, idx)), shape=(self.N, self.N))
            self.faces.append(dict(m=m, nu=nu, idx=idx, Hf=Hf, Jhat=Jhat, n=n, P=P, h1=self.op[m].H[0]))
        self.A = self._assemble()

    # ------------------------------------------------------------------ tensor-product helpers
    def kr(self, i, A):
        """The 1-D matrix A (square or rectangular) acting along direction i of the 3-D grid."""
        I1, I2, I3 = self.I
        if i == 0:
            return sp.kron(I3, sp.kron(I2, A), format="csr")
        if i == 1:
            return sp.kron(I3, sp.kron(A, I1), format="csr")
        return sp.kron(A, sp.kron(I2, I1), format="csr")

    def kvec(self, i, v):
        """A 1-D vector along direction i spread over the grid."""
        o = [np.ones(n) for n in self.Ns]
        o[i] = np.asarray(v, dtype=float)
        return np.kron(o[2], np.kron(o[1], o[0]))

    # ------------------------------------------------------------------ operator pieces
    def narrow(self, i, b):
        """D_ii^FC(b) on every grid line of direction i (Sec. 4.4)."""
        op = self.op[i]
        Bm = _diag(b)
        Dk, Hk, Bd, Hinv = self.kr(i, op.D), self.kr(i, op.Hm), self.kr(i, op.Bd), self.kr(i, op.Hinv)
        R = sp.csr_matrix((self.N, self.N))
        for alpha, c_alpha, Delta, hc, Avg in op.r_terms:
            Dl, Al = self.kr(i, Delta), self.kr(i, Avg)
            hcl = self.kvec(i, hc)
            R = R + (c_alpha / op.h ** 2) * (Dl.T @ _diag(hcl * (Al @ b)) @ Dl)
        return Hinv @ (-Dk.T @ Hk @ Bm @ Dk - R + Bd @ Bm @ Dk)

    def DD(self, i, k, b):
        if i == k:
            return self.narrow(i, b)
        return self.Dr[i] @ _diag(b) @ self.Dr[k]

    def volume_operator(self):
        """3 x 3 blocks K[j][l] = sum_ik DD_ik(c_ijkl) (Sec. 4.6)."""
        K = [[None] * 3 for _ in range(3)]
        for j in range(3):
            for l in range(3):
                acc = sp.csr_matrix((self.N, self.N))
                for i in range(3):
                    for k in range(3):
                        acc = acc + self.DD(i, k, self.c[i, j, k, l])
                K[j][l] = acc.tocsr()
        return K

    def traction_rows(self, f):
        """T[J][L]: rows at face f give nu_i c_iJkL D_k = J^ n_I C_IJKL (D_K u_L) (eq. n-C_conversion)."""
        m, nu = self.faces[f]["m"], self.faces[f]["nu"]
        T = [[None] * 3 for _ in range(3)]
        for J in range(3):
            for L in range(3):
                acc = sp.csr_matrix((self.N, self.N))
                for k in range(3):
                    acc = acc + _diag(nu * self.c[m, J, k, L]) @ self.Dr[k]
                T[J][L] = acc.tocsr()
        return T

    def traction_transpose(self, f):
        """Tt[J][L] = sum_k D_k^T diag(nu c_mLkJ); applied to P_f w it gives (T_LJ)^T e_f J^ H_f w."""
        m, nu = self.faces[f]["m"], self.faces[f]["nu"]
        Tt = [[None] * 3 for _ in range(3)]
        for J in range(3):
            for L in range(3):
                acc = sp.csr_matrix((self.N, self.N))
                for k in range(3):
                    acc = acc + self.Dr[k].T @ _diag(nu * self.c[m, L, k, J])
                Tt[J][L] = acc.tocsr()
        return Tt

    def _assemble(self):
        K = self.volume_operator()
        M = [[K[j][l] for l in range(3)] for j in range(3)]
        beta, d = self.blk.beta, D_DIM
        for f, kind in enumerate(self.blk.faces):
            fc = self.faces[f]
            m, P = fc["m"], fc["P"]
            if kind == "open":
                continue                       # a crop edge: no SAT (oracle windows of a larger block)
            if kind == "traction":
                T = self.traction_rows(f)
                for J in range(3):
                    for L in range(3):
                        M[J][L] = M[J][L] - self.Hinv @ P @ T[J][L]
            elif kind == "displacement":
                Tt = self.traction_transpose(f)
                for J in range(3):
                    for L in range(3):
                        JZ = beta * d / fc["h1"] * self.c[m, J, m, L]
                        M[J][L] = M[J][L] + self.Hinv @ (Tt[J][L] @ P - P @ _diag(JZ))
            else:
                raise ValueError(kind)
        return sp.bmat(M, format="csr")

    # ------------------------------------------------------------------ layout and time stepping
    def pack(self, u):
        return np.asarray(u, dtype=float).reshape(3, -1).ravel()

    def unpack(self, vec):
        N1, N2, N3 = self.Ns
        return vec.reshape(3, N3, N2, N1)

    @property
    def wvec(self):
        return np.concatenate([self.w] * 3)

    @property
    def hvec(self):
        return np.concatenate([self.Hvec] * 3)

    def accel(self, u):
        """u'' = diag(1 / (rho J)) A u."""
        return self.unpack(self.wvec * (self.A @ self.pack(u)))

    def leapfrog(self, u_prev, u_cur, dt, nsteps):
        """u^{n+1} = 2 u^n - u^{n-1} + dt^2 diag(1 / (rho J)) A u^n (the scheme's time stepping, Sec. 7)."""
        a, b = self.pack(u_prev), self.pack(u_cur)
        w = self.wvec
        for _ in range(nsteps):
            a, b = b, 2 * b - a + dt * dt * (w * (self.A @ b))
        return self.unpack(a), self.unpack(b)

    def energy(self, u_prev, u_cur, dt):
        """Leapfrog energy: kinetic term of the centred velocity plus the strain energy of the two
        levels, (1/2)[ v^T M v - u_cur^T (HA) u_prev ],  v = (u_cur - u_prev)/dt, M = diag(H rho J)."""
        a, b = self.pack(u_prev), self.pack(u_cur)
        mass = np.concatenate([self.Hvec * self.rho * self.J] * 3)
        v = (b - a) / dt
        HA = self.hvec * (self.A @ a)
        return 0.5 * (v @ (mass * v) - b @ HA)

    def max_rate(self):
        """Largest |eigenvalue| of diag(1/(rho J)) A (a symmetric similarity of diag(H) A)."""
        import scipy.sparse.linalg as spla
        s = np.sqrt(self.wvec / self.hvec)
        Sym = _diag(s) @ (_diag(self.hvec) @ self.A) @ _diag(s)
        lam = spla.eigsh(Sym, k=1, which="LM", return_eigenvectors=False, tol=1e-8)
        return float(abs(lam[0]))

    def suggest_dt(self, cfl=0.9):
        """Leapfrog is stable for dt < 2 / sqrt(max rate)."""
        return cfl * 2.0 / np.sqrt(self.max_rate())
