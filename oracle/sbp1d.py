"""1-D diagonal-norm summation-by-parts operators (Sec. 4, 4.1) -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

First derivative (Sec. 4): a diagonal norm H_x = h diag(h_1, ..., h_nb, 1, ..., 1, h_nb, ..., h_1)
and D_x with H_x D_x = -D_x^T H_x - e_0 e_0^T + e_N e_N^T, a repeating central interior stencil
of order 2q and boundary rows exact for polynomials of degree <= q (the Mattsson-Nordstrom
operators the paper cites).  The paper does not print the coefficients, so they are derived
here from exactly those defining conditions by an exact rational solve.  Writing
Q = h H_x D_x, the conditions are linear in the unknown norm weights and the unknown entries
of Q's boundary block.  Order 2 and 4 have a unique solution; order 6 has one free parameter,
fixed by Q[4,5] = 342523/518400 (the choice that gives the published rational operator).

Second derivative (Sec. 4, 4.1): the fully compatible narrow operator
    H_x D_xx^FC(b) = -D_x^T H_x b D_x - R_xx(b) - e_0 e_0^T b D_x + e_N e_N^T b D_x,
with R_xx(b) = sum_alpha c_alpha h^(2 alpha - 2) D_alpha^T H_alpha B_alpha(b) D_alpha (Sec. 4 structure,
D_alpha = undivided alpha-th difference / h^alpha on the rows where it fits, H_alpha the norm at the
stencil centre, B_alpha(b) a convex average of b around the centre, alpha = q+1 .. 2q).  The c_alpha and
averages are the ones for which the interior row of D_xx^FC collapses to a (2q+1)-point stencil in u
and equals the textbook central 2q-order stencil for constant b (reading (ii) of the coefficient
question; Mattsson's own closures are not in the paper).
"""
from __future__ import annotations

from fractions import Fraction as Fr
from math import comb

import numpy as np
import scipy.sparse as sp

# boundary block shape (rows, cols) of D_x for interior order 2q
BLOCK = {2: (1, 2), 4: (4, 6), 6: (6, 9)}
FREE_PARAM = {6: ((4, 5), Fr(342523, 518400))}

# R_xx(b) terms: alpha -> (c_alpha, averaging offsets of b around the centre)
#   even alpha: centre node c = s + alpha/2, weights over c+offsets
#   odd alpha : centre between c0 = s + (alpha-1)/2 and c0 + 1, offsets relative to c0
R_TERMS = {
    2: {2: (Fr(1, 4), [0])},
    4: {3: (Fr(1, 18), [0, 1]), 4: (Fr(1, 144), [0])},
    6: {4: (Fr(1, 80), [-1, 0, 1]), 5: (Fr(1, 600), [0, 1]), 6: (Fr(1, 3600), [0])},
}


def _solve_exact(rows, rhs, nunk):
    """Gaussian elimination over the rationals; returns one solution (raises if inconsistent
    or if the solution is not unique)."""
    A = [list(r) + [b] for r, b in zip(rows, rhs)]
    piv_cols = []
    r = 0
    for c in range(nunk):
        p = next((i for i in range(r, len(A)) if A[i][c] != 0), None)
        if p is None:
            continue
        A[r], A[p] = A[p], A[r]
        inv = 1 / A[r][c]
        A[r] = [v * inv for v in A[r]]
        for i in range(len(A)):
            if i != r and A[i][c] != 0:
                f = A[i][c]
                A[i] = [vi - f * vr for vi, vr in zip(A[i], A[r])]
        piv_cols.append(c)
        r += 1
    for i in range(r, len(A)):
        if A[i][nunk] != 0:
            raise ValueError("inconsistent SBP conditions")
    if len(piv_cols) != nunk:
        raise ValueError("SBP conditions leave free parameters")
    x = [Fr(0)] * nunk
    for i, c in enumerate(piv_cols):
        x[c] = A[i][nunk]
    return x


def central_coefficients(q):
    """a_1..a_q with sum_k a_k (u_{i+k} - u_{i-k}) exact for polynomials of degree 2q."""
    rows, rhs = [], []
    for p in range(1, 2 * q, 2):
        rows.append([2 * Fr(k) ** p for k in range(1, q + 1)])
        rhs.append(Fr(1) if p == 1 else Fr(0))
    return _solve_exact(rows, rhs, q)


def derive_first_derivative(order):
    """Return (hw, Q, a): norm weights hw[0..nb-1] (units of h), boundary block Q (nb x ncol)
    of h*H*D, and interior central coefficients a[0..q-1]."""
    q = order // 2
    nb, ncol = BLOCK[order]
    a = central_coefficients(q)
    # unknowns: hw_0..hw_{nb-1}, then S[i][j] for i < nb, i < j < ncol
    sidx = {}
    for i in range(nb):
        for j in range(i + 1, ncol):
            sidx[(i, j)] = nb + len(sidx)
    nunk = nb + len(sidx)
    npts = ncol + q + 2

    def qrow(i):
        """Q[i][j] for j in range(npts) as linear forms (coef vector, const)."""
        out = []
        for j in range(npts):
            v = [Fr(0)] * nunk
            const = Fr(0)
            if i < nb and j < ncol:
                if i == j:
                    const = Fr(-1, 2) if i == 0 else Fr(0)
                elif j > i:
                    v[sidx[(i, j)]] = Fr(1)
                else:
                    v[sidx[(j, i)]] = Fr(-1)
            elif i >= nb:
                k = j - i
                if 1 <= abs(k) <= q:
                    const = a[abs(k) - 1] * (1 if k > 0 else -1)
            out.append((v, const))
        return out

    rows, rhs = [], []
    # (i) interior rows reaching into the block: Q[i][j] = -Q[j][i]
    for i in range(nb, ncol):
        for j in range(nb):
            k = i - j
            target = -a[k - 1] if 1 <= k <= q else Fr(0)
            v = [Fr(0)] * nunk
            if (j, i) in sidx:
                v[sidx[(j, i)]] = Fr(-1)
                rows.append(v)
                rhs.append(target)
            elif target != 0:
                raise ValueError("block too narrow")
    # (ii) boundary rows exact for x^p, p = 0..q: sum_j Q[i][j] x_j^p = hw_i p x_i^(p-1)
    for i in range(nb):
        qi = qrow(i)
        for p in range(q + 1):
            v = [Fr(0)] * nunk
            const = Fr(0)
            for j, (cv, cc) in enumerate(qi):
                xp = Fr(j) ** p
                v = [x + y * xp for x, y in zip(v, cv)]
                const += cc * xp
            if p > 0:
                v[i] -= p * Fr(i) ** (p - 1)
            rows.append(v)
            rhs.append(-const)
    if order in FREE_PARAM:
        (i, j), val = FREE_PARAM[order]
        v = [Fr(0)] * nunk
        v[sidx[(i, j)]] = Fr(1)
        rows.append(v)
        rhs.append(val)
    x = _solve_exact(rows, rhs, nunk)
    hw = x[:nb]
    Q = [[Fr(0)] * ncol for _ in range(nb)]
    for i in range(nb):
        for j in range(ncol):
            if i == j:
                Q[i][j] = Fr(-1, 2) if i == 0 else Fr(0)
            elif j > i:
                Q[i][j] = x[sidx[(i, j)]]
            else:
                Q[i][j] = -x[sidx[(j, i)]]
    return hw, Q, a


_CACHE = {}


def tables(order):
    if order not in _CACHE:
        _CACHE[order] = derive_first_derivative(order)
    return _CACHE[order]


MIN_N = {2: 5, 4: 18, 6: 27}


class SBP1D:
    """H_x, D_x and the fully compatible D_xx^FC(b) for N nodes with spacing h."""

    def __init__(self, order: int, N: int, h: float):
        if order not in BLOCK:
            raise ValueError("order must be 2, 4 or 6")
        if N < MIN_N[order]:
            raise ValueError(f"need N >= {MIN_N[order]} for order {order}")
        self.order, self.N, self.h = order, N, h
        self.q = order // 2
        hw, Q, a = tables(order)
        nb, ncol = BLOCK[order]
        Hd = np.ones(N)
        Hd[:nb] = [float(v) for v in hw]
        Hd[N - nb:] = [float(v) for v in reversed(hw)]
        self.H = h * Hd
        D = np.zeros((N, N))
        for i in range(N):
            for k in range(1, self.q + 1):
                if 0 <= i + k < N:
                    D[i, i + k] = float(a[k - 1])
                if 0 <= i - k < N:
                    D[i, i - k] = -float(a[k - 1])
        for i in range(nb):
            D[i, :] = 0.0
            D[N - 1 - i, :] = 0.0
            for j in range(ncol):
                D[i, j] = float(Q[i][j] / hw[i])
                D[N - 1 - i, N - 1 - j] = -float(Q[i][j] / hw[i])
        self.D = sp.csr_matrix(D / h)
        Bd = np.zeros(N)
        Bd[0], Bd[-1] = -1.0, 1.0
        self.Bd = sp.diags(Bd)
        self.Hm = sp.diags(self.H)
        self.Hinv = sp.diags(1.0 / self.H)
        # R_xx pieces: for each alpha the undivided difference, centre norm and averaging map
        self.r_terms = []
        for alpha, (c_alpha, offs) in R_TERMS[order].items():
            nrow = N - alpha
            rows, cols, vals = [], [], []
            arows, acols, avals = [], [], []
            hc = np.zeros(nrow)
            for s in range(nrow):
                for t in range(alpha + 1):
                    rows.append(s)
                    cols.append(s + t)
                    vals.append((-1) ** (alpha - t) * comb(alpha, t))
                if alpha % 2 == 0:
                    c = s + alpha // 2
                    hc[s] = self.H[c]
                    for o in offs:
                        arows.append(s)
                        acols.append(c + o)
                        avals.append(1.0 / len(offs))
                else:
                    c0 = s + (alpha - 1) // 2
                    hc[s] = 0.5 * (self.H[c0] + self.H[c0 + 1])
                    for o in offs:
                        arows.append(s)
                        acols.append(c0 + o)
                        avals.append(1.0 / len(offs))
            Delta = sp.csr_matrix((vals, (rows, cols)), shape=(nrow, N))
            Avg = sp.csr_matrix((avals, (arows, acols)), shape=(nrow, N))
            self.r_terms.append((alpha, float(c_alpha), Delta, hc, Avg))

    def R(self, b):
        """R_xx(b) = sum_alpha c_alpha h^(2 alpha - 2) D_alpha^T H_alpha B_alpha(b) D_alpha, D_alpha = Delta/h^alpha."""
        out = sp.csr_matrix((self.N, self.N))
        for alpha, c_alpha, Delta, hc, Avg in self.r_terms:
            # h^(2a-2) * (Delta/h^a)^T diag(hc * Avg b) (Delta/h^a) = h^-2 Delta^T diag(...) Delta
            out = out + (c_alpha / self.h ** 2) * (Delta.T @ sp.diags(hc * (Avg @ b)) @ Delta)
        return out.tocsr()

    def Dxx_fc(self, b):
        """D_xx^FC(b) = H^-1 ( -D^T H b D - R(b) - e_0 e_0^T b D + e_N e_N^T b D )."""
        B = sp.diags(b)
        M = -self.D.T @ self.Hm @ B @ self.D - self.R(b) + self.Bd @ B @ self.D
        return (self.Hinv @ M).tocsr()
