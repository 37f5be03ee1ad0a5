"""Pins of the oracle's wide-stencil variant (Sec. 7.1: first-derivative SBP operators applied
twice, D_i c D_k for every i, k, with the narrow scheme's SATs): self-adjoint and negative
semidefinite like the narrow scheme; the difference from the narrow operator is exactly the
symmetric negative semidefinite remainder term that annihilates linear fields; and the paper's
comparison -- the narrow operator has the slightly larger spectral radius and is the more
accurate one."""
import dataclasses
import math

import numpy as np
import pytest
import scipy.sparse.linalg as sla

import workloads as W
from oracle.scheme import Oracle

NSMALL = {2: (12, 11), 4: (20, 19), 6: (28, 27)}
CASES = [
    (("robin",) * 4, False, False),
    (("displacement",) * 4, False, False),
    (("robin", "displacement", "displacement", "robin"), True, False),
    (("displacement", "robin", "robin", "displacement"), True, True),
]


def _wide(P):
    return dataclasses.replace(P, stencil="wide")


@pytest.mark.parametrize("order", (2, 4, 6))
@pytest.mark.parametrize("case", range(len(CASES)))
def test_wide_scheme_self_adjoint_and_negative_semidefinite(order, case):
    kinds, two, rev = CASES[case]
    P = _wide(W.random_problem(kinds=kinds, n=NSMALL[order], order=order, two_blocks=two, reversed_interface=rev))
    A = Oracle(P).symmetric_matrix().toarray()
    scale = np.abs(A).max()
    assert np.abs(A - A.T).max() / scale < 1e-14
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).max() < 1e-12 * scale


@pytest.mark.parametrize("order", (2, 4, 6))
def test_narrow_minus_wide_is_the_remainder_term(order):
    """H (A_narrow - A_wide) = -sum R(c) (the SATs are identical): symmetric, negative
    semidefinite, not zero, and zero on displacement fields linear in each block's reference
    coordinates (R acts along grid lines through differences of order >= q + 1 >= 2)."""
    P = W.random_problem(kinds=("robin", "displacement", "displacement", "robin"), n=NSMALL[order], order=order,
                         two_blocks=True)
    On, Ow = Oracle(P), Oracle(_wide(P))
    Dm = (On.symmetric_matrix() - Ow.symmetric_matrix()).toarray()
    scale = np.abs(On.symmetric_matrix().toarray()).max()
    assert np.abs(Dm).max() > 1e-3 * scale
    assert np.abs(Dm - Dm.T).max() < 1e-13 * scale
    assert np.linalg.eigvalsh(0.5 * (Dm + Dm.T)).max() < 1e-12 * scale
    for coef in ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.3, -0.7, 0.2)):
        refs = [W.ref_grid(b.N1, b.N2) for b in P.blocks]
        lin = [np.stack([coef[0] + coef[1] * x1 + coef[2] * x2, coef[2] - coef[0] * x1 + coef[1] * x2])
               for (x1, x2) in refs]
        v = On.pack(lin)
        assert np.abs(Dm @ v).max() < 1e-10 * scale * np.abs(v).max()


def test_wide_leapfrog_energy_conserved():
    P = _wide(W.random_problem(kinds=("robin", "displacement", "displacement", "robin"), n=NSMALL[4], order=4,
                               two_blocks=True))
    O = Oracle(P)
    dt = O.suggest_dt(0.3)
    u0 = O.pack(W.smooth_state(P, seed=4, amplitude=0.1))
    up, u = u0, u0
    E0 = None
    for _ in range(50):
        up2, u2, _ = O.leapfrog(up, u, 0.0, dt, 1, homogeneous=True)
        E = O.energy_leapfrog(up2, u2, dt)
        E0 = E if E0 is None else E0
        assert abs(E - E0) <= 1e-12 * abs(E0)
        up, u = up2, u2


def test_narrow_spectral_radius_slightly_larger():
    """Sec. 7.1: the spectral radius of the spatial operator is slightly larger for the narrow
    scheme than for the wide one, most so at second order (the paper: 5.34 / 1.28 / 1.23 % on its
    domain at h = 0.01; this domain and grid differ, so only the ordering is pinned)."""
    rel = {}
    for order in (2, 4, 6):
        P = W.mms_problem(31, order, kinds=("robin", "displacement", "robin", "displacement"), two_blocks=True)
        rho = {}
        for st, Q in (("narrow", P), ("wide", _wide(P))):
            O = Oracle(Q)
            M = O.A.multiply(O.wvec[:, None]).tocsr()
            rho[st] = abs(sla.eigs(M, k=1, which="LM", return_eigenvectors=False)[0])
        rel[order] = rho["narrow"] / rho["wide"] - 1
        assert 0 < rel[order] < 0.25, (order, rel[order])
    assert rel[2] > rel[4] and rel[2] > rel[6]


@pytest.mark.slow
def test_narrow_more_accurate_than_wide():
    """Sec. 7.1: with the same SATs, the narrow scheme is the more accurate one at every order
    (manufactured solution of Sec. 7.1, RK4 to T = 0.5)."""
    for order in (2, 4, 6):
        P = W.mms_problem(31, order, kinds=("robin", "displacement", "robin", "displacement"), two_blocks=True)
        errs = []
        for Q in (P, _wide(P)):
            O = Oracle(Q)
            dt = O.suggest_dt(0.25)
            n = int(math.ceil(0.5 / dt))
            dt = 0.5 / n
            u0 = O.pack([Q.exact(b, 0.0) for b in Q.blocks])
            v0 = O.pack([np.stack([-W.MMS_W[L] * np.cos(W.MMS_K[L, 0] * b.X[0] + W.MMS_K[L, 1] * b.X[1])
                                   for L in range(2)]) for b in Q.blocks])
            u, _, t = O.rk4(u0, v0, 0.0, dt, n)
            errs.append(O.l2_error(u, t))
        assert errs[1] > 2 * errs[0], (order, errs)
