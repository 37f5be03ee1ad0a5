"""Pins of the oracle's 1-D SBP operators (Sec. 4, 4.1) against the defining identities,
published coefficient values, textbook special cases and polynomial exactness."""
import json
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle.sbp1d import SBP1D, tables, BLOCK

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ORDERS = (2, 4, 6)


def _op(order, N=41):
    return SBP1D(order, N, 1.0 / (N - 1))


@pytest.mark.parametrize("order", ORDERS)
def test_published_norm_and_first_row(order):
    gold = json.load(open(os.path.join(GOLD, "sbp_published.json")))[str(order)]
    hw, Q, a = tables(order)
    assert [Fr(s) for s in gold["norm"]] == list(hw)
    row0 = [Q[0][j] / hw[0] for j in range(BLOCK[order][1])]
    assert [Fr(s) for s in gold["row0"]] == row0


@pytest.mark.parametrize("order", ORDERS)
def test_first_derivative_sbp_identity(order):
    op = _op(order)
    D, H = op.D.toarray(), np.diag(op.H)
    Bd = np.zeros_like(D)
    Bd[0, 0], Bd[-1, -1] = -1, 1
    assert np.abs(H @ D + D.T @ H - Bd).max() < 1e-13


@pytest.mark.parametrize("order", ORDERS)
def test_first_derivative_accuracy(order):
    q = order // 2
    N = 41
    op = _op(order, N)
    x = np.linspace(0, 1, N)
    D = op.D.toarray()
    nb = BLOCK[order][0]
    for p in range(order + 1):
        err = np.abs(D @ x ** p - (p * x ** (p - 1) if p else 0 * x))
        if p <= q:
            assert err.max() < 1e-11, (p, err.max())
        assert err[nb:-nb].max() < 1e-10, (p, err[nb:-nb].max())
    # and NOT exact one degree beyond the interior order (the stencil really is order 2q)
    p = order + 1
    assert np.abs(D @ x ** p - p * x ** (p - 1))[nb:-nb].max() > 1e-10


def test_second_order_is_textbook():
    """Order 2 is fully specified: H = h diag(1/2, 1, .., 1/2), D = central, boundary rows (-1, 1)/h,
    and H D_xx^FC(b) = -M(b) - e_0 b_0 d_0^T + e_N b_N d_N^T with M the cell-average stiffness."""
    N = 9
    h = 1.0 / (N - 1)
    op = SBP1D(2, N, h)
    rng = np.random.default_rng(1)
    b = 1 + rng.random(N)
    Hx = h * np.array([0.5] + [1.0] * (N - 2) + [0.5])
    assert np.allclose(op.H, Hx, atol=0, rtol=1e-15)
    M = np.zeros((N, N))
    for i in range(N - 1):
        bb = 0.5 * (b[i] + b[i + 1]) / h
        M[i, i] += bb
        M[i + 1, i + 1] += bb
        M[i, i + 1] -= bb
        M[i + 1, i] -= bb
    d0 = np.zeros(N)
    d0[:2] = [-1 / h, 1 / h]
    dN = np.zeros(N)
    dN[-2:] = [-1 / h, 1 / h]
    ref = -M
    ref[0] -= b[0] * d0
    ref[-1] += b[-1] * dN
    got = np.diag(op.H) @ op.Dxx_fc(b).toarray()
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("order", ORDERS)
def test_narrow_interior_constant_b_is_textbook(order):
    """For b = 1 the interior row is the (2q+1)-point central stencil of order 2q."""
    text = {2: [1, -2, 1], 4: [-1 / 12, 4 / 3, -5 / 2, 4 / 3, -1 / 12],
            6: [1 / 90, -3 / 20, 3 / 2, -49 / 18, 3 / 2, -3 / 20, 1 / 90]}[order]
    N = 41
    h = 1.0 / (N - 1)
    op = SBP1D(order, N, h)
    row = op.Dxx_fc(np.ones(N)).toarray()[N // 2] * h * h
    q = order // 2
    assert np.allclose(row[N // 2 - q:N // 2 + q + 1], text, atol=1e-12)
    assert np.abs(row[:N // 2 - q]).max() < 1e-14 and np.abs(row[N // 2 + q + 1:]).max() < 1e-14


@pytest.mark.parametrize("order", ORDERS)
def test_narrow_interior_variable_b_width(order):
    """Variable b: u-support of interior rows stays 2q+1 wide (narrow stencil)."""
    N = 45
    op = _op(order, N)
    rng = np.random.default_rng(3)
    b = 1 + rng.random(N)
    A = op.Dxx_fc(b).toarray()
    q = order // 2
    for i in range(15, N - 15):
        nz = np.nonzero(np.abs(A[i]) > 1e-9 * np.abs(A[i]).max())[0]
        assert nz.min() >= i - q and nz.max() <= i + q


@pytest.mark.parametrize("order", ORDERS)
def test_second_derivative_sbp_identity_and_R(order):
    """H D_xx^FC(b) + D^T H b D - B b D = -R(b), R symmetric positive semidefinite (Sec. 4, Lemma 1)."""
    N = 40
    op = _op(order, N)
    rng = np.random.default_rng(5)
    b = 0.5 + rng.random(N)
    D, H = op.D.toarray(), np.diag(op.H)
    Bd = np.zeros((N, N))
    Bd[0, 0], Bd[-1, -1] = -1, 1
    R = -(H @ op.Dxx_fc(b).toarray() + D.T @ H @ np.diag(b) @ D - Bd @ np.diag(b) @ D)
    assert np.abs(R - R.T).max() < 1e-12 * np.abs(R).max()
    assert np.linalg.eigvalsh(R).min() > -1e-12 * np.abs(R).max()
    assert np.abs(R - op.R(b).toarray()).max() < 1e-12 * np.abs(R).max()
    # R is zero to order 2q on smooth functions: u^T R v scales as h^(2q)
    vals = []
    for N in (41, 81):
        opn = _op(order, N)
        x = np.linspace(0, 1, N)
        bb = 1 + 0.3 * np.sin(2 * x)
        vals.append(np.sin(3 * x) @ opn.R(bb).toarray() @ np.cos(2 * x))
    rate = np.log2(abs(vals[0]) / abs(vals[1]))
    assert rate > order - 1.2


@pytest.mark.parametrize("order", ORDERS)
def test_second_derivative_accuracy(order):
    """Interior order 2q for variable b; boundary rows consistent to order q - 1 (adapted fully
    compatible operators, Sec. 4.1): check rates on a smooth (b, u)."""
    q = order // 2
    errs_int, errs_bnd = [], []
    for N in (41, 81):
        op = _op(order, N)
        x = np.linspace(0, 1, N)
        b = 1 + 0.5 * np.sin(3 * x)
        u = np.sin(2 * x + 0.3)
        ex = 1.5 * np.cos(3 * x) * 2 * np.cos(2 * x + 0.3) - b * 4 * np.sin(2 * x + 0.3)
        e = np.abs(op.Dxx_fc(b) @ u - ex)
        errs_int.append(e[12:-12].max())
        errs_bnd.append(e.max())
    assert np.log2(errs_int[0] / errs_int[1]) > order - 0.3
    assert np.log2(errs_bnd[0] / errs_bnd[1]) > q - 1 - 0.3


@pytest.mark.parametrize("order", ORDERS)
def test_second_derivative_exact_on_low_polynomials(order):
    """Constant b: exact on polynomials of degree <= q at every row (degree q - 1 would suffice)."""
    q = order // 2
    N = 40
    op = _op(order, N)
    x = np.linspace(0, 1, N)
    A = op.Dxx_fc(np.ones(N)).toarray()
    for p in range(q + 1):
        ex = p * (p - 1) * x ** max(p - 2, 0) if p >= 2 else 0 * x
        assert np.abs(A @ x ** p - ex).max() < 1e-8 * (1 + np.abs(A).max() * 1e-6)
