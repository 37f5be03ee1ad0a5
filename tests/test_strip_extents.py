"""The boundary-strip kernel stages, per tile, the strip of S = max(NCLOS, NCOL) nodes plus
HN = Q nodes across the face and HT = Q - LO (rounded up to 4) nodes along it, and applies the
closure rows of D_xx^FC as matrices NCLOSJ columns wide; the last band tile of a block stages the
window of the last 32 columns.  These extents (the compile-time constants of the coefficient
tables the kernels include) are checked here against the oracle's operators (Sec. 4, 4.1): for
every row, the nodes it reads through u and through b (D_xx^FC(b) is linear in b, so the b
columns of row i are the k with D_xx^FC(e_k)[i] != 0), and the columns of D."""
import os
import re

import numpy as np
import pytest

from oracle.sbp1d import SBP1D, BLOCK

TABLES = os.path.join(os.path.dirname(__file__), "..", "paper_2003_12811_gb300", "csrc", "sbp_tables.inc")
ORDERS = (2, 4, 6)
N = 48


def _consts(order):
    txt = open(TABLES).read()
    d = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define SBP%d_(\w+) (-?\d+)" % order, txt)}
    S = max(d["NCLOS"], d["NCOL"])
    return dict(d, S=S, HN=d["Q"], HT=(d["Q"] - d["ELO"] + 3) // 4 * 4)


def _reads(order):
    """reads[i] = sorted nodes row i of D_xx^FC(b) reads through u or b (random b > 0)."""
    op = SBP1D(order, N, 1.0 / (N - 1))
    b = 1 + np.random.default_rng(order).random(N)
    A = op.Dxx_fc(b).toarray()
    tol = 1e-12 * np.abs(A).max()
    reads = [set(np.nonzero(np.abs(A[i]) > tol)[0]) for i in range(N)]
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        Ak = op.Dxx_fc(e).toarray()
        for i in np.nonzero(np.abs(Ak).max(axis=1) > 1e-12 * np.abs(Ak).max())[0]:
            reads[i].add(k)
    return [sorted(r) for r in reads], op


@pytest.mark.parametrize("order", ORDERS)
def test_tables_match_the_oracle_block_sizes(order):
    c = _consts(order)
    nb, ncol = BLOCK[order]
    assert (c["NB"], c["NCOL"], c["Q"]) == (nb, ncol, order // 2)


@pytest.mark.parametrize("order", ORDERS)
def test_strip_rows_read_inside_the_staged_region(order):
    """Rows 0 .. S-1 (the strip) read nothing beyond S - 1 + HN; the mirrored end likewise."""
    c = _consts(order)
    reads, _ = _reads(order)
    for i in range(c["S"]):
        assert max(reads[i]) <= c["S"] - 1 + c["HN"], (i, reads[i])
        j = N - 1 - i
        assert min(reads[j]) >= N - c["S"] - c["HN"], (j, reads[j])


@pytest.mark.parametrize("order", ORDERS)
def test_closure_rows_fit_the_matrix_width_and_the_corner_window(order):
    """Closure rows (i < NCLOS) read only columns < NCLOSJ (the width of the precomputed closure
    matrices), and NCLOSJ <= 32, so the 32-column window of the last band tile holds them."""
    c = _consts(order)
    reads, _ = _reads(order)
    for i in range(c["NCLOS"]):
        assert max(reads[i]) < c["NCLOSJ"], (i, reads[i])
    assert c["NCLOSJ"] <= 32
    # the first row outside the closure is the interior stencil: it reaches no closer to the
    # boundary than i - (Q - LO)
    i = c["NCLOS"]
    assert min(reads[i]) >= i - (c["Q"] - c["ELO"])


@pytest.mark.parametrize("order", ORDERS)
def test_interior_rows_reach_at_most_the_halos(order):
    """Away from the ends a row reads i - (Q - LO) .. i + Q: inside HT behind and HN ahead (along
    a face the tile is staged HT on both sides)."""
    c = _consts(order)
    reads, _ = _reads(order)
    for i in range(c["NCLOS"], N - c["NCLOS"]):
        back, ahead = i - min(reads[i]), max(reads[i]) - i
        assert back <= c["Q"] - c["ELO"] <= c["HT"], (i, back)
        assert ahead <= max(c["Q"], c["EHI"]) <= c["HN"] <= c["HT"], (i, ahead)


@pytest.mark.parametrize("order", ORDERS)
def test_first_derivative_stays_inside_the_strip(order):
    """D (mixed terms, tractions): boundary rows read columns < NCOL <= S, interior rows i +- Q."""
    c = _consts(order)
    _, op = _reads(order)
    D = op.D.toarray()
    for i in range(N):
        nz = np.nonzero(np.abs(D[i]) > 1e-12 * np.abs(D).max())[0]
        if i < c["NB"]:
            assert nz.max() < c["NCOL"] <= c["S"]
        elif i >= N - c["NB"]:
            assert nz.min() >= N - c["NCOL"]
        else:
            assert nz.min() >= i - c["Q"] and nz.max() <= i + c["Q"]
