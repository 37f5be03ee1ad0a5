"""Generate ``sbp_tables.inc``: the SBP coefficient tables the CUDA kernels use.

Run at development time (needs sympy):  python paper_2003_12811_gb300/csrc/gen_tables.py
The output is committed, so building the library does not need sympy.

What is derived (Sec. 4 and 4.1 of Almquist & Dunham; coefficients are not printed there):
* D_x: diagonal norm H_x = h diag(hw_0, .., hw_{nb-1}, 1, ..), repeating central interior
  stencil of order 2q, boundary rows exact for degree <= q, SBP property
  H D + D^T H = diag(-1, 0, .., 0, 1).  Order 6 has one free parameter, fixed at
  Q[4][5] = 342523/518400 (h H D = Q).  Solved with sympy's linear solver.
* D_xx^FC(b) = D b D - H^-1 R(b) (the fully compatible form of the paper's SBP property), with
  R(b) = sum_alpha c_alpha h^-2 Delta_alpha^T diag(Hc_alpha * Avg_alpha b) Delta_alpha:
  Delta_alpha the undivided alpha-th difference on every row where it fits, Hc the norm weight at
  the stencil centre (mean of the two centre weights for odd alpha), Avg the centred convex
  average of b (order 2: alpha=2 -> b_c, c=1/4; order 4: alpha=3 -> mean of 2, c=1/18,
  alpha=4 -> b_c, c=1/144; order 6: alpha=4 -> mean of 3, c=1/80, alpha=5 -> mean of 2,
  c=1/600, alpha=6 -> b_c, c=1/3600).
* Tables emitted: the D boundary block, the norm weights, the closure rows of D_xx^FC(b) as
  sparse (u-column, b-column, coefficient) triples, and the interior row written through
  "edge weights": row i = sum_{m=1..q} E_m(i) (u_{i+m} - u_i) + E_m(i-m) (u_{i-m} - u_i),
  E_m(i) = sum_k e_{m,k} b_{i+k}.  For gradients with respect to b near an end: per node k the
  (row, u-column, coefficient) list of d(row)/d b_k, and per column k the non-zeros of D.
  Every FP64 table has an FP32 twin (suffix _F) holding exactly the values a cast of the FP64
  entry gives, so FP32 kernels read single-precision constants without converting them.
"""
import os
from math import comb

import sympy as sp

BLOCK = {2: (1, 2), 4: (4, 6), 6: (6, 9)}
RDEF = {
    2: [(2, sp.Rational(1, 4), [0])],
    4: [(3, sp.Rational(1, 18), [0, 1]), (4, sp.Rational(1, 144), [0])],
    6: [(4, sp.Rational(1, 80), [-1, 0, 1]), (5, sp.Rational(1, 600), [0, 1]), (6, sp.Rational(1, 3600), [0])],
}
NGEN = 48


def first_derivative(order):
    q = order // 2
    nb, ncol = BLOCK[order]
    a = sp.symbols("a1:%d" % (q + 1))
    sol = sp.solve([sum(2 * a[k - 1] * sp.Integer(k) ** p for k in range(1, q + 1)) - (1 if p == 1 else 0)
                    for p in range(1, 2 * q, 2)], a, dict=True)[0]
    acoef = [sol[x] for x in a]
    hs = sp.symbols("hw0:%d" % nb)
    S = {(i, j): sp.Symbol("s_%d_%d" % (i, j)) for i in range(nb) for j in range(i + 1, ncol)}

    def Q(i, j):
        if i < nb and j < ncol:
            if i == j:
                return sp.Rational(-1, 2) if i == 0 else sp.Integer(0)
            return S[(i, j)] if j > i else -S[(j, i)]
        if i >= nb:
            k = j - i
            if 1 <= abs(k) <= q:
                return acoef[abs(k) - 1] * (1 if k > 0 else -1)
        return sp.Integer(0)

    eqs = []
    for i in range(nb, ncol):
        for j in range(nb):
            k = i - j
            eqs.append(-S[(j, i)] - (-acoef[k - 1] if 1 <= k <= q else 0))
    for i in range(nb):
        for p in range(q + 1):
            lhs = sum(Q(i, j) * sp.Integer(j) ** p for j in range(ncol + q + 2))
            rhs = hs[i] * p * sp.Integer(i) ** (p - 1) if p > 0 else 0
            eqs.append(lhs - rhs)
    if order == 6:
        eqs.append(S[(4, 5)] - sp.Rational(342523, 518400))
    unknowns = list(hs) + list(S.values())
    sol = sp.solve(eqs, unknowns, dict=True)
    assert len(sol) == 1
    sol = sol[0]
    hw = [sp.Rational(sol[x]) for x in hs]
    Dq = [[sp.Rational(Q(i, j).subs(sol) / hw[i]) for j in range(ncol)] for i in range(nb)]
    for row in Dq:
        for v in row:
            assert v.is_Rational
    return hw, Dq, acoef


def full_D(order, N):
    hw, Dq, a = first_derivative(order)
    q = order // 2
    nb, ncol = BLOCK[order]
    D = sp.zeros(N, N)
    for i in range(N):
        for k in range(1, q + 1):
            if i + k < N:
                D[i, i + k] = a[k - 1]
            if i - k >= 0:
                D[i, i - k] = -a[k - 1]
    for i in range(nb):
        for j in range(N):
            D[i, j] = 0
            D[N - 1 - i, j] = 0
        for j in range(ncol):
            D[i, j] = Dq[i][j]
            D[N - 1 - i, N - 1 - j] = -Dq[i][j]
    Hd = [sp.Integer(1)] * N
    for i in range(nb):
        Hd[i] = hw[i]
        Hd[N - 1 - i] = hw[i]
    return D, Hd, hw, Dq, a


def second_derivative_coeffs(order, N):
    """W[i][(j, k)] = coefficient of b_k u_j in row i of h^2 D_xx^FC(b)."""
    D, Hd, hw, Dq, a = full_D(order, N)
    W = [dict() for _ in range(N)]

    def add(i, j, k, v):
        if v != 0:
            W[i][(j, k)] = W[i].get((j, k), 0) + v

    # D b D
    for i in range(N):
        for m in range(N):
            if D[i, m] == 0:
                continue
            for j in range(N):
                if D[m, j] != 0:
                    add(i, j, m, D[i, m] * D[m, j])
    # - H^-1 R(b)
    for alpha, c_alpha, offs in RDEF[order]:
        for s in range(N - alpha):
            st = {s + t: (-1) ** (alpha - t) * comb(alpha, t) for t in range(alpha + 1)}
            if alpha % 2 == 0:
                c = s + alpha // 2
                hc = Hd[c]
                avg = [(c + o, sp.Rational(1, len(offs))) for o in offs]
            else:
                c0 = s + (alpha - 1) // 2
                hc = (Hd[c0] + Hd[c0 + 1]) / 2
                avg = [(c0 + o, sp.Rational(1, len(offs))) for o in offs]
            for i, di in st.items():
                for j, dj in st.items():
                    for k, wk in avg:
                        add(i, j, k, -c_alpha * di * dj * hc * wk / Hd[i])
    for i in range(N):
        W[i] = {key: v for key, v in W[i].items() if v != 0}
    return W, hw, Dq, a


def analyse(order):
    N = NGEN
    q = order // 2
    W, hw, Dq, a = second_derivative_coeffs(order, N)
    mid = N // 2
    pattern = {(j - mid, k - mid): v for (j, k), v in W[mid].items()}

    def is_interior(i):
        shifted = {(j - i, k - i): v for (j, k), v in W[i].items()}
        return shifted == pattern

    nclos = 0
    while not is_interior(nclos):
        nclos += 1
    for i in range(nclos, N - nclos):
        assert is_interior(i), (order, i)
    # mirror symmetry of the closures
    for i in range(nclos):
        mirrored = {(N - 1 - j, N - 1 - k): v for (j, k), v in W[i].items()}
        assert mirrored == W[N - 1 - i], (order, i)
    # edge weights: coefficient of u_{i+m} in row i, as a function of b offsets
    edges = []
    for m in range(1, q + 1):
        e = {k: v for (j, k), v in pattern.items() if j == m}
        edges.append(e)
        em = {k: v for (j, k), v in pattern.items() if j == -m}
        # E_m(i - m) expressed around i must equal the coefficient of u_{i-m}
        assert {k - m: v for k, v in e.items()} == em, (order, m)
    # diagonal consistency: coefficient of u_i = -sum of off-diagonal coefficients
    diag = {k: v for (j, k), v in pattern.items() if j == 0}
    tot = {}
    for m, e in enumerate(edges, start=1):
        for k, v in e.items():
            tot[k] = tot.get(k, 0) - v
            tot[k - m] = tot.get(k - m, 0) - v
    assert {k: v for k, v in tot.items() if v != 0} == diag
    clos = [sorted(W[i].items()) for i in range(nclos)]
    # transposed views for the gradient with respect to b near the left end (node k < GS = nclos + q):
    # every (row, u-column, coefficient) with d(row of h^2 D_xx(b) u)/d b_k = sum coefficient * u_j,
    # and every (row, D[row][k] h) of the column k of D
    gs = nclos + q
    D, _, _, _, _ = full_D(order, N)
    gn, dt = [], []
    for k in range(gs):
        gn.append(sorted((i, j, v) for i in range(N) for (j, kk), v in W[i].items() if kk == k))
        dt.append([(r, D[r, k]) for r in range(N) if D[r, k] != 0])
    return dict(hw=hw, Dq=Dq, a=a, nclos=nclos, clos=clos, edges=edges, gs=gs, gn=gn, dt=dt)


def cnum(v):
    v = sp.Rational(v)
    return "(%d.0/%d.0)" % (v.p, v.q) if v.q != 1 else "%d.0" % v.p


def fnum(v):
    """The FP32 value a CUDA cast of the FP64 table entry produces (round to nearest), exactly."""
    import numpy as np
    f = np.float32(float(sp.Rational(v)))
    return "%sf" % np.format_float_scientific(f, unique=True, exp_digits=2) if f != 0 else "0.0f"


def table(out, typ, name, vals, dims):
    """Emit a double table and its FP32 twin (name_F)."""
    shape = "".join("[%d]" % d for d in dims)
    if len(dims) == 2:
        n = dims[1]
        body = ", ".join("{%s}" % ", ".join(cnum(v) for v in vals[r * n:(r + 1) * n]) for r in range(dims[0]))
        fbody = ", ".join("{%s}" % ", ".join(fnum(v) for v in vals[r * n:(r + 1) * n]) for r in range(dims[0]))
    else:
        body = ", ".join(cnum(v) for v in vals)
        fbody = ", ".join(fnum(v) for v in vals)
    out.append("SBP_TABLE double %s%s = {%s};" % (name, shape, body))
    out.append("SBP_TABLE float %s_F%s = {%s};" % (name, shape, fbody))


def emit():
    out = ["// Generated by gen_tables.py -- SBP coefficient tables (Sec. 4, 4.1). Do not edit.",
           "// included twice by sbp.cu: with SBP_TABLE = static __constant__ (device) and static const (host)", ""]
    for order in (2, 4, 6):
        t = analyse(order)
        nb, ncol = BLOCK[order]
        q = order // 2
        P = "SBP%d" % order
        out.append("// ---- interior order %d" % order)
        out.append("#define %s_Q %d" % (P, q))
        out.append("#define %s_NB %d" % (P, nb))
        out.append("#define %s_NCOL %d" % (P, ncol))
        out.append("#define %s_NCLOS %d" % (P, t["nclos"]))
        table(out, "double", "%s_HW" % P.lower(), t["hw"], [nb])
        table(out, "double", "%s_A" % P.lower(), t["a"], [q])
        table(out, "double", "%s_DQ" % P.lower(), [v for r in t["Dq"] for v in r], [nb, ncol])
        starts, js, ks, cs = [0], [], [], []
        for row in t["clos"]:
            for (j, k), v in row:
                js.append(j)
                ks.append(k)
                cs.append(v)
            starts.append(len(js))
        out.append("SBP_TABLE int %s_CLOS_START[%d] = {%s};" % (P.lower(), len(starts), ", ".join(map(str, starts))))
        out.append("SBP_TABLE int %s_CLOS_J[%d] = {%s};" % (P.lower(), len(js), ", ".join(map(str, js))))
        out.append("SBP_TABLE int %s_CLOS_K[%d] = {%s};" % (P.lower(), len(ks), ", ".join(map(str, ks))))
        table(out, "double", "%s_CLOS_C" % P.lower(), cs, [len(cs)])
        # columns 0 .. NCLOSJ-1 hold every j and k of the closure triples
        out.append("#define %s_NCLOSJ %d" % (P, max(max(js), max(ks)) + 1))
        # edge weights as an inline device function
        out.append("// interior edge weights E_m(i) = sum_k e_{m,k} b_{i+k}; B(k) reads b_{i+k}")
        for m, e in enumerate(t["edges"], start=1):
            terms = " + ".join("T(%s) * B(%d)" % (cnum(v), k) for k, v in sorted(e.items()))
            out.append("#define %s_E%d(B) (%s)" % (P, m, terms))
        # gradient tables: node k < GS from the left end (the right end is the mirror image, with
        # the sign of D flipped)
        out.append("#define %s_GS %d" % (P, t["gs"]))
        for name, tab in (("GN", t["gn"]), ("DT", t["dt"])):
            starts, rows, js, cs = [0], [], [], []
            for ent in tab:
                for e in ent:
                    rows.append(e[0])
                    if name == "GN":
                        js.append(e[1])
                    cs.append(e[-1])
                starts.append(len(rows))
            out.append("SBP_TABLE int %s_%s_START[%d] = {%s};" % (P.lower(), name, len(starts), ", ".join(map(str, starts))))
            out.append("SBP_TABLE int %s_%s_ROW[%d] = {%s};" % (P.lower(), name, len(rows), ", ".join(map(str, rows))))
            if name == "GN":
                out.append("SBP_TABLE int %s_GN_J[%d] = {%s};" % (P.lower(), len(js), ", ".join(map(str, js))))
            table(out, "double", "%s_%s_C" % (P.lower(), name), cs, [len(cs)])
        lo = min(min(e) for e in t["edges"])
        hi = max(max(e) for e in t["edges"])
        out.append("#define %s_ELO %d" % (P, lo))
        out.append("#define %s_EHI %d" % (P, hi))
        out.append("")
    return "\n".join(out) + "\n"


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "sbp_tables.inc"), "w") as fh:
        fh.write(emit())
    print("wrote sbp_tables.inc")
