"""Seeded synthetic inputs for the 2-D anisotropic elastic wave problems.

This module is the ONLY code shared by the FP64 oracle (``oracle/``) and the CUDA path
(``paper_2003_12811_gb300``).  It describes continuous problems -- block geometry
(physical node coordinates), density and stiffness fields, boundary/interface topology,
boundary data, body forces, point sources and initial states -- and holds none of the
SBP-SAT method's arithmetic (no difference operators, metric terms, SATs or time
stepping).  Every random draw is seeded.

Conventions
-----------
* A block has ``N1 x N2`` nodes; fields are numpy arrays of shape ``(N2, N1)`` (x1 fastest).
* Faces are numbered 0: x1=0, 1: x1=1, 2: x2=0, 3: x2=1 (reference coordinates).  The
  tangential node index along faces 0/1 is i2, along faces 2/3 it is i1.
* The stiffness tensor is stored in full, ``C[I, J, K, L]`` of shape ``(2, 2, 2, 2, N2, N1)``
  (major symmetry C_IJKL = C_KLIJ; minor symmetry is NOT assumed, Sec. 3).
* Time-dependent data (boundary data g, body force f) is separable in time:
  ``value(t) = sum_k coef[k] * T_k(t)`` with the basis ``Problem.time_basis``, a list of
  ``(kind, omega)`` with kind 'sin' or 'cos'.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional, Tuple

import numpy as np

SEED = 2003_12811

FACE_NAMES = ("x1=0", "x1=1", "x2=0", "x2=1")


# ----------------------------------------------------------------------------- data types
@dataclass
class Face:
    """Boundary condition of one block face.

    kind: 'displacement' (Sec. 5.2), 'robin' (Sec. 5.1, traction when U = 0),
          'interface' (Sec. 6) or 'open' (a crop edge: no SAT; oracle windows only).
    U:    (3, Nf) physical Robin matrix entries (U11, U12, U22) per face node, or None (= 0).
    g:    (2, K, Nf) harmonic coefficients of the boundary data (displacement g_J for
          'displacement', physical traction data g_J for 'robin'), or None (= 0).
    nbr:  for 'interface': (block, face, reversed) -- node s of this face touches node
          s (or Nf-1-s when reversed) of the neighbour's face.
    """
    kind: str
    U: Optional[np.ndarray] = None
    g: Optional[np.ndarray] = None
    nbr: Optional[Tuple[int, int, bool]] = None
    V: Optional[np.ndarray] = None    # 'robin': (3, Nf) symmetric PSD damping V (V11, V12, V22) of T u + U u + V du/dt = g


@dataclass
class Block:
    X: np.ndarray                     # (2, N2, N1) physical coordinates X_1, X_2
    rho: np.ndarray                   # (N2, N1)
    C: np.ndarray                     # (2, 2, 2, 2, N2, N1)
    faces: List[Face]
    h: Optional[Tuple[float, float]] = None   # reference spacing; default 1/(N-1)
    origin: Tuple[int, int] = (0, 0)  # index of node (0,0) inside the uncropped block
    forcing: Optional[np.ndarray] = None      # (2, K, N2, N1) harmonic coefficients of f_J
    sponge: Optional[np.ndarray] = None       # (N2, N1) >= 0: super-grid layer dissipation coefficient s

    @property
    def N1(self) -> int:
        return self.X.shape[2]

    @property
    def N2(self) -> int:
        return self.X.shape[1]

    @property
    def spacing(self) -> Tuple[float, float]:
        if self.h is not None:
            return self.h
        return (1.0 / (self.N1 - 1), 1.0 / (self.N2 - 1))


@dataclass
class PointSource:
    """Point force f_J = dir_J * amplitude * W(t) * delta(X - X0) (Sec. 7.4), W = Ricker.

    x_ref is the source position in the reference coordinates of ``block`` ([0,1]^2)."""
    block: int
    x_ref: Tuple[float, float]
    direction: Tuple[float, float]
    amplitude: float
    alpha_p: float                    # Ricker peak frequency (Hz)
    t0: float


@dataclass
class Problem:
    name: str
    order: int                        # interior order 2q in {2, 4, 6}
    blocks: List[Block]
    time_basis: List[Tuple[str, float]] = field(default_factory=list)
    sources: List[PointSource] = field(default_factory=list)
    beta: float = 1.0                 # SAT penalty factor (Sec. 5.2, 6; beta = 1 in the paper)
    stencil: str = "narrow"           # 'narrow' (D_xx^FC, the paper's scheme) or 'wide' (D_i c D_i, Sec. 7.1)
    exact: Optional[Callable] = None  # exact solution u(block, t) -> (2, N2, N1), if known

    @property
    def n_nodes(self) -> int:
        return sum(b.N1 * b.N2 for b in self.blocks)


def eval_time_basis(basis, t: float) -> np.ndarray:
    return np.array([np.sin(w * t) if k == "sin" else np.cos(w * t) for (k, w) in basis])


def face_tangent_count(b: Block, f: int) -> int:
    return b.N2 if f < 2 else b.N1


def face_slice(f: int):
    """Index into a (N2, N1) array selecting face f in tangential order."""
    return {0: (slice(None), 0), 1: (slice(None), -1), 2: (0, slice(None)), 3: (-1, slice(None))}[f]


# ----------------------------------------------------------------------------- materials
def voigt_to_tensor(cv: np.ndarray) -> np.ndarray:
    """2-D Voigt (3x3: 1 <-> 11, 2 <-> 22, 3 <-> 12/21) to the full tensor C_IJKL.

    The result is a view of the 4x4 pair matrix M[2I+J, 2K+L] reshaped to (2, 2, 2, 2, ...)."""
    v = [0, 2, 2, 1]                       # pair index p = 2I+J -> Voigt index
    M = np.empty((4, 4) + cv.shape[2:], dtype=cv.dtype)
    for p in range(4):
        for q in range(4):
            M[p, q] = cv[v[p], v[q]]
    return M.reshape((2, 2, 2, 2) + cv.shape[2:])


def pair10_to_tensor(m: np.ndarray) -> np.ndarray:
    """Symmetric 4x4 pair matrix over (IJ) in order 11, 12, 21, 22 -> C_IJKL (Cosserat)."""
    return np.ascontiguousarray(m).reshape((2, 2, 2, 2) + m.shape[2:])


def rotate_tensor(C: np.ndarray, theta) -> np.ndarray:
    """C'_IJKL = R_Ia R_Jb R_Kc R_Ld C_abcd, R the rotation by theta (array or scalar),
    evaluated in pair form M' = Rp M Rp^T with Rp[2I+J, 2a+b] = R_Ia R_Jb."""
    c, s = np.cos(theta), np.sin(theta)
    R = [[c, -s], [s, c]]
    M = C.reshape((4, 4) + C.shape[4:])
    Rp = [[R[p // 2][a // 2] * R[p % 2][a % 2] for a in range(4)] for p in range(4)]
    T = [[sum(Rp[p][a] * M[a, b] for a in range(4)) for b in range(4)] for p in range(4)]
    out = np.empty(np.broadcast(M[0, 0], np.asarray(c)).shape, dtype=np.result_type(c, C))
    out = np.empty((4, 4) + out.shape, dtype=out.dtype)
    for p in range(4):
        for q in range(4):
            out[p, q] = sum(T[p][b] * Rp[q][b] for b in range(4))
    return out.reshape((2, 2, 2, 2) + out.shape[2:])


def vti_voigt(rho, vp, vs, eps, delta):
    """2-D (x1 horizontal, x2 vertical symmetry axis) VTI Voigt matrix from Thomsen parameters."""
    c33 = rho * vp ** 2
    c55 = rho * vs ** 2
    c11 = c33 * (1 + 2 * eps)
    c13 = np.sqrt(2 * delta * c33 * (c33 - c55) + (c33 - c55) ** 2) - c55
    cv = np.zeros((3, 3) + np.shape(rho))
    cv[0, 0] = c11
    cv[1, 1] = c33
    cv[0, 1] = cv[1, 0] = c13
    cv[2, 2] = c55
    return cv


def paper_mms_material(X1, X2):
    """Material of the convergence study (Sec. 7.1): rho and the Cosserat C_IJKL."""
    rho = 2 + np.sin((X1 + X2) / 2)
    C = np.zeros((2, 2, 2, 2) + np.shape(X1), dtype=np.result_type(X1, X2))
    for I in range(1, 3):
        for J in range(1, 3):
            for K in range(1, 3):
                for L in range(1, 3):
                    if I == K and J == L:
                        val = 8 + np.sin(I * X1 + J * X2) + 0.5 * np.sin(K * X1 - L * X2)
                    else:
                        val = (np.sin(I * X1 + J * X2) + np.sin(K * X1 + L * X2)) / 8 + \
                              (np.sin(I * X1 - J * X2) + np.sin(K * X1 - L * X2)) / 16
                    C[I - 1, J - 1, K - 1, L - 1] = val
    return rho, C


def random_material(shape, rng):
    """Random material of the self-adjointness test (Sec. 7.2): rho = 1 + U(0,1); the 10
    independent entries of C~ ~ U(0,1); +4 on the entries with I = K and J = L."""
    rho = 1 + rng.random(shape)
    m = np.zeros((4, 4) + tuple(shape))
    for a in range(4):
        for b in range(a, 4):
            m[a, b] = m[b, a] = rng.random(shape)
    for a in range(4):
        m[a, a] += 4
    return rho, pair10_to_tensor(m)


# ----------------------------------------------------------------------------- manufactured solution
MMS_K = np.array([[2.0, 3.0], [3.0, 2.0]])   # u_L = sin(k_L . X - omega_L t)  (Sec. 7.1)
MMS_W = np.array([1.0, 2.0])
MMS_BASIS = [("sin", 1.0), ("cos", 1.0), ("sin", 2.0), ("cos", 2.0)]


def mms_u(X1, X2, t):
    return np.stack([np.sin(MMS_K[L, 0] * X1 + MMS_K[L, 1] * X2 - MMS_W[L] * t) for L in range(2)])


def _harm_sin(a, L):
    """coefficients of sin(a - w_L t) on the basis MMS_BASIS -> (4, ...)"""
    out = np.zeros((4,) + np.shape(a))
    out[2 * L + 0] = -np.cos(a)      # sin(a)cos(wt) - cos(a)sin(wt)
    out[2 * L + 1] = np.sin(a)
    return out


def _harm_cos(a, L):
    out = np.zeros((4,) + np.shape(a))
    out[2 * L + 0] = np.sin(a)       # cos(a)cos(wt) + sin(a)sin(wt)
    out[2 * L + 1] = np.cos(a)
    return out


def mms_displacement_data(X1, X2):
    """(2, 4, ...) harmonic coefficients of u_J on the given points."""
    return np.stack([_harm_sin(MMS_K[J, 0] * X1 + MMS_K[J, 1] * X2, J) for J in range(2)])


def mms_traction_data(X1, X2, C, n):
    """(2, 4, ...) harmonic coefficients of tau_J = n_I C_IJKL d_K u_L; n (2, ...) exact normal."""
    out = np.zeros((2, 4) + np.shape(X1))
    for J in range(2):
        for L in range(2):
            coef = sum(n[I] * C[I, J, K, L] * MMS_K[L, K] for I in range(2) for K in range(2))
            out[J] += coef * _harm_cos(MMS_K[L, 0] * X1 + MMS_K[L, 1] * X2, L)
    return out


def mms_forcing(X1, X2, rho, C_fun):
    """(2, 4, N2, N1) harmonic coefficients of f_J = rho u_J'' - d_I(C_IJKL d_K u_L)
    for the manufactured solution; dC/dX by complex-step differentiation of C_fun."""
    eps = 1e-30
    C = C_fun(X1, X2)
    dC = [np.imag(C_fun(X1 + 1j * eps, X2 + 0j)) / eps, np.imag(C_fun(X1 + 0j, X2 + 1j * eps)) / eps]
    out = np.zeros((2, 4) + np.shape(X1))
    for J in range(2):
        for L in range(2):
            kL = MMS_K[L]
            S = sum(C[I, J, K, L] * kL[I] * kL[K] for I in range(2) for K in range(2))
            if J == L:
                S = S - rho * MMS_W[J] ** 2
            P = -sum(dC[I][I, J, K, L] * kL[K] for I in range(2) for K in range(2))
            a = kL[0] * X1 + kL[1] * X2
            out[J] += S * _harm_sin(a, L) + P * _harm_cos(a, L)
    return out


# ----------------------------------------------------------------------------- geometry helpers
def ref_grid(N1, N2, i1=None, i2=None):
    """Reference coordinates (x1, x2) of nodes, optionally of an index window."""
    i1 = np.arange(N1) if i1 is None else i1
    i2 = np.arange(N2) if i2 is None else i2
    x1 = i1 / (N1 - 1)
    x2 = i2 / (N2 - 1)
    return np.meshgrid(x1, x2)


# ----------------------------------------------------------------------------- config 1
def config1(N: int = 101, order: int = 4) -> Problem:
    """Single Cartesian block on [0,1]^2, constant anisotropic C (Voigt c11=4, c22=3, c33=1,
    c12=1, c13=0.2, c23=0.1), rho = 1, manufactured solution (Sec. 7.1), displacement SATs."""
    x1, x2 = ref_grid(N, N)
    X = np.stack([x1, x2])
    cv = np.array([[4.0, 1.0, 0.2], [1.0, 3.0, 0.1], [0.2, 0.1, 1.0]])
    C = voigt_to_tensor(cv.reshape(3, 3, 1, 1) * np.ones((1, 1, N, N)))
    rho = np.ones((N, N))
    Cfun = lambda a, b: voigt_to_tensor(cv.reshape(3, 3, 1, 1) * np.ones((1, 1) + np.shape(a)))
    faces = []
    for f in range(4):
        sl = face_slice(f)
        faces.append(Face("displacement", g=mms_displacement_data(X[0][sl], X[1][sl])))
    blk = Block(X=X, rho=rho, C=C, faces=faces, forcing=mms_forcing(X[0], X[1], rho, Cfun))
    return Problem("config1", order, [blk], time_basis=list(MMS_BASIS),
                   exact=lambda b, t, P=None: mms_u(X[0], X[1], t))


# ----------------------------------------------------------------------------- config 2
def _c2_map(x, y):
    bump = 0.05 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    return x + bump, y + bump


def c2_material(X1, X2):
    base = np.zeros((3, 3) + np.shape(X1), dtype=np.result_type(X1, X2, float))
    base[0, 0], base[1, 1], base[2, 2] = 4.0, 3.0, 1.0
    theta = (np.pi / 6) * np.sin(2 * np.pi * X1) * np.sin(2 * np.pi * X2)
    return rotate_tensor(voigt_to_tensor(base), theta)


def c2_rho(X1, X2):
    return 2 + np.sin(2 * np.pi * (X1 + X2)) * np.cos(np.pi * X1)


def config2(n: int = 801, order: int = 6, window=None, nbx: int = 2, nby: int = 2) -> Problem:
    """2x2 (nbx x nby) curvilinear blocks of n x n nodes on [0,1]^2 with X = x + 0.05 sin(2 pi x) sin(2 pi y) (1,1);
    C(X) = rotation by theta(X) = (pi/6) sin(2 pi X1) sin(2 pi X2) of diag Voigt (4, 3, 1);
    rho = 2 + sin(2 pi (X1+X2)) cos(pi X1) in [1, 3]; welded interfaces, traction on the outer
    faces with manufactured data; manufactured forcing.

    window: optional {block: (i1_lo, i1_hi, i2_lo, i2_hi)} crop (oracle sampling)."""
    blocks = []
    idx = lambda bx, by: by * nbx + bx
    for by in range(nby):
        for bx in range(nbx):
            b = idx(bx, by)
            i1 = np.arange(n)
            i2 = np.arange(n)
            if window is not None:
                if b not in window:
                    continue
                lo1, hi1, lo2, hi2 = window[b]
                i1, i2 = np.arange(lo1, hi1), np.arange(lo2, hi2)
            xi1, xi2 = ref_grid(n, n, i1, i2)
            x, y = (bx + xi1) / nbx, (by + xi2) / nby
            X1, X2 = _c2_map(x, y)
            X = np.stack([X1, X2])
            rho = c2_rho(X1, X2)
            C = c2_material(X1, X2)
            faces = []
            for f in range(4):
                sl = face_slice(f)
                on_real = _window_touches(window, b, f, n, n)
                outer = (f == 0 and bx == 0) or (f == 1 and bx == nbx - 1) or (f == 2 and by == 0) or (f == 3 and by == nby - 1)
                if not on_real:
                    faces.append(Face("open"))
                elif outer:
                    nrm = np.zeros((2,) + X1[sl].shape)
                    nrm[f // 2] = -1.0 if f % 2 == 0 else 1.0
                    faces.append(Face("robin", g=mms_traction_data(X1[sl], X2[sl], C[(slice(None),) * 4 + sl], nrm)))
                else:
                    nb_b = {0: idx(bx - 1, by), 1: idx(bx + 1, by), 2: idx(bx, by - 1), 3: idx(bx, by + 1)}[f]
                    nb_f = {0: 1, 1: 0, 2: 3, 3: 2}[f]
                    faces.append(Face("interface", nbr=(nb_b, nb_f, False)))
            blk = Block(X=X, rho=rho, C=C, faces=faces, h=(1.0 / (n - 1), 1.0 / (n - 1)),
                        origin=(int(i1[0]), int(i2[0])),
                        forcing=mms_forcing(X1, X2, rho, c2_material))
            blocks.append(blk)
    if window is not None:
        _remap_window_interfaces(blocks, sorted(window))
    return Problem("config2", order, blocks, time_basis=list(MMS_BASIS),
                   exact=lambda b, t, P=None: mms_u(b.X[0], b.X[1], t))


def _window_touches(window, b, f, N1, N2):
    if window is None:
        return True
    lo1, hi1, lo2, hi2 = window[b]
    return {0: lo1 == 0, 1: hi1 == N1, 2: lo2 == 0, 3: hi2 == N2}[f]


def _remap_window_interfaces(blocks, kept):
    """Renumber interface neighbours after cropping; drop interfaces to blocks not kept."""
    pos = {b: k for k, b in enumerate(kept)}
    for blk in blocks:
        for f, face in enumerate(blk.faces):
            if face.kind == "interface":
                nb, nf, rev = face.nbr
                if nb in pos:
                    face.nbr = (pos[nb], nf, rev)
                else:
                    blk.faces[f] = Face("open")


# ----------------------------------------------------------------------------- config 3
C3_W = 8.0     # km, width
C3_D = 8.0     # km, depth below the reference surface


def c3_topography(seed=SEED):
    rng = np.random.default_rng(seed)
    xs = rng.uniform(0.1, 0.9, 5) * C3_W
    amp = rng.uniform(0.03, 0.15, 5) * C3_D
    wid = rng.uniform(0.03, 0.10, 5) * C3_W
    return lambda x: sum(a * np.exp(-((x - c) / w) ** 2) for a, c, w in zip(amp, xs, wid))


def c3_tilt(seed=SEED):
    rng = np.random.default_rng(seed + 1)
    kx = rng.uniform(0.5, 2.0, 3) * 2 * np.pi / C3_W
    ky = rng.uniform(0.5, 2.0, 3) * 2 * np.pi / C3_D
    ph = rng.uniform(0, 2 * np.pi, 3)
    return lambda X1, X2: (np.pi / 6) * np.tanh(sum(np.sin(a * X1 + b * X2 + p) for a, b, p in zip(kx, ky, ph)) / 1.5)


C3_RHO, C3_VP, C3_VS = 2.3, 3.5, 2.0          # g/cm^3, km/s (Sec. 7.4 constant model)
C3_EPS, C3_DELTA = 0.2, 0.1


def c3_map(block, xi1, xi2, topo):
    """Transfinite interpolation (Sec. 7.4): uniform in X1; block 0 from the flat bottom to
    the interface y_I = D/2 + h/2, block 1 from y_I to the surface y_s = D + h."""
    X1 = C3_W * xi1
    hx = topo(X1)
    if block == 0:
        yb, yt = 0.0 * X1, C3_D / 2 + 0.5 * hx
    else:
        yb, yt = C3_D / 2 + 0.5 * hx, C3_D + hx
    return X1, yb + xi2 * (yt - yb)


def c3_material(X1, X2, tilt):
    cv = vti_voigt(C3_RHO * np.ones(np.shape(X1)), C3_VP, C3_VS, C3_EPS, C3_DELTA)
    return rotate_tensor(voigt_to_tensor(cv), tilt(X1, X2))


def config3(n1: int = 4001, n2: int = 2001, order: int = 6, window=None,
            robin_length: float = C3_D, f_peak: float = 8.0) -> Problem:
    """Topography model: 2 stacked curvilinear blocks of n1 x n2 nodes; surface y = D + h(x),
    h a sum of 5 seeded Gaussian hills (<= 15% of D); tilted VTI C (Thomsen eps=0.2,
    delta=0.1; seeded tilt field within +-30 deg); traction-free top; Robin
    U = (1/L) n C n on the other outer faces; vertical Ricker point force (8 Hz) at the surface."""
    topo, tilt = c3_topography(), c3_tilt()
    blocks = []
    for b in range(2):
        i1, i2 = np.arange(n1), np.arange(n2)
        if window is not None:
            if b not in window:
                continue
            lo1, hi1, lo2, hi2 = window[b]
            i1, i2 = np.arange(lo1, hi1), np.arange(lo2, hi2)
        xi1, xi2 = ref_grid(n1, n2, i1, i2)
        X1, X2 = c3_map(b, xi1, xi2, topo)
        X = np.stack([X1, X2])
        C = c3_material(X1, X2, tilt)
        rho = C3_RHO * np.ones_like(X1)
        faces = []
        for f in range(4):
            sl = face_slice(f)
            if not _window_touches(window, b, f, n1, n2):
                faces.append(Face("open"))
                continue
            if (b == 0 and f == 3) or (b == 1 and f == 2):
                faces.append(Face("interface", nbr=(1 - b, 5 - f, False)))
                continue
            if b == 1 and f == 3:
                faces.append(Face("robin"))          # traction-free surface
                continue
            nrm = np.zeros((2,) + X1[sl].shape)
            nrm[f // 2] = -1.0 if f % 2 == 0 else 1.0
            Cf = C[(slice(None),) * 4 + sl]
            nCn = np.einsum("i...,ijkl...,k...->jl...", nrm, Cf, nrm) / robin_length
            U = np.stack([nCn[0, 0], nCn[0, 1], nCn[1, 1]])
            faces.append(Face("robin", U=U))
        blocks.append(Block(X=X, rho=rho, C=C, faces=faces, h=(1.0 / (n1 - 1), 1.0 / (n2 - 1)),
                            origin=(int(i1[0]), int(i2[0]))))
    if window is not None:
        _remap_window_interfaces(blocks, sorted(window))
    srcs = []
    src_i1, src_i2 = 0.5 * (n1 - 1), float(n2 - 1)          # surface, mid-width, in block 1
    keep = window is None or (1 in window and window[1][0] <= src_i1 < window[1][1] - 1
                              and window[1][2] <= src_i2 < window[1][3])
    if keep:
        bidx = 1 if window is None else sorted(window).index(1)
        lo1, lo2 = (0, 0) if window is None else (window[1][0], window[1][2])
        xr = ((src_i1 - lo1) / (n1 - 1), (src_i2 - lo2) / (n2 - 1))
        srcs.append(PointSource(block=bidx, x_ref=xr, direction=(0.0, -1.0),
                                amplitude=1.0, alpha_p=f_peak, t0=1.0 / f_peak))
    return Problem("config3", order, blocks, sources=srcs)


# ----------------------------------------------------------------------------- small synthetic problems
def random_problem(kinds=("robin", "robin", "displacement", "robin"), n=(14, 12), order=4,
                   seed=SEED, curved=True, two_blocks=False, reversed_interface=False) -> Problem:
    """Small problem with the random material of Sec. 7.2 on a (mildly) curvilinear grid.
    With two_blocks, a second block sits to the right (interface along x1 = 1 of block 0)."""
    rng = np.random.default_rng(seed)
    blocks = []
    nblk = 2 if two_blocks else 1
    for b in range(nblk):
        N1, N2 = n
        x1, x2 = ref_grid(N1, N2)
        gx = 0.5 * (b + x1)
        gy = x2
        if reversed_interface and b == 1:
            gx, gy = 0.5 * (2 - x1), 1 - x2        # block 1 is rotated by 180 degrees
        if curved:
            bump = 0.04 * np.sin(np.pi * gx) * np.sin(np.pi * gy) + 0.03 * gx * gy
            X1 = gx + bump + 0.1 * gy * gy
            X2 = 0.8 * gy + 0.5 * bump + 0.05 * gx
        else:
            X1, X2 = gx, gy
        rho, C = random_material((N2, N1), rng)
        faces = [Face(k) for k in kinds]
        for f, face in enumerate(faces):
            if face.kind == "robin":
                Nf = N2 if f < 2 else N1
                a, c = rng.random(Nf), rng.random(Nf)
                face.U = np.stack([a + 0.5, 0.3 * (a - c), c + 0.5])
        blocks.append(Block(X=np.stack([X1, X2]), rho=rho, C=C, faces=faces))
    if two_blocks:
        if reversed_interface:
            blocks[0].faces[1] = Face("interface", nbr=(1, 1, True))
            blocks[1].faces[1] = Face("interface", nbr=(0, 1, True))
        else:
            blocks[0].faces[1] = Face("interface", nbr=(1, 0, False))
            blocks[1].faces[0] = Face("interface", nbr=(0, 1, False))
    return Problem("random", order, blocks)


def smooth_state(problem: Problem, seed=SEED, amplitude=1.0):
    """Seeded smooth displacement field per block (sum of low Fourier modes of X)."""
    rng = np.random.default_rng(seed + 7)
    k = rng.uniform(1.0, 4.0, (2, 3, 2))
    ph = rng.uniform(0, 2 * np.pi, (2, 3))
    out = []
    for b in problem.blocks:
        u = np.zeros((2, b.N2, b.N1))
        for J in range(2):
            for m in range(3):
                u[J] += amplitude * np.sin(k[J, m, 0] * b.X[0] + k[J, m, 1] * b.X[1] + ph[J, m]) / (m + 1)
        out.append(u)
    return out


def random_state(problem: Problem, seed=SEED):
    rng = np.random.default_rng(seed + 11)
    return [rng.standard_normal((2, b.N2, b.N1)) for b in problem.blocks]


def mms_problem(N: int, order: int, kinds=("displacement",) * 4, curved=True, two_blocks=False,
                material="paper") -> Problem:
    """Manufactured-solution problem (Sec. 7.1 solution and material) on one block, or on two
    blocks sharing an interface at reference x1 = 1 of block 0, on a smoothly curved grid."""
    nblk = 2 if two_blocks else 1
    blocks = []
    for b in range(nblk):
        x1, x2 = ref_grid(N, N)
        gx = (b + x1) / nblk
        gy = x2
        if curved:
            X1 = gx + 0.06 * np.sin(np.pi * gy) * np.sin(np.pi * gx)
            X2 = gy + 0.05 * np.sin(np.pi * gx) + 0.04 * gx * gy
        else:
            X1, X2 = gx, gy
        if material == "paper":
            rho, C = paper_mms_material(X1, X2)
            Cfun = lambda a, c: paper_mms_material(a, c)[1]
        else:
            cv = np.array([[4.0, 1.0, 0.2], [1.0, 3.0, 0.1], [0.2, 0.1, 1.0]])
            C = voigt_to_tensor(cv.reshape(3, 3, 1, 1) * np.ones((1, 1) + X1.shape))
            rho = np.ones_like(X1)
            Cfun = lambda a, c: voigt_to_tensor(cv.reshape(3, 3, 1, 1) * np.ones((1, 1) + np.shape(a)))
        faces = []
        for f in range(4):
            sl = face_slice(f)
            kind = kinds[f]
            if two_blocks and ((b == 0 and f == 1) or (b == 1 and f == 0)):
                faces.append(Face("interface", nbr=(1 - b, 1 - f, False)))
            elif kind == "displacement":
                faces.append(Face("displacement", g=mms_displacement_data(X1[sl], X2[sl])))
            else:
                # exact physical outward normal of the mapped face (from the exact mapping derivative)
                eps = 1e-30
                if f < 2:      # face along x2: tangent = dX/dgy
                    tx, ty = _mms_tangent(gx[sl], gy[sl], curved, along="y")
                    nrm = np.stack([ty, -tx]) * (-1.0 if f == 0 else 1.0)
                else:
                    tx, ty = _mms_tangent(gx[sl], gy[sl], curved, along="x")
                    nrm = np.stack([-ty, tx]) * (-1.0 if f == 2 else 1.0)
                nrm = nrm / np.sqrt(nrm[0] ** 2 + nrm[1] ** 2)
                faces.append(Face("robin", g=mms_traction_data(X1[sl], X2[sl], C[(slice(None),) * 4 + sl], nrm)))
        blocks.append(Block(X=np.stack([X1, X2]), rho=rho, C=C, faces=faces,
                            forcing=mms_forcing(X1, X2, rho, Cfun)))
    return Problem("mms", order, blocks, time_basis=list(MMS_BASIS),
                   exact=lambda blk, t, P=None: mms_u(blk.X[0], blk.X[1], t))


def _mms_tangent(gx, gy, curved, along):
    if not curved:
        return (np.ones_like(gx), np.zeros_like(gx)) if along == "x" else (np.zeros_like(gx), np.ones_like(gx))
    if along == "x":   # d/dgx of (X1, X2)
        return (1 + 0.06 * np.sin(np.pi * gy) * np.pi * np.cos(np.pi * gx),
                0.05 * np.pi * np.cos(np.pi * gx) + 0.04 * gy)
    return (0.06 * np.pi * np.cos(np.pi * gy) * np.sin(np.pi * gx), 1 + 0.04 * gx)


# ----------------------------------------------------------------------------- config 4 (served batch)
def _smooth_field(X1, X2, rng, nmodes=3, kmax=3.0):
    """Seeded smooth field in [0, 1]: normalised sum of low Fourier modes of X."""
    f = np.zeros_like(X1)
    for _ in range(nmodes):
        k1, k2 = rng.uniform(-kmax, kmax, 2) * np.pi
        f += np.sin(k1 * X1 + k2 * X2 + rng.uniform(0, 2 * np.pi))
    return 0.5 + 0.5 * f / nmodes


def _smooth_field_sep(g1, g2, rng, nmodes=3, kmax=3.0, out=None):
    """Seeded smooth field in [0, 1] on the tensor grid g1 (x1, along the row) x g2 (x2): the
    normalised sum 1/2 + 1/(2 nmodes) sum_j sin(k1_j x1 + k2_j x2 + phi_j) of low Fourier modes,
    each split as sin(k1 x1 + phi) cos(k2 x2) + cos(k1 x1 + phi) sin(k2 x2), so the field is one
    rank-(2 nmodes + 1) product of O(n) factors."""
    A = np.empty((g2.size, 2 * nmodes + 1))
    Bm = np.empty((2 * nmodes + 1, g1.size))
    for j in range(nmodes):
        k1, k2 = rng.uniform(-kmax, kmax, 2) * np.pi
        ph = rng.uniform(0, 2 * np.pi)
        A[:, 2 * j] = np.cos(k2 * g2) * (0.5 / nmodes)
        A[:, 2 * j + 1] = np.sin(k2 * g2) * (0.5 / nmodes)
        Bm[2 * j] = np.sin(k1 * g1 + ph)
        Bm[2 * j + 1] = np.cos(k1 * g1 + ph)
    A[:, -1] = 0.5
    Bm[-1] = 1.0
    if out is None:
        return A @ Bm
    np.matmul(A, Bm, out=out)
    return out


def shot_problem(side: int, seed: int, order: int = 6, f_peak: float = 4.0) -> Problem:
    """One served shot: a single curvilinear block side x side on a unit square perturbed by a
    seeded smooth mapping; smooth random material after the Sec. 7.2 recipe (rho = 1 + r,
    the 10 independent pair entries of C~ smooth in [0,1], +4 on I=K, J=L; the smooth fields are
    sums of low Fourier modes of the reference coordinates); traction-free top, displacement
    elsewhere; a vertical Ricker point force at a seeded interior point."""
    rng = np.random.default_rng(seed)
    g = np.linspace(0.0, 1.0, side)
    a1, a2 = rng.uniform(0.02, 0.05, 2)
    X1 = g[None, :] + a1 * np.multiply.outer(np.sin(2 * np.pi * g), np.sin(np.pi * g))
    X2 = g[:, None] + a2 * np.multiply.outer(np.sin(np.pi * g), np.sin(2 * np.pi * g))
    rho = 1 + _smooth_field_sep(g, g, rng)
    m = np.zeros((4, 4, side, side))
    for a in range(4):
        for b in range(a, 4):
            _smooth_field_sep(g, g, rng, out=m[a, b])
            if b != a:
                m[b, a] = m[a, b]
    for a in range(4):
        m[a, a] += 4
    C = pair10_to_tensor(m)
    faces = [Face("displacement"), Face("displacement"), Face("displacement"), Face("robin")]
    src = PointSource(block=0, x_ref=(float(rng.uniform(0.3, 0.7)), float(rng.uniform(0.3, 0.7))),
                      direction=(0.0, -1.0), amplitude=1.0, alpha_p=f_peak, t0=1.0 / f_peak)
    return Problem(f"shot{seed}", order, [Block(X=np.stack([X1, X2]), rho=rho, C=C, faces=faces)], sources=[src])


def config4_requests(nshots: int = 256, side_range=(201, 2001), rate: float = 1.0, seed: int = SEED,
                     steps_per_side: float = 2.0, step_multiple: int = 2):
    """Served batch: nshots requests with Poisson arrivals (rate per second), side lengths uniform
    in side_range, steps = steps_per_side * side (rounded up to step_multiple).  Returns a list of
    (arrival, problem, nsteps); problems are built lazily by calling the returned factory."""
    rng = np.random.default_rng(seed + 4)
    t = 0.0
    out = []
    for i in range(nshots):
        t += rng.exponential(1.0 / rate)
        side = int(rng.integers(side_range[0], side_range[1] + 1))
        n = int(np.ceil(steps_per_side * side / step_multiple) * step_multiple)
        out.append((t, side, seed + 100 + i, n))
    return out


# ----------------------------------------------------------------------------- misfit-gradient workload
def config5(n: int = 1001, order: int = 6, blob: bool = False, nrec: int = 64, seed: int = SEED,
            f_peak: float = 15.0):
    """Misfit-gradient workload: one curvilinear block n x n on a perturbed unit square; smooth
    tilted VTI stiffness (Thomsen eps = 0.2, delta = 0.1) and density 2.3 scaled by a smooth
    seeded field within +-10 %; with ``blob`` a Gaussian inclusion (radius 0.08, centre 0.3 below
    the surface) raises rho and C by 10 % at its centre.  Traction-free top, displacement (no data)
    elsewhere; a vertical Ricker point force 0.05 below the surface at mid-width; ``nrec`` receivers
    evenly spaced on the surface nodes.  Returns (problem, receivers) with receivers as
    (block, i1, i2) node indices."""
    rng = np.random.default_rng(seed + 5)
    x1, x2 = ref_grid(n, n)
    X1 = x1 + 0.03 * np.sin(np.pi * x1) * np.sin(2 * np.pi * x2)
    X2 = x2 + 0.02 * np.sin(2 * np.pi * x1) * np.sin(np.pi * x2)
    scale = 0.9 + 0.2 * _smooth_field(X1, X2, rng)
    tilt = (np.pi / 8) * (2 * _smooth_field(X1, X2, rng) - 1)
    if blob:
        cx, cy, r = 0.5, float(X2.max()) - 0.3, 0.08
        scale = scale * (1 + 0.1 * np.exp(-((X1 - cx) ** 2 + (X2 - cy) ** 2) / (2 * r * r)))
    rho = C3_RHO * scale
    cv = vti_voigt(rho, C3_VP, C3_VS, C3_EPS, C3_DELTA)
    C = rotate_tensor(voigt_to_tensor(cv), tilt)
    faces = [Face("displacement"), Face("displacement"), Face("displacement"), Face("robin")]
    src = PointSource(block=0, x_ref=(0.5, 0.95), direction=(0.0, -1.0), amplitude=1.0,
                      alpha_p=f_peak, t0=1.0 / f_peak)
    prob = Problem("config5" + ("_blob" if blob else ""), order,
                   [Block(X=np.stack([X1, X2]), rho=rho, C=C, faces=faces)], sources=[src])
    idx = np.unique(np.round(np.linspace(0.05, 0.95, nrec) * (n - 1)).astype(int))
    receivers = [(0, int(i), n - 1) for i in idx]
    return prob, receivers
