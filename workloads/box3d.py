"""Seeded synthetic inputs for the 3-D operator: one curvilinear block of N1 x N2 x N3 nodes.

Like the rest of ``workloads`` this module only describes continuous problems (node coordinates,
density, stiffness, face kinds, states) and holds none of the SBP-SAT arithmetic.

Conventions
-----------
* Fields are numpy arrays of shape ``(N3, N2, N1)`` (x1 fastest); vector fields ``(3, N3, N2, N1)``.
* Faces are numbered 0: x1=0, 1: x1=1, 2: x2=0, 3: x2=1, 4: x3=0, 5: x3=1 (reference coordinates).
  A face is 'traction' (the Robin face of Sec. 5.1 with U = 0 and g = 0) or 'displacement'
  (Sec. 5.2 with g = 0); 'open' marks the cut edge of a crop (no SAT; oracle windows only).
* The stiffness is stored in full, ``C[I, J, K, L]`` of shape ``(3, 3, 3, 3, N3, N2, N1)`` (major
  symmetry; minor symmetry not assumed).  ``pair45`` packs it into the 45 entries of the upper
  triangle of the 9 x 9 pair matrix over (IJ) = 11, 12, 13, 21, ..., 33, the layout the C-ABI takes.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Tuple

import numpy as np

from . import SEED

VOIGT3 = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))    # Voigt index -> tensor pair


@dataclass
class Block3D:
    X: np.ndarray                     # (3, N3, N2, N1) physical coordinates X_1, X_2, X_3
    rho: np.ndarray                   # (N3, N2, N1)
    C: np.ndarray                     # (3, 3, 3, 3, N3, N2, N1)
    faces: Tuple[str, ...]            # six kinds, 'traction' or 'displacement'
    order: int = 6
    beta: float = 1.0                 # SAT penalty factor (beta = 1 in the paper)
    h: Optional[Tuple[float, float, float]] = None   # reference spacing; default 1/(N_i - 1)

    @property
    def shape(self) -> Tuple[int, int, int]:
        return self.X.shape[1:]

    @property
    def N(self) -> Tuple[int, int, int]:
        """(N1, N2, N3)."""
        return (self.X.shape[3], self.X.shape[2], self.X.shape[1])

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.X.shape[1:]))


def voigt6_to_tensor(cv: np.ndarray) -> np.ndarray:
    """3-D Voigt (6 x 6, order 11 22 33 23 13 12) to the full tensor C_IJKL (minor symmetric)."""
    idx = np.empty((3, 3), dtype=int)
    for v, (a, b) in enumerate(VOIGT3):
        idx[a, b] = idx[b, a] = v
    C = np.empty((3, 3, 3, 3) + cv.shape[2:], dtype=float)
    for I in range(3):
        for J in range(3):
            for K in range(3):
                for L in range(3):
                    C[I, J, K, L] = cv[idx[I, J], idx[K, L]]
    return C


def pair45(C: np.ndarray) -> np.ndarray:
    """(45, ...) upper triangle (row-major) of the 9 x 9 pair matrix M[3I+J, 3K+L] = C_IJKL."""
    M = C.reshape((9, 9) + C.shape[4:])
    return np.stack([M[p, q] for p in range(9) for q in range(p, 9)])


def tensor_from_pair45(P: np.ndarray) -> np.ndarray:
    M = np.empty((9, 9) + P.shape[1:], dtype=P.dtype)
    t = 0
    for p in range(9):
        for q in range(p, 9):
            M[p, q] = M[q, p] = P[t]
            t += 1
    return M.reshape((3, 3, 3, 3) + P.shape[1:])


def ref_grid3(N1: int, N2: int, N3: int):
    """Reference node coordinates (x1, x2, x3) on [0,1]^3, each (N3, N2, N1)."""
    g3, g2, g1 = np.meshgrid(np.linspace(0, 1, N3), np.linspace(0, 1, N2), np.linspace(0, 1, N1), indexing="ij")
    return g1, g2, g3


def _rotation(a, b, c):
    """Rotation matrix from three angles (z-y-z), for tilting a transversely isotropic medium."""
    def rz(t):
        return np.array([[np.cos(t), -np.sin(t), 0], [np.sin(t), np.cos(t), 0], [0, 0, 1]])

    def ry(t):
        return np.array([[np.cos(t), 0, np.sin(t)], [0, 1, 0], [-np.sin(t), 0, np.cos(t)]])
    return rz(a) @ ry(b) @ rz(c)


def rotate_tensor3(C: np.ndarray, R: np.ndarray) -> np.ndarray:
    """C'_IJKL = R_Ia R_Jb R_Kc R_Ld C_abcd with one constant rotation R."""
    return np.einsum("ia,jb,kc,ld,abcd...->ijkl...", R, R, R, R, C)


def _tti_basis(R):
    """pair45 images of the five Voigt patterns of tti_voigt, rotated by R: the stiffness is
    c11 B0 + c13 B1 + c33 B2 + c44 B3 + c66 B4 (c12 = c11 - 2 c66 is folded into B0, B4)."""
    pats = []
    for name in ("c11", "c13", "c33", "c44", "c66"):
        V = np.zeros((6, 6))
        if name == "c11":
            V[0, 0] = V[1, 1] = V[0, 1] = V[1, 0] = 1.0
        elif name == "c13":
            V[0, 2] = V[2, 0] = V[1, 2] = V[2, 1] = 1.0
        elif name == "c33":
            V[2, 2] = 1.0
        elif name == "c44":
            V[3, 3] = V[4, 4] = 1.0
        else:
            V[5, 5] = 1.0
            V[0, 1] = V[1, 0] = -2.0
        pats.append(pair45(rotate_tensor3(voigt6_to_tensor(V), R)))
    return np.array(pats)                         # (5, 45)


def material3_planes(N, seed=SEED, k0=0, k1=None, aniso=True):
    """Density (k, N2, N1) and stiffness pair45 (45, k, N2, N1) of the x3-planes k0 <= i3 < k1 of
    a smoothly varying, tilted transversely isotropic medium (SPD, minor symmetric); isotropic
    when ``aniso`` is False.  Planes can be made in chunks: the values do not depend on k0, k1."""
    N1, N2, N3 = N
    k1 = N3 if k1 is None else k1
    rng = np.random.default_rng([seed, 2])
    ph = rng.uniform(0, 2 * np.pi, 6)
    angles = rng.uniform(-0.6, 0.6, 3)
    x3 = np.linspace(0, 1, N3)[k0:k1][:, None, None]
    x2 = np.linspace(0, 1, N2)[None, :, None]
    x1 = np.linspace(0, 1, N1)[None, None, :]
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x1 + ph[0]) * np.cos(np.pi * x2 + ph[1]) + 0.1 * np.sin(np.pi * x3 + ph[2])
    vp = 2.0 + 0.3 * np.sin(np.pi * x2 + ph[3]) * np.cos(np.pi * x3 + ph[4])
    vs = 1.1 + 0.15 * np.cos(np.pi * x1 + ph[5])
    shape = (k1 - k0, N2, N1)
    rho = np.broadcast_to(rho, shape)
    vp = np.broadcast_to(vp, shape)
    vs = np.broadcast_to(vs, shape)
    eps, delta, gamma = (0.15, 0.08, 0.1) if aniso else (0.0, 0.0, 0.0)
    c33 = rho * vp ** 2
    c44 = rho * vs ** 2
    c11 = c33 * (1 + 2 * eps)
    c66 = c44 * (1 + 2 * gamma)
    c13 = np.sqrt(np.maximum((c33 - c44) * (2 * delta * c33 + c33 - c44), 0.0)) - c44
    B = _tti_basis(_rotation(*angles) if aniso else np.eye(3))
    moduli = np.stack([c11, c13, c33, c44, c66]).reshape(5, -1)
    P = (B.T @ moduli).reshape((45,) + shape)
    return np.ascontiguousarray(rho), P


def random_material3(N, seed=SEED, aniso=True):
    """Density (N3, N2, N1) and full stiffness C_IJKL of material3_planes over all planes."""
    rho, P = material3_planes(N, seed, aniso=aniso)
    return rho, tensor_from_pair45(P)


def block3_coords(N, seed=SEED, curved=True):
    """Node coordinates (3, N3, N2, N1) of the random block: curved_map3, or the plain box."""
    N1, N2, N3 = N
    if curved:
        return curved_map3(N1, N2, N3, np.random.default_rng([seed, 1]))
    x1, x2, x3 = ref_grid3(N1, N2, N3)
    return np.array([1.0 * x1, 1.2 * x2, 0.9 * x3])


def curved_map3(N1, N2, N3, rng, L=(1.0, 1.2, 0.9), amp=0.04):
    """Physical coordinates of a smoothly deformed box: X_I = L_I x_I plus low-mode bumps
    (a topography-like top face and gently curved sides)."""
    x1, x2, x3 = ref_grid3(N1, N2, N3)
    a = rng.uniform(-1, 1, 6) * amp
    X1 = L[0] * x1 + a[0] * np.sin(np.pi * x2) * np.sin(np.pi * x3) + a[1] * x1 * (1 - x1) * x2
    X2 = L[1] * x2 + a[2] * np.sin(np.pi * x1) * np.cos(np.pi * x3) + a[3] * x2 * (1 - x2) * x3
    topo = a[4] * np.sin(2 * np.pi * x1) * np.sin(np.pi * x2) + a[5] * np.cos(np.pi * x1 + 0.3) * x2
    X3 = L[2] * x3 + topo * x3
    return np.array([X1, X2, X3])


def random_block3(N=(12, 10, 9), order=6, faces=("traction", "displacement", "displacement", "traction",
                                                 "displacement", "traction"),
                  seed=SEED, curved=True, aniso=True, beta=1.0) -> Block3D:
    """A random curvilinear block with variable density and tilted transversely isotropic stiffness."""
    N1, N2, N3 = N
    X = block3_coords(N, seed, curved)
    rho, C = random_material3(N, seed, aniso)
    return Block3D(X=X, rho=rho, C=C, faces=tuple(faces), order=order, beta=beta)


def extrude_block(b2, N3: int, L3: float = 0.7, C33=None, C_out=None) -> Block3D:
    """A 2-D block (workloads.Block) extruded along X3 = L3 x3.  The 3-D stiffness keeps the 2-D
    in-plane tensor in its (1, 2) components and adds out-of-plane entries that do not couple
    in-plane motion to x3 (a monoclinic medium with the x3 = const mirror plane):
    C_33aa = C33[a], C_3a3b = C_out[a][b], everything with an odd number of 3's zero."""
    N2, N1 = b2.X.shape[1:]
    x3 = np.linspace(0, 1, N3)
    X = np.empty((3, N3, N2, N1))
    X[0] = b2.X[0][None]
    X[1] = b2.X[1][None]
    X[2] = (L3 * x3)[:, None, None]
    rho = np.broadcast_to(b2.rho, (N3, N2, N1)).copy()
    C = np.zeros((3, 3, 3, 3, N3, N2, N1))
    C[:2, :2, :2, :2] = b2.C[:, :, :, :, None]
    C33 = (1.3, 1.1, 3.0) if C33 is None else C33           # C_3311, C_3322, C_3333
    C_out = ((0.9, 0.1), (0.1, 0.8)) if C_out is None else C_out   # C_3a3b (a, b in-plane)
    for a in range(2):
        C[2, 2, a, a] = C[a, a, 2, 2] = C33[a]
    C[2, 2, 2, 2] = C33[2]
    for a in range(2):
        for b in range(2):
            v = C_out[a][b]
            # C_{3a3b} and every minor-symmetric twin (a3 3b, 3a b3, a3 b3)
            C[2, a, 2, b] = C[a, 2, 2, b] = C[2, a, b, 2] = C[a, 2, b, 2] = v
    return Block3D(X=X, rho=rho, C=C, faces=("traction",) * 6, order=6)


def smooth_state3(b: Block3D, seed=SEED, amplitude=1.0, nmodes=3):
    """A smooth random displacement (3, N3, N2, N1) of low Fourier modes."""
    N1, N2, N3 = b.N
    rng = np.random.default_rng(seed)
    x1, x2, x3 = ref_grid3(N1, N2, N3)
    u = np.zeros((3, N3, N2, N1))
    for c in range(3):
        for _ in range(nmodes):
            k = rng.uniform(0.5, 2.5, 3)
            ph = rng.uniform(0, 2 * np.pi, 3)
            u[c] += rng.normal() * np.sin(np.pi * k[0] * x1 + ph[0]) * np.sin(np.pi * k[1] * x2 + ph[1]) \
                * np.sin(np.pi * k[2] * x3 + ph[2])
    return amplitude * u


def random_state3(b: Block3D, seed=SEED):
    rng = np.random.default_rng(seed)
    N1, N2, N3 = b.N
    return rng.standard_normal((3, N3, N2, N1))


def bench_block3(n=(256, 256, 256), order=6, seed=SEED) -> Block3D:
    """The 3-D bench workload: a deformed box with topography on x3 = 1, tilted TTI medium with
    smooth heterogeneity, traction on the top face and displacement faces elsewhere."""
    return random_block3(N=n, order=order, faces=("displacement",) * 5 + ("traction",), seed=seed)


def crop_block3(b: Block3D, lo, hi) -> Block3D:
    """The nodes lo[i] <= i_i < hi[i] of ``b`` as a block of its own, keeping the spacing of ``b``.
    A face that cuts through ``b`` becomes 'open'; a face on the boundary of ``b`` keeps its kind."""
    N = b.N
    sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
    faces = []
    for f in range(6):
        m, side = f // 2, f % 2
        on_bdry = lo[m] == 0 if side == 0 else hi[m] == N[m]
        faces.append(b.faces[f] if on_bdry else "open")
    h = b.h if b.h is not None else tuple(1.0 / (n - 1) for n in N)
    return Block3D(X=b.X[(slice(None),) + sl].copy(), rho=b.rho[sl].copy(), C=b.C[(slice(None),) * 4 + sl].copy(),
                   faces=tuple(faces), order=b.order, beta=b.beta, h=h)


def random_block3_crop(N, lo, hi, order=6, faces=("displacement",) * 5 + ("traction",), seed=SEED,
                       curved=True, aniso=True, beta=1.0) -> Block3D:
    """crop_block3 of random_block3(N, ...) without forming the whole block's stiffness."""
    X = block3_coords(N, seed, curved)
    rho, P = material3_planes(N, seed, lo[2], hi[2], aniso)
    sl = (slice(lo[1], hi[1]), slice(lo[0], hi[0]))
    rho = rho[(slice(None),) + sl]
    C = tensor_from_pair45(P[(slice(None), slice(None)) + sl])
    full = Block3D(X=X[:, lo[2]:hi[2]][(slice(None), slice(None)) + sl], rho=rho, C=C, faces=tuple(faces),
                   order=order, beta=beta)
    out = []
    for f in range(6):
        m, side = f // 2, f % 2
        on_bdry = lo[m] == 0 if side == 0 else hi[m] == N[m]
        out.append(faces[f] if on_bdry else "open")
    full.faces = tuple(out)
    full.h = tuple(1.0 / (n - 1) for n in N)
    return full
