"""Pins of the oracle's velocity-dependent terms: the dissipative Robin term of the remark in Sec. 5.1
(T u + U u + V u' = g) and the super-grid layer dissipation of Sec. 7.3 (zero outside the layers,
H E symmetric negative semidefinite inside), on their own and in the time steppers."""
import numpy as np
import pytest

import workloads as W
from oracle.scheme import Oracle

NS = {2: (12, 11), 4: (20, 19), 6: (28, 27)}


def _damped_problem(order, V=True, sponge=True, seed=3):
    P = W.random_problem(kinds=("robin", "displacement", "robin", "robin"), n=NS[order], order=order,
                         two_blocks=True, seed=seed)
    rng = np.random.default_rng(seed)
    for b in P.blocks:
        for f, face in enumerate(b.faces):
            face.g = None
            if face.kind == "robin" and V:
                nf = b.N2 if f < 2 else b.N1
                a, c = 0.5 + rng.random(nf), 0.5 + rng.random(nf)
                bb = 0.4 * np.sqrt(a * c) * (2 * rng.random(nf) - 1)
                face.V = np.stack([a, bb, c])                     # symmetric positive definite
        if sponge:
            x1, x2 = W.ref_grid(b.N1, b.N2)
            b.sponge = 0.05 * np.clip((x1 - 0.6) / 0.4, 0, 1) ** 2   # a layer along the x1 = 1 side
    return P


@pytest.mark.parametrize("order", (2, 4, 6))
def test_robin_damping_leapfrog_energy_identity(order):
    """Leapfrog with the centred velocity in the Robin damping term loses exactly
    (1 / (4 dt)) |u^{n+1} - u^{n-1}|^2_{H Bv} of the leapfrog energy per step (homogeneous data)."""
    P = _damped_problem(order, V=True, sponge=False)
    O = Oracle(P)
    dt = O.suggest_dt(0.3)
    up = O.pack(W.smooth_state(P, seed=5, amplitude=0.1))
    u = up + dt * O.pack(W.smooth_state(P, seed=6, amplitude=0.1))
    E_prev = O.energy_leapfrog(up, u, dt)
    HB = O.hvec[:, None] * O.Bv.toarray()
    assert np.abs(HB - HB.T).max() < 1e-13 * np.abs(HB).max()
    assert np.linalg.eigvalsh(0.5 * (HB + HB.T)).min() > -1e-12 * np.abs(HB).max()
    for n in range(40):
        u_prev0 = up
        up, u, _ = O.leapfrog(up, u, 0.0, dt, 1, homogeneous=True)
        E = O.energy_leapfrog(up, u, dt)
        d = u - u_prev0
        loss = float(d @ (HB @ d)) / (4 * dt)
        assert loss >= 0
        assert abs((E_prev - E) - loss) <= 1e-11 * abs(E_prev), (n, E_prev - E, loss)
        E_prev = E


@pytest.mark.parametrize("order", (2, 4, 6))
def test_layer_dissipation_symmetric_psd_and_confined(order):
    P = _damped_problem(order, V=False, sponge=True)
    O = Oracle(P)
    assert O.Bs.nnz > 0 and O.Bv.nnz == 0
    HB = (O.hvec[:, None] * O.Bs.toarray())
    scale = np.abs(HB).max()
    assert np.abs(HB - HB.T).max() < 1e-14 * scale
    assert np.linalg.eigvalsh(0.5 * (HB + HB.T)).min() > -1e-13 * scale
    # nodes whose 3-point neighbourhoods see no layer carry no dissipation
    for b, bo in enumerate(O.bops):
        s = P.blocks[b].sponge
        near = np.zeros_like(s, dtype=bool)
        for d1 in (-2, -1, 0, 1, 2):
            near |= np.roll(s, d1, axis=1) > 0
        for d2 in (-2, -1, 0, 1, 2):
            near |= np.roll(s, d2, axis=0) > 0
        rows = O.offsets[b] + np.flatnonzero(~near.ravel())
        assert np.abs(O.Bs[rows]).max() == 0.0


def test_layer_damps_grid_scale_content():
    """Grid-scale content placed inside the layer loses its energy much faster with the layer's
    dissipation than without it (RK4, layer coefficient s = eta rho c h1 h2 / (32 h), eta = 0.5: a
    damping rate eta c / h of the grid-scale checkerboard), and with the layer the energy never
    grows."""
    energies = {}
    for on in (False, True):
        P = _damped_problem(4, V=False, sponge=True)
        for b in P.blocks:
            h1, h2 = b.spacing
            b.sponge = (0.5 * b.rho * 3.0 * h1 * h2 / (32 * min(h1, h2))) * (b.sponge > 0) * on
            for face in b.faces:
                if face.kind == "robin":
                    face.U = None
        O = Oracle(P)
        dt = O.suggest_dt(0.4)
        fields = []
        for b in P.blocks:
            x1, x2 = W.ref_grid(b.N1, b.N2)
            i1, i2 = np.meshgrid(np.arange(b.N1), np.arange(b.N2))
            bump = np.exp(-((x1 - 0.85) / 0.08) ** 2 - ((x2 - 0.5) / 0.2) ** 2)
            fields.append(np.stack([bump * (-1.0) ** (i1 + i2), bump * (-1.0) ** i1]) * 1e-3)
        u = O.pack(fields)
        v = 0 * u
        es = [O.energy_semidiscrete(u, v)]
        for _ in range(10):
            u, v, _ = O.rk4(u, v, 0.0, dt, 4)
            es.append(O.energy_semidiscrete(u, v))
        energies[on] = es
    assert energies[True][-1] < 0.5 * energies[False][-1], (energies[True][-1], energies[False][-1])
    assert all(b <= a * (1 + 1e-9) for a, b in zip(energies[True], energies[True][1:]))
