"""ctypes binding of libsbp (include/sbp.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts numpy arrays to the
C layouts, calls the C entry points by the same names, and raises on non-zero status.
The library must be built (``paper_2003_12811_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsbp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "sbp.h")
HEADER3 = os.path.join(os.path.dirname(HERE), "include", "sbp3.h")

SBP_OK = 0
STATUS = {0: "SBP_OK", -1: "SBP_E_INVALID_ARG", -2: "SBP_E_JACOBIAN_NONPOSITIVE",
          -3: "SBP_E_NONCONFORMING_INTERFACE", -4: "SBP_E_OOM", -5: "SBP_E_CUDA", -6: "SBP_E_TIMEOUT",
          -7: "SBP_E_UNSTABLE", -8: "SBP_E_STATE"}
FP64, FP32 = 0, 1
BC = {"displacement": 0, "robin": 1, "interface": 2}
FIELD_PREV, FIELD_CUR, FIELD_APPLY, FIELD_VELOCITY = 0, 1, 2, 3
C_PAIR10, C_VOIGT6 = 0, 1
STENCIL = {"narrow": 0, "wide": 1}
PROF_FAMILIES = 8      # SBP_PROF_FAMILIES


class SbpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class FaceDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("nbr_block", C.c_int), ("nbr_face", C.c_int), ("reversed", C.c_int)]


class BlockDesc(C.Structure):
    _fields_ = [("n1", C.c_int), ("n2", C.c_int), ("x1", C.POINTER(C.c_double)), ("x2", C.POINTER(C.c_double)),
                ("h1", C.c_double), ("h2", C.c_double), ("faces", FaceDesc * 4)]


class GridDesc(C.Structure):
    _fields_ = [("order", C.c_int), ("precision", C.c_int), ("nblocks", C.c_int),
                ("blocks", C.POINTER(BlockDesc)), ("beta", C.c_double), ("stencil", C.c_int)]


_lib = None
_DP = C.POINTER(C.c_double)


def header_functions():
    """Names of the functions declared in include/sbp.h and include/sbp3.h."""
    txt = open(HEADER).read() + open(HEADER3).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\s*\*)\s+(sbp3?_\w+)\s*\(", txt, re.M)))


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsbp.so is not built (run __graft_entry__.build()); no fallback exists")
        L = C.CDLL(LIB_PATH)
        L.sbp_grid_create.argtypes = [C.POINTER(GridDesc), C.POINTER(C.c_void_p)]
        L.sbp_destroy.argtypes = [C.c_void_p]
        L.sbp_last_error.argtypes = [C.c_void_p]
        L.sbp_last_error.restype = C.c_char_p
        L.sbp_set_material.argtypes = [C.c_void_p, C.c_int, _DP, _DP, C.c_int]
        L.sbp_set_robin.argtypes = [C.c_void_p, C.c_int, C.c_int, _DP]
        L.sbp_set_time_basis.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int), _DP]
        L.sbp_set_robin_damping.argtypes = [C.c_void_p, C.c_int, C.c_int, _DP]
        L.sbp_set_layer_dissipation.argtypes = [C.c_void_p, C.c_int, _DP]
        L.sbp_set_boundary_data.argtypes = [C.c_void_p, C.c_int, C.c_int, _DP]
        L.sbp_set_forcing.argtypes = [C.c_void_p, C.c_int, _DP]
        L.sbp_add_point_source.argtypes = [C.c_void_p, C.c_int] + [C.c_double] * 7
        L.sbp_set_state.argtypes = [C.c_void_p, C.c_int, _DP, _DP, C.c_double]
        L.sbp_set_state_device.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_longlong, C.c_double,
                                           C.c_void_p]
        L.sbp_get_field_device.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_longlong, C.c_void_p]
        L.sbp_step.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_void_p]
        L.sbp_set_state_rk4.argtypes = [C.c_void_p, C.c_int, _DP, _DP, C.c_double]
        L.sbp_step_rk4.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_void_p]
        L.sbp_apply.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.sbp_get_field.argtypes = [C.c_void_p, C.c_int, C.c_int, _DP]
        L.sbp_energy.argtypes = [C.c_void_p, C.c_double, _DP]
        L.sbp_suggest_dt.argtypes = [C.c_void_p, C.c_double, _DP]
        L.sbp_get_time.argtypes = [C.c_void_p, _DP]
        L.sbp_profile.argtypes = [C.c_void_p, C.c_int]
        L.sbp_step_graph.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_void_p]
        L.sbp_grid_footprint.argtypes = [C.POINTER(GridDesc), C.POINTER(C.c_longlong)]
        L.sbp_autotune.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.sbp_set_tuning.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.sbp_apply_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_void_p]
        L.sbp_profile_read.argtypes = [C.c_void_p, _DP, C.POINTER(C.c_longlong)]
        L.sbp_get_info.argtypes = [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.sbp_check.argtypes = [C.c_void_p]
        L.sbp_l2_diff.argtypes = [C.c_void_p, C.c_int, C.POINTER(_DP), _DP, _DP]
        L.sbp_debug_wait_probe.argtypes = [C.c_void_p, C.c_int]
        L.sbp_batch_create.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_void_p)]
        L.sbp_batch_destroy.argtypes = [C.c_void_p]
        L.sbp_batch_last_error.argtypes = [C.c_void_p]
        L.sbp_batch_last_error.restype = C.c_char_p
        L.sbp_batch_add.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_int)]
        L.sbp_batch_step.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.sbp_batch_poll.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.c_void_p]
        L.sbp_batch_remove.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.sbp_batch_set_rows.argtypes = [C.c_void_p, C.c_int]
        L.sbp_batch_autotune.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]
        L.sbp_set_receivers.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int)]
        L.sbp_record.argtypes = [C.c_void_p, C.c_int, C.c_double, _DP]
        L.sbp_misfit_gradient.argtypes = [C.c_void_p, C.c_int, C.c_double, _DP, C.c_int, _DP,
                                          C.POINTER(_DP), C.POINTER(_DP), C.c_int]
        L.sbp3_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _DP, C.POINTER(C.c_int), C.c_double,
                                  C.POINTER(C.c_void_p)]
        L.sbp3_destroy.argtypes = [C.c_void_p]
        L.sbp3_last_error.argtypes = [C.c_void_p]
        L.sbp3_last_error.restype = C.c_char_p
        L.sbp3_footprint.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_longlong)]
        L.sbp3_set_material.argtypes = [C.c_void_p, C.c_int, C.c_int, _DP, _DP]
        L.sbp3_set_state.argtypes = [C.c_void_p, _DP, _DP]
        L.sbp3_get_state.argtypes = [C.c_void_p, _DP, _DP]
        L.sbp3_apply.argtypes = [C.c_void_p, _DP, _DP]
        L.sbp3_step.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_void_p]
        L.sbp3_profile.argtypes = [C.c_void_p, C.c_int]
        L.sbp3_set_tuning.argtypes = [C.c_void_p, C.c_int]
        L.sbp3_autotune.argtypes = [C.c_void_p, C.POINTER(C.c_int), _DP]
        L.sbp3_profile_read.argtypes = [C.c_void_p, _DP, C.POINTER(C.c_longlong)]
        L.sbp3_get_info.argtypes = [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_DP)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def pair10(Cfull):
    """Full tensor C[I,J,K,L,...] -> 10 planes: upper triangle of M[p][q], p = 2I+J, q = 2K+L."""
    planes = []
    for p in range(4):
        for q in range(p, 4):
            planes.append(Cfull[p // 2, p % 2, q // 2, q % 2])
    return np.stack(planes)


def grid_desc(problem, precision="fp64"):
    """Build the C grid descriptor of a ``workloads.Problem``; returns (desc, arrays kept alive)."""
    keep = []
    blocks = (BlockDesc * len(problem.blocks))()
    for b, blk in enumerate(problem.blocks):
        x1, x2 = _f64(blk.X[0]), _f64(blk.X[1])
        keep += [x1, x2]
        bd = blocks[b]
        bd.n1, bd.n2 = blk.N1, blk.N2
        bd.x1, bd.x2 = _ptr(x1), _ptr(x2)
        bd.h1, bd.h2 = blk.spacing
        for f, face in enumerate(blk.faces):
            if face.kind not in BC:
                raise ValueError(f"face kind {face.kind!r} is not supported by libsbp")
            fd = bd.faces[f]
            fd.kind = BC[face.kind]
            if face.kind == "interface":
                fd.nbr_block, fd.nbr_face, fd.reversed = face.nbr[0], face.nbr[1], int(bool(face.nbr[2]))
            else:
                fd.nbr_block, fd.nbr_face, fd.reversed = -1, -1, 0
    keep.append(blocks)
    prec = FP64 if precision == "fp64" else FP32
    stencil = STENCIL[getattr(problem, "stencil", "narrow")]
    return GridDesc(problem.order, prec, len(problem.blocks), blocks, problem.beta, stencil), keep


def footprint_bytes(problem, precision="fp32"):
    """Device bytes a Solver for ``problem`` will hold (sbp_grid_footprint)."""
    desc, keep = grid_desc(problem, precision)
    out = C.c_longlong()
    rc = lib().sbp_grid_footprint(C.byref(desc), C.byref(out))
    if rc != SBP_OK:
        raise SbpError(rc, "footprint query failed")
    return int(out.value)


class Solver:
    """A libsbp handle built from a ``workloads.Problem``."""

    def __init__(self, problem, precision="fp64"):
        self.L = lib()
        self.problem = problem
        self.precision = FP64 if precision == "fp64" else FP32
        desc, self._keep = grid_desc(problem, precision)
        h = C.c_void_p()
        rc = self.L.sbp_grid_create(C.byref(desc), C.byref(h))
        if rc != SBP_OK:
            raise SbpError(rc, self.L.sbp_last_error(None).decode())
        self.h = h
        try:
            self._setup()
        except Exception:
            self.close()
            raise

    def _check(self, rc):
        if rc != SBP_OK:
            raise SbpError(rc, self.L.sbp_last_error(self.h).decode())

    def _setup(self):
        P = self.problem
        if P.time_basis:
            kinds = (C.c_int * len(P.time_basis))(*[0 if k == "sin" else 1 for k, _ in P.time_basis])
            om = _f64([w for _, w in P.time_basis])
            self._check(self.L.sbp_set_time_basis(self.h, len(P.time_basis), kinds, _ptr(om)))
        for b, blk in enumerate(P.blocks):
            self.sbp_set_material(b, blk.rho, pair10(blk.C), C_PAIR10)
            for f, face in enumerate(blk.faces):
                if face.kind == "robin" and face.U is not None:
                    U = _f64(face.U)
                    self._check(self.L.sbp_set_robin(self.h, b, f, _ptr(U)))
                if face.kind == "robin" and getattr(face, "V", None) is not None:
                    V = _f64(face.V)
                    self._check(self.L.sbp_set_robin_damping(self.h, b, f, _ptr(V)))
                if face.g is not None and face.kind in ("robin", "displacement"):
                    g = _f64(face.g)
                    self._check(self.L.sbp_set_boundary_data(self.h, b, f, _ptr(g)))
            if getattr(blk, "sponge", None) is not None:
                sp_ = _f64(blk.sponge)
                self._check(self.L.sbp_set_layer_dissipation(self.h, b, _ptr(sp_)))
            if blk.forcing is not None:
                fo = _f64(blk.forcing)
                self._check(self.L.sbp_set_forcing(self.h, b, _ptr(fo)))
        for s in P.sources:
            self._check(self.L.sbp_add_point_source(self.h, s.block, s.x_ref[0], s.x_ref[1], s.direction[0],
                                                    s.direction[1], s.amplitude, s.alpha_p, s.t0))

    # ---------------------------------------------------------------- C entry points
    def sbp_set_material(self, block, rho, Cplanes, layout=C_PAIR10):
        """rho (N2, N1); Cplanes (10, N2, N1) pair layout or (6, N2, N1) Voigt layout."""
        r, c = _f64(rho), _f64(Cplanes)
        self._check(self.L.sbp_set_material(self.h, int(block), _ptr(r), _ptr(c), int(layout)))

    def sbp_set_state_device(self, block, u_prev_ptr, u_cur_ptr, pitch, t, stream=None):
        """Device addresses of caller buffers: 2 planes of N2 rows x pitch elements each."""
        s = None if stream is None else C.c_void_p(stream)
        self._check(self.L.sbp_set_state_device(self.h, int(block), C.c_void_p(u_prev_ptr), C.c_void_p(u_cur_ptr),
                                                int(pitch), float(t), s))

    def sbp_get_field_device(self, block, which, dst_ptr, pitch, stream=None):
        s = None if stream is None else C.c_void_p(stream)
        self._check(self.L.sbp_get_field_device(self.h, int(block), int(which), C.c_void_p(dst_ptr), int(pitch), s))

    def sbp_set_state(self, u_prev, u_cur, t):
        for b, (up, uc) in enumerate(zip(u_prev, u_cur)):
            a, c = _f64(up), _f64(uc)
            self._check(self.L.sbp_set_state(self.h, b, _ptr(a), _ptr(c), float(t)))

    def sbp_step(self, nsteps, dt, stream=None):
        s = None if stream is None else C.c_void_p(stream)
        self._check(self.L.sbp_step(self.h, int(nsteps), float(dt), s))

    def sbp_set_state_rk4(self, u, v, t):
        for b, (ub, vb) in enumerate(zip(u, v)):
            a, c = _f64(ub), _f64(vb)
            self._check(self.L.sbp_set_state_rk4(self.h, b, _ptr(a), _ptr(c), float(t)))

    def sbp_step_rk4(self, nsteps, dt, stream=None):
        s = None if stream is None else C.c_void_p(stream)
        self._check(self.L.sbp_step_rk4(self.h, int(nsteps), float(dt), s))

    def state_rk4(self):
        """(u, v) of the RK4 state."""
        return self.sbp_get_field(FIELD_CUR), self.sbp_get_field(FIELD_VELOCITY)

    def sbp_step_graph(self, nsteps, dt, stream=None):
        s = None if stream is None else C.c_void_p(stream)
        self._check(self.L.sbp_step_graph(self.h, int(nsteps), float(dt), s))

    def sbp_autotune(self):
        """Returns (rows_per_cta, overlap) chosen for this grid."""
        r, o = C.c_int(), C.c_int()
        self._check(self.L.sbp_autotune(self.h, C.byref(r), C.byref(o)))
        return r.value, o.value

    def sbp_set_tuning(self, rows_per_cta, overlap=-1):
        self._check(self.L.sbp_set_tuning(self.h, int(rows_per_cta), int(overlap)))

    def sbp_apply(self, with_data=False, t=0.0):
        self._check(self.L.sbp_apply(self.h, int(bool(with_data)), float(t)))

    def sbp_get_field(self, which):
        out = []
        for b, blk in enumerate(self.problem.blocks):
            dst = np.empty((2, blk.N2, blk.N1))
            self._check(self.L.sbp_get_field(self.h, b, which, _ptr(dst)))
            out.append(dst)
        return out

    def sbp_energy(self, dt):
        E = C.c_double()
        self._check(self.L.sbp_energy(self.h, float(dt), C.byref(E)))
        return E.value

    def sbp_suggest_dt(self, cfl):
        dt = C.c_double()
        self._check(self.L.sbp_suggest_dt(self.h, float(cfl), C.byref(dt)))
        return dt.value

    def sbp_get_time(self):
        t = C.c_double()
        self._check(self.L.sbp_get_time(self.h, C.byref(t)))
        return t.value

    def sbp_apply_noalloc(self, u_ptr, r_ptr, with_data=False, t=0.0, stream=None):
        """u_ptr, r_ptr: device addresses of buffers in the library layout (see include/sbp.h)."""
        s = None if stream is None else C.c_void_p(stream)
        self._check(self.L.sbp_apply_noalloc(self.h, C.c_void_p(u_ptr), C.c_void_p(r_ptr), int(bool(with_data)),
                                             float(t), s))

    def sbp_set_receivers(self, receivers):
        """receivers: sequence of (block, i1, i2) node indices."""
        rec = np.ascontiguousarray(np.asarray(receivers, dtype=np.int32).reshape(-1, 3))
        self._nrec = rec.shape[0]
        self._check(self.L.sbp_set_receivers(self.h, self._nrec, rec.ctypes.data_as(C.POINTER(C.c_int))))

    def sbp_record(self, nsteps, dt):
        """Step nsteps times; returns the receiver traces (nsteps, nrec, 2)."""
        out = np.empty((int(nsteps), getattr(self, "_nrec", 0), 2))
        self._check(self.L.sbp_record(self.h, int(nsteps), float(dt), _ptr(out)))
        return out

    def sbp_misfit_gradient(self, nsteps, dt, observed, checkpoint_every=0, rho=True, stiffness=True, layout=C_PAIR10):
        """Returns (misfit, [dPhi/drho (N2, N1)] or None, [dPhi/dC (10 or 6, N2, N1) in `layout`] or None)."""
        obs = _f64(observed)
        nb = len(self.problem.blocks)
        ncp = 6 if layout == C_VOIGT6 else 10
        gr = [np.empty((b.N2, b.N1)) for b in self.problem.blocks] if rho else None
        gc = [np.empty((ncp, b.N2, b.N1)) for b in self.problem.blocks] if stiffness else None
        pr = (_DP * nb)(*[_ptr(a) for a in gr]) if rho else None
        pc = (_DP * nb)(*[_ptr(a) for a in gc]) if stiffness else None
        phi = C.c_double()
        self._check(self.L.sbp_misfit_gradient(self.h, int(nsteps), float(dt), _ptr(obs), int(checkpoint_every),
                                               C.byref(phi), pr, pc, int(layout)))
        return phi.value, gr, gc

    def sbp_l2_diff(self, which, ref):
        """(sum (u-ref)^T JH (u-ref), sum ref^T JH ref) over blocks for field `which`."""
        arrs = [_f64(r) for r in ref]
        ptrs = (_DP * len(arrs))(*[_ptr(a) for a in arrs])
        e, r = C.c_double(), C.c_double()
        self._check(self.L.sbp_l2_diff(self.h, int(which), ptrs, C.byref(e), C.byref(r)))
        return e.value, r.value

    def sbp_check(self):
        self._check(self.L.sbp_check(self.h))

    def sbp_debug_wait_probe(self, polls):
        self._check(self.L.sbp_debug_wait_probe(self.h, int(polls)))

    def sbp_profile(self, enable):
        self._check(self.L.sbp_profile(self.h, int(bool(enable))))

    def sbp_profile_read(self):
        ms = np.zeros(PROF_FAMILIES)
        n = (C.c_longlong * PROF_FAMILIES)()
        self._check(self.L.sbp_profile_read(self.h, _ptr(ms), n))
        return ms, np.array(list(n), dtype=np.int64)

    # ---------------------------------------------------------------- conveniences
    set_state = sbp_set_state
    step = sbp_step
    energy = sbp_energy
    suggest_dt = sbp_suggest_dt

    def apply(self, with_data=False, t=0.0):
        self.sbp_apply(with_data, t)
        return self.sbp_get_field(FIELD_APPLY)

    def state(self):
        return self.sbp_get_field(FIELD_PREV), self.sbp_get_field(FIELD_CUR)

    def close(self):
        if getattr(self, "h", None):
            self.L.sbp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A batch of resident shots advanced by the persistent tile-queue kernel (sbp_batch_*)."""

    def __init__(self, order, max_shots):
        self.L = lib()
        self.max_shots = int(max_shots)
        b = C.c_void_p()
        rc = self.L.sbp_batch_create(int(order), self.max_shots, C.byref(b))
        if rc != SBP_OK:
            raise SbpError(rc, "sbp_batch_create failed")
        self.b = b
        self._rem = (C.c_int * self.max_shots)()

    def _check(self, rc):
        if rc != SBP_OK:
            raise SbpError(rc, self.L.sbp_batch_last_error(self.b).decode())

    @staticmethod
    def _s(stream):
        return None if stream is None else C.c_void_p(stream)

    def sbp_batch_add(self, solver, nsteps, dt):
        slot = C.c_int()
        self._check(self.L.sbp_batch_add(self.b, solver.h, int(nsteps), float(dt), C.byref(slot)))
        return slot.value

    def sbp_batch_step(self, ksteps, stream=None):
        self._check(self.L.sbp_batch_step(self.b, int(ksteps), self._s(stream)))

    def sbp_batch_poll(self, stream=None):
        """Steps left per slot (-1: free slot); synchronises the stream."""
        self._check(self.L.sbp_batch_poll(self.b, self._rem, self._s(stream)))
        return list(self._rem)

    def sbp_batch_remove(self, slot, stream=None):
        self._check(self.L.sbp_batch_remove(self.b, int(slot), self._s(stream)))

    def sbp_batch_set_rows(self, rows):
        self._check(self.L.sbp_batch_set_rows(self.b, int(rows)))

    def sbp_batch_autotune(self, solver):
        rows = C.c_int()
        self._check(self.L.sbp_batch_autotune(self.b, solver.h, C.byref(rows)))
        return rows.value

    def close(self):
        if getattr(self, "b", None):
            self.L.sbp_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- 3-D operator (include/sbp3.h)
BC3 = {"displacement": 0, "traction": 1}
PROF3_FAMILIES = 3     # SBP3_PROF_FAMILIES: k3_flux, k3_div_int, k3_div_shell (with the face SATs)


def footprint3_bytes(N, precision="fp32", order=6):
    out = C.c_longlong()
    rc = lib().sbp3_footprint(order, FP64 if precision == "fp64" else FP32, N[0], N[1], N[2], C.byref(out))
    if rc != SBP_OK:
        raise SbpError(rc, lib().sbp3_last_error(None).decode())
    return int(out.value)


class Solver3D:
    """A 3-D libsbp handle (include/sbp3.h) for one block.  ``X`` is (3, N3, N2, N1); the material
    is given per chunk of x3-planes with ``sbp3_set_material`` (rho (k, N2, N1), C45 (45, k, N2, N1)),
    or at once from a ``workloads.box3d.Block3D`` through ``from_block``."""

    def __init__(self, X, faces, order=6, precision="fp64", beta=1.0):
        self.L = lib()
        X = _f64(X)
        self.shape = X.shape[1:]
        self.N = (X.shape[3], X.shape[2], X.shape[1])
        self.precision = FP64 if precision == "fp64" else FP32
        kinds = (C.c_int * 6)(*[BC3[f] for f in faces])
        h = C.c_void_p()
        rc = self.L.sbp3_create(order, self.precision, self.N[0], self.N[1], self.N[2], _ptr(X), kinds, float(beta),
                                C.byref(h))
        if rc != SBP_OK:
            raise SbpError(rc, self.L.sbp3_last_error(None).decode())
        self.h = h

    @classmethod
    def from_block(cls, blk, precision="fp64", pair45=None):
        S = cls(blk.X, blk.faces, blk.order, precision, blk.beta)
        try:
            P = pair45(blk.C) if pair45 is not None else _pair45(blk.C)
            S.sbp3_set_material(0, blk.shape[0], blk.rho, P)
        except Exception:
            S.close()
            raise
        return S

    def _check(self, rc):
        if rc != SBP_OK:
            raise SbpError(rc, self.L.sbp3_last_error(self.h).decode())

    def sbp3_set_material(self, i3_begin, i3_count, rho, C45):
        rho, C45 = _f64(rho), _f64(C45)
        self._check(self.L.sbp3_set_material(self.h, i3_begin, i3_count, _ptr(rho), _ptr(C45)))

    def set_state(self, u_prev, u_cur):
        a, b = _f64(u_prev), _f64(u_cur)
        self._check(self.L.sbp3_set_state(self.h, _ptr(a), _ptr(b)))

    def state(self):
        a = np.empty((3,) + tuple(self.shape))
        b = np.empty_like(a)
        self._check(self.L.sbp3_get_state(self.h, _ptr(a), _ptr(b)))
        return a, b

    def apply(self, u):
        u = _f64(u)
        out = np.empty_like(u)
        self._check(self.L.sbp3_apply(self.h, _ptr(u), _ptr(out)))
        return out

    def step(self, nsteps, dt, stream=None):
        self._check(self.L.sbp3_step(self.h, int(nsteps), float(dt), stream))

    def sbp3_set_tuning(self, variant):
        self._check(self.L.sbp3_set_tuning(self.h, int(variant)))

    def sbp3_autotune(self):
        """Selects the fastest launch shape of the interior kernel; returns (variant, ms per variant)."""
        v = C.c_int()
        ms = (C.c_double * 4)()
        self._check(self.L.sbp3_autotune(self.h, C.byref(v), ms))
        return int(v.value), list(ms)

    def profile(self, enable):
        self._check(self.L.sbp3_profile(self.h, int(enable)))

    def profile_read(self):
        ms = (C.c_double * PROF3_FAMILIES)()
        n = (C.c_longlong * PROF3_FAMILIES)()
        self._check(self.L.sbp3_profile_read(self.h, ms, n))
        return list(ms), list(n)

    def close(self):
        if getattr(self, "h", None):
            self.L.sbp3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _pair45(Cfull):
    """Full tensor C[I,J,K,L,...] -> 45 planes: upper triangle of M[p][q], p = 3I+J, q = 3K+L."""
    M = Cfull.reshape((9, 9) + Cfull.shape[4:])
    return np.stack([M[p, q] for p in range(9) for q in range(p, 9)])
