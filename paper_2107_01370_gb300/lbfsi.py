"""Thin ctypes binding of liblbfsi.so (C ABI declared in include/lbfsi.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  There is no CPU fallback; if the library is missing the import
of this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbfsi.so")

FP64 = 0
FP32 = 1
FIELD_MOMENTS, FIELD_POPULATIONS = 0, 1

OK, EINVAL, ENOMEM, ECUDA, EDEPARTURE, ENONPHYS, ETIMEOUT, ESTATE, EBOUNDS = 0, -1, -2, -3, -4, -5, -6, -7, -8
_NAMES = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", EDEPARTURE: "EDEPARTURE",
          ENONPHYS: "ENONPHYS", ETIMEOUT: "ETIMEOUT", ESTATE: "ESTATE", EBOUNDS: "EBOUNDS"}

EXPORTED = ["lbfsi_create_mesh", "lbfsi_destroy_mesh", "lbfsi_init_fields", "lbfsi_blend_mesh",
            "lbfsi_step", "lbfsi_body_forces", "lbfsi_advance_bodies", "lbfsi_get_body_state",
            "lbfsi_get_fields", "lbfsi_get_populations", "lbfsi_set_populations",
            "lbfsi_synchronize", "lbfsi_launch_count", "lbfsi_last_error",
            "lbfsi_wall_loads_noalloc", "lbfsi_batch_create", "lbfsi_batch_destroy",
            "lbfsi_batch_add", "lbfsi_batch_step", "lbfsi_batch_poll", "lbfsi_batch_get",
            "lbfsi_batch_remove", "lbfsi_batch_memory", "lbfsi_step_variants",
            "lbfsi_set_schedule", "lbfsi_get_schedule", "lbfsi_set_graph_steps", "lbfsi_autotune",
            "lbfsi_batch_set_schedule", "lbfsi_batch_get_schedule", "lbfsi_batch_set_graph_steps",
            "lbfsi_batch_autotune", "lbfsi_checkpoint_bytes", "lbfsi_checkpoint", "lbfsi_restore",
            "lbfsi_create_mesh_xy", "lbfsi_step_record", "lbfsi_batch_add_xy",
            "lbfsi_create_mesh_cgrid", "lbfsi_batch_add_cgrid", "lbfsi_field_ptr",
            "lbfsi_create_mesh_box", "lbfsi_create_mesh_cgrid_walls",
            "lbfsi_create_mesh_elements", "lbfsi_emesh_destroy", "lbfsi_emesh_init_fields",
            "lbfsi_emesh_blend_mesh", "lbfsi_emesh_step", "lbfsi_emesh_synchronize",
            "lbfsi_emesh_body_forces", "lbfsi_emesh_get_body_state", "lbfsi_emesh_get_fields",
            "lbfsi_emesh_get_populations", "lbfsi_emesh_launch_count"]


class LbfsiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class BodyDesc(ctypes.Structure):
    _fields_ = [("dof", ctypes.c_int), ("xc", ctypes.c_double), ("yc", ctypes.c_double),
                ("xp", ctypes.c_double), ("yp", ctypes.c_double), ("r_in", ctypes.c_double),
                ("r_out", ctypes.c_double), ("length", ctypes.c_double),
                ("m_star", ctypes.c_double), ("v_r", ctypes.c_double), ("zeta", ctypes.c_double),
                ("x_alpha", ctypes.c_double), ("r_alpha", ctypes.c_double),
                ("wh_wa", ctypes.c_double), ("pitch_amp", ctypes.c_double),
                ("forced_periods", ctypes.c_double)]


class FlowParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("ma", "re", "t_inf", "gamma", "pr", "rho_inf", "dt", "length")]


class MeshDesc(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("ntheta", ctypes.c_int),
                ("r", ctypes.POINTER(ctypes.c_double)), ("e", ctypes.POINTER(ctypes.c_double)),
                ("xc", ctypes.c_double), ("yc", ctypes.c_double), ("precision", ctypes.c_int),
                ("nbatch", ctypes.c_int), ("bodies", ctypes.POINTER(BodyDesc))]


class MeshXYDesc(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("ntheta", ctypes.c_int),
                ("X", ctypes.POINTER(ctypes.c_double)),
                ("xc", ctypes.c_double), ("yc", ctypes.c_double), ("precision", ctypes.c_int),
                ("nbatch", ctypes.c_int), ("bodies", ctypes.POINTER(BodyDesc))]


class _DeviceArray:
    """Device memory of a handle exposed through __cuda_array_interface__
    (keeps the handle alive); row0: slot of node (0, 0) in each component."""

    def __init__(self, ptr, shape, typestr, owner, row0):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None, "stream": None}
        self.owner = owner
        self.row0 = row0


class MeshBoxDesc(ctypes.Structure):
    _fields_ = [("ni", ctypes.c_int), ("nj", ctypes.c_int), ("X", ctypes.POINTER(ctypes.c_double)),
                ("shift_i", ctypes.c_double * 2), ("shift_j", ctypes.c_double * 2),
                ("precision", ctypes.c_int), ("nbatch", ctypes.c_int), ("bodies", ctypes.POINTER(BodyDesc))]


class MeshCGridWallsDesc(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("ntheta", ctypes.c_int), ("nwalls", ctypes.c_int),
                ("walls", ctypes.POINTER(ctypes.c_int)), ("X", ctypes.POINTER(ctypes.c_double)),
                ("xc", ctypes.c_double), ("yc", ctypes.c_double), ("precision", ctypes.c_int),
                ("nbatch", ctypes.c_int), ("bodies", ctypes.POINTER(BodyDesc)),
                ("nbody", ctypes.c_int), ("wall_body", ctypes.POINTER(ctypes.c_int))]


class MeshElementsDesc(ctypes.Structure):
    _fields_ = [("nnode", ctypes.c_int), ("X", ctypes.POINTER(ctypes.c_double)),
                ("nelem", ctypes.c_int), ("elements", ctypes.POINTER(ctypes.c_int)),
                ("nwall", ctypes.c_int), ("wall", ctypes.POINTER(ctypes.c_int)),
                ("nfar", ctypes.c_int), ("far", ctypes.POINTER(ctypes.c_int)),
                ("grid_ij", ctypes.POINTER(ctypes.c_int)), ("grid_nr", ctypes.c_int),
                ("grid_nt", ctypes.c_int), ("nbatch", ctypes.c_int),
                ("bodies", ctypes.POINTER(BodyDesc)), ("precision", ctypes.c_int)]


class MeshCGridDesc(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("ntheta", ctypes.c_int), ("n_cut", ctypes.c_int),
                ("X", ctypes.POINTER(ctypes.c_double)),
                ("xc", ctypes.c_double), ("yc", ctypes.c_double), ("precision", ctypes.c_int),
                ("nbatch", ctypes.c_int), ("bodies", ctypes.POINTER(BodyDesc))]


class SolveCGridDesc(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("ntheta", ctypes.c_int), ("n_cut", ctypes.c_int),
                ("X", ctypes.POINTER(ctypes.c_double)),
                ("xc", ctypes.c_double), ("yc", ctypes.c_double), ("body", BodyDesc),
                ("flow", FlowParams), ("rho_u_T", ctypes.POINTER(ctypes.c_double)),
                ("steps", ctypes.c_int)]


class SolveXYDesc(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("ntheta", ctypes.c_int),
                ("X", ctypes.POINTER(ctypes.c_double)),
                ("xc", ctypes.c_double), ("yc", ctypes.c_double), ("body", BodyDesc),
                ("flow", FlowParams), ("rho_u_T", ctypes.POINTER(ctypes.c_double)),
                ("steps", ctypes.c_int)]


class SolveDesc(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("ntheta", ctypes.c_int),
                ("r", ctypes.POINTER(ctypes.c_double)), ("e", ctypes.POINTER(ctypes.c_double)),
                ("xc", ctypes.c_double), ("yc", ctypes.c_double), ("body", BodyDesc),
                ("flow", FlowParams), ("rho_u_T", ctypes.POINTER(ctypes.c_double)),
                ("steps", ctypes.c_int)]


class BodyState(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("alpha", ctypes.c_double), ("hdot", ctypes.c_double),
                ("adot", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblbfsi.so and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"liblbfsi.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    lib.lbfsi_create_mesh.argtypes = [ctypes.POINTER(MeshDesc), P, ctypes.POINTER(P)]
    lib.lbfsi_destroy_mesh.argtypes = [P]
    lib.lbfsi_init_fields.argtypes = [P, ctypes.POINTER(FlowParams), dp]
    lib.lbfsi_blend_mesh.argtypes = [P, ctypes.POINTER(BodyState), ctypes.POINTER(BodyState)]
    lib.lbfsi_step.argtypes = [P, ctypes.c_int]
    lib.lbfsi_body_forces.argtypes = [P, dp]
    lib.lbfsi_advance_bodies.argtypes = [P, dp, ctypes.c_double]
    lib.lbfsi_get_body_state.argtypes = [P, ctypes.POINTER(BodyState)]
    lib.lbfsi_get_fields.argtypes = [P, dp]
    lib.lbfsi_get_populations.argtypes = [P, ctypes.c_int, dp, dp]
    lib.lbfsi_set_populations.argtypes = [P, dp, dp, dp]
    lib.lbfsi_synchronize.argtypes = [P]
    lib.lbfsi_launch_count.argtypes = [P]
    lib.lbfsi_launch_count.restype = ctypes.c_int64
    lib.lbfsi_wall_loads_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             P, P, ctypes.c_double, ctypes.c_double, P, P, P,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             P, P]
    sz = ctypes.c_size_t
    ip = ctypes.POINTER(ctypes.c_int)
    lib.lbfsi_batch_create.argtypes = [sz, ctypes.c_int, P, ctypes.POINTER(P)]
    lib.lbfsi_batch_destroy.argtypes = [P]
    lib.lbfsi_batch_add.argtypes = [P, ctypes.POINTER(SolveDesc), ip]
    lib.lbfsi_batch_step.argtypes = [P, ctypes.c_int, ip]
    lib.lbfsi_batch_poll.argtypes = [P, ctypes.c_int, ip, ip]
    lib.lbfsi_batch_get.argtypes = [P, ctypes.c_int, dp, dp, ctypes.POINTER(BodyState)]
    lib.lbfsi_batch_remove.argtypes = [P, ctypes.c_int]
    lib.lbfsi_batch_memory.argtypes = [P, ctypes.POINTER(sz), ctypes.POINTER(sz)]
    lib.lbfsi_last_error.argtypes = []
    lib.lbfsi_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("lbfsi_launch_count", "lbfsi_last_error", "lbfsi_checkpoint_bytes",
                        "lbfsi_emesh_launch_count"):
            getattr(lib, name).restype = ctypes.c_int
    lib.lbfsi_field_ptr.argtypes = [P, ctypes.c_int, ctypes.POINTER(P), ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_int64)]
    lib.lbfsi_create_mesh_elements.argtypes = [ctypes.POINTER(MeshElementsDesc), P, ctypes.POINTER(P)]
    lib.lbfsi_emesh_destroy.argtypes = [P]
    lib.lbfsi_emesh_init_fields.argtypes = [P, ctypes.POINTER(FlowParams), dp]
    lib.lbfsi_emesh_blend_mesh.argtypes = [P, ctypes.POINTER(BodyState), ctypes.POINTER(BodyState)]
    lib.lbfsi_emesh_step.argtypes = [P, ctypes.c_int]
    lib.lbfsi_emesh_synchronize.argtypes = [P]
    lib.lbfsi_emesh_body_forces.argtypes = [P, dp]
    lib.lbfsi_emesh_get_body_state.argtypes = [P, ctypes.POINTER(BodyState)]
    lib.lbfsi_emesh_get_fields.argtypes = [P, dp]
    lib.lbfsi_emesh_get_populations.argtypes = [P, ctypes.c_int, dp, dp]
    lib.lbfsi_emesh_launch_count.argtypes = [P]
    lib.lbfsi_emesh_launch_count.restype = ctypes.c_int64
    lib.lbfsi_checkpoint_bytes.restype = ctypes.c_size_t
    lib.lbfsi_checkpoint_bytes.argtypes = [ctypes.c_void_p]
    lib.lbfsi_checkpoint.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
    lib.lbfsi_restore.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
    _lib = lib
    return lib


def _check(rc):
    if rc != OK:
        raise LbfsiError(rc, _lib.lbfsi_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def wall_loads_noalloc(nr, ntheta, nbatch, precision, r_dev, e_dev, centre, f_dev, g_dev,
                       body_ref_dev, mu, dt, gamma, loads_dev, stream=0):
    """Allocation-free wall loads; every array argument is a device pointer
    (int) owned by the caller (see include/lbfsi.h)."""
    lib = load()
    _check(lib.lbfsi_wall_loads_noalloc(nr, ntheta, nbatch, precision, r_dev, e_dev, centre[0],
                                        centre[1], f_dev, g_dev, body_ref_dev, mu, dt, gamma,
                                        loads_dev, stream))


def body_desc(spec) -> BodyDesc:
    """BodyDesc from any object carrying the BodySpec attribute names."""
    return BodyDesc(int(spec.dof), spec.xc, spec.yc, spec.xp, spec.yp, spec.r_in, spec.r_out,
                    spec.length, spec.m_star, spec.v_r, spec.zeta, spec.x_alpha, spec.r_alpha,
                    spec.wh_wa, getattr(spec, "pitch_amp", 0.0), getattr(spec, "forced_periods", 0.0))


def flow_params(flow) -> FlowParams:
    return FlowParams(flow.ma, flow.re, flow.t_inf, flow.gamma, flow.pr, flow.rho_inf, flow.dt,
                      flow.length)


def step_variants(precision) -> int:
    """Number of tile shapes of the step kernel for a precision."""
    n = load().lbfsi_step_variants(int(precision))
    if n < 0:
        raise LbfsiError(n, _lib.lbfsi_last_error().decode())
    return n


class Mesh:
    """Handle of one O-grid mesh with nbatch independent solves."""

    nbody = 1   # bodies per solve (several: independent bodies of a C-grid)

    @property
    def _bshape(self):
        # leading shape of the per-(solve, body) arrays
        return (self.nbatch,) if self.nbody == 1 else (self.nbatch, self.nbody)

    @property
    def _nslots(self):
        return self.nbatch * self.nbody

    def __init__(self, r, e, bodies, precision=FP64, centre=(0.0, 0.0), stream=None):
        lib = load()
        self._lib = lib
        self.r = np.ascontiguousarray(r, dtype=np.float64)
        self.e = np.ascontiguousarray(e, dtype=np.float64).reshape(-1, 2)
        self.nr, self.nt = self.r.size, self.e.shape[0]
        self.N = self.nr * self.nt
        self.nbatch = len(bodies)
        self.precision = precision
        self._bodies = (BodyDesc * self.nbatch)(*[body_desc(b) for b in bodies])
        d = MeshDesc(self.nr, self.nt, _dptr(self.r), _dptr(self.e), centre[0], centre[1],
                     precision, self.nbatch, self._bodies)
        h = ctypes.c_void_p()
        _check(lib.lbfsi_create_mesh(ctypes.byref(d), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        self.h = h

    @classmethod
    def xy(cls, X, bodies, precision=FP64, centre=(0.0, 0.0), stream=None):
        """Handle of an O-grid given by node coordinates X [nr, ntheta, 2]
        (lbfsi_create_mesh_xy)."""
        self = cls.__new__(cls)
        lib = load()
        self._lib = lib
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.r = self.e = None
        self.nr, self.nt = self.X.shape[0], self.X.shape[1]
        self.N = self.nr * self.nt
        self.nbatch = len(bodies)
        self.precision = precision
        self._bodies = (BodyDesc * self.nbatch)(*[body_desc(b) for b in bodies])
        d = MeshXYDesc(self.nr, self.nt, _dptr(self.X), centre[0], centre[1], precision, self.nbatch,
                       self._bodies)
        h = ctypes.c_void_p()
        self.h = None
        _check(lib.lbfsi_create_mesh_xy(ctypes.byref(d), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        self.h = h
        return self

    @classmethod
    def box(cls, X, shift_i, shift_j, nbatch=1, precision=FP64, stream=None):
        """Handle of a doubly periodic box: node coordinates X [ni, nj, 2] of
        one period and the period vectors (lbfsi_create_mesh_box); no wall,
        fixed bodies."""
        self = cls.__new__(cls)
        lib = load()
        self._lib = lib
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.r = self.e = None
        self.nr, self.nt = self.X.shape[0], self.X.shape[1]
        self.N = self.nr * self.nt
        self.nbatch = int(nbatch)
        self.precision = precision
        self._bodies = (BodyDesc * self.nbatch)()
        d = MeshBoxDesc(self.nr, self.nt, _dptr(self.X), (ctypes.c_double * 2)(*shift_i),
                        (ctypes.c_double * 2)(*shift_j), precision, self.nbatch, self._bodies)
        h = ctypes.c_void_p()
        self.h = None
        _check(lib.lbfsi_create_mesh_box(ctypes.byref(d), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        self.h = h
        return self

    @classmethod
    def cgrid(cls, X, n_cut, bodies, precision=FP64, centre=(0.0, 0.0), stream=None):
        """Handle of a C-grid given by node coordinates X [nr, ntheta, 2]
        (ntheta odd) whose first and last n_cut row-0 nodes lie on the wake
        cut (lbfsi_create_mesh_cgrid)."""
        self = cls.__new__(cls)
        lib = load()
        self._lib = lib
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.r = self.e = None
        self.nr, self.nt = self.X.shape[0], self.X.shape[1]
        self.N = self.nr * self.nt
        self.nbatch = len(bodies)
        self.precision = precision
        self._bodies = (BodyDesc * self.nbatch)(*[body_desc(b) for b in bodies])
        d = MeshCGridDesc(self.nr, self.nt, int(n_cut), _dptr(self.X), centre[0], centre[1], precision,
                          self.nbatch, self._bodies)
        h = ctypes.c_void_p()
        self.h = None
        _check(lib.lbfsi_create_mesh_cgrid(ctypes.byref(d), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        self.h = h
        return self

    @classmethod
    def cgrid_walls(cls, X, walls, bodies, precision=FP64, centre=(0.0, 0.0), stream=None, wall_body=None):
        """Handle of a C-grid around several bodies: node coordinates X
        [nr, ntheta, 2] and the wall chains as inclusive column ranges
        [(first, last), ...] (lbfsi_create_mesh_cgrid_walls).  Without
        wall_body the walls move as the solve's one body (bodies: one per
        solve); with wall_body (the body index of each chain) the bodies are
        independent and bodies holds one list of nbody bodies per solve; the
        body accessors then take and return [nbatch, nbody, ...]."""
        self = cls.__new__(cls)
        lib = load()
        self._lib = lib
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.r = self.e = None
        self.nr, self.nt = self.X.shape[0], self.X.shape[1]
        self.N = self.nr * self.nt
        self.nbatch = len(bodies)
        self.precision = precision
        if wall_body is None:
            flat, wb = list(bodies), None
        else:
            self.nbody = len(bodies[0])
            if any(len(bs) != self.nbody for bs in bodies):
                raise ValueError("the same number of bodies for every solve")
            flat = [b for bs in bodies for b in bs]
            wb = (ctypes.c_int * len(wall_body))(*[int(k) for k in wall_body])
        self._wall_body = wb
        self._bodies = (BodyDesc * len(flat))(*[body_desc(b) for b in flat])
        w = [int(v) for ab in walls for v in ab]
        self._walls = (ctypes.c_int * len(w))(*w)
        d = MeshCGridWallsDesc(self.nr, self.nt, len(walls), self._walls, _dptr(self.X), centre[0], centre[1],
                               precision, self.nbatch, self._bodies, self.nbody, wb)
        h = ctypes.c_void_p()
        self.h = None
        _check(lib.lbfsi_create_mesh_cgrid_walls(ctypes.byref(d), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        self.h = h
        return self

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _check(self._lib.lbfsi_destroy_mesh(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, flow, rho_u_T=None):
        p = flow_params(flow)
        if rho_u_T is None:
            _check(self._lib.lbfsi_init_fields(self.h, ctypes.byref(p), None))
        else:
            a = np.ascontiguousarray(rho_u_T, dtype=np.float64).reshape(self.nbatch, 4, self.N)
            _check(self._lib.lbfsi_init_fields(self.h, ctypes.byref(p), _dptr(a)))

    def blend_mesh(self, states, prev=None):
        """states, prev: one (h, alpha, hdot, adot) per solve (per solve and
        body, flat in that order, for independent bodies)."""
        s = (BodyState * self._nslots)(*[BodyState(*x) for x in states])
        pv = None if prev is None else (BodyState * self._nslots)(*[BodyState(*x) for x in prev])
        _check(self._lib.lbfsi_blend_mesh(self.h, s, pv))

    def step(self, n=1):
        _check(self._lib.lbfsi_step(self.h, int(n)))

    def step_record(self, n, states=False):
        """Advance n steps; per-step loads [n, nbatch, 3] (and body states
        [n, nbatch, 4] as (h, alpha, hdot, adot) if states); [n, nbatch,
        nbody, ...] for independent bodies."""
        loads = np.empty((n, *self._bshape, 3))
        st = (BodyState * (n * self._nslots))() if states else None
        _check(self._lib.lbfsi_step_record(self.h, int(n), _dptr(loads), st))
        if not states:
            return loads
        arr = np.array([(s.h, s.alpha, s.hdot, s.adot) for s in st]).reshape(n, *self._bshape, 4)
        return loads, arr

    def synchronize(self):
        _check(self._lib.lbfsi_synchronize(self.h))

    def field_ptr(self, which=FIELD_MOMENTS):
        """Device pointer, slots per component and the slot of node (0, 0) of
        the current moment field or populations (lbfsi_field_ptr)."""
        ptr = ctypes.c_void_p()
        slots = ctypes.c_int64()
        row0 = ctypes.c_int64()
        _check(self._lib.lbfsi_field_ptr(self.h, int(which), ctypes.byref(ptr), ctypes.byref(slots),
                                         ctypes.byref(row0)))
        return ptr.value, slots.value, row0.value

    def field_view(self, which=FIELD_MOMENTS):
        """The current moment field [nbatch, 4, slots] or populations
        [nbatch, 9, slots, 2] as a CUDA array interface over the handle's own
        memory (torch.as_tensor(view, device="cuda") wraps it without a copy);
        valid as the current state until the next step, read after
        synchronize()."""
        ptr, slots, row0 = self.field_ptr(which)
        shape = (self.nbatch, 4, slots) if which == FIELD_MOMENTS else (self.nbatch, 9, slots, 2)
        return _DeviceArray(ptr, shape, "<f8" if self.precision == FP64 else "<f4", self, row0)

    def body_forces(self, out=None):
        out = np.empty((*self._bshape, 3)) if out is None else out
        _check(self._lib.lbfsi_body_forces(self.h, _dptr(out)))
        return out

    def advance_bodies(self, loads=None, dt=0.0):
        if loads is None:
            _check(self._lib.lbfsi_advance_bodies(self.h, None, float(dt)))
        else:
            a = np.ascontiguousarray(loads, dtype=np.float64).reshape(self._nslots, 3)
            _check(self._lib.lbfsi_advance_bodies(self.h, _dptr(a), float(dt)))

    def body_state(self):
        """Body states, one dict per solve (a list of nbody dicts per solve
        for independent bodies)."""
        out = (BodyState * self._nslots)()
        _check(self._lib.lbfsi_get_body_state(self.h, out))
        d = [dict(h=s.h, alpha=s.alpha, hdot=s.hdot, adot=s.adot) for s in out]
        return d if self.nbody == 1 else [d[k * self.nbody:(k + 1) * self.nbody] for k in range(self.nbatch)]

    def get_fields(self):
        out = np.empty((self.nbatch, 4, self.nr, self.nt))
        _check(self._lib.lbfsi_get_fields(self.h, _dptr(out)))
        return out

    def get_populations(self, which=0):
        f = np.empty((self.nbatch, 9, self.nr, self.nt))
        g = np.empty_like(f)
        _check(self._lib.lbfsi_get_populations(self.h, int(which), _dptr(f), _dptr(g)))
        return f, g

    def set_populations(self, f, g, rho_u_T):
        fa = np.ascontiguousarray(f, dtype=np.float64)
        ga = np.ascontiguousarray(g, dtype=np.float64)
        ma = np.ascontiguousarray(rho_u_T, dtype=np.float64)
        _check(self._lib.lbfsi_set_populations(self.h, _dptr(fa), _dptr(ga), _dptr(ma)))

    def checkpoint(self) -> bytes:
        """The handle's whole step state (see lbfsi_checkpoint)."""
        n = self._lib.lbfsi_checkpoint_bytes(self.h)
        buf = ctypes.create_string_buffer(n)
        _check(self._lib.lbfsi_checkpoint(self.h, buf, n))
        return buf.raw

    def restore(self, ckpt: bytes):
        _check(self._lib.lbfsi_restore(self.h, ckpt, len(ckpt)))

    def set_schedule(self, variant, order=0):
        _check(self._lib.lbfsi_set_schedule(self.h, int(variant), int(order)))

    def schedule(self):
        v, o = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.lbfsi_get_schedule(self.h, ctypes.byref(v), ctypes.byref(o)))
        return v.value, o.value

    def set_graph_steps(self, n):
        _check(self._lib.lbfsi_set_graph_steps(self.h, int(n)))

    def autotune(self, steps_per_trial=20):
        """Returns (variant, order, ms per step [variants][2])."""
        nv = step_variants(self.precision)
        ms = (ctypes.c_float * (2 * nv))()
        v, o = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.lbfsi_autotune(self.h, int(steps_per_trial), ctypes.byref(v), ctypes.byref(o), ms))
        return v.value, o.value, np.array(ms, dtype=np.float64).reshape(nv, 2)

    def launch_count(self) -> int:
        return int(self._lib.lbfsi_launch_count(self.h))


class Batch:
    """Batch runtime: solves on meshes of different sizes admitted into one
    device pool and advanced together (see include/lbfsi.h)."""

    def __init__(self, pool_bytes, precision=FP32, stream=None):
        lib = load()
        self._lib = lib
        self.precision = precision
        h = ctypes.c_void_p()
        _check(lib.lbfsi_batch_create(int(pool_bytes), precision, ctypes.c_void_p(stream or 0),
                                      ctypes.byref(h)))
        self.h = h
        self._shapes = {}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _check(self._lib.lbfsi_batch_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, r, e, body, flow, steps, rho_u_T=None, centre=(0.0, 0.0)):
        """Admit a solve; returns its slot, or None if the pool has no room now."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        e = np.ascontiguousarray(e, dtype=np.float64).reshape(-1, 2)
        m = None if rho_u_T is None else np.ascontiguousarray(rho_u_T, dtype=np.float64)
        d = SolveDesc(r.size, e.shape[0], _dptr(r), _dptr(e), centre[0], centre[1], body_desc(body),
                      flow_params(flow), None if m is None else _dptr(m), int(steps))
        slot = ctypes.c_int(-1)
        rc = self._lib.lbfsi_batch_add(self.h, ctypes.byref(d), ctypes.byref(slot))
        if rc == ENOMEM:
            return None
        _check(rc)
        self._shapes[slot.value] = (r.size, e.shape[0])
        return slot.value

    def add_xy(self, X, body, flow, steps, rho_u_T=None, centre=(0.0, 0.0)):
        """Admit a solve on an O-grid given by node coordinates X [nr, ntheta, 2];
        returns its slot, or None if the pool has no room now."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        m = None if rho_u_T is None else np.ascontiguousarray(rho_u_T, dtype=np.float64)
        d = SolveXYDesc(X.shape[0], X.shape[1], _dptr(X), centre[0], centre[1], body_desc(body),
                        flow_params(flow), None if m is None else _dptr(m), int(steps))
        slot = ctypes.c_int(-1)
        rc = self._lib.lbfsi_batch_add_xy(self.h, ctypes.byref(d), ctypes.byref(slot))
        if rc == ENOMEM:
            return None
        _check(rc)
        self._shapes[slot.value] = (X.shape[0], X.shape[1])
        return slot.value

    def add_cgrid(self, X, n_cut, body, flow, steps, rho_u_T=None, centre=(0.0, 0.0)):
        """Admit a solve on a C-grid X [nr, ntheta, 2] with n_cut cut nodes
        per side; returns its slot, or None if the pool has no room now."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        m = None if rho_u_T is None else np.ascontiguousarray(rho_u_T, dtype=np.float64)
        d = SolveCGridDesc(X.shape[0], X.shape[1], int(n_cut), _dptr(X), centre[0], centre[1],
                           body_desc(body), flow_params(flow), None if m is None else _dptr(m), int(steps))
        slot = ctypes.c_int(-1)
        rc = self._lib.lbfsi_batch_add_cgrid(self.h, ctypes.byref(d), ctypes.byref(slot))
        if rc == ENOMEM:
            return None
        _check(rc)
        self._shapes[slot.value] = (X.shape[0], X.shape[1])
        return slot.value

    def step(self, n=1):
        act = ctypes.c_int(0)
        _check(self._lib.lbfsi_batch_step(self.h, int(n), ctypes.byref(act)))
        return act.value

    def poll(self, slot):
        done = ctypes.c_int(0)
        fin = ctypes.c_int(0)
        _check(self._lib.lbfsi_batch_poll(self.h, slot, ctypes.byref(done), ctypes.byref(fin)))
        return done.value, bool(fin.value)

    def get(self, slot, fields=True):
        nr, nt = self._shapes[slot]
        f = np.empty((4, nr, nt)) if fields else None
        loads = np.empty(3)
        st = BodyState()
        _check(self._lib.lbfsi_batch_get(self.h, slot, None if f is None else _dptr(f), _dptr(loads),
                                         ctypes.byref(st)))
        return f, loads, dict(h=st.h, alpha=st.alpha, hdot=st.hdot, adot=st.adot)

    def remove(self, slot):
        _check(self._lib.lbfsi_batch_remove(self.h, slot))
        self._shapes.pop(slot, None)

    def set_schedule(self, variant, order=0):
        _check(self._lib.lbfsi_batch_set_schedule(self.h, int(variant), int(order)))

    def schedule(self):
        v, o = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.lbfsi_batch_get_schedule(self.h, ctypes.byref(v), ctypes.byref(o)))
        return v.value, o.value

    def set_graph_steps(self, n):
        _check(self._lib.lbfsi_batch_set_graph_steps(self.h, int(n)))

    def autotune(self, steps_per_trial=20):
        """Returns (variant, order, ns per node update [variants][2])."""
        nv = step_variants(self.precision)
        ns = (ctypes.c_float * (2 * nv))()
        v, o = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.lbfsi_batch_autotune(self.h, int(steps_per_trial), ctypes.byref(v), ctypes.byref(o), ns))
        return v.value, o.value, np.array(ns, dtype=np.float64).reshape(nv, 2)

    def memory(self):
        fb = ctypes.c_size_t(0)
        lg = ctypes.c_size_t(0)
        _check(self._lib.lbfsi_batch_memory(self.h, ctypes.byref(fb), ctypes.byref(lg)))
        return fb.value, lg.value


class ElementMesh:
    """Handle of an unstructured Q2 element list (lbfsi_create_mesh_elements):
    X [N, 2], elements [Ne, 3, 3] node indices, wall and far chains (node
    indices, counterclockwise), bodies (one per solve); grid_ij [N, 2] with
    grid (nr, nt) selects the structured gradient stencil (reading R18)."""

    def __init__(self, X, elements, wall, far, bodies, precision=FP64, stream=None, grid_ij=None,
                 grid=(0, 0)):
        lib = load()
        self._lib = lib
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.E = np.ascontiguousarray(elements, dtype=np.int32)
        self.wall = np.ascontiguousarray(wall, dtype=np.int32)
        self.far = np.ascontiguousarray(far, dtype=np.int32)
        self.N = self.X.shape[0]
        self.nbatch = len(bodies)
        self.precision = precision
        ip = ctypes.POINTER(ctypes.c_int)
        self._bodies = (BodyDesc * self.nbatch)(*[body_desc(b) for b in bodies])
        gij = None if grid_ij is None else np.ascontiguousarray(grid_ij, dtype=np.int32)
        d = MeshElementsDesc(self.N, _dptr(self.X), self.E.shape[0], self.E.ctypes.data_as(ip),
                             len(self.wall), self.wall.ctypes.data_as(ip), len(self.far),
                             self.far.ctypes.data_as(ip), None if gij is None else gij.ctypes.data_as(ip),
                             int(grid[0]), int(grid[1]), self.nbatch, self._bodies, precision)
        h = ctypes.c_void_p()
        _check(lib.lbfsi_create_mesh_elements(ctypes.byref(d), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self._lib.lbfsi_emesh_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def init_fields(self, flow, rho_u_T=None):
        fp = flow_params(flow)
        if rho_u_T is None:
            _check(self._lib.lbfsi_emesh_init_fields(self.h, ctypes.byref(fp), None))
        else:
            a = np.ascontiguousarray(rho_u_T, dtype=np.float64).reshape(self.nbatch, 4, self.N)
            _check(self._lib.lbfsi_emesh_init_fields(self.h, ctypes.byref(fp), _dptr(a)))

    def blend_mesh(self, states, prev=None):
        s = (BodyState * self.nbatch)(*[BodyState(*x) for x in states])
        pv = None if prev is None else (BodyState * self.nbatch)(*[BodyState(*x) for x in prev])
        _check(self._lib.lbfsi_emesh_blend_mesh(self.h, s, pv))

    def step(self, n=1):
        _check(self._lib.lbfsi_emesh_step(self.h, int(n)))

    def synchronize(self):
        _check(self._lib.lbfsi_emesh_synchronize(self.h))

    def body_forces(self):
        out = np.empty((self.nbatch, 3))
        _check(self._lib.lbfsi_emesh_body_forces(self.h, _dptr(out)))
        return out

    def body_state(self):
        out = (BodyState * self.nbatch)()
        _check(self._lib.lbfsi_emesh_get_body_state(self.h, out))
        return [dict(h=s.h, alpha=s.alpha, hdot=s.hdot, adot=s.adot) for s in out]

    def get_fields(self):
        out = np.empty((self.nbatch, 4, self.N))
        _check(self._lib.lbfsi_emesh_get_fields(self.h, _dptr(out)))
        return out

    def get_populations(self, which=0):
        f = np.empty((self.nbatch, 9, self.N))
        g = np.empty_like(f)
        _check(self._lib.lbfsi_emesh_get_populations(self.h, int(which), _dptr(f), _dptr(g)))
        return f, g

    def launch_count(self):
        return int(self._lib.lbfsi_emesh_launch_count(self.h))
