"""ctypes binding of the solver's C ABI (``include/hqn.h``).

Argument marshalling only: every step of the method runs inside the CUDA
library.  The library must be built (``build.build_library()``); importing
this module without it raises, and there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

HQN_OK = 0
HQN_WARN_LS_EXHAUSTED = 1
HQN_WARN_NONDESCENT = 2
LAYOUT_F32X4, LAYOUT_F64X4 = 1, 2
HQN_ERR_ARG = -1
HQN_ERR_DEGENERATE_TET = -2
HQN_ERR_NONFINITE = -3
HQN_ERR_NOT_SPD = -4
HQN_ERR_CUDA = -5
HQN_ERR_NO_MEMORY = -6
HQN_ERR_UNSUPPORTED = -7
HQN_ERR_DEVICE_TIMEOUT = -8
STATIC_MAX_TETS, STATIC_MAX_VERTS = 65536, 262144

NEOHOOKEAN, STVK, SPLINE_VL, COROTATED, POLY4 = 0, 1, 2, 3, 4
STAGE_TET, STAGE_GATHER, STAGE_SOLVE, STAGE_LS_PASS, STAGE_TWO_LOOP = 0, 1, 2, 3, 4
FP64_PLAIN, FP32_MIXED = 0, 1
MAX_HISTORY, MAX_ITERS = 128, 512

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_up = C.POINTER(C.c_uint8)


class Mesh(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tets", C.c_int32), ("rest_pos", _dp),
                ("tets", _ip), ("clamped", _up), ("n_materials", C.c_int32), ("tet_material", _ip)]


MAX_MATERIALS = 16


class Material(C.Structure):
    _fields_ = [("kind", C.c_int32), ("E", C.c_double), ("nu", C.c_double),
                ("density", C.c_double), ("spline", _dp), ("kappa", C.c_double),
                ("fiber", C.c_double * 3)]


MAX_COLLIDERS = 4
COLLIDER_PLANE, COLLIDER_SPHERE, COLLIDER_TORUS = 1, 2, 3


class Collider(C.Structure):
    _fields_ = [("kind", C.c_int32), ("point", C.c_double * 3), ("normal", C.c_double * 3),
                ("radius", C.c_double), ("major_radius", C.c_double)]


class Params(C.Structure):
    _fields_ = [("h", C.c_double), ("gamma", C.c_double), ("backtrack", C.c_double),
                ("x_start", C.c_double), ("x_end", C.c_double), ("gravity", C.c_double * 3),
                ("iters", C.c_int32), ("history_m", C.c_int32), ("ls_max", C.c_int32),
                ("precision", C.c_int32), ("leaf_size", C.c_int32), ("use_graph", C.c_int32),
                ("tet_block", C.c_int32), ("ls_batch", C.c_int32), ("solve_threads", C.c_int32),
                ("solve_item_kb", C.c_int32), ("solve_items", C.c_int32), ("solve_leaf_kb", C.c_int32),
                ("solve_leaf_threads", C.c_int32), ("solve_dense_top", C.c_int32), ("solve_prefetch", C.c_int32),
                ("solve_dense_prefetch", C.c_int32), ("n_colliders", C.c_int32), ("contact_scale", C.c_double),
                ("colliders", Collider * MAX_COLLIDERS), ("a0_solver", C.c_int32), ("pcg_iters", C.c_int32),
                ("direction", C.c_int32), ("cheb_S", C.c_int32), ("cheb_rho", C.c_double),
                ("merge_depths", C.c_int32), ("wait_polls", C.c_int32), ("fault_test", C.c_int32),
                ("tune_cache", C.c_char_p)]


class StepStats(C.Structure):
    _fields_ = [("steps", C.c_int32), ("iters", C.c_int32), ("status", C.c_int32),
                ("trials_total", C.c_int32), ("iters_total", C.c_int32),
                ("trials", C.c_int32 * MAX_ITERS), ("g0", C.c_double),
                ("g", C.c_double * MAX_ITERS), ("ls_passes_total", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tets", C.c_int32), ("n_free", C.c_int32),
                ("n_supernodes", C.c_int32), ("n_levels", C.c_int32),
                ("factor_entries", C.c_int64), ("factor_nnz", C.c_int64),
                ("stiffness_k", C.c_double), ("setup_seconds", C.c_double),
                ("device_bytes", C.c_int64), ("precision", C.c_int32),
                ("graph_mode", C.c_int32), ("n_update_entries", C.c_int64),
                ("chained_sweeps", C.c_int32), ("solve_threads", C.c_int32), ("solve_item_kb", C.c_int32),
                ("solve_items", C.c_int32), ("solve_leaf_kb", C.c_int32), ("solve_leaf_threads", C.c_int32),
                ("solve_prefetch", C.c_int32), ("solve_dense_prefetch", C.c_int32), ("solve_dense_top", C.c_int32),
                ("dense_top_cols", C.c_int32), ("n_sims", C.c_int32)]


_lib = None


def library(path: str | None = None):
    """Loads libhqn.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.build_library()
    if not os.path.exists(path):
        raise RuntimeError(f"solver library not found at {path}")
    lib = C.CDLL(path)
    lib.hqn_default_params.argtypes = [C.POINTER(Params)]
    lib.hqn_default_params.restype = None
    lib.sim_create.argtypes = [C.POINTER(Mesh), C.POINTER(Material), C.POINTER(Params), C.c_void_p,
                               C.POINTER(C.c_void_p)]
    lib.sim_create.restype = C.c_int
    lib.sim_batch_create.argtypes = [C.c_int32, C.POINTER(Mesh), C.POINTER(Material), C.POINTER(Params),
                                     C.c_void_p, C.POINTER(C.c_void_p)]
    lib.sim_batch_create.restype = C.c_int
    lib.sim_batch_count.argtypes = [C.c_void_p]
    lib.sim_batch_count.restype = C.c_int32
    lib.sim_batch_set_state.argtypes = [C.c_void_p, C.c_int32, _dp, _dp]
    lib.sim_batch_get_state.argtypes = [C.c_void_p, C.c_int32, _dp, _dp]
    lib.sim_batch_get_stats.argtypes = [C.c_void_p, C.c_int32, C.POINTER(StepStats)]
    lib.sim_set_state.argtypes = [C.c_void_p, _dp, _dp]
    lib.sim_get_state.argtypes = [C.c_void_p, _dp, _dp]
    lib.sim_step.argtypes = [C.c_void_p, C.c_int32, C.POINTER(StepStats)]
    lib.sim_energy_grad.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
    lib.sim_solve_A0.argtypes = [C.c_void_p, _dp, _dp]
    lib.sim_energy_grad_device.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, _dp, C.c_void_p]
    lib.sim_energy_grad_device.restype = C.c_int
    lib.sim_direction.argtypes = [C.c_void_p, _dp, C.c_int32, _dp, _dp, _dp]
    lib.sim_get_info.argtypes = [C.c_void_p, C.POINTER(Info)]
    lib.hqn_measure_peak.argtypes = [C.c_int32, _dp]
    lib.hqn_measure_peak.restype = C.c_int
    lib.sim_set_solve_shapes.argtypes = [C.c_void_p, C.POINTER(Params)]
    lib.sim_set_solve_shapes.restype = C.c_int
    lib.hqn_mesh_key.argtypes = [C.POINTER(Mesh)]
    lib.hqn_mesh_key.restype = C.c_uint64
    lib.hqn_tune_lookup.argtypes = [C.c_char_p, C.c_char_p, C.c_uint64, C.c_int32, C.POINTER(Params)]
    lib.hqn_tune_lookup.restype = C.c_int
    lib.hqn_analyse.argtypes = [C.POINTER(Mesh), C.POINTER(Material), C.POINTER(Params), C.POINTER(Info)]
    lib.sim_positions_device.argtypes = [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int32)]
    lib.sim_time_stage.argtypes = [C.c_void_p, C.c_int32, C.c_int32, _dp]
    lib.sim_destroy.argtypes = [C.c_void_p]
    lib.sim_destroy.restype = None
    lib.sim_strerror.argtypes = [C.c_int]
    lib.sim_strerror.restype = C.c_char_p
    lib.hqn_last_error.argtypes = []
    lib.hqn_last_error.restype = C.c_char_p
    lib.hqn_energy_grad_static.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.POINTER(Material), C.c_double,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.hqn_energy_grad_static.restype = C.c_int
    for f in ("sim_set_state", "sim_get_state", "sim_step", "sim_energy_grad", "sim_solve_A0",
              "sim_direction", "sim_get_info", "sim_time_stage", "sim_batch_set_state",
              "sim_batch_get_state", "sim_batch_get_stats"):
        getattr(lib, f).restype = C.c_int
    _lib = lib
    return lib


class HQNError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def _check(code, what):
    if code < 0:
        lib = library()
        raise HQNError(code, f"{what}: {lib.sim_strerror(code).decode()}: "
                             f"{lib.hqn_last_error().decode()}")
    return code


def _ptr(a, ctype=_dp):
    return a.ctypes.data_as(ctype)


def measure_peak(precision=FP32_MIXED) -> float:
    """``hqn_measure_peak``: the current device's non-tensor FMA FLOP/s."""
    v = C.c_double()
    _check(library().hqn_measure_peak(precision, C.byref(v)), "hqn_measure_peak")
    return v.value


def default_params(**kw) -> Params:
    p = Params()
    library().hqn_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "gravity":
            p.gravity[:] = list(v)
        elif k == "tune_cache":
            p.tune_cache = None if v is None else os.fsencode(v)
        elif k == "colliders":
            cols = list(v)
            if len(cols) > MAX_COLLIDERS:
                raise ValueError(f"at most {MAX_COLLIDERS} colliders")
            p.n_colliders = len(cols)
            for i, c in enumerate(cols):
                # workloads.Collider or a ("plane", point, normal) / ("sphere", centre, radius) /
                # ("torus", centre, axis, ring radius, tube radius) tuple
                t = c.as_tuple() if hasattr(c, "as_tuple") else tuple(c)
                cc = p.colliders[i]
                cc.point[:] = list(t[1])
                if t[0] == "plane":
                    cc.kind = COLLIDER_PLANE
                    cc.normal[:] = list(t[2])
                elif t[0] == "sphere":
                    cc.kind = COLLIDER_SPHERE
                    cc.radius = float(t[2])
                elif t[0] == "torus":
                    cc.kind = COLLIDER_TORUS
                    cc.normal[:] = list(t[2])
                    cc.major_radius = float(t[3])
                    cc.radius = float(t[4])
                else:
                    raise ValueError(f"unknown collider {t[0]!r}")
        else:
            setattr(p, k, v)
    return p


def _material_struct(m, keep):
    """hqn_material of a workloads.Material (its spline array kept in `keep`)."""
    sp = None if m.spline is None else np.ascontiguousarray(m.spline, dtype=np.float64)
    keep.append(sp)
    return Material(m.kind, m.E, m.nu, m.density, None if sp is None else _ptr(sp),
                    float(getattr(m, "kappa", 0.0)), (C.c_double * 3)(*getattr(m, "fiber", (0.0, 0.0, 0.0))))


class _MeshArgs:
    """hqn_mesh and hqn_material views of caller arrays (kept alive here).
    extra_materials (workloads.Material) and tet_material: several materials
    in the mesh, material 0 being the one given by kind, E, nu, ...."""

    def __init__(self, rest_pos, tets, clamped, kind, E, nu, density, spline, kappa, fiber,
                 extra_materials=(), tet_material=None):
        self.X = np.ascontiguousarray(rest_pos, dtype=np.float64)
        self.tets = np.ascontiguousarray(tets, dtype=np.int32)
        self.n = self.X.shape[0]
        self.cl = None if clamped is None else np.ascontiguousarray(clamped, dtype=np.uint8)
        nm = 1 + len(extra_materials)
        self.tm = None if nm == 1 else np.ascontiguousarray(tet_material, dtype=np.int32)
        self.mesh = Mesh(self.n, self.tets.shape[0], _ptr(self.X), _ptr(self.tets, _ip),
                         None if self.cl is None else _ptr(self.cl, _up), nm,
                         None if self.tm is None else _ptr(self.tm, _ip))
        self.spline = None if spline is None else np.ascontiguousarray(spline, dtype=np.float64)
        self._keep = []
        self.mats = (Material * nm)()
        self.mats[0] = Material(kind, E, nu, density, None if self.spline is None else _ptr(self.spline),
                                float(kappa), (C.c_double * 3)(*fiber))
        for i, m in enumerate(extra_materials):
            self.mats[1 + i] = _material_struct(m, self._keep)
        self.mat = self.mats[0]


def _workload_kwargs(w, pkw):
    """Mesh, material and parameter keywords of a workloads.Workload."""
    m = w.material
    pkw.setdefault("iters", w.iters)
    pkw.setdefault("history_m", w.history)
    pkw.setdefault("h", w.h)
    pkw.setdefault("gravity", w.gravity)
    if getattr(w, "colliders", ()):
        pkw.setdefault("colliders", w.colliders)
        pkw.setdefault("contact_scale", w.contact_scale)
    extra = tuple(getattr(w, "extra_materials", ()))
    if extra:
        pkw.setdefault("extra_materials", extra)
        pkw.setdefault("tet_material", w.tet_material)
    return (w.rest_pos, w.tets, w.clamped), dict(kind=m.kind, E=m.E, nu=m.nu, density=m.density,
                                                 spline=m.spline, kappa=getattr(m, "kappa", 0.0),
                                                 fiber=getattr(m, "fiber", (0.0, 0.0, 0.0)), **pkw)


def analyse(rest_pos, tets, clamped=None, *, kind=NEOHOOKEAN, E=1e5, nu=0.45, density=1000.0,
            spline=None, kappa=0.0, fiber=(0.0, 0.0, 0.0), extra_materials=(), tet_material=None,
            params: Params | None = None, **pkw) -> dict:
    """Host-only set-up statistics of one mesh (``hqn_analyse``; no GPU):
    the factor's supernodes, levels and entries, the fitted stiffness."""
    a = _MeshArgs(rest_pos, tets, clamped, kind, E, nu, density, spline, kappa, fiber, extra_materials,
                  tet_material)
    p = params if params is not None else default_params(**pkw)
    i = Info()
    _check(library().hqn_analyse(C.byref(a.mesh), a.mats, C.byref(p), C.byref(i)), "hqn_analyse")
    return {f: getattr(i, f) for f, _ in Info._fields_}


def analyse_workload(w, **pkw) -> dict:
    args, kw = _workload_kwargs(w, pkw)
    return analyse(*args, **kw)


class Sim:
    """One simulation handle (``sim_create`` ... ``sim_destroy``)."""

    def __init__(self, rest_pos, tets, clamped=None, *, kind=NEOHOOKEAN, E=1e5, nu=0.45,
                 density=1000.0, spline=None, kappa=0.0, fiber=(0.0, 0.0, 0.0), extra_materials=(),
                 tet_material=None, params: Params | None = None, stream=None, **pkw):
        lib = library()
        self._args = _MeshArgs(rest_pos, tets, clamped, kind, E, nu, density, spline, kappa, fiber,
                               extra_materials, tet_material)
        self.n = self._args.n
        self.params = params if params is not None else default_params(**pkw)
        h = C.c_void_p()
        _check(lib.sim_create(C.byref(self._args.mesh), self._args.mats, C.byref(self.params),
                              C.c_void_p(stream or 0), C.byref(h)), "sim_create")
        self._h = h
        self.last_status = 0

    @classmethod
    def from_workload(cls, w, **pkw):
        args, kw = _workload_kwargs(w, pkw)
        return cls(*args, **kw)

    def close(self):
        if getattr(self, "_h", None):
            library().sim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _vec(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != (self.n, 3):
            raise ValueError(f"expected shape ({self.n}, 3), got {a.shape}")
        return a

    def set_state(self, q_cur, q_prev=None):
        qc = self._vec(q_cur)
        qp = None if q_prev is None else self._vec(q_prev)
        _check(library().sim_set_state(self._h, _ptr(qc), None if qp is None else _ptr(qp)),
               "sim_set_state")

    def get_state(self):
        qc = np.empty((self.n, 3))
        qp = np.empty((self.n, 3))
        _check(library().sim_get_state(self._h, _ptr(qc), _ptr(qp)), "sim_get_state")
        return qc, qp

    def step(self, nsteps=1, stats=False):
        st = StepStats()
        rc = _check(library().sim_step(self._h, nsteps, C.byref(st) if stats else None), "sim_step")
        self.last_status = rc
        if not stats:
            return rc
        k = st.iters
        return rc, {"steps": st.steps, "iters": k, "status": st.status,
                    "trials_total": st.trials_total, "iters_total": st.iters_total,
                    "trials": list(st.trials[:k]), "g0": st.g0, "g": list(st.g[:k]),
                    "ls_passes_total": st.ls_passes_total}

    def energy_grad(self, x, y):
        x, y = self._vec(x), self._vec(y)
        g = C.c_double()
        grad = np.empty((self.n, 3))
        _check(library().sim_energy_grad(self._h, _ptr(x), _ptr(y), C.byref(g), _ptr(grad)),
               "sim_energy_grad")
        return g.value, grad

    def energy_grad_device(self, x, y, grad=None):
        """``sim_energy_grad_device``: x, y are torch float64 CUDA tensors
        (n x 3, caller order); returns (g, grad) with grad a torch tensor on
        the same device (the given one if passed)."""
        import torch
        for t in (x, y):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and tuple(t.shape) == (self.n, 3)):
                raise ValueError("expected contiguous float64 CUDA tensors of shape (n, 3)")
        if grad is None:
            grad = torch.empty_like(x)
        g = C.c_double()
        _check(library().sim_energy_grad_device(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                                C.byref(g), C.c_void_p(grad.data_ptr())), "sim_energy_grad_device")
        return g.value, grad

    def solve_A0(self, q):
        q = self._vec(q)
        r = np.empty((self.n, 3))
        _check(library().sim_solve_A0(self._h, _ptr(q), _ptr(r)), "sim_solve_A0")
        return r

    def direction(self, grad, s_list=(), t_list=()):
        grad = self._vec(grad)
        npairs = len(s_list)
        d = np.empty((self.n, 3))
        if npairs:
            s = np.ascontiguousarray(np.stack([self._vec(v) for v in s_list]))
            t = np.ascontiguousarray(np.stack([self._vec(v) for v in t_list]))
            sp, tp = _ptr(s), _ptr(t)
        else:
            sp = tp = None
        _check(library().sim_direction(self._h, _ptr(grad), npairs, sp, tp, _ptr(d)),
               "sim_direction")
        return d

    def set_solve_shapes(self, **shapes):
        """``sim_set_solve_shapes``: re-plans the sweeps on this handle with the
        given solve_* fields (the others at their defaults)."""
        p = Params()
        for k, v in shapes.items():
            if not k.startswith("solve_") or k == "solve_dense_top":
                raise ValueError(f"not a re-plannable sweep shape: {k}")
            setattr(p, k, v)
        _check(library().sim_set_solve_shapes(self._h, C.byref(p)), "sim_set_solve_shapes")

    def time_stage(self, stage, reps=20):
        """Mean device milliseconds of one launch of a stage (CUDA events on the
        handle's stream)."""
        ms = C.c_double()
        _check(library().sim_time_stage(self._h, stage, reps, C.byref(ms)), "sim_time_stage")
        return ms.value

    def info(self) -> dict:
        i = Info()
        _check(library().sim_get_info(self._h, C.byref(i)), "sim_get_info")
        return {f: getattr(i, f) for f, _ in Info._fields_}

    def positions_device(self):
        """``sim_positions_device``: a torch view (n x 4, float32 or float64,
        caller's vertex order, w = 0) of the handle's device copy of q_l.
        The view borrows the handle's buffer: it is valid until the next
        positions_device, step, set_state or close."""
        import torch
        ptr, layout = C.c_void_p(), C.c_int32()
        _check(library().sim_positions_device(self._h, C.byref(ptr), C.byref(layout)), "sim_positions_device")
        typestr = {LAYOUT_F32X4: "<f4", LAYOUT_F64X4: "<f8"}[layout.value]

        class _View:
            __cuda_array_interface__ = {"shape": (self.n, 4), "typestr": typestr,
                                        "data": (ptr.value, False), "version": 3, "strides": None}
        return torch.as_tensor(_View(), device="cuda")


class Batch:
    """A batch of independent simulations advanced together (``sim_batch_create``).

    ``workloads`` is a list of objects with the fields of ``workloads.Workload``
    (mesh, clamps, material); the parameters (h, iterations, history window,
    precision, ...) are shared and come from ``pkw`` / ``params``.
    """

    def __init__(self, workloads, *, params: Params | None = None, stream=None, **pkw):
        lib = library()
        ws = list(workloads)
        if not ws:
            raise ValueError("empty batch")
        self._keep = []
        meshes = (Mesh * len(ws))()
        all_mats = []
        self.n = []
        for k, w in enumerate(ws):
            X = np.ascontiguousarray(w.rest_pos, dtype=np.float64)
            tets = np.ascontiguousarray(w.tets, dtype=np.int32)
            cl = None if w.clamped is None else np.ascontiguousarray(w.clamped, dtype=np.uint8)
            ms = (w.material,) + tuple(getattr(w, "extra_materials", ()))
            tm = None if len(ms) == 1 else np.ascontiguousarray(w.tet_material, dtype=np.int32)
            self._keep += [X, tets, cl, tm]
            meshes[k] = Mesh(X.shape[0], tets.shape[0], _ptr(X), _ptr(tets, _ip),
                             None if cl is None else _ptr(cl, _up), len(ms), None if tm is None else _ptr(tm, _ip))
            all_mats += [_material_struct(m, self._keep) for m in ms]
            self.n.append(X.shape[0])
        mats = (Material * len(all_mats))(*all_mats)
        w0 = ws[0]
        pkw.setdefault("iters", w0.iters)
        pkw.setdefault("history_m", w0.history)
        pkw.setdefault("h", w0.h)
        pkw.setdefault("gravity", w0.gravity)
        if getattr(w0, "colliders", ()):
            pkw.setdefault("colliders", w0.colliders)
            pkw.setdefault("contact_scale", w0.contact_scale)
        self.params = params if params is not None else default_params(**pkw)
        h = C.c_void_p()
        _check(lib.sim_batch_create(len(ws), meshes, mats, C.byref(self.params), C.c_void_p(stream or 0),
                                    C.byref(h)), "sim_batch_create")
        self._h = h
        self.count = len(ws)

    def close(self):
        if getattr(self, "_h", None):
            library().sim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _vec(self, i, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != (self.n[i], 3):
            raise ValueError(f"expected shape ({self.n[i]}, 3), got {a.shape}")
        return a

    def set_state(self, i, q_cur, q_prev=None):
        qc = self._vec(i, q_cur)
        qp = None if q_prev is None else self._vec(i, q_prev)
        _check(library().sim_batch_set_state(self._h, i, _ptr(qc), None if qp is None else _ptr(qp)),
               "sim_batch_set_state")

    def get_state(self, i):
        qc = np.empty((self.n[i], 3))
        qp = np.empty((self.n[i], 3))
        _check(library().sim_batch_get_state(self._h, i, _ptr(qc), _ptr(qp)), "sim_batch_get_state")
        return qc, qp

    def step(self, nsteps=1):
        st = StepStats()
        rc = _check(library().sim_step(self._h, nsteps, C.byref(st)), "sim_step")
        return rc, {"trials_total": st.trials_total, "iters_total": st.iters_total,
                    "ls_passes_total": st.ls_passes_total, "status": st.status}

    def stats(self, i):
        st = StepStats()
        _check(library().sim_batch_get_stats(self._h, i, C.byref(st)), "sim_batch_get_stats")
        k = st.iters
        return {"steps": st.steps, "iters": k, "status": st.status, "trials_total": st.trials_total,
                "iters_total": st.iters_total, "trials": list(st.trials[:k]), "g0": st.g0,
                "g": list(st.g[:k]), "ls_passes_total": st.ls_passes_total}

    def time_stage(self, stage, reps=20):
        ms = C.c_double()
        _check(library().sim_time_stage(self._h, stage, reps, C.byref(ms)), "sim_time_stage")
        return ms.value

    def info(self) -> dict:
        i = Info()
        _check(library().sim_get_info(self._h, C.byref(i)), "sim_get_info")
        return {f: getattr(i, f) for f, _ in Info._fields_}
