"""Thin ctypes binding of libcgks (include/cgks.h).

Argument marshalling only: every step of the solver runs in the CUDA
library.  PyTorch supplies device memory (through the allocator callback)
and the stream the library synchronises with.  There is no CPU fallback:
if libcgks.so is missing or no CUDA device is usable, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

TRI, QUAD, TET, PRISM, PYRAMID, HEX = 0, 1, 2, 3, 4, 5
BC_SLIP, BC_NOSLIP, BC_FARFIELD, BC_DIRICHLET, BC_OUTFLOW = 0, 1, 2, 3, 4
S1O2, S2O4 = 0, 1
FP64, MIXED = 0, 1
FLUX_KFVS, FLUX_LF = 0, 1
FLUX_SMOOTH, FLUX_FULL = 0, 1
WENO_CONSERVATIVE, WENO_CHARACTERISTIC = 0, 1
SWEEP_COLOUR, SWEEP_PARTITIONED = 0, 1
MAX_BC = 16
OK, EINVAL, ENOMEM, EMESH, ECUDA, EDIVERGED, ETIMEOUT, EBUDGET = 0, -1, -2, -3, -4, -5, -6, -7

STATUS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "mesh rejected", -4: "CUDA error",
          -5: "diverged", -6: "timeout", -7: "memory budget exceeded"}


class CgksError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {lib().cgks_strerror(status).decode()} ({status})")


class CgksBC(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad_", C.c_int32), ("u_wall", C.c_double * 3),
                ("rho", C.c_double), ("u", C.c_double * 3), ("p", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class CgksParams(C.Structure):
    _fields_ = [("gamma", C.c_double), ("mu", C.c_double), ("alpha", C.c_double),
                ("cfl_hi", C.c_double), ("cfl_lo", C.c_double),
                ("n_implicit", C.c_int32), ("n_sweeps", C.c_int32), ("time_scheme", C.c_int32),
                ("precision", C.c_int32), ("n_bc", C.c_int32), ("use_graph", C.c_int32),
                ("low_order_fused", C.c_int32), ("autotune", C.c_int32), ("programmatic_launch", C.c_int32),
                ("flux_lo", C.c_int32), ("flux_hi", C.c_int32), ("weno_vars", C.c_int32),
                ("sweep_order", C.c_int32), ("sweep_part_cells", C.c_int32),
                ("lo_viscous", C.c_int32), ("pad2_", C.c_int32),
                ("tau_c1", C.c_double), ("tau_c2", C.c_double), ("weno_eps", C.c_double), ("weno_g0", C.c_double),
                ("bc", CgksBC * MAX_BC),
                ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p)]


TUNE_KERNELS = 4
TUNE_SHAPES = 5
TUNE_NAMES = ("k_recon", "k_face", "k_lo_face", "k_sweep")


class CgksTuning(C.Structure):
    _fields_ = [("shape", C.c_int32 * TUNE_KERNELS), ("done", C.c_int32 * TUNE_KERNELS),
                ("ms", (C.c_double * TUNE_SHAPES) * TUNE_KERNELS)]


def _tuning_dict(t: CgksTuning) -> dict:
    return {name: dict(shape=int(t.shape[k]), done=bool(t.done[k]), ms=[float(x) for x in t.ms[k]])
            for k, name in enumerate(TUNE_NAMES)}


class CgksMeshInfo(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("n_faces", C.c_int64), ("n_bfaces", C.c_int64),
                ("n_colours", C.c_int32), ("dim", C.c_int32), ("device_bytes", C.c_int64)]


_dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")

# every entry point of include/cgks.h with its ctypes signature
SIGNATURES = {
    "cgks_default_params": (None, [C.POINTER(CgksParams)]),
    "cgks_strerror": (C.c_char_p, [C.c_int]),
    "cgks_mesh_create": (C.c_int, [C.c_int, C.c_int64, _dp, C.c_int64, _u8p, _i64p, _i64p, C.c_int64,
                                   _i64p, _i64p, _i32p, C.POINTER(C.c_void_p)]),
    "cgks_mesh_info": (C.c_int, [C.c_void_p, C.POINTER(CgksMeshInfo)]),
    "cgks_mesh_ordering": (C.c_int, [C.c_void_p, _i64p, _i32p]),
    "cgks_mesh_destroy": (C.c_int, [C.c_void_p]),
    "cgks_solver_create": (C.c_int, [C.c_void_p, C.POINTER(CgksParams), C.POINTER(C.c_void_p)]),
    "cgks_solver_destroy": (C.c_int, [C.c_void_p]),
    "cgks_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "cgks_set_state_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "cgks_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "cgks_get_state_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "cgks_highorder_step": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_double)]),
    "cgks_explicit_steps": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "cgks_loworder_smooth": (C.c_int, [C.c_void_p]),
    "cgks_pmg_cycle": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "cgks_residual": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "cgks_get_rp0": (C.c_int, [C.c_void_p, _dp]),
    "cgks_set_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "cgks_get_timing": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_char_p), C.c_void_p, C.c_void_p]),
    "cgks_reset_timing": (C.c_int, [C.c_void_p]),
    "cgks_launch_count": (C.c_int64, [C.c_void_p]),
    "cgks_launches_per_call": (C.c_int, [C.c_void_p, C.c_int]),
    "cgks_wall_loads": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_int64), C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p]),
    "cgks_tune_shape": (C.c_int, [C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "cgks_get_tuning": (C.c_int, [C.c_void_p, C.POINTER(CgksTuning)]),
    "cgks_set_tuning": (C.c_int, [C.c_void_p, _i32p]),
    "cgks_set_barrier_spin_limit": (C.c_int, [C.c_void_p, C.c_int64]),
    "cgks_density_residual_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
}


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libcgks.so (building it with nvcc if absent or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing and _build.needs_build():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libcgks.so is not built; run paper_2109_09965_gb300/build.py")
            L = C.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc, what):
    if rc != 0:
        raise CgksError(rc, what)


def _check_or(rc, what, ok):
    if rc not in ok:
        raise CgksError(rc, what)


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


class Mesh:
    """Mesh handle built from raw node / cell / boundary arrays (meshgen.Mesh)."""

    def __init__(self, m):
        L = lib()
        h = C.c_void_p()
        rc = L.cgks_mesh_create(int(m.dim), m.nodes.shape[0], np.ascontiguousarray(m.nodes, np.float64),
                                m.cell_type.shape[0], np.ascontiguousarray(m.cell_type, np.uint8),
                                np.ascontiguousarray(m.cell_ptr, np.int64),
                                np.ascontiguousarray(m.cell_nodes, np.int64), m.bface_tag.shape[0],
                                np.ascontiguousarray(m.bface_ptr, np.int64),
                                np.ascontiguousarray(m.bface_nodes, np.int64),
                                np.ascontiguousarray(m.bface_tag, np.int32), C.byref(h))
        _check(rc, "cgks_mesh_create")
        self._h = h
        info = CgksMeshInfo()
        _check(L.cgks_mesh_info(h, C.byref(info)), "cgks_mesh_info")
        self.n_cells = info.n_cells
        self.n_faces = info.n_faces
        self.n_bfaces = info.n_bfaces
        self.n_colours = info.n_colours
        self.dim = info.dim
        self.nv = info.dim + 2
        self.device_bytes = info.device_bytes

    def ordering(self):
        rcm = np.zeros(self.n_cells, np.int64)
        col = np.zeros(self.n_cells, np.int32)
        _check(lib().cgks_mesh_ordering(self._h, rcm, col), "cgks_mesh_ordering")
        return rcm, col

    def close(self):
        if getattr(self, "_h", None):
            lib().cgks_mesh_destroy(self._h)
            self._h = None

    __del__ = close


def make_params(spec: dict, stream=None, allocator=None) -> CgksParams:
    """Problem settings from a plain dict (same keys as the bench configs):
    gamma, mu, alpha, cfl_hi, cfl_lo, n_implicit, n_sweeps, time_scheme,
    precision, use_graph, flux_lo ('kfvs' | 'lf'), flux_hi ('smooth' |
    'full'), tau_c1, tau_c2, weno_eps (0: linear weights), weno_g0,
    weno_vars ('conservative' | 'characteristic'), sweep_order ('colour' |
    'partitioned'), sweep_part_cells,
    bcs=[{kind ('slip' | 'noslip' | 'farfield' | 'dirichlet' | 'outflow'),
    uw, rho, u, p}]."""
    P = CgksParams()
    lib().cgks_default_params(C.byref(P))
    for key in ("gamma", "mu", "alpha", "cfl_hi", "cfl_lo", "tau_c1", "tau_c2", "weno_eps", "weno_g0"):
        if key in spec:
            setattr(P, key, float(spec[key]))
    for key in ("n_implicit", "n_sweeps", "use_graph", "low_order_fused", "autotune", "programmatic_launch",
                "sweep_part_cells", "lo_viscous"):
        if key in spec:
            setattr(P, key, int(spec[key]))
    P.sweep_order = {"colour": SWEEP_COLOUR, "partitioned": SWEEP_PARTITIONED}[spec.get("sweep_order", "colour")]
    P.time_scheme = {"S1O2": S1O2, "S2O4": S2O4}[spec.get("time_scheme", "S1O2")]
    P.flux_lo = {"kfvs": FLUX_KFVS, "lf": FLUX_LF}[spec.get("flux_lo", "kfvs")]
    P.flux_hi = {"smooth": FLUX_SMOOTH, "full": FLUX_FULL}[spec.get("flux_hi", "smooth")]
    P.weno_vars = {"conservative": WENO_CONSERVATIVE,
                   "characteristic": WENO_CHARACTERISTIC}[spec.get("weno_vars", "conservative")]
    P.precision = {"fp64": FP64, "mixed": MIXED}[spec.get("precision", "fp64")]
    bcs = spec.get("bcs", [])
    P.n_bc = len(bcs)
    kinds = {"slip": BC_SLIP, "noslip": BC_NOSLIP, "farfield": BC_FARFIELD, "dirichlet": BC_DIRICHLET,
             "outflow": BC_OUTFLOW}
    def vec3(x):
        x = [float(v) for v in x]
        return x + [0.0] * (3 - len(x))
    for i, b in enumerate(bcs):
        P.bc[i].kind = kinds[b["kind"]]
        P.bc[i].u_wall[:] = vec3(b.get("uw", (0.0, 0.0)))
        P.bc[i].rho = float(b.get("rho", 1.0))
        P.bc[i].u[:] = vec3(b.get("u", (0.0, 0.0)))
        P.bc[i].p = float(b.get("p", 1.0 / P.gamma))
    if stream is not None:
        P.stream = C.c_void_p(stream)
    if allocator is not None:
        P.alloc, P.free, P.alloc_ctx = allocator.alloc_fn, allocator.free_fn, None
    return P


class TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.blocks = {}
        self.alloc_fn = ALLOC_FN(self._alloc)
        self.free_fn = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except RuntimeError:
            return None
        p = t.data_ptr()
        self.blocks[p] = t
        return p

    def _free(self, ptr, ctx):
        self.blocks.pop(ptr, None)


class Solver:
    """One steady solve on one mesh; state lives on the device."""

    def __init__(self, mesh: Mesh, spec: dict, use_torch: bool = True):
        L = lib()
        self.mesh = mesh
        self.n_cells = mesh.n_cells
        self.dim, self.nv = mesh.dim, mesh.nv
        stream, self._alloc = None, None
        if use_torch:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("libcgks needs a CUDA device; none is available")
            self._alloc = TorchAllocator()
            stream = torch.cuda.current_stream().cuda_stream
        self.params = make_params(spec, stream=stream, allocator=self._alloc)
        h = C.c_void_p()
        _check(L.cgks_solver_create(mesh._h, C.byref(self.params), C.byref(h)), "cgks_solver_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().cgks_solver_destroy(self._h)
            self._h = None

    __del__ = close

    # -- state --------------------------------------------------------
    def set_state(self, W, Wx=None):
        W = np.ascontiguousarray(W, np.float64).reshape(self.n_cells, self.nv)
        Wx = None if Wx is None else np.ascontiguousarray(Wx, np.float64).reshape(self.n_cells, self.dim, self.nv)
        _check(lib().cgks_set_state(self._h, _ptr(W), _ptr(Wx)), "cgks_set_state")

    def set_state_device(self, W_ptr: int, Wx_ptr: int | None = None):
        _check(lib().cgks_set_state_device(self._h, C.c_void_p(W_ptr), C.c_void_p(Wx_ptr) if Wx_ptr else None),
               "cgks_set_state_device")

    def get_state(self):
        W = np.zeros((self.n_cells, self.nv))
        Wx = np.zeros((self.n_cells, self.dim, self.nv))
        _check(lib().cgks_get_state(self._h, _ptr(W), _ptr(Wx)), "cgks_get_state")
        return W, Wx

    def get_state_device(self, W_ptr: int, Wx_ptr: int | None = None):
        _check(lib().cgks_get_state_device(self._h, C.c_void_p(W_ptr), C.c_void_p(Wx_ptr) if Wx_ptr else None),
               "cgks_get_state_device")

    # -- hot path -----------------------------------------------------
    def highorder_step(self, dt: float = -1.0) -> float:
        used = C.c_double()
        _check(lib().cgks_highorder_step(self._h, float(dt), C.byref(used)), "cgks_highorder_step")
        return used.value

    def explicit_steps(self, n: int, record=True):
        r = np.zeros(max(n, 1)) if record else None
        _check(lib().cgks_explicit_steps(self._h, int(n), _ptr(r)), "cgks_explicit_steps")
        return r[:n] if record else None

    def pmg_cycle(self, n: int, record=True):
        r = np.zeros(max(n, 1)) if record else None
        _check(lib().cgks_pmg_cycle(self._h, int(n), _ptr(r)), "cgks_pmg_cycle")
        return r[:n] if record else None

    def loworder_smooth(self):
        _check(lib().cgks_loworder_smooth(self._h), "cgks_loworder_smooth")

    def residual(self):
        res = C.c_double()
        rl2 = np.zeros(self.nv)
        _check(lib().cgks_residual(self._h, C.byref(res), _ptr(rl2)), "cgks_residual")
        return res.value, rl2

    def rp0(self):
        R = np.zeros((self.n_cells, self.nv))
        _check(lib().cgks_get_rp0(self._h, R.reshape(-1)), "cgks_get_rp0")
        return R

    # -- instrumentation ----------------------------------------------
    def set_timing(self, on: bool):
        _check(lib().cgks_set_timing(self._h, int(bool(on))), "cgks_set_timing")

    def timing(self):
        names = (C.c_char_p * 32)()
        ms = np.zeros(32)
        cnt = np.zeros(32, np.int64)
        k = lib().cgks_get_timing(self._h, 32, names, _ptr(ms), _ptr(cnt))
        return {names[i].decode(): (float(ms[i]), int(cnt[i])) for i in range(k)}

    def reset_timing(self):
        _check(lib().cgks_reset_timing(self._h), "cgks_reset_timing")

    def launch_count(self) -> int:
        return int(lib().cgks_launch_count(self._h))

    def launches_per_call(self, cycle: bool) -> int:
        return int(lib().cgks_launches_per_call(self._h, int(bool(cycle))))

    def wall_loads(self, tag: int) -> dict:
        """Boundary faces of one tag at the current state: centre x, unit
        normal n (out of the fluid), length / area S and the momentum flux
        `traction` the fluid exerts there (pressure and viscous stress)."""
        k = C.c_int64(0)
        _check_or(lib().cgks_wall_loads(self._h, int(tag), 0, C.byref(k), None, None, None, None),
                  "cgks_wall_loads", ok=(0, -1))
        m = k.value
        x, n = np.zeros((m, self.dim)), np.zeros((m, self.dim))
        S, t = np.zeros(m), np.zeros((m, self.dim))
        _check(lib().cgks_wall_loads(self._h, int(tag), m, C.byref(k), _ptr(x), _ptr(n), _ptr(S), _ptr(t)),
               "cgks_wall_loads")
        return dict(x=x, n=n, S=S, traction=t)

    def tuning(self) -> dict:
        """Per tunable kernel: shape index in use, whether it is final, and
        the mean timed launch (ms) of every shape tried."""
        t = CgksTuning()
        _check(lib().cgks_get_tuning(self._h, C.byref(t)), "cgks_get_tuning")
        return _tuning_dict(t)

    def set_tuning(self, shapes):
        """Fix the four launch shapes (indices 0 .. TUNE_SHAPES-1)."""
        a = np.ascontiguousarray(shapes, np.int32)
        if a.shape != (TUNE_KERNELS,):
            raise ValueError("one shape per tunable kernel")
        _check(lib().cgks_set_tuning(self._h, a), "cgks_set_tuning")

    def set_barrier_spin_limit(self, polls: int):
        """Polls per grid-barrier wait of the persistent low-order launch
        before it gives up (0: the default)."""
        _check(lib().cgks_set_barrier_spin_limit(self._h, int(polls)), "cgks_set_barrier_spin_limit")


def tune_shape(shape: int):
    """(block size, items per thread, minimum resident blocks per SM)."""
    b, i, m = C.c_int32(0), C.c_int32(0), C.c_int32(0)
    _check(lib().cgks_tune_shape(int(shape), C.byref(b), C.byref(i), C.byref(m)), "cgks_tune_shape")
    return b.value, i.value, m.value


# ---------------------------------------------------------------- serving
class CgksServerOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("time_scheme", C.c_int32), ("cfl_hi", C.c_double),
                ("cfl_lo", C.c_double), ("n_implicit", C.c_int32), ("n_sweeps", C.c_int32),
                ("max_active", C.c_int32), ("max_cycles", C.c_int32), ("use_graph", C.c_int32),
                ("low_order_fused", C.c_int32), ("autotune", C.c_int32), ("programmatic_launch", C.c_int32),
                ("flux_lo", C.c_int32), ("lo_viscous", C.c_int32), ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p)]


class CgksReqStatus(C.Structure):
    _fields_ = [("state", C.c_int32), ("cycles", C.c_int32), ("res_first", C.c_double),
                ("res_last", C.c_double), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("n_cells", C.c_int64)]


REQ_STATES = {0: "queued", 1: "active", 2: "converged", 3: "stopped", 4: "diverged", 5: "rejected"}

SIGNATURES.update({
    "cgks_server_default_opts": (None, [C.POINTER(CgksServerOpts)]),
    "cgks_server_create": (C.c_int, [C.c_size_t, C.POINTER(CgksServerOpts), C.POINTER(C.c_void_p)]),
    "cgks_server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(CgksParams), _dp, C.c_double,
                                     C.c_int32, C.POINTER(C.c_int64)]),
    "cgks_server_step": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "cgks_server_poll": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(CgksReqStatus), C.c_void_p, C.c_int]),
    "cgks_server_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32)]),
    "cgks_server_footprint": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]),
    "cgks_server_destroy": (C.c_int, [C.c_void_p]),
    "cgks_server_get_tuning": (C.c_int, [C.c_void_p, C.POINTER(CgksTuning)]),
})


class Server:
    """Continuous batching of steady solves: submit requests, step the
    server (one batched V-cycle per step), poll for finished states."""

    def __init__(self, hbm_budget: int, precision="fp64", time_scheme="S1O2", max_active=64,
                 max_cycles=20000, use_torch: bool = True, **kw):
        L = lib()
        o = CgksServerOpts()
        L.cgks_server_default_opts(C.byref(o))
        o.precision = {"fp64": FP64, "mixed": MIXED}[precision]
        o.time_scheme = {"S1O2": S1O2, "S2O4": S2O4}[time_scheme]
        o.flux_lo = {"kfvs": FLUX_KFVS, "lf": FLUX_LF}[kw.get("flux_lo", "kfvs")]
        o.max_active, o.max_cycles = int(max_active), int(max_cycles)
        for key in ("cfl_hi", "cfl_lo"):
            if key in kw:
                setattr(o, key, float(kw[key]))
        for key in ("n_implicit", "n_sweeps", "use_graph", "low_order_fused", "autotune", "programmatic_launch",
                    "lo_viscous"):
            if key in kw:
                setattr(o, key, int(kw[key]))
        self._alloc = None
        if use_torch:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("libcgks needs a CUDA device; none is available")
            self._alloc = TorchAllocator()
            o.stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
            o.alloc, o.free, o.alloc_ctx = self._alloc.alloc_fn, self._alloc.free_fn, None
        self.opts = o
        self.n_cells = {}
        h = C.c_void_p()
        _check(L.cgks_server_create(int(hbm_budget), C.byref(o), C.byref(h)), "cgks_server_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().cgks_server_destroy(self._h)
            self._h = None

    __del__ = close

    def submit(self, mesh: Mesh, spec: dict, W0, res_drop: float, max_cycles: int = 0) -> int:
        """Queue a solve; returns its id.  Raises CgksError(-7) when the
        request alone exceeds the budget (the id is then still pollable)."""
        P = make_params(spec)
        W0 = np.ascontiguousarray(W0, np.float64).reshape(-1)
        rid = C.c_int64(0)
        rc = lib().cgks_server_submit(self._h, mesh._h, C.byref(P), W0, float(res_drop), int(max_cycles),
                                      C.byref(rid))
        self.n_cells[rid.value] = mesh.n_cells
        _check(rc, "cgks_server_submit")
        return rid.value

    def step(self) -> int:
        n = C.c_int32(0)
        _check(lib().cgks_server_step(self._h, C.byref(n)), "cgks_server_step")
        return n.value

    def poll(self, rid: int, timeout_ms: int = 0, want_state=True):
        """(status dict, W or None).  With timeout_ms > 0 the server is
        stepped until the request is done (CgksError -6 on timeout)."""
        st = CgksReqStatus()
        W = np.zeros((self.n_cells[rid], 4)) if want_state else None
        _check(lib().cgks_server_poll(self._h, int(rid), C.byref(st), _ptr(W), int(timeout_ms)),
               "cgks_server_poll")
        d = {k: getattr(st, k) for k, _ in CgksReqStatus._fields_}
        d["state"] = REQ_STATES[st.state]
        done = d["state"] in ("converged", "stopped", "diverged", "rejected")
        return d, (W if done and d["state"] != "rejected" else None)

    def footprint(self, mesh: Mesh) -> int:
        b = C.c_int64(0)
        _check(lib().cgks_server_footprint(self._h, mesh._h, C.byref(b)), "cgks_server_footprint")
        return b.value

    def info(self):
        b, q, a = C.c_int64(0), C.c_int32(0), C.c_int32(0)
        _check(lib().cgks_server_info(self._h, C.byref(b), C.byref(q), C.byref(a)), "cgks_server_info")
        return dict(device_bytes=b.value, n_queued=q.value, n_active=a.value)

    def tuning(self) -> dict:
        t = CgksTuning()
        _check(lib().cgks_server_get_tuning(self._h, C.byref(t)), "cgks_server_get_tuning")
        return _tuning_dict(t)
