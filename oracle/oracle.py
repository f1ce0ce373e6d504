"""ctypes wrapper of the serial FP64 CPU oracle (``cgks_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use this module; the CUDA library never does.
It depends on numpy and ctypes only and imports nothing from the product
package.  Problem settings arrive as a plain dict (see ``make_params``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cgks_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NV = 4
BC_SLIP, BC_NOSLIP, BC_FARFIELD, BC_DIRICHLET, BC_OUTFLOW = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu99", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrBC(C.Structure):
    _fields_ = [("kind", C.c_int), ("pad_", C.c_int), ("uw", C.c_double * 2),
                ("rho", C.c_double), ("u", C.c_double * 2), ("p", C.c_double)]


class OrParams(C.Structure):
    _fields_ = [("gamma", C.c_double), ("mu", C.c_double), ("alpha", C.c_double), ("cfl_hi", C.c_double),
                ("cfl_lo", C.c_double), ("n_implicit", C.c_int), ("n_sweeps", C.c_int),
                ("time_scheme", C.c_int), ("restrict_mode", C.c_int), ("n_bc", C.c_int),
                ("flux_lo", C.c_int), ("sweep_order", C.c_int), ("n_parts", C.c_int),
                ("flux_hi", C.c_int), ("pad_", C.c_int), ("tau_c1", C.c_double), ("tau_c2", C.c_double),
                ("weno_eps", C.c_double), ("weno_g0", C.c_double), ("weno_char", C.c_int), ("pad2_", C.c_int),
                ("bc", OrBC * 16), ("lo_viscous", C.c_int), ("pad3_", C.c_int)]


_dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            vp, P = C.c_void_p, C.POINTER(OrParams)
            L.or_mesh_create.restype = vp
            L.or_mesh_create.argtypes = [C.c_long, _dp, C.c_long, _u8p, _i64p, _i64p, C.c_long,
                                         _i64p, _i64p, _i32p, C.POINTER(C.c_int)]
            L.or_mesh_destroy.argtypes = [vp]
            L.or_mesh_nfaces.restype = C.c_long
            L.or_mesh_nfaces.argtypes = [vp]
            L.or_mesh_ncolours.argtypes = [vp]
            L.or_mesh_geometry.argtypes = [vp, _dp, _dp]
            L.or_mesh_faces.argtypes = [vp, _i64p, _i64p, _i32p, _dp, _dp, _dp]
            L.or_mesh_ordering.argtypes = [vp, _i64p, _i32p]
            L.or_solver_create.restype = vp
            L.or_solver_create.argtypes = [vp, P]
            L.or_solver_destroy.argtypes = [vp]
            L.or_set_state.argtypes = [vp, _dp, vp]
            L.or_get_state.argtypes = [vp, _dp, _dp]
            L.or_last_residual.restype = C.c_double
            L.or_last_residual.argtypes = [vp]
            L.or_status.argtypes = [vp]
            L.or_highorder_step.restype = C.c_double
            L.or_highorder_step.argtypes = [vp, C.c_double]
            L.or_explicit_dt.restype = C.c_double
            L.or_explicit_dt.argtypes = [vp]
            L.or_pmg_cycle.argtypes = [vp, C.c_int, _dp]
            L.or_explicit_steps.argtypes = [vp, C.c_int, _dp]
            L.or_loworder_smooth.argtypes = [vp]
            L.or_hi_residual.argtypes = [vp, C.c_double, _dp]
            L.or_reconstruct.argtypes = [vp]
            L.or_recon_eval.argtypes = [vp, C.c_long, _dp, _dp, _dp]
            L.or_face_side_eval.argtypes = [vp, C.c_long, C.c_int, _dp, _dp, _dp]
            L.or_lo_residual.argtypes = [vp, _dp, _dp]
            L.or_lo_lambda.argtypes = [vp, _dp, _dp]
            L.or_lo_diag.argtypes = [vp, _dp, _dp]
            L.or_lo_relax.argtypes = [vp, _dp, _dp, C.c_int, _dp]
            L.or_set_rp0.argtypes = [vp, _dp]
            L.or_get_rp0.argtypes = [vp, _dp]
            L.or_gks_flux_point.argtypes = [P, _dp, _dp, _dp, _dp, _dp, C.c_double, _dp, _dp, _dp, _dp]
            L.or_gks_full_flux_point.argtypes = [P, _dp, _dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                                 _dp, _dp, _dp, _dp]
            L.or_kfvs.argtypes = [P, _dp, _dp, _dp, _dp]
            L.or_euler_right_eigvecs.argtypes = [C.c_double, _dp, _dp, _dp]
            L.or_euler_flux.argtypes = [C.c_double, _dp, _dp, _dp]
            L.or_ghost.argtypes = [P, C.c_int, _dp, _dp, _dp, _dp, _dp]
            L.or_micro_slope.argtypes = [C.c_double, _dp, _dp, _dp]
            L.or_wall_loads.restype = C.c_long
            L.or_wall_loads.argtypes = [vp, C.c_int, C.c_double, C.c_long, _dp, _dp, _dp, _dp]
            _lib = L
    return _lib


def make_params(spec: dict) -> OrParams:
    """spec keys: gamma, mu, cfl_hi, cfl_lo, n_implicit, n_sweeps,
    time_scheme ('S1O2'|'S2O4'), alpha (jump coefficient, default 1/2),
    flux_lo ('kfvs' default | 'lf': low-level flux), lo_viscous (1: the
    low-order residual carries a first-order viscous flux), sweep_order ('colour'
    default | 'index' | 'partitioned' with n_parts index partitions, default
    8 | 'partitioned_colour': n_parts partitions of the RCM order, colour
    classes inside, exchange lagged by one sweep),
    flux_hi ('smooth' default | 'full': Eq. (2nd-flux) with
    tau_n = tau + tau_c1 dt + tau_c2 dt |p_l - p_r| / (p_l + p_r), defaults
    0.01 and 1), weno_eps (> 0: nonlinear compact WENO weights, default 0 =
    linear weights), weno_g0 (linear weight of the quadratic, default 0.95),
    weno_vars ('conservative' default | 'characteristic': weights per
    characteristic field of the face normal, per face side),
    bcs: list of dicts {kind: 'slip'|'noslip'|'farfield'|'dirichlet'|
    'outflow', uw=(u,v), rho, u=(u,v), p}."""
    P = OrParams()
    P.gamma = float(spec.get("gamma", 1.4))
    P.mu = float(spec.get("mu", 0.0))
    P.alpha = float(spec.get("alpha", 0.5))
    P.cfl_hi = float(spec.get("cfl_hi", 0.4))
    P.cfl_lo = float(spec.get("cfl_lo", 1000.0))
    P.n_implicit = int(spec.get("n_implicit", 6))
    P.n_sweeps = int(spec.get("n_sweeps", 2))
    P.time_scheme = {"S1O2": 0, "S2O4": 1}[spec.get("time_scheme", "S1O2")]
    P.restrict_mode = 0
    P.flux_lo = {"kfvs": 0, "lf": 1}[spec.get("flux_lo", "kfvs")]
    P.lo_viscous = int(spec.get("lo_viscous", 0))
    P.sweep_order = {"colour": 0, "index": 1, "partitioned": 2,
                     "partitioned_colour": 3}[spec.get("sweep_order", "colour")]
    P.n_parts = int(spec.get("n_parts", 8))
    P.flux_hi = {"smooth": 0, "full": 1}[spec.get("flux_hi", "smooth")]
    P.tau_c1 = float(spec.get("tau_c1", 0.01))
    P.tau_c2 = float(spec.get("tau_c2", 1.0))
    P.weno_eps = float(spec.get("weno_eps", 0.0))
    P.weno_g0 = float(spec.get("weno_g0", 0.95))
    P.weno_char = {"conservative": 0, "characteristic": 1}[spec.get("weno_vars", "conservative")]
    bcs = spec.get("bcs", [])
    P.n_bc = len(bcs)
    for i, b in enumerate(bcs):
        P.bc[i].kind = {"slip": BC_SLIP, "noslip": BC_NOSLIP, "farfield": BC_FARFIELD, "dirichlet": BC_DIRICHLET,
                        "outflow": BC_OUTFLOW}[b["kind"]]
        uw = b.get("uw", (0.0, 0.0))
        P.bc[i].uw[0], P.bc[i].uw[1] = float(uw[0]), float(uw[1])
        P.bc[i].rho = float(b.get("rho", 1.0))
        u = b.get("u", (0.0, 0.0))
        P.bc[i].u[0], P.bc[i].u[1] = float(u[0]), float(u[1])
        P.bc[i].p = float(b.get("p", 1.0 / P.gamma))
    return P


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


class OracleMesh:
    """Oracle-side mesh built from raw node/cell/boundary arrays."""

    def __init__(self, mesh):
        L = lib()
        err = C.c_int(0)
        self._m = L.or_mesh_create(
            mesh.nodes.shape[0], _f64(mesh.nodes), mesh.cell_type.shape[0],
            np.ascontiguousarray(mesh.cell_type, np.uint8), np.ascontiguousarray(mesh.cell_ptr, np.int64),
            np.ascontiguousarray(mesh.cell_nodes, np.int64), mesh.bface_tag.shape[0],
            np.ascontiguousarray(mesh.bface_ptr, np.int64), np.ascontiguousarray(mesh.bface_nodes, np.int64),
            np.ascontiguousarray(mesh.bface_tag, np.int32), C.byref(err))
        if not self._m:
            raise ValueError(f"oracle mesh rejected (code {err.value})")
        self.n_cells = int(mesh.cell_type.shape[0])
        self.n_faces = int(L.or_mesh_nfaces(self._m))
        self.n_colours = int(L.or_mesh_ncolours(self._m))

    def __del__(self):
        if getattr(self, "_m", None):
            lib().or_mesh_destroy(self._m)
            self._m = None

    def geometry(self):
        vol = np.zeros(self.n_cells)
        xc = np.zeros((self.n_cells, 2))
        lib().or_mesh_geometry(self._m, vol, xc)
        return vol, xc

    def faces(self):
        nf = self.n_faces
        c0 = np.zeros(nf, np.int64); c1 = np.zeros(nf, np.int64); tag = np.zeros(nf, np.int32)
        n = np.zeros((nf, 2)); S = np.zeros(nf); xg = np.zeros((nf, 2, 2))
        lib().or_mesh_faces(self._m, c0, c1, tag, n, S, xg)
        return dict(c0=c0, c1=c1, tag=tag, n=n, S=S, xg=xg)

    def ordering(self):
        rcm = np.zeros(self.n_cells, np.int64)
        colour = np.zeros(self.n_cells, np.int32)
        lib().or_mesh_ordering(self._m, rcm, colour)
        return rcm, colour


class OracleSolver:
    """Serial FP64 solver state on an OracleMesh."""

    def __init__(self, omesh: OracleMesh, spec: dict):
        self.mesh = omesh
        self.params = make_params(spec)
        self._s = lib().or_solver_create(omesh._m, C.byref(self.params))
        self.nc = omesh.n_cells

    def __del__(self):
        if getattr(self, "_s", None):
            lib().or_solver_destroy(self._s)
            self._s = None

    def set_state(self, W, Wx=None):
        W = _f64(W, (self.nc, NV))
        if Wx is None:
            lib().or_set_state(self._s, W, None)
        else:
            Wx = _f64(Wx, (self.nc, 2, NV))
            lib().or_set_state(self._s, W, Wx.ctypes.data_as(C.c_void_p))

    def get_state(self):
        W = np.zeros((self.nc, NV)); Wx = np.zeros((self.nc, 2, NV))
        lib().or_get_state(self._s, W, Wx)
        return W, Wx

    def status(self) -> int:
        return int(lib().or_status(self._s))

    def explicit_dt(self) -> float:
        return float(lib().or_explicit_dt(self._s))

    def highorder_step(self, dt: float = -1.0) -> float:
        return float(lib().or_highorder_step(self._s, dt))

    def explicit_steps(self, n: int) -> np.ndarray:
        r = np.zeros(max(n, 1))
        rc = lib().or_explicit_steps(self._s, n, r)
        if rc:
            raise FloatingPointError(f"oracle explicit steps failed (status {rc})")
        return r[:n]

    def pmg_cycles(self, n: int) -> np.ndarray:
        r = np.zeros(max(n, 1))
        rc = lib().or_pmg_cycle(self._s, n, r)
        if rc:
            raise FloatingPointError(f"oracle p-multigrid cycle failed (status {rc})")
        return r[:n]

    def loworder_smooth(self):
        lib().or_loworder_smooth(self._s)

    def residual(self) -> float:
        return float(lib().or_last_residual(self._s))

    def wall_loads(self, tag: int) -> dict:
        """Face centres, normals, lengths and momentum flux F0 of the
        boundary faces with this tag at the current state (oracle face
        order); dt of the full flux from CFL_hi."""
        dt = self.explicit_dt()
        nf = int(lib().or_wall_loads(self._s, int(tag), dt, 0, np.zeros(1), np.zeros(1), np.zeros(1), np.zeros(1)))
        x, n, t = np.zeros((max(nf, 1), 2)), np.zeros((max(nf, 1), 2)), np.zeros((max(nf, 1), 2))
        S = np.zeros(max(nf, 1))
        lib().or_wall_loads(self._s, int(tag), dt, nf, x, n, S, t)
        return dict(x=x[:nf], n=n[:nf], S=S[:nf], traction=t[:nf])

    def hi_residual(self, dt: float) -> np.ndarray:
        R = np.zeros((self.nc, NV))
        lib().or_hi_residual(self._s, dt, R)
        return R

    def reconstruct(self):
        lib().or_reconstruct(self._s)

    def recon_eval(self, cell: int, x):
        v = np.zeros(NV); g = np.zeros((2, NV))
        lib().or_recon_eval(self._s, int(cell), _f64(x), v, g)
        return v, g

    def face_side_eval(self, face: int, side: int, x):
        """Polynomial the face flux uses on one side of a face (after
        reconstruct()): value and gradient at x."""
        v = np.zeros(NV); g = np.zeros(2 * NV)
        lib().or_face_side_eval(self._s, int(face), int(side), _f64(x), v, g)
        return v, g.reshape(2, NV)

    def lo_residual(self, U):
        R = np.zeros((self.nc, NV))
        lib().or_lo_residual(self._s, _f64(U, (self.nc, NV)), R)
        return R

    def lo_lambda(self, U):
        lam = np.zeros(self.mesh.n_faces)
        lib().or_lo_lambda(self._s, _f64(U, (self.nc, NV)), lam)
        return lam

    def lo_diag(self, U):
        D = np.zeros(self.nc)
        lib().or_lo_diag(self._s, _f64(U, (self.nc, NV)), D)
        return D

    def lo_relax(self, U, R, n_sweeps: int):
        dU = np.zeros((self.nc, NV))
        lib().or_lo_relax(self._s, _f64(U, (self.nc, NV)), _f64(R, (self.nc, NV)), int(n_sweeps), dU)
        return dU

    def set_rp0(self, R):
        lib().or_set_rp0(self._s, _f64(R, (self.nc, NV)))

    def get_rp0(self):
        R = np.zeros((self.nc, NV))
        lib().or_get_rp0(self._s, R)
        return R


def gks_flux_point(spec, Wl, Wr, gl, gr, n, delta=0.0):
    P = make_params(spec)
    F0 = np.zeros(NV); F1 = np.zeros(NV); Wc = np.zeros(NV); Wt = np.zeros(NV)
    lib().or_gks_flux_point(C.byref(P), _f64(Wl), _f64(Wr), _f64(gl, (2 * NV,)), _f64(gr, (2 * NV,)),
                            _f64(n), float(delta), F0, F1, Wc, Wt)
    return F0, F1, Wc, Wt


def gks_full_flux_point(spec, Wl, Wr, gl, gr, n, delta, dt):
    """Full flux, Eq. (2nd-flux), as F0 + t F1 and W^c + t W_t over [0, dt]."""
    P = make_params(spec)
    F0 = np.zeros(NV); F1 = np.zeros(NV); Wc = np.zeros(NV); Wt = np.zeros(NV)
    lib().or_gks_full_flux_point(C.byref(P), _f64(Wl), _f64(Wr), _f64(gl, (2 * NV,)), _f64(gr, (2 * NV,)),
                                 _f64(n), float(delta), float(dt), F0, F1, Wc, Wt)
    return F0, F1, Wc, Wt


def kfvs(spec, Wl, Wr, n):
    P = make_params(spec)
    F = np.zeros(NV)
    lib().or_kfvs(C.byref(P), _f64(Wl), _f64(Wr), _f64(n), F)
    return F


def euler_flux(gamma, W, n):
    F = np.zeros(NV)
    lib().or_euler_flux(float(gamma), _f64(W), _f64(n), F)
    return F


def ghost(spec, tag, W, grad, n):
    P = make_params(spec)
    Wg = np.zeros(NV); gg = np.zeros(2 * NV)
    lib().or_ghost(C.byref(P), int(tag), _f64(W), _f64(grad, (2 * NV,)), _f64(n), Wg, gg)
    return Wg, gg.reshape(2, NV)


def euler_right_eigvecs(gamma, W, n):
    R = np.zeros(NV * NV)
    lib().or_euler_right_eigvecs(float(gamma), _f64(W), _f64(n), R)
    return R.reshape(NV, NV)


def micro_slope(gamma, W, dW):
    s = np.zeros(NV)
    rc = lib().or_micro_slope(float(gamma), _f64(W), _f64(dW), s)
    if rc:
        raise np.linalg.LinAlgError("singular moment matrix")
    return s
