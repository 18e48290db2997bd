"""ctypes front end of the FP64 DI-LBM oracle (``dilbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use this module to produce expected values.  The product
path never imports it.  It shares no code with the CUDA library; both take
their inputs from ``paper_2106_08950_gb300.workloads``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dilbm_oracle.c")
_LIB = os.path.join(_HERE, "libdilbm_oracle.so")
_lock = threading.Lock()
_lib = None

SIDE_CODE = {"periodic": 0, "velocity": 1, "pressure": 2}


class OrcParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("side_kind", C.c_int * 4),
        ("side_ux", C.c_double * 4), ("side_uy", C.c_double * 4), ("side_rho", C.c_double * 4),
        ("tau", C.c_double), ("eps", C.c_double),
        ("gx", C.c_double), ("gy", C.c_double),
        ("rho_f", C.c_double),
        ("rho_init", C.c_double), ("u0x", C.c_double), ("u0y", C.c_double),
        ("force_model", C.c_int),
        ("eps_p", C.c_double), ("eps_p2", C.c_double), ("eps_w", C.c_double),
        ("eps_w2", C.c_double), ("xi", C.c_double),
        ("phi_cutoff", C.c_double),
        ("method", C.c_int),
    ]


class OrcParticle(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("r", C.c_double),
                ("ux", C.c_double), ("uy", C.c_double), ("omega", C.c_double),
                ("theta", C.c_double), ("rho_s", C.c_double), ("fixed", C.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE: no contraction into FMA)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                                   "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                                   _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcParticle), C.c_int]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_step.restype = C.c_int
        L.orc_step.argtypes = [C.c_void_p, C.c_longlong]
        L.orc_fields.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_forces.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_get_populations.argtypes = [C.c_void_p, dp]
        L.orc_set_populations.argtypes = [C.c_void_p, dp]
        L.orc_set_particles.argtypes = [C.c_void_p, C.POINTER(OrcParticle)]
        L.orc_equilibrium.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        L.orc_phi.restype = C.c_double
        L.orc_phi.argtypes = [C.c_double, C.c_double]
        L.orc_force_term.argtypes = [C.c_double] * 6 + [dp]
        L.orc_collide_node.argtypes = [C.c_double, dp, C.c_double, C.c_double, C.c_double, dp, dp, dp]
        L.orc_collide_node_ps.argtypes = [C.c_double, dp, C.c_double, C.c_double, C.c_double, dp, dp, dp]
        L.orc_cell_fraction.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_cell_fraction.restype = C.c_double
        L.orc_wan_turek.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcParticle), C.c_int, dp]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_max_threads.restype = C.c_int
        L.orc_steps_done.restype = C.c_longlong
        L.orc_steps_done.argtypes = [C.c_void_p]
        L.orc_set_moving_frame.restype = C.c_int
        L.orc_set_moving_frame.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.orc_frame_offset.restype = C.c_longlong
        L.orc_frame_offset.argtypes = [C.c_void_p]
        _lib = L
    return _lib


def make_params(prob, phi_cutoff: float = 0.0) -> OrcParams:
    p = OrcParams()
    p.nx, p.ny = prob.nx, prob.ny
    for k, side in enumerate((prob.west, prob.east, prob.south, prob.north)):
        p.side_kind[k] = SIDE_CODE[side.kind]
        p.side_ux[k], p.side_uy[k], p.side_rho[k] = side.ux, side.uy, side.rho
    p.tau, p.eps = prob.tau, prob.eps
    p.gx, p.gy = prob.gravity
    p.rho_f = prob.rho_f
    p.rho_init = prob.rho_init
    p.u0x, p.u0y = prob.u0
    p.force_model = prob.force_model
    p.eps_p, p.eps_p2, p.eps_w, p.eps_w2, p.xi = prob.wan_turek
    p.phi_cutoff = phi_cutoff
    p.method = getattr(prob, "method", 0)
    return p


def make_particles(parts) -> "C.Array":
    arr = (OrcParticle * max(1, len(parts)))()
    for k, q in enumerate(parts):
        arr[k] = OrcParticle(q.x, q.y, q.r, q.ux, q.uy, q.omega, q.theta, q.rho_s, int(q.fixed))
    return arr


def particles_to_array(arr, n) -> np.ndarray:
    """(n, 8) float64: x, y, r, ux, uy, omega, theta, rho_s."""
    out = np.zeros((n, 8))
    for k in range(n):
        q = arr[k]
        out[k] = (q.x, q.y, q.r, q.ux, q.uy, q.omega, q.theta, q.rho_s)
    return out


class OracleSim:
    """FP64 DI-LBM on the host.  ``phi_cutoff`` > 0 skips, at each node, the
    particles whose signed distance is below -phi_cutoff (phi < 1.1e-7 beyond
    4 interface widths); 0 evaluates every particle at every node."""

    def __init__(self, prob, phi_cutoff: float = 0.0, threads: int = 0):
        self.L = lib()
        if threads:
            self.L.orc_set_threads(threads)
        self.prob = prob
        self.np = len(prob.particles)
        self._p = make_params(prob, phi_cutoff)
        self._parts = make_particles(prob.particles)
        h = self.L.orc_create(C.byref(self._p), self._parts, self.np)
        if not h:
            raise ValueError("oracle rejected the problem")
        self.h = C.c_void_p(h)

    def close(self):
        if getattr(self, "h", None):
            self.L.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1) -> None:
        rc = self.L.orc_step(self.h, int(n))
        if rc != 0:
            raise FloatingPointError(f"oracle step failed ({rc}): unstable state")

    @property
    def steps_done(self) -> int:
        return int(self.L.orc_steps_done(self.h))

    def set_moving_frame(self, particle: int, x_ref: float) -> None:
        """Moving computational domain (Sec. 3.5): the frame follows particle
        ``particle`` (-1: off) about ``x_ref``, one column at a time."""
        if self.L.orc_set_moving_frame(self.h, int(particle), float(x_ref)) != 0:
            raise ValueError("bad moving-frame particle or reference")

    def frame_offset(self) -> int:
        """Columns the frame has moved: lab x = frame x + offset."""
        return int(self.L.orc_frame_offset(self.h))

    def fields(self):
        """rho, ux, uy, phi as (ny, nx) float64 and the owner map (int32)."""
        n = self.prob.nx * self.prob.ny
        rho, ux, uy, phi = (np.empty(n) for _ in range(4))
        own = np.empty(n, dtype=np.int32)
        self.L.orc_fields(self.h, rho.ctypes.data, ux.ctypes.data, uy.ctypes.data,
                          phi.ctypes.data, own.ctypes.data)
        sh = (self.prob.ny, self.prob.nx)
        return rho.reshape(sh), ux.reshape(sh), uy.reshape(sh), phi.reshape(sh), own.reshape(sh)

    def forces(self):
        """(np, 3) hydrodynamic Fx, Fy, T of the last step, (np, 2) Wan-Turek
        force of the last step, (np, 8) particle state."""
        F = np.zeros((max(1, self.np), 3))
        Fc = np.zeros((max(1, self.np), 2))
        st = (OrcParticle * max(1, self.np))()
        self.L.orc_forces(self.h, F.ctypes.data, Fc.ctypes.data, st)
        return F[: self.np], Fc[: self.np], particles_to_array(st, self.np)

    def populations(self) -> np.ndarray:
        out = np.empty(9 * self.prob.nx * self.prob.ny)
        self.L.orc_get_populations(self.h, out)
        return out.reshape(9, self.prob.ny, self.prob.nx)

    def set_populations(self, f: np.ndarray) -> None:
        self.L.orc_set_populations(self.h, np.ascontiguousarray(f, dtype=np.float64).ravel())

    def set_particles(self, parts) -> None:
        arr = make_particles(parts)
        self.L.orc_set_particles(self.h, arr)


def equilibrium(rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.empty(9)
    lib().orc_equilibrium(rho, ux, uy, out)
    return out


def phi(l: float, eps: float) -> float:
    return float(lib().orc_phi(l, eps))


def force_term(tau, rho, usx, usy, uax, uay) -> np.ndarray:
    out = np.empty(9)
    lib().orc_force_term(tau, rho, usx, usy, uax, uay, out)
    return out


def collide_node(tau, f, phi_, usx, usy):
    fo, Fi, mom = np.empty(9), np.empty(9), np.empty(5)
    lib().orc_collide_node(tau, np.ascontiguousarray(f, dtype=np.float64), phi_, usx, usy, fo, Fi, mom)
    return fo, Fi, mom


def collide_node_ps(tau, f, B, usx, usy):
    """PS-LBM collision (Eq. 7 with Omega^s of Eq. 9): (f', Omega^s, (rho, u*x, u*y))."""
    fo, om, mom = np.empty(9), np.empty(9), np.empty(3)
    lib().orc_collide_node_ps(tau, np.ascontiguousarray(f, dtype=np.float64), B, usx, usy, fo, om, mom)
    return fo, om, mom


def cell_fraction(dx: float, dy: float, r: float) -> float:
    """Area of the unit cell centred at (dx, dy) covered by the disc of radius r at the origin."""
    return float(lib().orc_cell_fraction(dx, dy, r))


def wan_turek(prob) -> np.ndarray:
    p = make_params(prob)
    parts = make_particles(prob.particles)
    out = np.zeros(2 * max(1, len(prob.particles)))
    lib().orc_wan_turek(C.byref(p), parts, len(prob.particles), out)
    return out[: 2 * len(prob.particles)].reshape(-1, 2)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())
