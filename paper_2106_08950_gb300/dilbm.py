"""Python binding of the C ABI in ``include/dilbm.h``.

Argument marshalling only: every step of the DI-LBM path runs in the CUDA
library ``libdilbm.so``.  The binding refuses to work when that library is
missing or cannot be loaded; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdilbm.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_CUDA = -3
ERR_UNSTABLE = -4
ERR_TIMEOUT = -5
ERR_OVERFLOW = -6
MAX_CANDIDATES = 32

FP32, FP16_DEV, BF16_DEV = 0, 1, 2
STORAGE = {"fp32": FP32, "fp16": FP16_DEV, "bf16": BF16_DEV}
STORAGE_PER_JOB = -1          # server: each job keeps its own storage
STORAGE_AUTO = -2             # server: FP16 where the job's tau and disc area allow, else FP32
SIDE = {W.PERIODIC: 0, W.VELOCITY: 1, W.PRESSURE: 2}


class DilbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dilbm error {code}: {msg}")
        self.code = code


class Side(C.Structure):
    _fields_ = [("kind", C.c_int), ("ux", C.c_double), ("uy", C.c_double), ("rho", C.c_double)]


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int),
                ("west", Side), ("east", Side), ("south", Side), ("north", Side),
                ("gravity", C.c_double * 2), ("rho_f", C.c_double), ("rho_init", C.c_double),
                ("u0", C.c_double * 2), ("storage", C.c_int), ("force_model", C.c_int),
                ("wan_turek", C.c_double * 5), ("method", C.c_int)]


class Particle(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("r", C.c_double),
                ("ux", C.c_double), ("uy", C.c_double), ("omega", C.c_double),
                ("theta", C.c_double), ("rho_s", C.c_double), ("fixed", C.c_int)]


class ServerConfig(C.Structure):
    _fields_ = [("storage", C.c_int), ("max_jobs", C.c_int), ("macro_steps", C.c_longlong),
                ("memory_budget", C.c_double), ("policy", C.c_int),
                ("auto_tau_max", C.c_double), ("auto_area_max", C.c_double)]


class Job(C.Structure):
    _fields_ = [("grid", Grid), ("tau", C.c_double), ("interface_width", C.c_double),
                ("particles", C.POINTER(Particle)), ("np", C.c_int), ("nsteps", C.c_longlong),
                ("mean_window", C.c_longlong), ("arrival", C.c_double)]


class JobStatus(C.Structure):
    _fields_ = [("state", C.c_int), ("error", C.c_int), ("np", C.c_int), ("steps_done", C.c_longlong),
                ("arrival", C.c_double), ("admitted", C.c_double), ("finished", C.c_double),
                ("footprint", C.c_ulonglong), ("storage", C.c_int)]


class ServerStats(C.Structure):
    _fields_ = [("running", C.c_int), ("queued", C.c_int), ("done", C.c_longlong), ("failed", C.c_longlong),
                ("macro_steps", C.c_longlong), ("node_updates", C.c_double), ("busy_seconds", C.c_double),
                ("form_seconds", C.c_double), ("admit_seconds", C.c_double), ("wait_seconds", C.c_double),
                ("retire_seconds", C.c_double), ("memory_in_use", C.c_ulonglong), ("launches", C.c_longlong)]


JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED = 0, 1, 2, 3
ADMIT_FIFO, ADMIT_FIRST_FIT = 0, 1

_lib = None


def load_library(path: Optional[str] = None):
    """Load ``libdilbm.so`` (building it in-tree first if it is missing or
    older than its sources) and declare the C signatures."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    if path is None:
        from . import build as _build
        if _build.stale():
            _build.build()
        path = LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not found at {path}: run paper_2106_08950_gb300.build")
    L = C.CDLL(path)
    vp, ip, dp, fp = C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_float)
    L.dilbm_create.argtypes = [C.POINTER(Grid), ip, C.c_double, C.c_double, C.POINTER(Particle), ip, vp,
                               C.POINTER(vp)]
    L.dilbm_step.argtypes = [vp, C.c_longlong]
    L.dilbm_forces.argtypes = [vp, vp, vp, vp]
    L.dilbm_fields.argtypes = [vp, vp, vp, vp, vp, ip]
    L.dilbm_get_populations.argtypes = [vp, vp]
    L.dilbm_set_populations.argtypes = [vp, vp]
    L.dilbm_set_particles.argtypes = [vp, C.POINTER(Particle), ip]
    L.dilbm_sync.argtypes = [vp]
    L.dilbm_destroy.argtypes = [vp]
    L.dilbm_destroy.restype = None
    L.dilbm_last_error.restype = C.c_char_p
    L.dilbm_set_timing.argtypes = [vp, ip]
    L.dilbm_sweep_time.argtypes = [vp, dp, C.POINTER(C.c_longlong)]
    L.dilbm_launch_count.argtypes = [vp]
    L.dilbm_launch_count.restype = C.c_longlong
    L.dilbm_batch_create.argtypes = [C.POINTER(vp), ip, vp, C.POINTER(vp)]
    L.dilbm_batch_step.argtypes = [vp, C.c_longlong]
    L.dilbm_batch_sync.argtypes = [vp, C.POINTER(C.c_int)]
    L.dilbm_batch_set_timing.argtypes = [vp, ip]
    L.dilbm_batch_sweep_time.argtypes = [vp, dp, C.POINTER(C.c_longlong)]
    L.dilbm_batch_launch_count.argtypes = [vp]
    L.dilbm_batch_launch_count.restype = C.c_longlong
    L.dilbm_batch_destroy.argtypes = [vp]
    L.dilbm_batch_destroy.restype = None
    L.dilbm_batch_errors.argtypes = [vp, C.POINTER(C.c_int)]
    ipp = C.POINTER(C.c_int)
    L.dilbm_autotune.argtypes = [vp, ip, ipp, ipp]
    L.dilbm_set_shape.argtypes = [vp, ip, ip]
    L.dilbm_batch_autotune.argtypes = [vp, ip, ipp, ipp]
    L.dilbm_batch_set_shape.argtypes = [vp, ip, ip]
    L.dilbm_footprint.argtypes = [C.POINTER(Grid), ip, C.POINTER(C.c_ulonglong)]
    L.dilbm_server_create.argtypes = [C.POINTER(ServerConfig), vp, C.POINTER(vp)]
    L.dilbm_server_submit.argtypes = [vp, C.POINTER(Job), C.POINTER(C.c_longlong)]
    L.dilbm_server_progress.argtypes = [vp, C.POINTER(ServerStats)]
    L.dilbm_server_status.argtypes = [vp, C.c_longlong, C.POINTER(JobStatus)]
    L.dilbm_server_result.argtypes = [vp, C.c_longlong, vp, vp, vp]
    L.dilbm_force_mean.argtypes = [vp, vp, C.POINTER(C.c_longlong)]
    L.dilbm_force_mean_reset.argtypes = [vp]
    L.dilbm_set_moving_frame.argtypes = [vp, C.c_int, C.c_double]
    L.dilbm_wait_probe.argtypes = [vp, C.POINTER(C.c_double)]
    L.dilbm_frame_offset.argtypes = [vp, C.POINTER(C.c_longlong)]
    L.dilbm_server_clock.argtypes = [vp]
    L.dilbm_server_clock.restype = C.c_double
    L.dilbm_create_strip.argtypes = [C.POINTER(Grid), ip, C.c_double, C.c_double, C.POINTER(Particle), ip, ip, ip,
                                     vp, C.POINTER(vp)]
    L.dilbm_strip_begin.argtypes = [vp]
    L.dilbm_strip_end.argtypes = [vp]
    L.dilbm_strip_buffers.argtypes = [vp] + [C.POINTER(vp)] * 5 + [C.POINTER(C.c_longlong)]
    L.dilbm_server_destroy.argtypes = [vp]
    L.dilbm_server_destroy.restype = None
    for name in ("dilbm_create", "dilbm_step", "dilbm_forces", "dilbm_fields", "dilbm_get_populations",
                 "dilbm_set_populations", "dilbm_set_particles", "dilbm_sync", "dilbm_set_timing",
                 "dilbm_sweep_time", "dilbm_batch_create", "dilbm_batch_step", "dilbm_batch_sync",
                 "dilbm_batch_set_timing", "dilbm_batch_sweep_time", "dilbm_batch_errors", "dilbm_footprint",
                 "dilbm_server_create", "dilbm_server_submit", "dilbm_server_progress", "dilbm_server_status",
                 "dilbm_server_result", "dilbm_force_mean", "dilbm_force_mean_reset", "dilbm_autotune",
                 "dilbm_set_shape", "dilbm_batch_autotune", "dilbm_batch_set_shape", "dilbm_set_moving_frame",
                 "dilbm_frame_offset", "dilbm_wait_probe", "dilbm_create_strip", "dilbm_strip_begin",
                 "dilbm_strip_end", "dilbm_strip_buffers"):
        getattr(L, name).restype = C.c_int
    if path == LIB_PATH:
        _lib = L
    return L


def last_error() -> str:
    """The library's message for the last failed call on this thread."""
    return load_library().dilbm_last_error().decode(errors="replace")


def check(rc: int) -> None:
    if rc != OK:
        raise DilbmError(rc, load_library().dilbm_last_error().decode(errors="replace"))


def _side(s: W.Side) -> Side:
    return Side(SIDE[s.kind], s.ux, s.uy, s.rho)


def make_grid(prob: W.Problem, storage: str = "fp32") -> Grid:
    g = Grid()
    g.nx, g.ny = prob.nx, prob.ny
    g.west, g.east, g.south, g.north = (_side(prob.west), _side(prob.east), _side(prob.south), _side(prob.north))
    g.gravity[0], g.gravity[1] = prob.gravity
    g.rho_f = prob.rho_f
    g.rho_init = prob.rho_init
    g.u0[0], g.u0[1] = prob.u0
    g.storage = STORAGE[storage]
    g.force_model = prob.force_model
    for k in range(5):
        g.wan_turek[k] = prob.wan_turek[k]
    g.method = getattr(prob, "method", W.METHOD_DI)
    return g


def make_particles(parts) -> "C.Array":
    arr = (Particle * max(1, len(parts)))()
    for k, q in enumerate(parts):
        arr[k] = Particle(q.x, q.y, q.r, q.ux, q.uy, q.omega, q.theta, q.rho_s, int(q.fixed))
    return arr


def particles_to_array(arr, n) -> np.ndarray:
    """(n, 8) float64: x, y, r, ux, uy, omega, theta, rho_s."""
    out = np.zeros((n, 8))
    for k in range(n):
        q = arr[k]
        out[k] = (q.x, q.y, q.r, q.ux, q.uy, q.omega, q.theta, q.rho_s)
    return out


def footprint(prob: W.Problem, storage: str = "fp32") -> int:
    """Device bytes ``dilbm_create`` allocates for ``prob`` (host arithmetic)."""
    g = make_grid(prob, storage)
    out = C.c_ulonglong()
    check(load_library().dilbm_footprint(C.byref(g), len(prob.particles), C.byref(out)))
    return int(out.value)


def wait_probe(stream: int):
    """Failure-detection check (no fault): a bounded device wait on a barrier
    nothing arrives at.  Returns (return code, seconds waited on the device);
    the expected code is ERR_TIMEOUT."""
    t = C.c_double()
    rc = load_library().dilbm_wait_probe(C.c_void_p(stream), C.byref(t))
    return int(rc), float(t.value)


def current_stream_handle() -> int:
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


class Simulation:
    """One DI-LBM lattice on the GPU (``dilbm_create`` .. ``dilbm_destroy``).

    ``stream``: an integer ``cudaStream_t`` (e.g. ``torch.cuda.Stream().cuda_stream``);
    None uses torch's current stream.
    """

    def __init__(self, prob: W.Problem, storage: str = "fp32", stream: Optional[int] = None):
        self.L = load_library()
        self.prob = prob
        self.storage = storage
        self.np = len(prob.particles)
        self.ny = prob.ny                # rows held (a strip holds fewer)
        if stream is None:
            stream = current_stream_handle()
        self.stream = stream
        self._grid = make_grid(prob, storage)
        self._parts = make_particles(prob.particles)
        h = C.c_void_p()
        check(self._create(h))
        self.h = h

    def _create(self, h) -> int:
        return self.L.dilbm_create(C.byref(self._grid), 0, self.prob.tau, self.prob.eps, self._parts, self.np,
                                   C.c_void_p(self.stream), C.byref(h))

    # -- lifetime
    def close(self) -> None:
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.dilbm_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- stepping
    def step(self, n: int = 1) -> None:
        check(self.L.dilbm_step(self.h, int(n)))

    def sync(self) -> None:
        check(self.L.dilbm_sync(self.h))

    # -- outputs
    def forces(self):
        """(np, 3) Fx, Fy, T of the last step; (np, 2) Wan-Turek force; (np, 8) state."""
        n = max(1, self.np)
        F = np.zeros((n, 3))
        Fc = np.zeros((n, 2))
        st = (Particle * n)()
        check(self.L.dilbm_forces(self.h, F.ctypes.data, Fc.ctypes.data, C.cast(st, C.c_void_p)))
        return F[: self.np], Fc[: self.np], particles_to_array(st, self.np)

    def force_mean(self):
        """(np, 3) mean Fx, Fy, T since create or the last reset, and the steps averaged."""
        n = max(1, self.np)
        M = np.zeros((n, 3))
        k = C.c_longlong()
        check(self.L.dilbm_force_mean(self.h, M.ctypes.data, C.byref(k)))
        return M[: self.np], int(k.value)

    def force_mean_reset(self) -> None:
        check(self.L.dilbm_force_mean_reset(self.h))

    def set_moving_frame(self, particle: int, x_ref: float = None) -> None:
        """Moving computational domain (Sec. 3.5): the frame follows particle
        ``particle`` (-1: off) about ``x_ref`` (default: its initial x)."""
        if x_ref is None:
            x_ref = self.prob.particles[particle].x if particle >= 0 else 0.0
        check(self.L.dilbm_set_moving_frame(self.h, int(particle), float(x_ref)))

    def frame_offset(self) -> int:
        """Columns the frame has moved: lab x = frame x + offset."""
        k = C.c_longlong()
        check(self.L.dilbm_frame_offset(self.h, C.byref(k)))
        return int(k.value)

    def forces_into(self, F: np.ndarray) -> None:
        """Copy Fx, Fy, T of the last step into a host array of np x 3 doubles."""
        check(self.L.dilbm_forces(self.h, F.ctypes.data, None, None))

    def fields(self):
        """rho, ux, uy, phi as (ny, nx) float32 host arrays."""
        sh = (self.ny, self.prob.nx)
        out = [np.empty(sh, dtype=np.float32) for _ in range(4)]
        check(self.L.dilbm_fields(self.h, *[o.ctypes.data for o in out], 0))
        return tuple(out)

    def fields_device(self, rho=None, ux=None, uy=None, phi=None) -> None:
        """Write the fields into caller-owned device buffers (torch float32
        tensors of ny x nx, or None)."""
        ptr = [t.data_ptr() if t is not None else None for t in (rho, ux, uy, phi)]
        check(self.L.dilbm_fields(self.h, *ptr, 1))

    def populations(self) -> np.ndarray:
        out = np.empty((9, self.ny, self.prob.nx))
        check(self.L.dilbm_get_populations(self.h, out.ctypes.data))
        return out

    def set_populations(self, f: np.ndarray) -> None:
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.size == 9 * self.prob.nx * self.ny
        check(self.L.dilbm_set_populations(self.h, f.ctypes.data))

    def set_particles(self, parts) -> None:
        self._parts = make_particles(parts)
        check(self.L.dilbm_set_particles(self.h, self._parts, len(parts)))

    def set_particles_raw(self, arr) -> None:
        """``arr``: a ctypes array of Particle (e.g. in pinned memory)."""
        check(self.L.dilbm_set_particles(self.h, arr, self.np))

    # -- launch shape
    def autotune(self, reps: int = 10):
        """Time the candidate sweep shapes on this lattice, keep the fastest;
        returns (warps per block, blocks per SM)."""
        w, b = C.c_int(), C.c_int()
        check(self.L.dilbm_autotune(self.h, int(reps), C.byref(w), C.byref(b)))
        return w.value, b.value

    def set_shape(self, warps: int, blocks_per_sm: int = 0) -> None:
        check(self.L.dilbm_set_shape(self.h, int(warps), int(blocks_per_sm)))

    # -- measurement
    def set_timing(self, on: bool) -> None:
        check(self.L.dilbm_set_timing(self.h, 1 if on else 0))

    def sweep_time(self):
        ms = C.c_double()
        n = C.c_longlong()
        check(self.L.dilbm_sweep_time(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    @property
    def launches(self) -> int:
        return int(self.L.dilbm_launch_count(self.h))


class Strip(Simulation):
    """Rows [y0, y1) of a lattice split over ranks (``dilbm_create_strip``).
    A step is ``begin()``, the caller's exchange of halo rows and force sums
    (see ``strips.py``), then ``end()``; ``buffers()`` gives the device
    addresses the exchange reads and writes."""

    def __init__(self, prob: W.Problem, y0: int, y1: int, storage: str = "fp32", stream: Optional[int] = None):
        self.y0, self.y1 = int(y0), int(y1)
        super().__init__(prob, storage, stream)
        self.ny = self.y1 - self.y0

    def _create(self, h) -> int:
        return self.L.dilbm_create_strip(C.byref(self._grid), 0, self.prob.tau, self.prob.eps, self._parts,
                                         self.np, self.y0, self.y1, C.c_void_p(self.stream), C.byref(h))

    def step(self, n: int = 1) -> None:
        raise DilbmError(ERR_INVALID_ARG, "a strip steps through begin(), the exchange and end()")

    def begin(self) -> None:
        check(self.L.dilbm_strip_begin(self.h))

    def end(self) -> None:
        check(self.L.dilbm_strip_end(self.h))

    def buffers(self):
        """Device addresses: fpart (np x 5 doubles), send_south, send_north,
        recv_south, recv_north (row_elems stored elements each), row_elems."""
        p = [C.c_void_p() for _ in range(5)]
        n = C.c_longlong()
        check(self.L.dilbm_strip_buffers(self.h, *[C.byref(q) for q in p], C.byref(n)))
        return tuple(q.value for q in p) + (int(n.value),)


class Batch:
    """Several Simulations advanced together (``dilbm_batch_*``): one sweep and
    one particle launch per step for all members, replayed from CUDA graphs.
    The members stay usable on their own; they must outlive the batch."""

    def __init__(self, sims):
        self.L = load_library()
        self.sims = list(sims)
        arr = (C.c_void_p * len(self.sims))(*[s.h.value for s in self.sims])
        h = C.c_void_p()
        check(self.L.dilbm_batch_create(arr, len(self.sims), None, C.byref(h)))
        self.h = h

    def close(self) -> None:
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.dilbm_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1) -> None:
        check(self.L.dilbm_batch_step(self.h, int(n)))

    def sync(self) -> None:
        bad = C.c_int(-1)
        rc = self.L.dilbm_batch_sync(self.h, C.byref(bad))
        if rc != OK:
            raise DilbmError(rc, f"member {bad.value}: " + self.L.dilbm_last_error().decode(errors="replace"))

    def autotune(self, reps: int = 10):
        w, b = C.c_int(), C.c_int()
        check(self.L.dilbm_batch_autotune(self.h, int(reps), C.byref(w), C.byref(b)))
        return w.value, b.value

    def set_shape(self, warps: int, blocks_per_sm: int = 0) -> None:
        check(self.L.dilbm_batch_set_shape(self.h, int(warps), int(blocks_per_sm)))

    def set_timing(self, on: bool) -> None:
        check(self.L.dilbm_batch_set_timing(self.h, 1 if on else 0))

    def sweep_time(self):
        ms = C.c_double()
        n = C.c_longlong()
        check(self.L.dilbm_batch_sweep_time(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    @property
    def launches(self) -> int:
        return int(self.L.dilbm_batch_launch_count(self.h))


class Server:
    """Continuous batching of DI-LBM jobs (``dilbm_server_*``): jobs are
    admitted by free slots and a device memory budget and every running job
    advances in one batch per macro-step."""

    def __init__(self, storage: str = "fp32", max_jobs: int = 256, macro_steps: int = 64,
                 memory_budget: float = 0.0, policy: int = ADMIT_FIFO):
        self.L = load_library()
        self.storage = storage
        code = {"per_job": STORAGE_PER_JOB, "auto": STORAGE_AUTO}.get(storage, None)
        code = STORAGE[storage] if code is None else code
        cfg = ServerConfig(code, int(max_jobs), int(macro_steps), float(memory_budget), int(policy), 0.0, 0.0)
        h = C.c_void_p()
        check(self.L.dilbm_server_create(C.byref(cfg), None, C.byref(h)))
        self.h = h
        self.np = {}

    def close(self) -> None:
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.dilbm_server_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def clock(self) -> float:
        return float(self.L.dilbm_server_clock(self.h))

    def submit(self, prob: W.Problem, nsteps: int, arrival: float = -1.0, mean_window: int = 0,
               storage: Optional[str] = None) -> int:
        """Queue a job; ``storage`` picks its storage on a "per_job" server
        (default "fp32") and is ignored otherwise (an "auto" server picks it)."""
        parts = make_particles(prob.particles)
        st = {"per_job": storage or "fp32", "auto": "fp32"}.get(self.storage, self.storage)
        job = Job(make_grid(prob, st), prob.tau, prob.eps, C.cast(parts, C.POINTER(Particle)),
                  len(prob.particles), int(nsteps), int(mean_window), float(arrival))
        jid = C.c_longlong()
        check(self.L.dilbm_server_submit(self.h, C.byref(job), C.byref(jid)))
        self.np[jid.value] = len(prob.particles)
        return int(jid.value)

    def progress(self) -> ServerStats:
        st = ServerStats()
        check(self.L.dilbm_server_progress(self.h, C.byref(st)))
        return st

    def status(self, jid: int) -> JobStatus:
        st = JobStatus()
        check(self.L.dilbm_server_status(self.h, int(jid), C.byref(st)))
        return st

    def result(self, jid: int, with_mean: bool = False):
        """(np, 3) Fx, Fy, T of the job's last step and its (np, 8) particle
        state (with ``with_mean``: also the (np, 3) mean force over the job's
        mean window, as the middle item); releases the job's record."""
        n = max(1, self.np[jid])
        F = np.zeros((n, 3))
        Fm = np.zeros((n, 3))
        st = (Particle * n)()
        check(self.L.dilbm_server_result(self.h, int(jid), F.ctypes.data, Fm.ctypes.data, C.cast(st, C.c_void_p)))
        k = self.np.pop(jid)
        if with_mean:
            return F[:k], Fm[:k], particles_to_array(st, k)
        return F[:k], particles_to_array(st, k)
