"""dilbm_step_static: a time step that allocates no device memory.

Callers that cannot call cudaMalloc where they step (a solver that owns a
fixed device memory pool, a stream-ordered pipeline in which an allocation
would synchronise the device) pass their own populations, particles and force
buffer; the library takes its scratch from a static device array.  The test
allocates those caller buffers with torch, calls the entry point through the
C ABI twice in a row, and checks each result against dilbm_step on the same
state within the FP32 parity tolerance.  It lives in its own file so that it
runs after every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2106_08950_gb300 import dilbm as D
from paper_2106_08950_gb300 import workloads as W
from tests import parity as PAR

pytestmark = pytest.mark.gpu

POP_OFFSET = 256          # DILBM_STATIC_POP_OFFSET


def pitch_of(nx):
    return (nx + 31) // 32 * 32                  # DILBM_STATIC_PITCH


def to_static_layout(f, nx, ny):
    """FP64 populations (9, ny, nx) -> the FP32 deviation buffer of
    DILBM_STATIC_POP_FLOATS(nx, ny) floats."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float32).astype(np.float64)
    p = pitch_of(nx)
    buf = np.zeros(9 * ny * p + 2 * POP_OFFSET, dtype=np.float32)
    planes = buf[POP_OFFSET:POP_OFFSET + 9 * ny * p].reshape(9, ny, p)
    planes[:, :, :nx] = (f - w[:, None, None]).astype(np.float32)
    return buf


def from_static_layout(buf, nx, ny):
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float32).astype(np.float64)
    p = pitch_of(nx)
    planes = buf[POP_OFFSET:POP_OFFSET + 9 * ny * p].reshape(9, ny, p)[:, :, :nx]
    return planes.astype(np.float64) + w[:, None, None]


@pytest.mark.parametrize("case", ["periodic", "walls"])
def test_static_step_matches_dilbm_step(case):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = D.load_library()
    L.dilbm_step_static.argtypes = [C.POINTER(D.Grid), C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    L.dilbm_step_static.restype = C.c_int

    if case == "periodic":
        prob = W.Problem(nx=160, ny=40, tau=0.7, eps=2.0, u0=(0.01, -0.004), gravity=(0.0, -2e-5),
                         wan_turek=W.wan_turek_defaults(5.0, 1.3, 1.0, 2e-5),
                         particles=[W.Particle(20.3, 12.7, 6.0, ux=0.02, uy=0.01, omega=0.002, rho_s=1.3),
                                    W.Particle(90.6, 27.4, 5.0, ux=-0.01, uy=0.015, rho_s=1.1),
                                    W.Particle(151.2, 3.1, 4.5, ux=0.005, rho_s=1.6)])
    else:
        prob = W.sedimentation(nx=64, ny=96, r=6.0, rho_s=1.5, g=2e-5, x0=6.3, y0=60.0)
    nx, ny, npart = prob.nx, prob.ny, len(prob.particles)

    stream = torch.cuda.Stream()
    ref = D.Simulation(prob, stream=int(stream.cuda_stream))
    ref.step(5)                                    # a non-uniform starting state
    _, _, st = ref.forces()
    start = [W.Particle(*row[:8], fixed=q.fixed) for row, q in zip(st, prob.particles)]

    # caller-owned device buffers (allocated here, by the caller)
    fa = torch.from_numpy(to_static_layout(ref.populations(), nx, ny)).cuda()
    fb = torch.zeros_like(fa)
    parts = D.make_particles(start)
    pdev = torch.from_numpy(np.frombuffer(bytes(parts), dtype=np.uint8).copy()).cuda()
    force = torch.zeros(npart * 3, dtype=torch.float64, device="cuda")
    grid = D.make_grid(prob, "fp32")
    torch.cuda.synchronize()

    for call in range(2):
        rc = L.dilbm_step_static(C.byref(grid), prob.tau, prob.eps, fa.data_ptr(), fb.data_ptr(),
                                 pdev.data_ptr(), npart, force.data_ptr(), int(stream.cuda_stream))
        assert rc == D.OK, L.dilbm_last_error().decode()
        ref.step(1)
        Fr, _, Sr = ref.forces()
        Fs = force.cpu().numpy().reshape(npart, 3)
        arr = (D.Particle * npart).from_buffer_copy(pdev.cpu().numpy().tobytes())
        Ss = D.particles_to_array(arr, npart)
        ok, e = PAR.compare_forces(Fs, Fr, PAR.TOL_FP32, max(q.r for q in prob.particles))
        assert ok, (call, e)
        ok, e = PAR.compare_state(Ss, Sr)
        assert ok, (call, e)
        fs = from_static_layout(fb.cpu().numpy(), nx, ny)
        fr = ref.populations()
        assert np.abs(fs - fr).max() <= PAR.TOL_FP32 * np.abs(fr).max(), call
        fa, fb = fb, fa


def test_static_step_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = D.load_library()
    L.dilbm_step_static.argtypes = [C.POINTER(D.Grid), C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    L.dilbm_step_static.restype = C.c_int
    prob = W.Problem(nx=2048, ny=2048, tau=0.8, eps=2.0)      # 16 x 256 tiles > 1024
    grid = D.make_grid(prob, "fp32")
    # small real buffers: the size check rejects the call before any work
    a = torch.zeros(64, dtype=torch.float32, device="cuda")
    b = torch.zeros(64, dtype=torch.float32, device="cuda")
    rc = L.dilbm_step_static(C.byref(grid), prob.tau, prob.eps, a.data_ptr(), b.data_ptr(), None, 0, None, None)
    assert rc == D.ERR_INVALID_ARG
    assert b"static scratch" in L.dilbm_last_error()


@pytest.mark.parametrize("bad", ["x_left_of_wall", "zero_radius", "nan_velocity", "inf_x_periodic",
                                 "huge_x_periodic", "huge_radius"])
def test_static_step_rejects_bad_particles_and_changes_nothing(bad):
    # The particles sit in device memory, so the entry point checks them on
    # the device before anything else runs: a bad one is reported as
    # INVALID_ARG, and the output populations and the particles are untouched.
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = D.load_library()
    L.dilbm_step_static.argtypes = [C.POINTER(D.Grid), C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    L.dilbm_step_static.restype = C.c_int
    good = W.Particle(20.3, 12.7, 6.0, ux=0.02, uy=0.01, omega=0.002, rho_s=1.3)
    if bad in ("inf_x_periodic", "huge_x_periodic"):
        prob = W.Problem(nx=160, ny=40, tau=0.7, eps=2.0, particles=[good])
    else:
        prob = W.sedimentation(nx=64, ny=96, r=6.0, rho_s=1.5, g=2e-5, x0=30.0, y0=60.0)
    q = W.Particle(30.0, 20.0, 5.0, rho_s=1.2)
    if bad == "x_left_of_wall":
        q.x = -3.0
    elif bad == "zero_radius":
        q.r = 0.0
    elif bad == "nan_velocity":
        q.ux = float("nan")
    elif bad == "inf_x_periodic":
        q.x = float("inf")
    elif bad == "huge_x_periodic":
        q.x = 1e17
    else:
        q.r = 1e4
    parts_in = list(prob.particles) + [q]
    npart, nx, ny = len(parts_in), prob.nx, prob.ny
    n = 9 * ny * pitch_of(nx) + 2 * POP_OFFSET
    fa = torch.zeros(n, dtype=torch.float32, device="cuda")
    fb = torch.full((n,), 7.0, dtype=torch.float32, device="cuda")
    raw = bytes(D.make_particles(parts_in))
    pdev = torch.from_numpy(np.frombuffer(raw, dtype=np.uint8).copy()).cuda()
    force = torch.zeros(npart * 3, dtype=torch.float64, device="cuda")
    grid = D.make_grid(prob, "fp32")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    rc = L.dilbm_step_static(C.byref(grid), prob.tau, prob.eps, fa.data_ptr(), fb.data_ptr(),
                             pdev.data_ptr(), npart, force.data_ptr(), int(stream.cuda_stream))
    torch.cuda.synchronize()
    assert rc == D.ERR_INVALID_ARG, (rc, L.dilbm_last_error())
    assert b"nothing was changed" in L.dilbm_last_error()
    assert bytes(pdev.cpu().numpy().tobytes()) == raw
    assert bool((fb == 7.0).all())
    assert bool((force == 0.0).all())
