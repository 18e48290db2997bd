"""Moving computational domain (Sec. 3.5) on the GPU against the FP64 oracle.

The frame follows one particle: after a step that started with the particle
one lattice unit or more from the reference x, the populations move by one
column (rolled on a periodic axis, the entering column repeating its
neighbour otherwise), every particle's x drops by one and the frame offset
grows by one.  Each case runs the CUDA path and the oracle in their moving
frames and compares offsets (exactly), fields, forces and particle state
with the FP32 tolerances.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_08950_gb300 import dilbm as D
from paper_2106_08950_gb300 import workloads as W
from tests import parity as PAR

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stream():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    D.load_library()
    return int(torch.cuda.Stream().cuda_stream)


def frame_box(method=W.METHOD_DI):
    prob = W.Problem(nx=96, ny=40, tau=0.8, eps=2.0, u0=(0.03, 0.004),
                     particles=[W.Particle(30.4, 20.3, 6.0, ux=0.07, uy=0.003, omega=0.001, rho_s=1.2),
                                W.Particle(71.8, 9.6, 4.0, ux=-0.02, uy=0.01, rho_s=1.5)])
    prob.method = method
    return prob


def frame_channel(method=W.METHOD_DI):
    # pressure-driven channel, walls on the first and last rows, a neutrally
    # buoyant disc released with the flow
    d = 0.01
    prob = W.Problem(nx=160, ny=33, tau=0.8, eps=2.0,
                     west=W.Side(W.PRESSURE, rho=1.0 + d / 2), east=W.Side(W.PRESSURE, rho=1.0 - d / 2),
                     south=W.wall(), north=W.wall(), u0=(0.02, 0.0),
                     particles=[W.Particle(70.3, 11.6, 4.5, ux=0.06, uy=0.002, rho_s=1.0)])
    prob.method = method
    return prob


def run_pair(prob, steps, track, x_ref, stream, storage="fp32"):
    g = D.Simulation(prob, storage=storage, stream=stream)
    o = O.OracleSim(prob, phi_cutoff=PAR.oracle_cutoff(prob))
    g.set_moving_frame(track, x_ref)
    o.set_moving_frame(track, x_ref)
    g.step(steps - 1)
    o.step(steps - 1)
    o.pre = PAR.oracle_pre(o)
    g.step(1)
    o.step(1)
    return g, o


def check_pair(g, o, tol=PAR.TOL_FP32):
    assert g.frame_offset() == o.frame_offset()
    fo = o.fields()
    ok, errs = PAR.compare_fields(g.fields(), fo, tol)
    assert ok, errs
    Fg, _, Sg = g.forces()
    Fo, _, So = o.forces()
    rmax = max(q.r for q in g.prob.particles)
    atol = PAR.ps_force_floor(fo[3], So) if g.prob.method == W.METHOD_PS else 0.0
    ok, e = PAR.compare_forces_terms(Fg, Fo, PAR.force_term_scales(g.prob, *o.pre), tol, atol, rmax)
    assert ok, e
    ok, e = PAR.compare_state(Sg, So)
    assert ok, e


@pytest.mark.parametrize("method", [W.METHOD_DI, W.METHOD_PS])
def test_frame_on_a_periodic_axis(stream, method):
    g, o = run_pair(frame_box(method), 200, 0, 30.4, stream)
    assert g.frame_offset() >= 5
    check_pair(g, o)


@pytest.mark.parametrize("method", [W.METHOD_DI, W.METHOD_PS])
def test_frame_in_a_pressure_driven_channel(stream, method):
    g, o = run_pair(frame_channel(method), 400, 0, 70.3, stream)
    assert g.frame_offset() >= 6
    check_pair(g, o)


def test_frame_is_a_relabelling_on_the_gpu(stream):
    # the moving-frame run equals the fixed-frame run rolled by the offset,
    # up to the FP32 rounding of the particle offsets
    prob = frame_box()
    a = D.Simulation(prob, stream=stream)
    b = D.Simulation(prob, stream=stream)
    b.set_moving_frame(0)
    a.step(200)
    b.step(200)
    off = b.frame_offset()
    assert off >= 8
    fa, fb = a.fields(), b.fields()
    for va, vb in zip(fa, fb):
        assert np.abs(np.roll(va, -off, axis=1) - vb).max() < 1e-5
    Sa, Sb = a.forces()[2], b.forces()[2]
    assert np.abs((Sb[:, 0] + off - Sa[:, 0] + 48.0) % 96.0 - 48.0).max() < 1e-5


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_frame_with_reduced_storage(stream, storage):
    # the column move copies stored values: reduced storage moves exactly as
    # FP32 does, so the frame offsets agree and the state stays within the
    # reduced-storage bound
    g, o = run_pair(frame_channel(), 300, 0, 70.3, stream, storage=storage)
    assert g.frame_offset() == o.frame_offset() >= 5
    ok, errs = PAR.compare_fields(g.fields(), o.fields(), 2e-2)
    assert ok, errs


def test_frame_switches_off_and_on(stream):
    prob = frame_box()
    g = D.Simulation(prob, stream=stream)
    o = O.OracleSim(prob, phi_cutoff=PAR.oracle_cutoff(prob))
    g.set_moving_frame(0, 30.4)
    o.set_moving_frame(0, 30.4)
    g.step(60)
    o.step(60)
    g.set_moving_frame(-1)
    o.set_moving_frame(-1, 0.0)
    g.step(60)
    o.step(60)
    off = g.frame_offset()
    # the second disc sits ~10 columns past 60: the frame moves on ten
    # consecutive steps, then follows it
    g.set_moving_frame(1, 60.0)
    o.set_moving_frame(1, 60.0)
    g.step(79)
    o.step(79)
    o.pre = PAR.oracle_pre(o)
    g.step(1)
    o.step(1)
    assert g.frame_offset() >= off + 10
    check_pair(g, o)


def test_frame_restrictions(stream):
    prob = frame_box()
    sim = D.Simulation(prob, stream=stream)
    with pytest.raises(D.DilbmError):
        sim.set_moving_frame(2, 10.0)
    with pytest.raises(D.DilbmError):
        sim.set_moving_frame(0, float("nan"))
    sim.set_moving_frame(0)
    with pytest.raises(D.DilbmError):
        D.Batch([sim])
    sim.set_moving_frame(-1)
    D.Batch([sim]).close()
    wide = W.Problem(nx=12289, ny=8, tau=0.8, eps=2.0, particles=[W.Particle(100.0, 4.0, 2.0)])
    w = D.Simulation(wide, stream=stream)
    with pytest.raises(D.DilbmError):
        w.set_moving_frame(0)
    w.close()
    sim.close()
