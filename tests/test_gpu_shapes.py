"""Launch shapes, the autotuner and graph replay change no result bit."""
import numpy as np
import pytest

from paper_2106_08950_gb300 import dilbm as D
from paper_2106_08950_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(2, 0), (4, 0), (8, 0), (8, 1), (4, 2), (2, 3)]


@pytest.fixture(scope="module")
def stream():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    D.load_library()
    return int(torch.cuda.Stream().cuda_stream)


def problems():
    return [W.periodic_suspension(n=300, count=10, seed=7, rmin=5, rmax=9),
            W.sedimentation(nx=150, ny=260, r=8.0, rho_s=1.5, g=2e-5, y0=150.0),
            W.cylinder_drag(nx=333, ny=70, r=9.0, cx=60.0, cy=35.0)]


def run(prob, storage, stream, shape=None, steps=9, single=False, tune=False):
    sim = D.Simulation(prob, storage=storage, stream=stream)
    if shape:
        sim.set_shape(*shape)
    if tune:
        sim.autotune(reps=2)
    if single:
        for _ in range(steps):
            sim.step(1)
    else:
        sim.step(steps)
    F, _, S = sim.forces()
    f = sim.populations()
    sim.close()
    return f, F, S


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_every_shape_gives_the_same_bits(stream, storage):
    for prob in problems():
        ref = run(prob, storage, stream, single=True)
        for shape in SHAPES:
            got = run(prob, storage, stream, shape=shape)
            for a, b in zip(ref, got):
                assert np.array_equal(a, b), (prob.name, shape)


def test_autotune_keeps_results_and_caches(stream):
    prob = problems()[1]
    ref = run(prob, "fp32", stream)
    got = run(prob, "fp32", stream, tune=True)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    sim = D.Simulation(prob, stream=stream)
    w, b = sim.autotune(reps=2)
    assert w in (2, 4, 8) and b >= 0
    l0 = sim.launches
    assert sim.autotune(reps=2) == (w, b)        # cached: nothing launched
    assert sim.launches == l0
    sim.close()


def test_graph_replay_matches_single_steps(stream):
    for prob in problems():
        for n in (2, 7):
            a = run(prob, "fp32", stream, steps=n)
            b = run(prob, "fp32", stream, steps=n, single=True)
            for x, y in zip(a, b):
                assert np.array_equal(x, y), (prob.name, n)


def test_batch_autotune_keeps_results(stream):
    probs = problems()
    alone = [run(p, "fp32", stream, steps=6) for p in probs]
    members = [D.Simulation(p, stream=stream) for p in probs]
    batch = D.Batch(members)
    batch.step(1)
    w, b = batch.autotune(reps=2)
    assert w in (2, 4, 8)
    batch.step(5)
    batch.sync()
    for m, ref in zip(members, alone):
        F, _, S = m.forces()
        assert np.array_equal(m.populations(), ref[0])
        assert np.array_equal(F, ref[1]) and np.array_equal(S, ref[2])
    batch.close()
    for m in members:
        m.close()


def test_bad_shapes_rejected(stream):
    sim = D.Simulation(problems()[0], stream=stream)
    for shape in ((3, 0), (16, 0), (8, -1)):
        with pytest.raises(D.DilbmError):
            sim.set_shape(*shape)
    sim.close()
