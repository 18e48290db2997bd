"""Batched stepping (many uneven lattices per launch): every member's result
is bit for bit the one it gets stepped alone, and alone matches the oracle."""
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


def mixed_problems():
    rng = np.random.default_rng(21)
    probs = [W.cylinder_drag(nx=150, ny=60, r=8.0, cx=40.0, cy=30.0),
             W.sedimentation(nx=70, ny=130, r=6.0, rho_s=1.5, g=2e-5, y0=80.0),
             W.periodic_suspension(n=200, count=6, seed=5, rmin=4, rmax=8),
             W.Problem(nx=37, ny=23, tau=0.8, eps=2.0, u0=(0.01, 0.0)),          # no particles, ragged
             W.cylinder_drag(nx=129, ny=45, r=7.0, cx=50.0, cy=22.0)]            # east edge alone in its segment
    probs += [W.random_job(rng, nx_range=(64, 300), ny_range=(64, 300), p_range=(1, 8)) for _ in range(4)]
    return probs


def state(sim):
    F, Fc, S = sim.forces() if sim.np else (np.zeros((0, 3)), np.zeros((0, 2)), np.zeros((0, 8)))
    return sim.populations(), F, S


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_batch_members_match_alone_bitwise(stream, storage):
    probs = mixed_problems()
    alone = [D.Simulation(p, storage=storage, stream=stream) for p in probs]
    members = [D.Simulation(p, storage=storage, stream=stream) for p in probs]
    batch = D.Batch(members)
    for s in alone:
        s.step(7)
    batch.step(7)              # odd: ends mid graph pair
    for s in alone:
        s.step(4)
    batch.step(4)
    batch.sync()
    for k, (a, m) in enumerate(zip(alone, members)):
        fa, Fa, Sa = state(a)
        fm, Fm, Sm = state(m)
        assert np.array_equal(fa, fm), k
        assert np.array_equal(Fa, Fm) and np.array_equal(Sa, Sm), k
    assert batch.launches == 11 * 2 + 1        # 11 steps of sweep + particles, one error gather at sync


def test_batch_mixed_with_member_calls(stream):
    # Members stepped on their own between batch steps (parity changes) and
    # read back mid-run stay consistent with running alone.
    probs = mixed_problems()[:4]
    alone = [D.Simulation(p, stream=stream) for p in probs]
    members = [D.Simulation(p, stream=stream) for p in probs]
    batch = D.Batch(members)
    batch.step(3)
    members[0].step(1)
    members[2].step(2)
    batch.step(2)
    steps = [3 + 1 + 2, 3 + 2, 3 + 2 + 2, 3 + 2]
    for s, n in zip(alone, steps):
        s.step(n)
    for k, (a, m) in enumerate(zip(alone, members)):
        assert np.array_equal(state(a)[0], state(m)[0]), k


def test_batch_member_matches_oracle(stream):
    # one member of a mixed batch against the FP64 oracle (cylinder, 600 steps)
    probs = mixed_problems()
    members = [D.Simulation(p, stream=stream) for p in probs]
    batch = D.Batch(members)
    batch.step(600)
    batch.sync()
    o = O.OracleSim(probs[0], phi_cutoff=PAR.oracle_cutoff(probs[0]))
    o.step(600)
    ok, errs = PAR.compare_fields(members[0].fields(), o.fields())
    assert ok, errs
    Fg, _, _ = members[0].forces()
    Fo, _, _ = o.forces()
    assert abs(Fg[0, 0] - Fo[0, 0]) <= PAR.TOL_FP32 * abs(Fo[0, 0])
    assert abs(Fg[0, 1] - Fo[0, 1]) <= PAR.TOL_FP32 * abs(Fo[0, 0])


def test_batch_rejects_mixed_storage(stream):
    p = W.Problem(nx=40, ny=40, tau=0.8, eps=2.0)
    a = D.Simulation(p, storage="fp32", stream=stream)
    b = D.Simulation(p, storage="fp16", stream=stream)
    with pytest.raises(D.DilbmError) as e:
        D.Batch([a, b])
    assert e.value.code == D.ERR_INVALID_ARG


def test_full_size_batch_workload_against_oracle(stream):
    # The benchmark's batch workload itself (64 uneven lattices, about 19 M
    # nodes, 1-32 discs each), autotuned as bench.py does, for 50 steps: every
    # member's forces and particle state, and 20k sampled nodes of each,
    # against the oracle (same 4-width phi cutoff).
    jobs = W.batch_lattices(seed=4)
    members = [D.Simulation(j, stream=stream) for j in jobs]
    batch = D.Batch(members)
    batch.autotune(reps=2)
    batch.step(50)
    batch.sync()
    rng = np.random.default_rng(1)
    for k, (p, m) in enumerate(zip(jobs, members)):
        o = O.OracleSim(p, phi_cutoff=4 * p.eps)
        o.step(49)
        pre = PAR.oracle_pre(o)
        o.step(1)
        Fg, _, Sg = m.forces()
        Fo, _, So = o.forces()
        ok, e = PAR.compare_forces_terms(Fg, Fo, PAR.force_term_scales(p, *pre))
        assert ok, (k, p.name, e)
        ok, e = PAR.compare_state(Sg, So)
        assert ok, (k, p.name, e)
        gf, of = m.fields(), o.fields()
        idx = rng.integers(0, p.nx * p.ny, size=20000)
        ok, errs = PAR.compare_fields([a.ravel()[idx] for a in gf[:4]], [a.ravel()[idx] for a in of[:4]])
        assert ok, (k, p.name, errs)
    batch.close()
