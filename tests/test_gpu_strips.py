"""One lattice split into strips over ranks, on the GPU.

Two or three processes share the one GPU, each running its strip through the
CUDA library (``dilbm_create_strip``); they exchange the rows beside each cut
and the per-particle force sums over gloo between steps (the host waits; no
kernel waits on another process).  Without particles a strip's arithmetic is
the whole lattice's, node for node, so the gathered populations must equal
the single-lattice run bit for bit.  With discs crossing the cuts the force
sums are added in another order, so the bound against the single lattice is
1e-6, and against the oracle the FP32 parity bound of the other tests.
"""
import os
import socket
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_08950_gb300 import dilbm as D
from paper_2106_08950_gb300 import workloads as W
from tests import parity as PAR

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def cases():
    return {
        # 12 tile rows: cuts at y = 48 (two strips) or 40, 72 (three); one
        # disc on the cut, one across the periodic edge y = 0, moving ones
        "periodic": W.Problem(nx=160, ny=96, tau=0.7, eps=2.0, u0=(0.01, -0.004), gravity=(0.0, -2e-5),
                              wan_turek=W.wan_turek_defaults(5.0, 1.3, 1.0, 2e-5),
                              particles=[W.Particle(20.3, 47.2, 6.0, ux=0.02, uy=0.01, omega=0.002, rho_s=1.3),
                                         W.Particle(90.6, 2.4, 5.0, ux=-0.01, uy=0.015, omega=-0.001, rho_s=1.1),
                                         W.Particle(140.2, 70.3, 4.5, ux=0.005, uy=-0.012, rho_s=1.6)]),
        # closed box: walls, corners; the disc falls through the cut at y = 48
        "walls": W.sedimentation(nx=64, ny=96, r=6.0, rho_s=1.5, g=4e-5, x0=30.7, y0=53.0),
        # no particles: the strips must reproduce the whole lattice bit for bit
        "channel": W.Problem(nx=150, ny=40, tau=0.9, eps=2.0, u0=(0.01, 0.0),
                             west=W.Side(W.VELOCITY, 0.02, 0.0, 1.0), east=W.Side(W.PRESSURE, rho=1.0),
                             south=W.wall(), north=W.wall(0.01, 0.0)),
    }


def rank_main(rank, world, port, name, steps, storage, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2106_08950_gb300 import strips as S
    try:
        torch.cuda.set_device(0)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        prob = cases()[name]
        sim = S.DecomposedSimulation(prob, storage=storage)
        sim.step(steps)
        sim.sync()
        F, Fc, St = sim.forces()
        pops = sim.populations()
        fields = sim.fields()
        if rank == 0:
            q.put(("ok", F, St, pops, fields))
        dist.barrier()
        sim.close()
        dist.destroy_process_group()
    except Exception as e:          # report, so that the parent does not wait for nothing
        q.put(("error", f"rank {rank}: {type(e).__name__}: {e}"))
        raise


def run_strips(name, world, steps, storage="fp32"):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, world, port, name, steps, storage, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
    assert res[0] == "ok", res
    for p in procs:
        assert p.exitcode == 0
    return res[1:]


@pytest.fixture(scope="module")
def stream():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    D.load_library()
    return int(torch.cuda.Stream().cuda_stream)


@pytest.mark.parametrize("world", [2, 3])
def test_strips_without_particles_are_bitwise_the_whole_lattice(stream, world):
    prob = cases()["channel"]
    F, St, pops, fields = run_strips("channel", world, 300)
    g = D.Simulation(prob, stream=stream)
    g.step(300)
    assert np.array_equal(pops, g.populations())
    g.close()


@pytest.mark.parametrize("name,world", [("periodic", 2), ("periodic", 3), ("walls", 2)])
def test_strips_match_the_whole_lattice_and_the_oracle(stream, name, world):
    steps = 300
    prob = cases()[name]
    F, St, pops, fields = run_strips(name, world, steps)
    # the same lattice in one piece
    g = D.Simulation(prob, stream=stream)
    g.step(steps)
    Fg, _, Sg = g.forces()
    gf = [a.astype(np.float64) for a in g.fields()]
    err = PAR.rel_l2_velocity(fields, gf)
    PAR.record("strips_vs_whole_vel", err, 1e-6)
    assert err <= 1e-6
    scale = np.abs(Fg[:, :2]).max()
    PAR.record("strips_vs_whole_force", np.abs(F[:, :2] - Fg[:, :2]).max() / scale, 1e-6)
    assert np.abs(F[:, :2] - Fg[:, :2]).max() <= 1e-6 * scale
    assert np.abs(St[:, :2] - Sg[:, :2]).max() <= 1e-6
    g.close()
    # and the oracle, with the sweep's phi cutoff
    o = O.OracleSim(prob, phi_cutoff=PAR.oracle_cutoff(prob))
    o.step(steps - 1)
    pre = PAR.oracle_pre(o)
    o.step(1)
    ok, errs = PAR.compare_fields(fields, o.fields())
    assert ok, errs
    Fo, _, So = o.forces()
    ok, e = PAR.compare_forces_terms(F, Fo, PAR.force_term_scales(prob, *pre))
    assert ok, e
    ok, e = PAR.compare_state(St, So)
    assert ok, e


def test_strips_in_fp16_match_the_whole_lattice(stream):
    prob = cases()["periodic"]
    F, St, pops, fields = run_strips("periodic", 2, 200, storage="fp16")
    g = D.Simulation(prob, storage="fp16", stream=stream)
    g.step(200)
    gf = [a.astype(np.float64) for a in g.fields()]
    err = PAR.rel_l2_velocity(fields, gf)
    PAR.record("strips_vs_whole_vel_fp16", err, 1e-6)
    assert err <= 1e-6
    g.close()


def test_strip_refusals(stream):
    prob = cases()["periodic"]
    with pytest.raises(D.DilbmError):
        D.Strip(prob, 4, 48)                  # a cut off the 8-row tiles
    with pytest.raises(D.DilbmError):
        D.Strip(prob, 0, 96)                  # the whole lattice is not a strip
    s = D.Strip(prob, 0, 48, stream=stream)
    with pytest.raises(D.DilbmError):
        s.step(1)                             # strips step through begin / end
    with pytest.raises(D.DilbmError):
        s.end()                               # no step begun
    s.begin()
    with pytest.raises(D.DilbmError):
        s.begin()                             # one step at a time
    s.end()
    s.sync()
    s.close()
