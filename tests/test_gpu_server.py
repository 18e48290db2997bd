"""Serving (continuous batching): jobs that join and leave a running mix get
bit for bit the result they get alone (also when the mix holds jobs of
different storage), admission respects the job slots and the memory budget,
and a job that fails leaves the others untouched."""
import numpy as np
import pytest

from paper_2106_08950_gb300 import dilbm as D
from paper_2106_08950_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stream():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    D.load_library()
    return int(torch.cuda.Stream().cuda_stream)


def small_jobs(seed, count):
    """Seeded cylinder / sedimentation jobs of uneven sizes and lengths."""
    rng = np.random.default_rng(seed)
    jobs = []
    for _ in range(count):
        prob = W.random_job(rng, nx_range=(64, 260), ny_range=(64, 260), p_range=(1, 6), r_range=(4.0, 9.0))
        jobs.append((prob, int(rng.integers(20, 120))))
    return jobs


def alone(prob, nsteps, storage, stream):
    sim = D.Simulation(prob, storage=storage, stream=stream)
    sim.step(nsteps)
    F, _, S = sim.forces()
    sim.close()
    return F, S


def drain(srv, pending, ids, check=None):
    """Submit ``pending`` (prob, nsteps, submit-after-macro-step) as their turn
    comes and progress the server until every job has finished."""
    macro = 0
    while True:
        for item in [p for p in pending if p[2] <= macro]:
            ids.append((srv.submit(item[0], item[1]), item[0], item[1]))
            pending.remove(item)
        st = srv.progress()
        macro += 1
        if check:
            check(st)
        if not pending and st.running == 0 and st.queued == 0:
            return st
        assert macro < 10000


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_jobs_in_the_mix_match_alone_bitwise(stream, storage):
    jobs = small_jobs(31, 8)
    # four jobs at the start, the rest join while others run
    pending = [(p, n, 0 if k < 4 else 1 + 2 * k) for k, (p, n) in enumerate(jobs)]
    srv = D.Server(storage, max_jobs=16, macro_steps=16)
    ids = []
    st = drain(srv, pending, ids)
    assert st.done == len(jobs) and st.failed == 0
    assert st.node_updates == sum(p.nx * p.ny * n for p, n in jobs)
    for jid, prob, n in ids:
        s = srv.status(jid)
        assert s.state == D.JOB_DONE and s.steps_done == n
        assert 0 <= s.arrival <= s.admitted <= s.finished
        F, S = srv.result(jid)
        Fa, Sa = alone(prob, n, storage, stream)
        assert np.array_equal(F, Fa), (jid, np.abs(F - Fa).max())
        assert np.array_equal(S, Sa), (jid, np.abs(S - Sa).max())
    srv.close()


def test_mixed_storage_jobs_match_alone_bitwise(stream):
    # one server, jobs in FP32, FP16 and BF16 storage: one batch per storage
    # type, all stepped by the same macro-steps; each job gets bit for bit the
    # result it gets alone in its storage
    jobs = small_jobs(38, 9)
    kinds = ["fp32", "fp16", "bf16"]
    srv = D.Server("per_job", max_jobs=16, macro_steps=16)
    ids = []
    for k, (p, n) in enumerate(jobs):
        ids.append((srv.submit(p, n, storage=kinds[k % 3]), p, n, kinds[k % 3]))
    seen = []
    drain(srv, [], [], check=lambda st: seen.append(st.running))
    assert max(seen) == len(jobs)
    for jid, p, n, st in ids:
        assert srv.status(jid).state == D.JOB_DONE
        F, S = srv.result(jid)
        Fa, Sa = alone(p, n, st, stream)
        assert np.array_equal(F, Fa), (jid, st, np.abs(F - Fa).max())
        assert np.array_equal(S, Sa), (jid, st)
    srv.close()


def test_automatic_storage_picks_fp32_for_viscous_or_packed_jobs(stream):
    # DILBM_STORAGE_AUTO: a job runs in FP16 unless its tau exceeds 0.6 or its
    # discs cover more than 5% of the lattice; each job then gets bit for bit
    # the result it gets alone in the storage it was given
    jobs = small_jobs(39, 8)
    srv = D.Server("auto", max_jobs=16, macro_steps=16)
    ids = [(srv.submit(p, n), p, n) for p, n in jobs]
    drain(srv, [], [])
    kinds = set()
    for jid, p, n in ids:
        st = srv.status(jid)
        assert st.state == D.JOB_DONE
        area = sum(np.pi * q.r ** 2 for q in p.particles) / (p.nx * p.ny)
        want = D.FP32 if (p.tau > 0.6 or area > 0.05) else D.FP16_DEV
        assert st.storage == want, (p.tau, area, st.storage)
        kinds.add(st.storage)
        F, S = srv.result(jid)
        Fa, Sa = alone(p, n, "fp32" if want == D.FP32 else "fp16", stream)
        assert np.array_equal(F, Fa) and np.array_equal(S, Sa), jid
    assert kinds == {D.FP32, D.FP16_DEV}         # the draw exercises both choices
    srv.close()


def test_jobs_overlap_on_the_device(stream):
    jobs = small_jobs(32, 6)
    srv = D.Server("fp32", max_jobs=8, macro_steps=8)
    ids = [srv.submit(p, n) for p, n in jobs]
    running = []
    drain(srv, [], [], check=lambda st: running.append(st.running))
    assert max(running) == len(jobs)        # every job resident at once
    spans = [(srv.status(j).admitted, srv.status(j).finished) for j in ids]
    for a0, a1 in spans:
        for b0, b1 in spans:
            assert a0 < b1 and b0 < a1        # all lifetimes intersect
    srv.close()


def test_admission_by_memory_budget(stream):
    rng = np.random.default_rng(33)
    jobs = [(W.random_job(rng, nx_range=(160, 160), ny_range=(200, 200), p_range=(1, 6), r_range=(4.0, 9.0)),
             int(rng.integers(20, 120))) for _ in range(6)]
    fps = [D.footprint(p) for p, _ in jobs]
    budget = 2.5 * max(fps)                    # two jobs of this size fit at once, three do not
    assert 3 * min(fps) > budget
    srv = D.Server("fp32", max_jobs=16, macro_steps=8, memory_budget=budget)
    ids = [srv.submit(p, n) for p, n in jobs]
    seen = []

    def check(st):
        assert st.memory_in_use <= budget
        assert st.running <= 2
        seen.append(st.running)

    drain(srv, [], [], check=check)
    assert max(seen) == 2
    adm = [srv.status(j).admitted for j in ids]
    assert adm == sorted(adm)                 # FIFO: admitted in arrival order
    for j, (p, n) in zip(ids, jobs):
        F, S = srv.result(j)
        Fa, Sa = alone(p, n, "fp32", stream)
        assert np.array_equal(F, Fa) and np.array_equal(S, Sa)
    srv.close()


def test_job_slots_limit_the_mix(stream):
    jobs = small_jobs(34, 5)
    srv = D.Server("fp16", max_jobs=2, macro_steps=32)
    for p, n in jobs:
        srv.submit(p, n)
    seen = []
    st = drain(srv, [], [], check=lambda st: seen.append(st.running))
    assert max(seen) == 2 and st.done == len(jobs)
    srv.close()


def test_failed_job_leaves_the_others_intact(stream):
    # a fixed disc in a fast flow at tau -> 1/2 goes unstable within a few
    # hundred steps; the job next to it must finish as it does alone
    bad = W.Problem(nx=64, ny=64, tau=0.501, eps=2.0, u0=(0.35, 0.25),
                    particles=[W.Particle(32.0, 32.0, 8.0, fixed=True)])
    good, n_good = small_jobs(35, 1)[0]
    srv = D.Server("fp32", max_jobs=4, macro_steps=50)
    jb = srv.submit(bad, 400)
    jg = srv.submit(good, n_good + 200)
    st = drain(srv, [], [])
    assert st.failed == 1 and st.done == 1
    sb = srv.status(jb)
    assert sb.state == D.JOB_FAILED and sb.error == D.ERR_UNSTABLE
    F, S = srv.result(jg)
    Fa, Sa = alone(good, n_good + 200, "fp32", stream)
    assert np.array_equal(F, Fa) and np.array_equal(S, Sa)
    srv.close()


def test_force_mean_is_the_mean_of_the_step_forces(stream):
    prob, _ = small_jobs(36, 1)[0]
    a = D.Simulation(prob, stream=stream)
    b = D.Simulation(prob, stream=stream)
    a.step(25)
    b.step(25)
    b.force_mean_reset()
    acc = np.zeros((len(prob.particles), 3))
    for _ in range(40):
        a.step(1)
        acc += a.forces()[0]
    b.step(40)
    M, n = b.force_mean()
    assert n == 40
    np.testing.assert_allclose(M, acc * (1.0 / 40), rtol=1e-13, atol=1e-18)
    a.close()
    b.close()


def test_server_mean_window_matches_alone(stream):
    jobs = small_jobs(37, 4)
    srv = D.Server("fp16", max_jobs=8, macro_steps=16)
    ids = [(srv.submit(p, n, mean_window=n // 3), p, n) for p, n in jobs]
    drain(srv, [], [])
    for jid, p, n in ids:
        F, Fm, S = srv.result(jid, with_mean=True)
        sim = D.Simulation(p, storage="fp16", stream=stream)
        sim.step(n - n // 3)
        sim.force_mean_reset()
        sim.step(n // 3)
        M, k = sim.force_mean()
        assert k == n // 3
        assert np.array_equal(Fm, M) and np.array_equal(F, sim.forces()[0])
        sim.close()
    srv.close()
