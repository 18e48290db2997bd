"""The C ABI library loads, exports every entry point of include/*.h, and
rejects bad arguments before touching the GPU (no compute call here)."""
import ctypes as C
import glob
import os
import re

import pytest

from paper_2106_08950_gb300 import build as B
from paper_2106_08950_gb300 import dilbm as D
from paper_2106_08950_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(dilbm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return D.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dilbm_create", "dilbm_step", "dilbm_forces", "dilbm_fields", "dilbm_sync",
                     "dilbm_destroy", "dilbm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_sizes_match_header_layout():
    # dilbm_side: int + 3 doubles (with padding) = 32 bytes; dilbm_particle: 8 doubles + int.
    assert C.sizeof(D.Side) == 32
    assert C.sizeof(D.Particle) == 72
    assert C.sizeof(D.Grid) == 8 + 4 * 32 + 16 + 8 + 8 + 16 + 8 + 40 + 8   # ... wan_turek, method (+ padding)


def _create(lib, prob, tau=None, eps=None, lattice=0, storage="fp32"):
    g = D.make_grid(prob, storage)
    parts = D.make_particles(prob.particles)
    h = C.c_void_p()
    rc = lib.dilbm_create(C.byref(g), lattice, prob.tau if tau is None else tau,
                          prob.eps if eps is None else eps, parts, len(prob.particles), None, C.byref(h))
    return rc, h


@pytest.mark.parametrize("kw", [dict(tau=0.5), dict(tau=0.3), dict(eps=0.0), dict(lattice=7)])
def test_bad_parameters_rejected(lib, kw):
    rc, h = _create(lib, W.cylinder_drag(), **kw)
    assert rc == D.ERR_INVALID_ARG and not h.value
    assert lib.dilbm_last_error()


def test_bad_geometry_rejected(lib):
    p = W.cylinder_drag()
    p.nx = 2
    assert _create(lib, p)[0] == D.ERR_INVALID_ARG
    p = W.cylinder_drag()
    p.east = W.Side()   # periodic on one side of the x axis only
    assert _create(lib, p)[0] == D.ERR_INVALID_ARG
    p = W.cylinder_drag()
    p.particles[0].x = 250.0   # outside the lattice
    assert _create(lib, p)[0] == D.ERR_INVALID_ARG
    p = W.cylinder_drag()
    p.particles[0].r = -1.0
    assert _create(lib, p)[0] == D.ERR_INVALID_ARG


def test_null_arguments_rejected(lib):
    assert lib.dilbm_create(None, 0, 0.8, 2.0, None, 0, None, None) == D.ERR_INVALID_ARG
    assert lib.dilbm_step(None, 1) == D.ERR_INVALID_ARG
    assert lib.dilbm_sync(None) == D.ERR_INVALID_ARG
    assert lib.dilbm_forces(None, None, None, None) == D.ERR_INVALID_ARG
    lib.dilbm_destroy(None)


def _c_layout():
    """sizeof / offsetof of the header's structs as a C compiler lays them out."""
    import subprocess
    import tempfile
    src = r'''
#include <stddef.h>
#include <stdio.h>
#include "dilbm.h"
int main(void) {
    printf("grid %zu\n", sizeof(dilbm_grid));
    printf("particle %zu\n", sizeof(dilbm_particle));
    printf("server_config %zu %zu %zu\n", sizeof(dilbm_server_config), offsetof(dilbm_server_config, macro_steps),
           offsetof(dilbm_server_config, policy));
    printf("job %zu %zu %zu %zu %zu\n", sizeof(dilbm_job), offsetof(dilbm_job, particles), offsetof(dilbm_job, nsteps), offsetof(dilbm_job, mean_window),
           offsetof(dilbm_job, arrival));
    printf("job_status %zu %zu %zu\n", sizeof(dilbm_job_status), offsetof(dilbm_job_status, steps_done),
           offsetof(dilbm_job_status, footprint));
    printf("server_stats %zu %zu %zu\n", sizeof(dilbm_server_stats), offsetof(dilbm_server_stats, node_updates),
           offsetof(dilbm_server_stats, launches));
    return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode()
    return {ln.split()[0]: [int(v) for v in ln.split()[1:]] for ln in out.strip().splitlines()}


def test_binding_structs_match_the_c_compiler():
    lay = _c_layout()
    assert lay["grid"] == [C.sizeof(D.Grid)]
    assert lay["particle"] == [C.sizeof(D.Particle)]
    assert lay["server_config"] == [C.sizeof(D.ServerConfig), D.ServerConfig.macro_steps.offset,
                                    D.ServerConfig.policy.offset]
    assert lay["job"] == [C.sizeof(D.Job), D.Job.particles.offset, D.Job.nsteps.offset, D.Job.mean_window.offset,
                          D.Job.arrival.offset]
    assert lay["job_status"] == [C.sizeof(D.JobStatus), D.JobStatus.steps_done.offset, D.JobStatus.footprint.offset]
    assert lay["server_stats"] == [C.sizeof(D.ServerStats), D.ServerStats.node_updates.offset,
                                   D.ServerStats.launches.offset]


def test_footprint_counts_both_population_buffers(lib):
    prob = W.cylinder_drag()
    f32, f16, b16 = (D.footprint(prob, s) for s in ("fp32", "fp16", "bf16"))
    pitch = (prob.nx + 31) // 32 * 32
    pops32 = 2 * 9 * pitch * prob.ny * 4
    assert f32 > pops32 and f16 == b16
    # the two storages differ by exactly half the population bytes (guards included)
    assert f32 - f16 == 2 * (9 * pitch * prob.ny + 2 * 256) * 2
    big = prob.copy(particles=prob.particles * 1)
    big.particles = [W.Particle(40.0 + 30 * k, 50.0, 5.0) for k in range(4)]
    assert D.footprint(big) > D.footprint(prob.copy(particles=[])) > 0
    g = D.make_grid(prob)
    out = C.c_ulonglong()
    assert lib.dilbm_footprint(None, 0, C.byref(out)) == D.ERR_INVALID_ARG
    assert lib.dilbm_footprint(C.byref(g), -1, C.byref(out)) == D.ERR_INVALID_ARG


def test_server_validates_jobs_on_the_host(lib):
    # a server with an explicit budget touches no device until progress()
    srv = D.Server("fp32", max_jobs=4, macro_steps=16, memory_budget=64e6)
    ok = W.cylinder_drag()
    a = srv.submit(ok, 100, arrival=0.5)
    b = srv.submit(ok, 50)
    assert (a, b) == (0, 1)
    st = srv.status(a)
    assert st.state == D.JOB_QUEUED and st.arrival == 0.5 and st.steps_done == 0
    assert st.footprint == D.footprint(ok)
    assert srv.status(b).arrival >= 0.0
    with pytest.raises(D.DilbmError):
        srv.submit(ok.copy(tau=0.5), 10)                 # tau must be > 0.5
    with pytest.raises(D.DilbmError):
        srv.submit(ok, 0)                                # at least one step
    with pytest.raises(D.DilbmError):
        srv.submit(ok, 10, mean_window=11)               # window longer than the job
    with pytest.raises(D.DilbmError):
        srv.submit(W.Problem(nx=4096, ny=4096, tau=0.8, eps=2.0), 10)   # beyond the budget
    with pytest.raises(D.DilbmError):
        srv.status(99)
    with pytest.raises(D.DilbmError):
        srv.result(a)                                    # not done
    srv.close()


def test_server_config_rejected(lib):
    for kw in (dict(max_jobs=0), dict(max_jobs=5000), dict(macro_steps=0), dict(policy=7)):
        with pytest.raises(D.DilbmError):
            D.Server("fp32", memory_budget=1e6, **kw)
