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
    assert C.sizeof(D.Grid) == 8 + 4 * 32 + 16 + 8 + 8 + 16 + 8 + 40


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
