"""Failure detection on the GPU without a fault.

Every device-side wait of the library is bounded by the device's global
timer: a sweep warp that waits longer than 1 s for its staged rows records
DILBM_ERR_TIMEOUT, waits (again bounded) for its own copies in flight and
returns, so the host reads an error instead of finding a hung GPU.  Here the
same bounded wait runs out on a barrier that nothing arrives at; the status
comes back and the device goes on working.  Instability (NaN or rho <= 0) and
tile overflow are reported the same way and are exercised in the parity and
server tests.
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


def test_bounded_wait_reports_timeout_and_the_device_stays_usable(stream):
    rc, waited = D.wait_probe(stream)
    assert rc == D.ERR_TIMEOUT
    assert 1.0 <= waited < 1.5                              # the 1 s limit, then out
    assert "gave up" in D.last_error()
    # the device and the library go on working: a fresh run matches the oracle
    prob = W.Problem(nx=64, ny=48, tau=0.8, eps=2.0, u0=(0.01, 0.0),
                     particles=[W.Particle(30.3, 20.6, 6.0, ux=0.02, rho_s=1.3)])
    g = D.Simulation(prob, stream=stream)
    o = O.OracleSim(prob, phi_cutoff=PAR.oracle_cutoff(prob))
    g.step(50)
    o.step(50)
    g.sync()
    ok, errs = PAR.compare_fields(g.fields(), o.fields())
    assert ok, errs
    g.close()
