"""Sec. 3.5 and Table 2: a neutrally buoyant disc in pressure-driven
Poiseuille flow, followed by the moving computational domain.

The paper's setup in lattice units: L x W = 20 x 4 with dx = 1/25, so a
500 x 100 channel (walls on rows 0 and 100), D = 1 -> r = 12.5, start at
(L/2, W/4) at rest, pressure drop 0.00267 (rho_in - rho_out = 3 x 0.00267),
tau = 0.75.  The channel flow is developed first without the disc (the
same library, 100k steps), the disc is then released into it and the frame
follows it.  The disc migrates to its equilibrium height within ~30k steps.

Table 2: DI-LBM 0.2876 (W from the lower wall), Li et al. 0.2874, Tao et
al. 0.2849; the paper's PS-LBM with the SP collision 0.50 (the centre line).
The paper gives no interface width; the equilibrium rises with it (0.2892
at eps = 1, 0.2943 at eps = 2, 0.3014 at eps = 3), toward the reference
values as the interface sharpens.  The exact-area PS-LBM here settles near
0.288, not on the centre line.
"""
import numpy as np
import pytest

from paper_2106_08950_gb300 import dilbm as D
from paper_2106_08950_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TABLE2_DI = 0.2876
DP = 0.00267


def channel(parts, eps=2.0, method=W.METHOD_DI):
    drho = 3.0 * DP
    prob = W.Problem(nx=501, ny=101, tau=0.75, eps=eps,
                     west=W.Side(W.PRESSURE, rho=1.0 + drho / 2), east=W.Side(W.PRESSURE, rho=1.0 - drho / 2),
                     south=W.wall(), north=W.wall(), particles=parts)
    prob.method = method
    return prob


@pytest.fixture(scope="module")
def developed():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    D.load_library()
    stream = int(torch.cuda.Stream().cuda_stream)
    dev = D.Simulation(channel([]), stream=stream)
    dev.step(100000)
    f = dev.populations()
    _, ux, uy, _ = dev.fields()
    dev.close()
    # the developed flow is the plane Poiseuille profile, up to what is left
    # of the start-up (the slowest mode decays as exp(-nu pi^2 t / W^2), e^-8
    # after 100k steps) and the compressibility of a pressure-driven lattice
    # flow (density falls by 0.8 % along the channel): a few 1e-4 of the peak
    y = np.arange(101)
    prof = ux[:, 250]
    fit = prof[50] * 4.0 * y * (100 - y) / 100.0 ** 2
    assert np.abs(prof - fit).max() < 3e-3 * prof[50]
    assert np.abs(uy).max() < 1e-4 * prof[50]
    return stream, f


def migrate(developed, y0, eps=2.0, method=W.METHOD_DI, steps=60000, every=5000):
    stream, f = developed
    sim = D.Simulation(channel([W.Particle(250.0, y0, 12.5, rho_s=1.0)], eps, method), stream=stream)
    sim.set_populations(f)
    sim.set_moving_frame(0, 250.0)
    ys = []
    for _ in range(steps // every):
        sim.step(every)
        ys.append(sim.forces()[2][0, 1] / 100.0)
    off = sim.frame_offset()
    sim.close()
    ys = np.array(ys)
    assert np.ptp(ys[-3:]) < 2e-4, ys            # settled
    # carried downstream near the mean flow speed: thousands of frame moves
    assert off > 0.03 * steps
    return ys[-1]


def test_di_equilibrium_matches_table2(developed):
    y2 = migrate(developed, 25.0, eps=2.0)
    y1 = migrate(developed, 25.0, eps=1.0)
    assert abs(y2 - TABLE2_DI) < 0.01, y2
    assert abs(y1 - TABLE2_DI) < 0.005, y1
    assert abs(y1 - TABLE2_DI) < abs(y2 - TABLE2_DI)   # sharper interface, closer to Table 2


def test_di_equilibrium_is_reached_from_either_side(developed):
    below = migrate(developed, 25.0)
    above = migrate(developed, 40.0)
    assert abs(below - above) < 1e-3


def test_ps_equilibrium(developed):
    y = migrate(developed, 25.0, method=W.METHOD_PS)
    assert abs(y - TABLE2_DI) < 0.01, y
    assert y < 0.4                                 # off the centre line
