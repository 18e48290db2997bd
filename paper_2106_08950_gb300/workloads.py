"""Seeded synthetic inputs for the DI-LBM hot path.

This module describes problems (lattice size, boundary sides, relaxation
time, interface width, particles) and draws the seeded random parts of
them.  It holds none of the method's arithmetic: no equilibrium, no
collision, no force term.  Both the CUDA path and the FP64 oracle take
their inputs from here, so a problem built once feeds both sides.

The shapes follow the workloads of the paper's Sec. 3 (a fixed cylinder in
a channel, a settling disc in a closed box) scaled to the sizes the
benchmarks use:

* ``cylinder_drag``  -- 200x100 channel, fixed disc r=10 at (50, 50), inlet
  U=0.05, Re=20 (Sec. 3.1 geometry type, Eq. 20 for Re).
* ``sedimentation``  -- 400x2000 closed box, one free disc r=12,
  rho_s/rho_f=1.5, g=1e-5, tau=0.8 (Sec. 3.2 geometry type).
* ``periodic_suspension`` -- 4096^2 periodic box, 2048 discs with radius
  uniform in [6, 12], rho_s/rho_f=1.2, g=1e-6, tau=0.8.
* ``batch_lattices`` -- 64 uneven lattices (log-uniform sizes), each a
  cylinder-drag or sedimentation job.
* ``request_stream`` -- Poisson arrivals of cylinder / sedimentation jobs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

PERIODIC = "periodic"
VELOCITY = "velocity"   # Dirichlet velocity side, density taken from the inner node
PRESSURE = "pressure"   # Dirichlet density side, velocity taken from the inner node

METHOD_DI = 0           # the diffuse-interface LBM (Eqs. 13-19)
METHOD_PS = 1           # the partially saturated LBM with the SP collision (Eqs. 7-11)
FORCE_EQ18 = 0          # hydrodynamic force as printed in Eq. 18
FORCE_MOMENTUM = 1      # momentum given up by the fluid in the collision


@dataclass(frozen=True)
class Side:
    kind: str = PERIODIC
    ux: float = 0.0
    uy: float = 0.0
    rho: float = 1.0


@dataclass
class Particle:
    x: float
    y: float
    r: float
    ux: float = 0.0
    uy: float = 0.0
    omega: float = 0.0
    theta: float = 0.0
    rho_s: float = 1.0
    fixed: bool = False


@dataclass
class Problem:
    nx: int
    ny: int
    tau: float
    eps: float                       # interface width of the solid fraction (Eq. 14)
    west: Side = field(default_factory=Side)
    east: Side = field(default_factory=Side)
    south: Side = field(default_factory=Side)
    north: Side = field(default_factory=Side)
    gravity: Tuple[float, float] = (0.0, 0.0)
    rho_f: float = 1.0               # fluid density in the buoyancy term of Eq. 22
    rho_init: float = 1.0
    u0: Tuple[float, float] = (0.0, 0.0)
    force_model: int = FORCE_EQ18
    method: int = 0                  # METHOD_DI (the paper's DI-LBM) or METHOD_PS (its PS-LBM comparison)
    # Wan-Turek stiffness (Eqs. 28-29): eps_P, eps_P', eps_W, eps_W', xi
    wan_turek: Tuple[float, float, float, float, float] = (1e30, 1e30, 5e29, 5e29, 1.0)
    particles: List[Particle] = field(default_factory=list)
    name: str = ""

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    def copy(self, **kw) -> "Problem":
        p = replace(self, **kw)
        if "particles" not in kw:
            p.particles = [replace(q) for q in self.particles]
        return p


def wall(ux: float = 0.0, uy: float = 0.0) -> Side:
    return Side(VELOCITY, ux, uy, 1.0)


def tau_for(re: float, u: float, d: float) -> float:
    """Relaxation time giving Reynolds number ``re`` for speed ``u`` and
    length ``d`` in lattice units (Re of Eq. 20, viscosity of Eq. 6)."""
    return 0.5 + 3.0 * u * d / re


def wan_turek_defaults(r_mean: float, rho_s: float, rho_f: float, g: float,
                       xi: float = 1.0) -> Tuple[float, float, float, float, float]:
    """Stiffness for Eqs. 28-29 in lattice units.

    The paper's 1e-7 is quoted without units; here eps_P is chosen so that two
    touching discs of the mean radius repel with the buoyant weight of one
    disc, eps_P' = eps_P, eps_W = eps_P/2, eps_W' = eps_P'/2 (the paper's
    ratios)."""
    w = abs(rho_s - rho_f) * math.pi * r_mean * r_mean * abs(g)
    if w <= 0.0:
        return (1e30, 1e30, 5e29, 5e29, xi)
    ep = 2.0 * r_mean * xi * xi / w
    return (ep, ep, ep / 2.0, ep / 2.0, xi)


# --------------------------------------------------------------------------
# Problem builders
# --------------------------------------------------------------------------

def cylinder_drag(nx: int = 200, ny: int = 100, r: float = 10.0,
                  cx: float = 50.0, cy: float = 50.0, u: float = 0.05,
                  re: float = 20.0, eps: float = 2.0,
                  force_model: int = FORCE_EQ18) -> Problem:
    """Flow past a fixed disc: velocity inlet (west), density outlet (east),
    periodic in y.  Fluid starts at the inlet velocity everywhere."""
    tau = tau_for(re, u, 2.0 * r)
    return Problem(nx=nx, ny=ny, tau=tau, eps=eps,
                   west=Side(VELOCITY, u, 0.0, 1.0), east=Side(PRESSURE, 0.0, 0.0, 1.0),
                   south=Side(), north=Side(), u0=(u, 0.0), force_model=force_model,
                   particles=[Particle(cx, cy, r, fixed=True)],
                   name=f"cylinder {nx}x{ny} r={r:g} Re={re:g}")


def sedimentation(nx: int = 400, ny: int = 2000, r: float = 12.0,
                  rho_s: float = 1.5, g: float = 1e-5, tau: float = 0.8,
                  eps: float = 2.0, x0: Optional[float] = None,
                  y0: Optional[float] = None,
                  force_model: int = FORCE_EQ18) -> Problem:
    """One free disc released from rest in a closed box (four no-slip walls)."""
    x0 = (nx - 1) / 2.0 if x0 is None else x0
    y0 = (ny - 1) / 2.0 if y0 is None else y0
    return Problem(nx=nx, ny=ny, tau=tau, eps=eps,
                   west=wall(), east=wall(), south=wall(), north=wall(),
                   gravity=(0.0, -g), force_model=force_model,
                   wan_turek=wan_turek_defaults(r, rho_s, 1.0, g),
                   particles=[Particle(x0, y0, r, rho_s=rho_s)],
                   name=f"sedimentation {nx}x{ny} r={r:g}")


def _place_discs(rng: np.random.Generator, nx: int, ny: int, n: int,
                 rmin: float, rmax: float, gap: float, periodic: bool,
                 margin: float = 0.0, max_tries: int = 2000000) -> List[Tuple[float, float, float]]:
    """Rejection sampling of non-overlapping discs (surface gap >= ``gap``),
    minimum-image distances on a periodic box, a cell grid for the test."""
    radii = rng.uniform(rmin, rmax, size=n)
    cell = 2.0 * rmax + gap
    gx, gy = max(1, int(nx // cell)), max(1, int(ny // cell))
    grid = {}
    out: List[Tuple[float, float, float]] = []
    tries = 0
    for r in radii:
        while True:
            tries += 1
            if tries > max_tries:
                raise RuntimeError("disc placement did not converge")
            lo = margin + r
            x = rng.uniform(lo, nx - 1 - lo) if not periodic else rng.uniform(0.0, nx)
            y = rng.uniform(lo, ny - 1 - lo) if not periodic else rng.uniform(0.0, ny)
            ci, cj = int(x / nx * gx) % gx, int(y / ny * gy) % gy
            ok = True
            for di in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    key = ((ci + di) % gx, (cj + dj) % gy)
                    for k in grid.get(key, ()):
                        qx, qy, qr = out[k]
                        dx, dy = x - qx, y - qy
                        if periodic:
                            dx -= nx * round(dx / nx)
                            dy -= ny * round(dy / ny)
                        if dx * dx + dy * dy < (r + qr + gap) ** 2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                grid.setdefault((ci, cj), []).append(len(out))
                out.append((float(x), float(y), float(r)))
                break
    return out


def periodic_suspension(n: int = 4096, count: int = 2048, seed: int = 3,
                        rmin: float = 6.0, rmax: float = 12.0, rho_s: float = 1.2,
                        g: float = 1e-6, tau: float = 0.8, eps: float = 2.0,
                        gap: float = 4.0, force_model: int = FORCE_EQ18,
                        ny: Optional[int] = None) -> Problem:
    """Fully periodic box with ``count`` free discs, radius uniform in
    [rmin, rmax], positions by seeded rejection sampling (surface gap >= gap)."""
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    discs = _place_discs(rng, n, ny, count, rmin, rmax, gap, periodic=True)
    parts = [Particle(x, y, r, rho_s=rho_s) for (x, y, r) in discs]
    rmean = 0.5 * (rmin + rmax)
    return Problem(nx=n, ny=ny, tau=tau, eps=eps, gravity=(0.0, -g),
                   force_model=force_model,
                   wan_turek=wan_turek_defaults(rmean, rho_s, 1.0, g),
                   particles=parts, name=f"periodic {n}x{ny} P={count}")


def _log_uniform_int(rng: np.random.Generator, lo: float, hi: float) -> int:
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def random_job(rng: np.random.Generator, nx_range=(128, 1024), ny_range=(128, 2048),
               p_range=(1, 32), r_range=(5.0, 15.0), re_range=(10.0, 100.0),
               u: float = 0.05, eps: float = 2.0) -> Problem:
    """One cylinder-drag or sedimentation job with seeded sizes and particles."""
    nx = _log_uniform_int(rng, *nx_range)
    ny = _log_uniform_int(rng, *ny_range)
    nparts = int(rng.integers(p_range[0], p_range[1] + 1))
    re = math.exp(rng.uniform(math.log(re_range[0]), math.log(re_range[1])))
    kind = "cylinder" if rng.random() < 0.5 else "sediment"
    rmax_fit = max(r_range[0], min(r_range[1], (min(nx, ny) - 2 * eps - 8) / 4.0))
    for _ in range(50):
        try:
            sub = np.random.default_rng(int(rng.integers(1 << 62)))
            discs = _place_discs(sub, nx, ny, nparts, r_range[0], rmax_fit, 4.0,
                                 periodic=False, margin=3.0 * eps, max_tries=20000)
            break
        except RuntimeError:
            nparts = max(1, nparts // 2)
    else:  # pragma: no cover - the loop above always succeeds for one disc
        raise RuntimeError("could not place discs")
    d = 2.0 * max(r for (_, _, r) in discs)
    tau = tau_for(re, u, d)
    uu = u
    if tau < 0.51:
        tau = 0.51
        uu = (tau - 0.5) * re / (3.0 * d)
    if kind == "cylinder":
        parts = [Particle(x, y, r, fixed=True) for (x, y, r) in discs]
        return Problem(nx=nx, ny=ny, tau=tau, eps=eps,
                       west=Side(VELOCITY, uu, 0.0, 1.0), east=Side(PRESSURE, 0.0, 0.0, 1.0),
                       u0=(uu, 0.0), particles=parts, name=f"cylinder {nx}x{ny} P={len(parts)}")
    g = 1e-5
    parts = [Particle(x, y, r, rho_s=1.5) for (x, y, r) in discs]
    rmean = sum(r for (_, _, r) in discs) / len(discs)
    return Problem(nx=nx, ny=ny, tau=tau, eps=eps,
                   west=wall(), east=wall(), south=wall(), north=wall(),
                   gravity=(0.0, -g), wan_turek=wan_turek_defaults(rmean, 1.5, 1.0, g),
                   particles=parts, name=f"sediment {nx}x{ny} P={len(parts)}")


def batch_lattices(count: int = 64, seed: int = 4, **kw) -> List[Problem]:
    """``count`` independent jobs with log-uniform lattice sizes."""
    rng = np.random.default_rng(seed)
    return [random_job(rng, **kw) for _ in range(count)]


@dataclass
class Request:
    arrival_s: float
    steps: int
    problem: Problem


def request_stream(count: int = 2000, rate_hz: float = 50.0, seed: int = 5,
                   n_range=(128, 2048), p_range=(1, 64),
                   steps_range=(1000, 20000)) -> List[Request]:
    """Poisson arrivals (exponential gaps) of random jobs."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        steps = _log_uniform_int(rng, *steps_range)
        prob = random_job(rng, nx_range=n_range, ny_range=n_range, p_range=p_range)
        out.append(Request(t, steps, prob))
    return out


def shear_wave(n: int = 64, amp: float = 1e-3, tau: float = 0.8, nx: int = 4) -> Tuple[Problem, np.ndarray]:
    """Periodic box with u_x = amp sin(2 pi y / n): returns the problem and
    the initial u_x profile over y (used with a custom initial state)."""
    y = np.arange(n)
    prof = amp * np.sin(2.0 * np.pi * y / n)
    return Problem(nx=nx, ny=n, tau=tau, eps=2.0, name="shear wave"), prof
