"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a closed form, a
conservation law, an analytic flow, a value printed in the paper, or a
brute-force recomputation written here in plain Python with a different
formula route (closed forms instead of the oracle's literal i-loops).
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_08950_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lattice():
    rows = []
    with open(os.path.join(GOLDEN, "d2q9_eq3_eq4.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            i, cx, cy, w = line.split()
            num, den = w.split("/")
            rows.append((int(cx), int(cy), float(num) / float(den)))
    c = np.array([[r[0], r[1]] for r in rows], dtype=float)
    w = np.array([r[2] for r in rows])
    return c, w


C_LAT, W_LAT = _golden_lattice()
CS2 = 1.0 / 3.0


def test_golden_lattice_matches_eq3_formula():
    # Eq. 3 written as cos/sin of multiples of pi/2 and pi/4.
    for i in range(9):
        if i == 0:
            c = (0.0, 0.0)
        elif i <= 4:
            a = (i - 1) * math.pi / 2
            c = (math.cos(a), math.sin(a))
        else:
            a = (2 * i - 1) * math.pi / 4
            c = (math.sqrt(2) * math.cos(a), math.sqrt(2) * math.sin(a))
        assert np.allclose(C_LAT[i], c, atol=1e-12)
    assert abs(W_LAT.sum() - 1.0) < 1e-15


def test_equilibrium_recovers_lattice_table():
    # f^eq(1, 0) = w_i; the odd part of f^eq in u is w_i c_i.u / cs^2.
    assert np.allclose(O.equilibrium(1.0, 0.0, 0.0), W_LAT, rtol=0, atol=1e-16)
    d = 1e-3
    for axis in (0, 1):
        up = O.equilibrium(1.0, d if axis == 0 else 0.0, d if axis == 1 else 0.0)
        dn = O.equilibrium(1.0, -d if axis == 0 else 0.0, -d if axis == 1 else 0.0)
        c_est = (up - dn) / (2 * d) * CS2 / W_LAT
        assert np.allclose(c_est, C_LAT[:, axis], atol=1e-12)


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.03, 0.05, -0.02), (0.97, -0.08, 0.11)])
def test_equilibrium_moments_A7(rho, ux, uy):
    # Eq. A.7: zeroth, first and second moments of f^eq.
    f = O.equilibrium(rho, ux, uy)
    u = np.array([ux, uy])
    assert abs(f.sum() - rho) < 1e-15
    assert np.allclose(C_LAT.T @ f, rho * u, atol=1e-16)
    pi2 = np.einsum("ia,ib,i->ab", C_LAT, C_LAT, f)
    assert np.allclose(pi2, CS2 * rho * np.eye(2) + rho * np.outer(u, u), atol=1e-15)


def test_phi_special_cases():
    eps = 2.0
    assert O.phi(0.0, eps) == 0.5                       # interface: l = 0
    assert abs(O.phi(50.0, eps) - 1.0) < 1e-15          # deep inside the solid
    assert O.phi(-50.0, eps) < 1e-40                    # far in the fluid
    for l in (0.3, 1.0, 2.5):
        assert abs(O.phi(l, eps) + O.phi(-l, eps) - 1.0) < 1e-15
    # (1 + tanh(1)) / 2 at l = eps / 2
    assert abs(O.phi(1.0, 2.0) - 0.8807970779778823) < 1e-15


RNG = np.random.default_rng(11)
CASES = [(0.8, 1.02, (0.04, -0.01), (0.01, 0.03)),
         (0.65, 0.99, (0.0, 0.0), (-0.05, 0.02)),
         (1.7, 1.0, (0.07, 0.06), (0.07, 0.06))]


@pytest.mark.parametrize("tau,rho,us,ua", CASES)
def test_force_term_moments(tau, rho, us, ua):
    # Eq. 15 with D2Q9 isotropy: sum F_i = 0, sum F_i c_i = (1 - 1/2tau) rho (u_s - u*),
    # sum F_i c_i c_i = (1 - 1/2tau) rho (u_s u_s - u* u*).
    Fi = O.force_term(tau, rho, us[0], us[1], ua[0], ua[1])
    k = (1.0 - 0.5 / tau) * rho
    us_, ua_ = np.array(us), np.array(ua)
    assert abs(Fi.sum()) < 1e-17
    assert np.allclose(C_LAT.T @ Fi, k * (us_ - ua_), rtol=1e-14, atol=1e-18)
    pi2 = np.einsum("ia,ib,i->ab", C_LAT, C_LAT, Fi)
    assert np.allclose(pi2, k * (np.outer(us_, us_) - np.outer(ua_, ua_)), rtol=1e-13, atol=1e-18)


@pytest.mark.parametrize("phi_", [0.0, 0.3, 1.0])
def test_collision_momentum_A8_A13(phi_):
    # The collision keeps mass and gives the fluid momentum phi rho (u_s - u*)
    # (Eq. A.8 with Eq. A.13).  With phi = 0 it is plain BGK (Eq. 1): the
    # second moment relaxes to cs^2 rho I + rho u* u* at rate 1/tau.
    tau = 0.8
    f = O.equilibrium(1.01, 0.03, -0.02) + RNG.uniform(-2e-3, 2e-3, size=9)
    us = (0.05, 0.01)
    fo, Fi, mom = O.collide_node(tau, f, phi_, *us)
    rho = f.sum()
    ua = (C_LAT.T @ f) / rho
    assert abs(mom[0] - rho) < 1e-15 and np.allclose(mom[1:3], ua, atol=1e-16)
    assert abs(fo.sum() - rho) < 1e-15
    assert np.allclose(C_LAT.T @ (fo - f), phi_ * rho * (np.array(us) - ua), atol=1e-16)
    if phi_ == 0.0:
        P = np.einsum("ia,ib,i->ab", C_LAT, C_LAT, f)
        Peq = CS2 * rho * np.eye(2) + rho * np.outer(ua, ua)
        Po = np.einsum("ia,ib,i->ab", C_LAT, C_LAT, fo)
        assert np.allclose(Po, P - (P - Peq) / tau, atol=1e-15)


def _moving_box(force_model=W.FORCE_EQ18, g=(0.0, 0.0)):
    prob = W.Problem(nx=48, ny=40, tau=0.7, eps=2.0, u0=(0.01, -0.005), gravity=g,
                     force_model=force_model,
                     particles=[W.Particle(14.3, 12.7, 6.0, ux=0.02, uy=0.01, omega=0.002, rho_s=1.3),
                                W.Particle(33.1, 27.4, 5.0, ux=-0.01, uy=0.015, omega=-0.001, rho_s=1.1)])
    return prob


def test_mass_conservation_periodic():
    # Eq. 13 with sum F_i = 0 and periodic streaming keeps total mass.
    sim = O.OracleSim(_moving_box())
    m0 = sim.populations().sum()
    for _ in range(5):
        sim.step(40)
        assert abs(sim.populations().sum() - m0) / m0 < 1e-12


@pytest.mark.parametrize("fm", [W.FORCE_EQ18, W.FORCE_MOMENTUM])
def test_total_momentum_invariant(fm):
    # The collision hands the fluid phi rho (u_s - u*) (Eq. A.13); the particle
    # receives the force of Eq. 18 = -(1 - 1/2tau) of that (or all of it with
    # momentum exchange).  Hence k P_fluid + sum m U is invariant, with
    # k = 1 - 1/2tau (Eq. 18) or k = 1 (momentum exchange).
    prob = _moving_box(force_model=fm)
    k = (1.0 - 0.5 / prob.tau) if fm == W.FORCE_EQ18 else 1.0
    sim = O.OracleSim(prob)
    masses = np.array([q.rho_s * math.pi * q.r ** 2 for q in prob.particles])

    def invariant():
        f = sim.populations()
        pf = np.array([np.einsum("i,iyx->", C_LAT[:, a], f) for a in (0, 1)])
        _, _, st = sim.forces()
        pp = (masses[:, None] * st[:, 3:5]).sum(axis=0)
        return k * pf + pp

    sim.step(1)
    i0 = invariant()
    sim.step(150)
    _, _, st = sim.forces()
    assert np.abs(st[:, 3:5]).max() > 1e-3     # the particles do interact
    assert np.allclose(invariant(), i0, rtol=0, atol=1e-11)


def test_degenerate_coupling_comoving():
    # u_s = u* everywhere: F_i = 0, no force, the uniform flow stays uniform and
    # the neutrally buoyant particle drifts with it.
    u0 = (0.02, 0.01)
    prob = W.Problem(nx=32, ny=24, tau=0.9, eps=2.0, u0=u0,
                     particles=[W.Particle(10.0, 12.0, 5.0, ux=u0[0], uy=u0[1], rho_s=1.0)])
    sim = O.OracleSim(prob)
    sim.step(50)
    rho, ux, uy, phi, _ = sim.fields()
    assert np.abs(ux - u0[0]).max() < 1e-14 and np.abs(uy - u0[1]).max() < 1e-14
    F, _, st = sim.forces()
    assert np.abs(F).max() < 1e-13
    assert abs(st[0, 0] - (10.0 + 50 * u0[0])) < 1e-12


def _brute_phi(prob, parts):
    """Pure-Python Eq. 14 over every node and particle (min-image), max rule."""
    ny, nx = prob.ny, prob.nx
    phi = np.zeros((ny, nx))
    own = -np.ones((ny, nx), dtype=int)
    rel = np.zeros((ny, nx, 2))
    for y in range(ny):
        for x in range(nx):
            best = 0.0
            for q, p in enumerate(parts):
                dx, dy = x - p.x, y - p.y
                dx -= nx * math.floor(dx / nx + 0.5)
                dy -= ny * math.floor(dy / ny + 0.5)
                l = p.r - math.hypot(dx, dy)
                v = 0.5 * (1.0 + math.tanh(2.0 * l / prob.eps))
                if v > best:
                    best, own[y, x], rel[y, x] = v, q, (dx, dy)
            phi[y, x] = best
    return phi, own, rel


def _brute_forces(prob, parts, rho, uax, uay, phi, own, rel):
    """Eqs. 18-19 via the closed form sum_i F_i c_i = (1-1/2tau) rho (u_s - u*)."""
    k = 1.0 - 0.5 / prob.tau
    F = np.zeros((len(parts), 3))
    for y in range(prob.ny):
        for x in range(prob.nx):
            q = own[y, x]
            if q < 0:
                continue
            p = parts[q]
            rx, ry = rel[y, x]
            usx, usy = p.ux - p.omega * ry, p.uy + p.omega * rx
            gx = -phi[y, x] * k * rho[y, x] * (usx - uax[y, x])
            gy = -phi[y, x] * k * rho[y, x] * (usy - uay[y, x])
            F[q] += (gx, gy, rx * gy - ry * gx)
    return F


def test_brute_force_phi_and_force_sums_tiny():
    # 12 x 10 periodic lattice, two particles (one straddling the edge).
    parts = [W.Particle(3.3, 4.6, 2.7, ux=0.01, uy=-0.02, omega=0.003, rho_s=1.2),
             W.Particle(10.2, 8.9, 2.1, ux=-0.015, uy=0.005, omega=-0.004, rho_s=1.4)]
    prob = W.Problem(nx=12, ny=10, tau=0.75, eps=1.5, u0=(0.012, 0.004), particles=parts)
    sim = O.OracleSim(prob)
    rho, ux, uy, phi, own = sim.fields()
    bphi, bown, rel = _brute_phi(prob, parts)
    assert np.abs(phi - bphi).max() < 1e-14
    assert (own == bown).all()
    # Step 1 collides the uniform initial state: rho = 1, u* = u0 exactly.
    sim.step(1)
    F, _, _ = sim.forces()
    one = np.ones((prob.ny, prob.nx))
    bF = _brute_forces(prob, parts, one, prob.u0[0] * one, prob.u0[1] * one, bphi, bown, rel)
    assert np.allclose(F, bF, rtol=1e-12, atol=1e-17)
    # Step 2 on a non-uniform state: stream the stored populations here
    # (np.roll) and recompute the moments and sums independently.
    _, _, st = sim.forces()
    parts2 = [W.Particle(*st[q, :8]) for q in range(2)]
    f = sim.populations()
    fs = np.stack([np.roll(np.roll(f[i], int(C_LAT[i, 1]), axis=0), int(C_LAT[i, 0]), axis=1)
                   for i in range(9)])
    r2 = fs.sum(axis=0)
    uax = np.einsum("i,iyx->yx", C_LAT[:, 0], fs) / r2
    uay = np.einsum("i,iyx->yx", C_LAT[:, 1], fs) / r2
    bphi2, bown2, rel2 = _brute_phi(prob, parts2)
    sim.step(1)
    F2, _, _ = sim.forces()
    bF2 = _brute_forces(prob, parts2, r2, uax, uay, bphi2, bown2, rel2)
    assert np.allclose(F2, bF2, rtol=1e-11, atol=1e-16)


def test_one_step_newton_euler_against_brute_force():
    # Eqs. 22-24 for one step from the uniform state, with the force and
    # torque recomputed here (pure Python, Eqs. 14, 18-19):
    #   U1 = U0 + (F + (rho_s - rho_f) pi r^2 g) / m,  m = rho_s pi r^2,
    #   omega1 = omega0 + T / I,  I = m r^2 / 2 (a disc of unit depth),
    #   X1 = X0 + U1,  theta1 = theta0 + omega1  (symplectic Euler, dt = 1).
    # A wrong moment of inertia (m r^2) or torque sign moves omega1 by
    # |T / I| ~ 1e-4 relative, far above the 1e-12 bound.
    g = (0.0, -1e-4)
    p0 = W.Particle(5.3, 4.6, 2.7, ux=0.01, uy=-0.02, omega=0.003, theta=0.4, rho_s=1.2)
    prob = W.Problem(nx=12, ny=10, tau=0.75, eps=1.5, u0=(0.012, 0.004), gravity=g, particles=[p0])
    sim = O.OracleSim(prob)
    sim.step(1)
    _, _, st = sim.forces()
    bphi, bown, rel = _brute_phi(prob, [p0])
    one = np.ones((prob.ny, prob.nx))
    F = _brute_forces(prob, [p0], one, prob.u0[0] * one, prob.u0[1] * one, bphi, bown, rel)[0]
    assert abs(F[2]) > 1e-4 * abs(p0.omega) * 0.5 * p0.rho_s * math.pi * p0.r ** 4   # the torque matters
    m = p0.rho_s * math.pi * p0.r ** 2
    inertia = 0.5 * m * p0.r ** 2
    u1 = p0.ux + (F[0] + (p0.rho_s - prob.rho_f) * math.pi * p0.r ** 2 * g[0]) / m
    v1 = p0.uy + (F[1] + (p0.rho_s - prob.rho_f) * math.pi * p0.r ** 2 * g[1]) / m
    w1 = p0.omega + F[2] / inertia
    assert st[0, 3] == pytest.approx(u1, rel=1e-12, abs=1e-17)
    assert st[0, 4] == pytest.approx(v1, rel=1e-12, abs=1e-17)
    assert st[0, 5] == pytest.approx(w1, rel=1e-12, abs=1e-17)
    assert st[0, 0] == pytest.approx(p0.x + u1, abs=1e-14)
    assert st[0, 1] == pytest.approx(p0.y + v1, abs=1e-14)
    assert st[0, 6] == pytest.approx(p0.theta + w1, abs=1e-14)
    # the angular update differs from a moment of inertia m r^2 or a flipped
    # torque by far more than the bound
    assert abs(st[0, 5] - (p0.omega + F[2] / m / p0.r ** 2)) > 1e3 * 1e-12 * abs(w1)
    assert abs(st[0, 5] - (p0.omega - F[2] / inertia)) > 1e3 * 1e-12 * abs(w1)


@pytest.mark.parametrize("fm", [W.FORCE_EQ18, W.FORCE_MOMENTUM])
def test_total_angular_momentum_invariant(fm):
    # Lattice BGK keeps sum_x x cross j exactly: streaming moves c_i f_i from
    # x to x + c_i, and (x + c_i) cross c_i = x cross c_i; the collision keeps
    # each node's momentum.  The coupled collision hands node n the momentum
    # m_n = phi rho (u_s - u*) (Eq. A.13), so the fluid gains sum x_n cross m_n;
    # the particle receives T = -k sum (x_n - X) cross m_n (Eqs. 18-19) and
    # F = -k sum m_n, and symplectic Euler gives its orbital part
    # d(X cross M U) = X cross F.  Hence
    #     k sum_x x cross j + I omega + X cross M U
    # is invariant, with k = 1 - 1/2tau (Eq. 18 as printed) or 1 (momentum
    # exchange), while the disturbance stays clear of the periodic edges: the
    # box is larger than twice the steps plus the reach r + 4 eps about the
    # disc.  A moment of inertia m r^2, a flipped torque or a dropped orbital
    # term breaks it by orders of magnitude more than the bound.
    steps = 30
    n = 2 * (steps + 6 + 8) + 12
    p0 = W.Particle(n / 2 + 0.3, n / 2 - 0.4, 6.0, ux=0.004, uy=-0.003, omega=0.01, rho_s=1.3)
    prob = W.Problem(nx=n, ny=n, tau=0.7, eps=2.0, force_model=fm, particles=[p0])
    k = (1.0 - 0.5 / prob.tau) if fm == W.FORCE_EQ18 else 1.0
    sim = O.OracleSim(prob)
    m = p0.rho_s * math.pi * p0.r ** 2
    inertia = 0.5 * m * p0.r ** 2
    ys, xs = np.mgrid[0:n, 0:n].astype(float)

    def parts():
        f = sim.populations()
        jx = np.einsum("i,iyx->yx", C_LAT[:, 0], f)
        jy = np.einsum("i,iyx->yx", C_LAT[:, 1], f)
        lf = (xs * jy - ys * jx).sum()
        _, _, st = sim.forces()
        X, Y, U, V, om = st[0, 0], st[0, 1], st[0, 3], st[0, 4], st[0, 5]
        return k * lf, inertia * om, m * (X * V - Y * U)

    a0 = parts()
    sim.step(steps)
    a1 = parts()
    assert abs(a1[1] - a0[1]) > 1e-3 * abs(a0[1])           # the disc's spin does change
    assert abs(sum(a1) - sum(a0)) < 1e-12 * abs(a0[1])
    # the readings a plausible slip would take instead
    assert abs(a1[0] + 2 * a1[1] + a1[2] - (a0[0] + 2 * a0[1] + a0[2])) > 1e3 * 1e-12 * abs(a0[1])
    assert abs(a1[0] - a1[1] + a1[2] - (a0[0] - a0[1] + a0[2])) > 1e3 * 1e-12 * abs(a0[1])
    assert abs(a1[0] + a1[1] - (a0[0] + a0[1])) > 1e3 * 1e-12 * abs(a0[1])


def test_translation_invariance():
    # An integer shift of every particle on a periodic box shifts the fields.
    prob = _moving_box()
    prob.u0 = (0.0, 0.0)
    a = O.OracleSim(prob)
    sh = (5, 3)
    prob2 = prob.copy()
    for q in prob2.particles:
        q.x += sh[0]
        q.y += sh[1]
    b = O.OracleSim(prob2)
    a.step(30)
    b.step(30)
    fa, fb = a.fields(), b.fields()
    for va, vb in zip(fa[:4], fb[:4]):
        assert np.abs(np.roll(np.roll(va, sh[1], axis=0), sh[0], axis=1) - vb).max() < 1e-13


def test_mirror_symmetry_cylinder():
    # A centred cylinder in a periodic channel: u_x even and u_y odd about the
    # centre line, zero lift.
    prob = W.cylinder_drag()
    sim = O.OracleSim(prob)
    sim.step(300)
    rho, ux, uy, _, _ = sim.fields()
    j = (100 - np.arange(100)) % 100
    assert np.abs(ux - ux[j]).max() < 1e-12
    assert np.abs(uy + uy[j]).max() < 1e-12
    assert np.abs(rho - rho[j]).max() < 1e-12
    F, _, _ = sim.forces()
    assert abs(F[0, 1]) < 1e-12 and F[0, 0] > 0


def test_couette_linear_profile():
    # No particle: plain BGK between a fixed and a moving wall (velocity
    # sides, non-equilibrium extrapolation) is exactly linear at steady state.
    U = 0.01
    prob = W.Problem(nx=4, ny=17, tau=0.8, eps=2.0, south=W.wall(), north=W.wall(U, 0.0))
    sim = O.OracleSim(prob)
    sim.step(30000)
    _, ux, uy, _, _ = sim.fields()
    y = np.arange(17)
    assert np.abs(ux - U * y[:, None] / 16.0).max() < 1e-10
    assert np.abs(uy).max() < 1e-12


def _poiseuille_error(ny, nx=32, tau=1.1, d=1e-4, steps=None):
    prob = W.Problem(nx=nx, ny=ny, tau=tau, eps=2.0,
                     west=W.Side(W.PRESSURE, rho=1.0 + d / 2), east=W.Side(W.PRESSURE, rho=1.0 - d / 2),
                     south=W.wall(), north=W.wall())
    sim = O.OracleSim(prob)
    sim.step(steps or 40 * (ny - 1) ** 2)
    rho, ux, uy, _, _ = sim.fields()
    nu = (tau - 0.5) / 3.0
    G = CS2 * d / (nx - 1)
    y = np.arange(ny)
    xm = nx // 2
    exact = G * y * (ny - 1 - y) / (2.0 * nu * rho[ny // 2, xm])
    assert np.abs(uy[:, xm]).max() < 1e-3 * exact.max()
    return np.linalg.norm(ux[:, xm] - exact) / np.linalg.norm(exact)


def test_poiseuille_pressure_driven():
    # Pressure inlet/outlet, walls on rows 0 and W: u(y) = G y (W - y) / (2 mu)
    # with G = cs^2 (rho_in - rho_out) / L.  The extrapolated walls converge at
    # second order or better: the error falls by > 3.5x when W doubles.
    e16 = _poiseuille_error(17)
    e32 = _poiseuille_error(33)
    assert e32 < 1e-3
    assert e16 / e32 > 3.5


def test_shear_wave_viscosity_eq6():
    # u_x = A sin(k y) decays as exp(-nu k^2 t) with nu = cs^2 (tau - 1/2) (Eq. 6).
    n, tau = 128, 0.8
    prob, prof = W.shear_wave(n=n, amp=1e-4, tau=tau)
    sim = O.OracleSim(prob)
    f0 = np.stack([np.tile(O.equilibrium(1.0, u, 0.0), (prob.nx, 1)).T for u in prof], axis=1)
    sim.set_populations(f0)
    k = 2.0 * np.pi / n
    s = np.sin(k * np.arange(n))

    def amp():
        _, ux, _, _, _ = sim.fields()
        return (ux[:, 0] @ s) / (s @ s)

    sim.step(200)
    a1 = amp()
    sim.step(2000)
    a2 = amp()
    nu_est = -math.log(a2 / a1) / (k * k * 2000)
    assert abs(nu_est / ((tau - 0.5) / 3.0) - 1.0) < 1e-3


def test_wan_turek_worked_examples():
    # Eq. 28: discs of radius 4 and 3 (r_i + r_j = 7), xi = 1, eps = 2.
    def prob_with(parts, **kw):
        return W.Problem(nx=200, ny=200, tau=0.8, eps=2.0, wan_turek=(2.0, 4.0, 1.0, 3.0, 1.0),
                         particles=parts, **kw)
    far = O.wan_turek(prob_with([W.Particle(50, 50, 4), W.Particle(58.1, 50, 3)]))
    assert np.abs(far).max() == 0.0                          # d = 8.1 > 8
    near = O.wan_turek(prob_with([W.Particle(50, 50, 4), W.Particle(57.5, 50, 3)]))
    # d = 7.5: (1/eps_P)(X_i - X_j)(7 + 1 - 7.5)^2 = (1/2)(-7.5)(0.25)
    assert np.allclose(near[0], (-0.9375, 0.0), atol=1e-15)
    assert np.allclose(near[1], (0.9375, 0.0), atol=1e-15)
    over = O.wan_turek(prob_with([W.Particle(50, 50, 4), W.Particle(50, 56.5, 3)]))
    # d = 6.5 <= 7: (1/eps_P')(X_i - X_j)(7 - 6.5) = (1/4)(-6.5)(0.5)
    assert np.allclose(over[0], (0.0, -0.8125), atol=1e-15)
    # Eq. 29, wall on row 0: image at y = -y_i, d' = 2 y_i.
    walls = dict(south=W.wall(), north=W.wall())
    wnear = O.wan_turek(prob_with([W.Particle(50, 4.25, 4)], **walls))
    # d' = 8.5, 2r = 8: (1/eps_W)(0, 8.5)(8 + 1 - 8.5)^2 = (0, 8.5 * 0.25)
    assert np.allclose(wnear[0], (0.0, 2.125), atol=1e-15)
    wover = O.wan_turek(prob_with([W.Particle(50, 195.0, 4)], **walls))
    # north wall on row 199: image at 2*199 - 195 = 203, d' = 8 -> branch 2 gives 0;
    # at 195.5: d' = 7, (1/eps_W')(0, -7)(8 - 7) = (0, -7/3)
    assert np.abs(wover).max() == 0.0 or np.allclose(wover[0], (0.0, -0.0))
    wover2 = O.wan_turek(prob_with([W.Particle(50, 195.5, 4)], **walls))
    assert np.allclose(wover2[0], (0.0, -7.0 / 3.0), atol=1e-14)


@pytest.mark.parametrize("widths", [4, 6])
def test_phi_cutoff_matches_full_sum(widths):
    # A particle reaches only the nodes within `widths` interface widths of its
    # surface; beyond, phi < 1/(1 + e^(4 widths)) (1.1e-7 at 4 widths), and the
    # fields and forces move by far less than the FP32 tolerance.
    prob = W.periodic_suspension(n=96, count=6, seed=7, rmin=4, rmax=7)
    for q in prob.particles:
        q.ux, q.uy = 0.01, -0.004
    a, b = O.OracleSim(prob), O.OracleSim(prob, phi_cutoff=widths * prob.eps)
    a.step(20)
    b.step(20)
    phi_cut = 1.0 / (1.0 + math.exp(4.0 * widths))      # phi where the reach ends
    for va, vb in zip(a.fields()[:4], b.fields()[:4]):
        assert np.abs(va - vb).max() <= max(1.01 * phi_cut, 1e-9)
    # the dropped tail: sum over l > cut of phi(l) rho |u_s - u*| along the
    # perimeter, phi(l) ~ phi_cut e^(-4 (l - cut) / eps): at most
    # 2 pi (r + cut) (eps / 4) phi_cut |du|, with |du| <= 0.05 here; twice that
    rmax = max(q.r for q in prob.particles)
    cut = widths * prob.eps
    bound = 2.0 * 2.0 * math.pi * (rmax + cut) * (prob.eps / 4.0) * phi_cut * 0.05
    Fa, Fb = a.forces()[0], b.forces()[0]
    assert np.abs(Fa[:, :2] - Fb[:, :2]).max() <= max(bound, 1e-13)
    assert np.abs(Fa[:, 2] - Fb[:, 2]).max() <= max(bound * (rmax + cut), 1e-13)


def test_settling_velocity_against_eq27():
    # Centre-line settling (Sec. 3.2) from rest toward the terminal velocity of
    # Eq. 27 with the wall factor K of Eq. 26.  With the momentum-exchange
    # force the disc reaches Eq. 27 within the error of a coarse (D = 8)
    # diffuse disc.  The force of Eq. 18 as printed carries an extra factor
    # (1 - 1/2tau), so at low Re its terminal velocity is larger by
    # 1 / (1 - 1/2tau).
    r, W_, rho_s, g, tau = 4.0, 48, 1.05, 2e-5, 0.8
    ws = W_ / (2 * r)
    K = 1.0 / (math.log(ws) - 0.9175 + 1.7244 / ws ** 2 - 1.7302 / ws ** 4
               + 2.4056 / ws ** 6 - 4.5913 / ws ** 8)
    mu = (tau - 0.5) / 3.0
    u_eq27 = (2 * r) ** 2 * (rho_s - 1.0) * g / (16 * K * mu)   # downward speed
    v = {}
    for fm in (W.FORCE_EQ18, W.FORCE_MOMENTUM):
        prob = W.sedimentation(nx=W_ + 1, ny=161, r=r, rho_s=rho_s, g=g, tau=tau, force_model=fm)
        sim = O.OracleSim(prob)
        sim.step(5000)
        _, _, st = sim.forces()
        v[fm] = -st[0, 4]
    assert 0.6 < v[W.FORCE_MOMENTUM] / u_eq27 < 1.2
    assert abs(v[W.FORCE_EQ18] / v[W.FORCE_MOMENTUM] * (1 - 0.5 / tau) - 1.0) < 0.05


# ---------------------------------------------------------------- PS-LBM (Sec. 2.2)
@pytest.mark.parametrize("r", [0.3, 0.5, 1.0, 2.5, 6.3, 12.9])
def test_cell_fraction_sums_to_the_disc_area(r):
    # The cells tile the plane, so the covered fractions of a disc anywhere sum
    # to pi r^2 (also when the circle touches cell edges).
    rng = np.random.default_rng(int(r * 100))
    for cx, cy in list(rng.uniform(-0.5, 0.5, size=(4, 2))) + [(0.0, 0.5 - r % 1.0), (0.5, 0.5)]:
        n = int(r) + 3
        tot = sum(O.cell_fraction(x - cx, y - cy, r) for x in range(-n, n + 1) for y in range(-n, n + 1))
        assert abs(tot - math.pi * r * r) <= 1e-12 * math.pi * r * r, (r, cx, cy, tot)


def test_cell_fraction_closed_forms():
    # cell fully inside / outside; a unit disc with the cell's corner at its
    # centre covers a quarter disc; a disc of radius 1/2 centred in the cell
    # lies inside it; a straight boundary (huge r) cuts the cell linearly.
    assert O.cell_fraction(0.0, 0.0, 5.0) == 1.0
    assert O.cell_fraction(7.0, 0.0, 5.0) == 0.0
    assert abs(O.cell_fraction(0.5, 0.5, 1.0) - math.pi / 4) < 1e-14
    assert abs(O.cell_fraction(0.0, 0.0, 0.5) - math.pi / 4) < 1e-14
    R = 1e5
    for t in (-0.4, -0.1, 0.0, 0.25):
        assert abs(O.cell_fraction(R + t, 0.0, R) - (0.5 - t)) < 1e-5
    # symmetries of the square and the disc
    for dx, dy, r in [(3.2, 1.7, 3.9), (-2.3, 4.4, 5.1), (0.4, -6.6, 6.5)]:
        e = O.cell_fraction(dx, dy, r)
        for ex in (O.cell_fraction(-dx, dy, r), O.cell_fraction(dx, -dy, r), O.cell_fraction(dy, dx, r)):
            assert abs(e - ex) < 1e-14


def test_cell_fraction_against_sampling():
    # 1500^2 midpoint samples of boundary cells: sampling error below 2e-4
    rng = np.random.default_rng(7)
    g = (np.arange(1500) + 0.5) / 1500 - 0.5
    X, Y = np.meshgrid(g, g)
    checked = 0
    while checked < 12:
        r = float(rng.uniform(2.5, 12.0))
        a = float(rng.uniform(0, 2 * math.pi))
        d = r + float(rng.uniform(-0.7, 0.7))
        dx, dy = d * math.cos(a), d * math.sin(a)
        e = O.cell_fraction(dx, dy, r)
        if not 0.0 < e < 1.0:
            continue
        bf = float(np.mean((X + dx) ** 2 + (Y + dy) ** 2 < r * r))
        assert abs(e - bf) < 2e-4, (dx, dy, r, e, bf)
        checked += 1


@pytest.mark.parametrize("B", [0.0, 0.37, 1.0])
def test_ps_collision_eq7_eq9_equals_eq12(B):
    # The paper gives the SP collision twice: Eq. 7 with Omega^s of Eq. 9, and
    # the single-term form Eq. 12.  They must agree; the collision keeps mass,
    # hands the fluid B rho (u_s - u*) of momentum, and sum_i Omega^s_i c_i =
    # rho (u_s - u*), so the force of Eq. 10 is -B rho (u_s - u*).  B = 0 is BGK.
    tau = 0.8
    f = O.equilibrium(1.02, 0.02, -0.03) + RNG.uniform(-2e-3, 2e-3, size=9)
    us = (0.05, -0.01)
    fo, om, mom = O.collide_node_ps(tau, f, B, *us)
    rho = f.sum()
    ua = (C_LAT.T @ f) / rho
    feq = O.equilibrium(rho, *ua)
    feqs = O.equilibrium(rho, *us)
    eq12 = f - (f - feq) / tau + B * (feqs - feq)
    assert np.allclose(fo, eq12, atol=1e-16)
    assert abs(fo.sum() - rho) < 1e-15
    assert np.allclose(C_LAT.T @ (fo - f), B * rho * (np.array(us) - ua), atol=1e-16)
    assert np.allclose(C_LAT.T @ om, rho * (np.array(us) - ua), atol=1e-16)
    if B == 0.0:
        assert np.allclose(fo, f - (f - feq) / tau, atol=1e-16)


def test_ps_periodic_box_conserves_mass_and_momentum():
    # PS-LBM force (Eq. 10) is exactly the momentum the collision hands the
    # fluid, so with periodic streaming P_fluid + sum m U stays constant, and
    # the total mass too.
    prob = _moving_box()
    prob.method = W.METHOD_PS
    sim = O.OracleSim(prob)
    masses = np.array([q.rho_s * math.pi * q.r ** 2 for q in prob.particles])

    def totals():
        f = sim.populations()
        pf = np.array([np.einsum("i,iyx->", C_LAT[:, a], f) for a in (0, 1)])
        _, _, st = sim.forces()
        return f.sum(), pf + (masses[:, None] * st[:, 3:5]).sum(axis=0)

    sim.step(1)
    m0, p0 = totals()
    sim.step(60)
    m1, p1 = totals()
    assert abs(m1 - m0) < 1e-10 * m0
    assert np.allclose(p1, p0, atol=1e-11)
    phi = sim.fields()[3]
    assert phi.max() == 1.0 and 0.0 < phi[(phi > 0) & (phi < 1)].min()   # interior and partial cells


def _frame_box():
    # periodic box, flow and discs moving in +x: the tracked disc crosses a
    # column every ~15 steps; the other disc moves against it
    return W.Problem(nx=96, ny=40, tau=0.8, eps=2.0, u0=(0.03, 0.004),
                     particles=[W.Particle(30.4, 20.3, 6.0, ux=0.07, uy=0.003, omega=0.001, rho_s=1.2),
                                W.Particle(71.8, 9.6, 4.0, ux=-0.02, uy=0.01, rho_s=1.5)])


def test_moving_frame_is_a_relabelling_on_a_periodic_axis():
    # Moving the frame on a periodic x axis only renames the columns: the run
    # in the moving frame equals the fixed-frame run rolled by the frame's
    # offset (fields, owners, forces; positions up to the integer offset).
    # A wrong direction for the populations, the particles or the offset, or
    # a move decided on the wrong particle, breaks the equality.
    prob = _frame_box()
    a = O.OracleSim(prob)
    b = O.OracleSim(prob)
    b.set_moving_frame(0, 30.4)
    a.step(200)
    b.step(200)
    off = b.frame_offset()
    assert off >= 8
    fa, fb = a.fields(), b.fields()
    for va, vb in zip(fa, fb):
        assert np.abs(np.roll(va, -off, axis=1).astype(np.float64) - vb).max() < 1e-12
    Fa, _, Sa = a.forces()
    Fb, _, Sb = b.forces()
    assert np.abs(Fa - Fb).max() < 1e-12
    assert np.abs((Sb[:, 0] + off - Sa[:, 0] + 48.0) % 96.0 - 48.0).max() < 1e-9
    assert np.abs(Sb[:, 1:] - Sa[:, 1:]).max() < 1e-12
    # the tracked disc stays within one column of its reference
    assert abs(((Sb[0, 0] - 30.4 + 48.0) % 96.0) - 48.0) < 1.0 + abs(Sb[0, 3]) + 1e-12


def test_moving_frame_keeps_the_channel_flow():
    # Pressure-driven channel (Sec. 3.5's setting at small size) with a
    # neutrally buoyant disc carried downstream; the frame follows it, so
    # columns leave at the inlet and enter at the outlet as zero-gradient
    # copies.  Each move displaces the channel's linear pressure field by one
    # column against the fixed inlet and outlet densities: a density step of
    # one gradient step g = (rho_in - rho_out) / (nx - 1) that the ends then
    # re-absorb within a few tens of steps.  So at every step the far columns
    # must match the same run in a fixed frame to within a few g in density
    # (an entering column taken from anywhere but its neighbour, the inlet
    # side say, puts a jump of the whole drop there) and to within a few
    # per cent of the peak velocity.
    d = 0.01
    nx = 120
    base = dict(nx=nx, ny=25, tau=0.8, eps=2.0,
                west=W.Side(W.PRESSURE, rho=1.0 + d / 2), east=W.Side(W.PRESSURE, rho=1.0 - d / 2),
                south=W.wall(), north=W.wall())
    s0 = O.OracleSim(W.Problem(**base))
    s0.step(12000)
    umax = s0.fields()[1].max()
    prob = W.Problem(**base, particles=[W.Particle(60.0, 12.0, 3.0, ux=0.8 * umax, rho_s=1.0)])
    fixed, moving = O.OracleSim(prob), O.OracleSim(prob)
    for sim in (fixed, moving):
        sim.set_populations(s0.populations())
    moving.set_moving_frame(0, 60.0)
    cols = np.r_[0:6, nx - 6:nx]
    g = d / (nx - 1)
    worst_rho = worst_u = 0.0
    for _ in range(600):
        fixed.step(1)
        moving.step(1)
        rf, uf, _, _, _ = fixed.fields()
        rm, um, _, _, _ = moving.fields()
        worst_u = max(worst_u, np.abs(um[:, cols] - uf[:, cols]).max() / umax)
        worst_rho = max(worst_rho, np.abs(rm[:, cols] - rf[:, cols]).max() / g)
    assert moving.frame_offset() >= 10
    assert 0.5 < worst_rho < 2.5, worst_rho
    assert worst_u < 0.02, worst_u
