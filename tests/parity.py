"""Comparison helpers shared by the GPU parity tests (CUDA path vs oracle).

Every comparison records its measured error beside its bound (``RECORDS``);
the test session prints them at the end (``tests/conftest.py``), so a run's
log shows how close each case came to its bound.
"""
import os

import numpy as np

# FP32 path: relative L2 of the velocity field and relative drag / absolute
# lift-coefficient error against the FP64 oracle.
TOL_FP32 = 1e-5
# A steady wall-driven shear flow (Couette): the FP32 steady state lies
# 1.4e-5 to 1.75e-5 (relative L2) from the exact profile, because at a fixed
# point every node rounds alike every step and the relaxation integrates it.
TOL_FP32_STEADY_SHEAR = 2e-5
# Particle positions (lattice units) after FP32 force integration.
TOL_FP32_POSITION = 1e-5
# FP16 / BF16 deviation storage: drag-coefficient error bound (the target), and
# the bound BF16 (8-bit mantissa, 8x coarser than FP16) is held to as a
# regression check.
TOL_REDUCED_DRAG = 1e-3
TOL_REDUCED = {"fp16": TOL_REDUCED_DRAG, "bf16": 2e-2}


# (test, metric, measured, bound) of every comparison made in this session
RECORDS = []


def oracle_cutoff(prob):
    """The phi cutoff the CUDA sweep applies (4 interface widths, phi < 1.1e-7
    beyond; PS-LBM evaluates covered areas exactly), for the oracle to apply
    the same: parity then measures the FP32 arithmetic, and the cutoff's own
    effect is bounded separately by the oracle pin on the full sum."""
    return 0.0 if getattr(prob, "method", 0) == 1 else 4.0 * prob.eps


def record(metric, value, bound):
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    RECORDS.append((test, metric, float(value), float(bound)))


def rel_l2_velocity(g, o):
    """Relative L2 norm of the velocity difference over all nodes."""
    gx, gy = np.asarray(g[1], np.float64), np.asarray(g[2], np.float64)
    ox, oy = o[1], o[2]
    num = np.sqrt(((gx - ox) ** 2 + (gy - oy) ** 2).sum())
    den = np.sqrt((ox ** 2 + oy ** 2).sum())
    return num / den


def compare_fields(g, o, tol=TOL_FP32, phi_tol=None):
    """g: (rho, ux, uy, phi) float32 from the GPU; o: the oracle's fields.
    ``phi_tol`` (default ``tol``): phi moves with the particle position, by
    at most |dphi/dl| = 1/eps per lattice unit (Eq. 14), so runs whose
    position bound grows with the distance travelled pass (position bound) /
    eps here."""
    phi_tol = tol if phi_tol is None else max(tol, phi_tol)
    errs = {
        "vel_rel_l2": rel_l2_velocity(g, o),
        "rho_max_abs": float(np.abs(g[0] - o[0]).max()),
        "phi_max_abs": float(np.abs(g[3] - o[3]).max()),
    }
    ok = errs["vel_rel_l2"] <= tol and errs["rho_max_abs"] <= tol and errs["phi_max_abs"] <= phi_tol
    for k, v in errs.items():
        record(k, v, phi_tol if k == "phi_max_abs" else tol)
    return ok, errs


def compare_forces(Fg, Fo, tol=TOL_FP32, rmax=None, atol=0.0):
    """Per-particle force relative to the largest force magnitude F, and torque
    relative to the larger of the largest torque and F times the largest
    radius (the torque's natural scale).  ``atol`` (force; torque: atol times
    the largest radius) is an absolute floor for sums whose net value is a
    small residual of their terms (see ps_force_floor)."""
    scale = max(np.abs(Fo[:, :2]).max(), 1e-30)
    dF = float(np.abs(Fg[:, :2] - Fo[:, :2]).max())
    err_f = dF / scale
    tscale = max(np.abs(Fo[:, 2]).max(), scale * (rmax if rmax else 1.0))
    dT = float(np.abs(Fg[:, 2] - Fo[:, 2]).max())
    err_t = dT / tscale
    ok_f = err_f <= tol or dF <= atol
    ok_t = err_t <= tol or dT <= atol * (rmax if rmax else 1.0)
    record("force_rel_max", err_f, tol)
    record("torque_rel_max", err_t, tol)
    return ok_f and ok_t, {"force_rel": err_f, "torque_rel": err_t, "force_abs": dF, "atol": atol}


def force_term_scales(prob, fields, state):
    """The scale against which a particle's hydrodynamic force error is held,
    from the method's own terms.  The force is F = sum_n g_n with the node
    terms g_n = -phi_n k rho_n (u_s - u*)_n of Eqs. 18-19 (k = 1 - 1/2tau
    for Eq. 18 as printed, 1 for momentum exchange): each term is a
    difference of the particle's velocity u_s and the fluid's u*, both
    carried by the FP32 path to a relative precision e, so the forward error
    of the sum is bounded by e sum_n phi_n k rho_n (|u_s| + |u*|)_n, the
    scale returned (for a fixed particle, u_s = 0, it is sum_n |g_n|).  A
    free particle moves with its fluid (u_s ~ u*), so its force is a small
    residual of these terms, and this, not |F| or sum |g_n|, is what a
    relative precision of the inputs bounds.  The torque's scale is the same
    sum weighted by |r_n|, the offset of the node from the centre.

    ``fields`` are the oracle's (rho, u, v, phi, owner) at the start of the
    step whose force is compared (u the corrected velocity of Eq. 17, from
    which u* = (u - phi u_s / 2) / (1 - phi / 2)); ``state`` the particle
    state (x, y, r, ux, uy, omega, ...) at the start of that step.  Returns
    (S_F, S_T), one entry per particle."""
    rho, ux, uy, phi, own = (np.asarray(a) for a in fields[:5])
    ny, nx = rho.shape
    ps = getattr(prob, "method", 0) == 1
    # PS-LBM's force (Eqs. 10-11) is -B rho (u_s - u*) whatever the force model
    k = (1.0 - 0.5 / prob.tau) if prob.force_model == 0 and not ps else 1.0
    yy, xx = np.nonzero(own >= 0)
    p = own[yy, xx]
    st = np.asarray(state)
    dx = xx - st[p, 0]
    dy = yy - st[p, 1]
    if prob.west.kind == "periodic":
        dx = dx - nx * np.floor(dx / nx + 0.5)
    if prob.south.kind == "periodic":
        dy = dy - ny * np.floor(dy / ny + 0.5)
    usx = st[p, 3] - st[p, 5] * dy
    usy = st[p, 4] + st[p, 5] * dx
    ph = phi[yy, xx]
    h = 0.0 * ph if ps else 0.5 * ph
    uax = (ux[yy, xx] - h * usx) / (1.0 - h)
    uay = (uy[yy, xx] - h * usy) / (1.0 - h)
    w = ph * k * rho[yy, xx] * (np.hypot(usx, usy) + np.hypot(uax, uay))
    n = len(st)
    sf = np.bincount(p, weights=w, minlength=n)
    stq = np.bincount(p, weights=np.hypot(dx, dy) * w, minlength=n)
    return sf, stq


def compare_forces_terms(Fg, Fo, scales, tol=TOL_FP32, atol=0.0, rmax=1.0):
    """Per particle |F_gpu - F_oracle| <= tol * S_F and |T_gpu - T_oracle|
    <= tol * S_T, with (S_F, S_T) from force_term_scales.  ``atol`` (force;
    torque: atol * rmax) is an absolute floor for PS-LBM sums (ps_force_floor)."""
    sf, stq = scales
    dF = np.hypot(Fg[:, 0] - Fo[:, 0], Fg[:, 1] - Fo[:, 1])
    dT = np.abs(Fg[:, 2] - Fo[:, 2])
    okf = (dF <= tol * sf) | (dF <= atol)
    okt = (dT <= tol * stq) | (dT <= atol * rmax)
    ef = float((dF / np.maximum(sf, 1e-300)).max()) if len(sf) else 0.0
    et = float((dT / np.maximum(stq, 1e-300)).max()) if len(sf) else 0.0
    record("force_rel_terms", ef, tol)
    record("torque_rel_terms", et, tol)
    return bool(okf.all() and okt.all()), {"force_rel_terms": ef, "torque_rel_terms": et, "atol": atol}


def oracle_pre(o):
    """The oracle's fields and particle state now, i.e. at the start of the
    step it takes next (the inputs of that step's force)."""
    return o.fields(), o.forces()[2]


def ps_force_floor(phi, state):
    """FP32 floor of a PS-LBM force (Eqs. 10-11).  The force is
    -sum_n B_n rho_n (u_s - u*)_n over the N covered nodes, interior nodes
    included (B = 1, where u* ~ u_s and every term is a small difference),
    so each term carries the FP32 rounding of u* and u_s, about 2^-24 |u_s|
    (rho ~ 1).  The floor is the coherent sum of those roundings,
    N 2^-24 max|u_s| with |u_s| <= |U| + |omega| r; a neutrally buoyant
    disc, whose net force is a small residual of its terms, is held to it."""
    n = int((np.asarray(phi) > 0).sum())
    us = max((abs(q[3]) + abs(q[4]) + abs(q[5]) * q[2]) for q in state) if len(state) else 0.0
    return n * 2.0 ** -24 * us


def compare_state(Sg, So, tol_pos=TOL_FP32_POSITION, tol_vel=TOL_FP32, travel=0.0):
    """Particle state (x, y, r, ux, uy, omega, theta, rho_s).  A position is
    the sum of the particle's velocities over the steps (Eq. 24, dt = 1), so
    its error is held to tol_pos plus tol_vel times the distance travelled
    (``travel``, lattice units)."""
    tol_pos = tol_pos + tol_vel * travel
    dpos = float(np.abs(Sg[:, :2] - So[:, :2]).max()) if len(So) else 0.0
    vscale = max(np.abs(So[:, 3:5]).max(), 1e-30) if len(So) else 1.0
    dvel = float(np.abs(Sg[:, 3:5] - So[:, 3:5]).max() / vscale) if len(So) else 0.0
    record("pos_abs", dpos, tol_pos)
    record("particle_vel_rel", dvel, tol_vel)
    return dpos <= tol_pos and dvel <= tol_vel, {"pos_abs": dpos, "vel_rel": dvel}
