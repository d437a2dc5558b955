"""Pins of the oracle's per-packet adaptive timestep with sub-cycling (Sec. 3,
timestep constraints: every CR constraint rescales by c/c~).

Each packet takes 2^k sub-steps of dt/2^k, k the smallest level whose
sub-step meets C min(1/Omega~, dx/|v_eff|, N/|dN/dt|); the deposit is the
time average over the global step.  Pinned by: the reduction to the plain step,
closed-form levels for each limit, the closed-form Boris phase of a
sub-cycled gyration, straight-line drift, and the exact exchange identities.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import rsol_inputs as ri


def _one(u, off=(0.5, 0.5, 0.5), cell=(1, 1, 1), w=1.0):
    return {"cell": np.array(cell, np.int32).reshape(3, 1), "off": np.array(off).reshape(3, 1),
            "u": np.array(u, dtype=np.float64).reshape(3, 1), "w": np.array([w])}


def _uniform(grid, E=(0, 0, 0), B=(0, 0, 0)):
    F = np.zeros((6,) + grid[::-1])
    for q in range(3):
        F[q] = E[q]
        F[3 + q] = B[q]
    return F


def test_level_rule():
    assert oracle.subcycle_level(8.0, 1.0, 10) == 3          # dt / 2^k <= limit, boundary included
    assert oracle.subcycle_level(8.0, 0.999, 10) == 4
    assert oracle.subcycle_level(8.0, 1e-9, 5) == 5          # capped
    assert oracle.subcycle_level(8.0, math.inf, 5) == 0
    assert oracle.subcycle_level(8.0, 8.0, 5) == 0


@pytest.mark.parametrize("shape", [1, 2])
def test_reduces_to_plain_step(shape):
    grid = (8, 8, 8)
    parts = ri.make_particles(300, grid, 21)
    modes = ri.alfven_modes(8, 21, L=(8.0,) * 3, kmax=2, dB_rms=0.3)
    F = ri.field_grid(grid, modes=modes, vA=0.01, u_gas=(0.0, 0.01, 0.0))
    p = oracle.params(grid, shape=shape, dt=2.0, c=1.0, c_tilde=0.1)
    for courant, max_level in ((1e30, 8), (0.01, 0)):
        A, B = oracle.Particles(parts), oracle.Particles(parts)
        G1 = oracle.step(p, F, A)
        G2, lev = oracle.step_subcycled(p, F, B, courant, max_level=max_level)
        assert np.all(lev == 0)
        assert np.array_equal(G1, G2)
        assert np.array_equal(A.u, B.u) and np.array_equal(A.off, B.off) and np.array_equal(A.cell, B.cell)


def test_gyro_level_and_phase_closed_form():
    """A slow packet in uniform B (E = 0): level ceil(log2(dt Omega~ / C)) and,
    over the global step, a rotation by 2^k * 2 atan(Omega~ dt_sub / 2)."""
    grid = (4, 4, 4)
    c, ct, qm, B0 = 1.0, 0.1, 1.0, 1.0
    u_perp = 0.05
    g = math.sqrt(1 + u_perp ** 2)
    omega = (ct / c) * qm * B0 / (g * c)
    C, dt = 0.1, 8.0
    p = oracle.params(grid, shape=2, dt=dt, c=c, c_tilde=ct, q_over_m=qm)
    P = oracle.Particles(_one((0.0, u_perp, 0.0)))
    lim = oracle.dt_limits(p, _uniform(grid, B=(B0, 0, 0)), P, C)[0]
    assert abs(lim - C / omega) <= 1e-14 * lim            # gyration binds (Courant: 200)
    G, lev = oracle.step_subcycled(p, _uniform(grid, B=(B0, 0, 0)), P, C)
    k = math.ceil(math.log2(dt * omega / C))
    assert lev[0] == k == 3
    theta = 2.0 ** k * 2.0 * math.atan(omega * (dt / 2 ** k) / 2.0)
    u1 = P.u[:, 0]
    assert abs(np.linalg.norm(u1) - u_perp) <= 1e-15
    ang = math.atan2(abs(u1[2]), u1[1])
    assert abs(ang - theta) <= 1e-13
    # finer sub-steps approach the exact phase Omega~ dt
    assert abs(theta - omega * dt) < abs(2 * math.atan(omega * dt / 2) - omega * dt) / 50


def test_courant_level_and_straight_line():
    grid = (16, 16, 16)
    ct, C = 0.1, 0.2
    u = 10.0
    beta = u / math.sqrt(1 + u * u)
    dt = 0.95 / ct                                          # c~ dt = 0.95 dx
    p = oracle.params(grid, shape=2, dt=dt, c=1.0, c_tilde=ct)
    P = oracle.Particles(_one((u, 0.0, 0.0), off=(0.25, 0.5, 0.5), cell=(3, 4, 5)))
    _, lev = oracle.step_subcycled(p, _uniform(grid), P, C)
    assert lev[0] == math.ceil(math.log2(ct * beta * dt / C)) == 3
    x = P.cell[0, 0] + P.off[0, 0]
    assert abs(x - (3.25 + ct * beta * dt)) <= 1e-13
    assert P.cell[1, 0] == 4 and P.cell[2, 0] == 5


def test_loss_limit_level():
    grid = (4, 4, 4)
    ct, c, C, sigma_nn = 0.1, 1.0, 0.5, 3.0
    u = 1.0
    beta = u / math.sqrt(2.0)
    dt = 2.0
    p = oracle.params(grid, shape=1, dt=dt, c=c, c_tilde=ct)
    P = oracle.Particles(_one((0.0, 0.0, u)))
    lim = oracle.dt_limits(p, _uniform(grid), P, C, sigma_nn)[0]
    t_loss = C / ((ct / c) * sigma_nn * c * beta)
    assert abs(lim - t_loss) <= 1e-14 * t_loss              # losses bind (Courant: 7.07)
    _, lev = oracle.step_subcycled(p, _uniform(grid), P, C, sigma_nn)
    assert lev[0] == math.ceil(math.log2(dt / t_loss))


@pytest.mark.parametrize("shape", [1, 2])
def test_exchange_identities_subcycled(shape):
    """Sum S dV = -(c/c~) sum N m c (u_end - u_start) / dt and the energy
    analogue hold exactly over a sub-cycled step (the sub-steps telescope)."""
    grid = (8, 8, 8)
    parts = ri.make_particles(400, grid, 22, p_range=(1.0, 100.0))
    modes = ri.alfven_modes(8, 22, L=(8.0,) * 3, kmax=2, dB_rms=0.5)
    F = ri.field_grid(grid, modes=modes, vA=0.02, u_gas=(0.0, 0.02, 0.0))
    c, ct = 1.0, 0.1
    dt = 1.0 / ct                                           # c~ dt = dx: packets must sub-cycle
    p = oracle.params(grid, shape=shape, dt=dt, c=c, c_tilde=ct)
    P = oracle.Particles(parts)
    u0 = P.u.copy()
    G, lev = oracle.step_subcycled(p, F, P, 0.2)
    assert len(np.unique(lev)) >= 2 and lev.max() >= 2
    m = 1.0
    dP = (c / ct) * m * c * (P.u - u0).sum(axis=1) / dt
    S = G[4:7].sum(axis=(1, 2, 3))
    assert np.all(np.abs(S + dP) <= 1e-12 * np.abs(dP).max())
    g0 = np.sqrt(1 + (u0 * u0).sum(axis=0))
    g1 = np.sqrt(1 + (P.u * P.u).sum(axis=0))
    dE = (c / ct) * m * c * c * (g1 - g0).sum() / dt
    assert abs(G[7].sum() + dE) <= 1e-10 * abs(dE)
    assert abs(G[0].sum() - parts["w"].sum()) <= 1e-12 * parts["w"].sum()


def test_substeps_match_separate_runs():
    """Each packet's sub-cycled step equals 2^k plain steps of dt/2^k taken on
    its own with its weight scaled by 2^-k."""
    grid = (8, 8, 8)
    parts = ri.make_particles(40, grid, 23)
    modes = ri.alfven_modes(8, 23, L=(8.0,) * 3, kmax=2, dB_rms=0.5)
    F = ri.field_grid(grid, modes=modes, vA=0.02)
    p = oracle.params(grid, shape=2, dt=8.0, c=1.0, c_tilde=0.1)
    P = oracle.Particles(parts)
    G, lev = oracle.step_subcycled(p, F, P, 0.3)
    Gsum = np.zeros_like(G)
    for j in range(40):
        one = {k: (v[:, j:j + 1] if v.ndim == 2 else v[j:j + 1]).copy() for k, v in parts.items()}
        one["w"] = one["w"] * 2.0 ** -lev[j]
        ps = oracle.params(grid, shape=2, dt=8.0 / 2 ** lev[j], c=1.0, c_tilde=0.1)
        Q = oracle.Particles(one)
        for _ in range(2 ** lev[j]):
            Gsum += oracle.step(ps, F, Q)
        assert np.array_equal(Q.u[:, 0], P.u[:, j]) and np.array_equal(Q.off[:, 0], P.off[:, j])
    assert np.allclose(Gsum, G, rtol=0, atol=1e-13 * np.abs(G).max())
