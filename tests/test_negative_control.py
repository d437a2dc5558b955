"""Negative control of the paper's central claim (Sec. 3, naive substitution).

Naive RSOL substitutes c~ for c everywhere (Lorentz force, Lorentz factor,
packet energy and momentum), i.e. the same step with c := c~.  The paper
lists what then goes wrong: the CR energy density carries c~^2 (item 1) and
the gyro radius changes with c~ (items 3-4), while the RSOL formulation keeps
both at their true values for every c~.  These tests run the FP64 oracle
(no GPU) and, marked gpu, the library through its C ABI.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import rsol_inputs as ri


def _gyro_radius(p, u_perp=2.0, B0=1.0, steps=12):
    """Gyro radius of one packet in uniform B, measured from its discrete orbit:
    the vertices lie on a circle (radius R from three consecutive vertices) and
    turn by theta per step, so r_g = R cos(theta / 2)."""
    g = (2, 2, 2)
    F = np.zeros((6, 2, 2, 2))
    F[3] = B0  # a uniform field needs no more nodes: the weights sum to one
    q = oracle.params(g, shape=1, dt=p.dt, c=p.c, c_tilde=p.c_tilde, q_over_m=p.q_over_m, q=p.q)
    parts = {"cell": np.zeros((3, 1), np.int32), "off": np.full((3, 1), 0.5),
             "u": np.array([[0.0], [u_perp], [0.0]]), "w": np.ones(1)}
    P = oracle.Particles(parts)
    pts = [np.array([0.5, 0.5])]
    for _ in range(steps):
        prev = pts[-1]
        oracle.step(q, F, P, deposit=False)
        cur = np.array([P.cell[1, 0] + P.off[1, 0], P.cell[2, 0] + P.off[2, 0]])
        pts.append(prev + ((cur - prev + 1) % 2 - 1))  # unwrap on the 2-cell box
    a, b, c = pts[3], pts[4], pts[5]
    ab, bc, ca = np.linalg.norm(b - a), np.linalg.norm(c - b), np.linalg.norm(a - c)
    area2 = abs((b - a)[0] * (c - a)[1] - (b - a)[1] * (c - a)[0])
    R = ab * bc * ca / (2 * area2)
    d1, d2 = b - a, c - b
    theta = math.acos(np.dot(d1, d2) / (np.linalg.norm(d1) * np.linalg.norm(d2)))
    return R * math.cos(theta / 2)


@pytest.mark.parametrize("c_tilde", [0.5, 0.1])
def test_gyro_radius_rsol_fixed_naive_scales(c_tilde):
    """RSOL: r_g does not depend on c~.  Naive (c := c~): r_g = u m c~^2/(qB) shrinks."""
    c = 1.0
    dt = 0.02 / c_tilde  # c~ dt fixed and small: many steps per orbit
    rs_ref = _gyro_radius(oracle.params((2, 2, 2), shape=1, dt=0.02, c=c, c_tilde=c))
    rs_rsol = _gyro_radius(oracle.params((2, 2, 2), shape=1, dt=dt, c=c, c_tilde=c_tilde))
    rs_naive = _gyro_radius(oracle.params((2, 2, 2), shape=1, dt=dt, c=c_tilde, c_tilde=c_tilde))
    r_g = 2.0 * 1.0 * c ** 2 / (1.0 * 1.0)  # |u_perp| m c^2 / (q B0)
    assert abs(rs_ref / r_g - 1) < 1e-9
    assert abs(rs_rsol / r_g - 1) < 1e-9
    assert abs(rs_naive / r_g - c_tilde ** 2) < 1e-9


def test_energy_density_rsol_true_naive_scaled():
    """Packet energy density: RSOL keeps N gamma m c^2 for every c~; naive gives
    N gamma m c~^2, off by (c~/c)^2 (Sec. 3 item 1)."""
    grid = (6, 6, 6)
    parts = ri.make_particles(400, grid, seed=3)
    dens = {}
    for name, c, ct in [("true", 1.0, 1.0), ("rsol", 1.0, 0.1), ("naive", 0.1, 0.1)]:
        p = oracle.params(grid, shape=2, dt=0.2 / ct, c=c, c_tilde=ct)
        dens[name] = oracle.state_moments(p, oracle.Particles(parts))[4]
    np.testing.assert_allclose(dens["rsol"], dens["true"], rtol=1e-14)
    np.testing.assert_allclose(dens["naive"], dens["true"] * 0.01, rtol=1e-12)


def test_back_reaction_rsol_c_tilde_free_naive_not():
    """Momentum source on the gas in static fields at fixed c~ dt: RSOL gives the
    same deposit sequence for c/c~ = 1 and 10; the naive scheme does not."""
    grid = (8, 8, 8)
    modes = ri.alfven_modes(8, 5, L=(8.0, 8.0, 8.0), kmax=2, dB_rms=0.3)
    F = ri.field_grid(grid, modes=modes, vA=0.01, u_gas=(0.0, 0.01, 0.0))
    parts = ri.make_particles(300, grid, seed=4)
    out = {}
    for name, c, ct in [("rsol1", 1.0, 1.0), ("rsol10", 1.0, 0.1), ("naive10", 0.1, 0.1)]:
        p = oracle.params(grid, shape=2, dt=0.2 / ct, c=c, c_tilde=ct)
        P = oracle.Particles(parts)
        G = [oracle.step(p, F, P) for _ in range(10)]
        out[name] = np.array(G)[:, 4:7]
    ref = out["rsol1"]
    assert np.abs(out["rsol10"] - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.linalg.norm(out["naive10"] - ref) > 0.1 * np.linalg.norm(ref)


@pytest.mark.gpu
def test_gpu_naive_vs_rsol_energy_source():
    """The same negative control through the C ABI (FP64): the RSOL feedback at
    c/c~ = 10 matches c/c~ = 1; with c := c~ it does not.  Fields are pure B
    (vA = u_gas = 0, so E = 0) and therefore the same in all three runs."""
    from tests.gpu_helpers import gpu_run, make_case, rel_l2
    grid = (12, 12, 12)
    res = {}
    for name, c, ct in [("rsol1", 1.0, 1.0), ("rsol10", 1.0, 0.1), ("naive10", 0.1, 0.1)]:
        params, parts, planes, _ = make_case(grid, 4000, seed=18, precision=64, c=c, c_tilde=ct,
                                             vA=0.0, u_gas=(0.0, 0.0, 0.0))
        g, f = gpu_run(params, parts, planes, 0.2 / ct, 10)
        res[name] = np.array(f)
    for q in range(8):
        assert rel_l2(res["rsol10"][:, q], res["rsol1"][:, q]) < 1e-12
    assert rel_l2(res["naive10"][:, 4:7], res["rsol1"][:, 4:7]) > 0.1
