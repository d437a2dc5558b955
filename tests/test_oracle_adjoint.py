"""Pins of the oracle's forward-mode tangent (the independent check of the
library's reverse-mode gradients of L = ||sum_n S^n||_2, S the deposited
momentum source of Sec. 2).

The tangent is pinned against central finite differences of the oracle's own
forward step (itself pinned by test_oracle), in FP64, along random directions
of a static field grid and of a time-dependent Alfven field sequence.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import rsol_inputs as ri

GRID = (8, 8, 8)


def _case(shape=2, n=256, seed=4, c_tilde=0.1):
    parts = ri.make_particles(n, GRID, seed)
    modes = ri.alfven_modes(16, seed, L=(8.0,) * 3, kmax=3, dB_rms=0.3)
    p = oracle.params(GRID, shape=shape, dt=0.2 / c_tilde, c=1.0, c_tilde=c_tilde)
    return p, parts, modes


def _fd(p, parts, F, dF, steps, h):
    Lp = oracle.momentum_source_loss(p, F + h * dF, oracle.Particles(parts), steps)
    Lm = oracle.momentum_source_loss(p, F - h * dF, oracle.Particles(parts), steps)
    return (Lp - Lm) / (2 * h)


def test_tangent_fd_static(steps=12, n_dirs=4):
    p, parts, modes = _case()
    F = ri.field_grid(GRID, modes=modes, vA=0.01, u_gas=(0.0, 0.01, 0.0))
    rng = np.random.default_rng(1)
    for _ in range(n_dirs):
        dF = rng.standard_normal(F.shape)
        dF /= np.linalg.norm(dF)
        L, dL = oracle.tangent(p, F, dF, oracle.Particles(parts), steps=steps)
        assert abs(L - oracle.momentum_source_loss(p, F, oracle.Particles(parts), steps)) <= 1e-13 * L
        fd = _fd(p, parts, F, dF, steps, 1e-6)
        assert abs(dL - fd) <= 1e-6 * max(abs(fd), 1e-3 * L), (dL, fd)


def test_tangent_fd_cic_static():
    p, parts, modes = _case(shape=1, seed=6)
    F = ri.field_grid(GRID, modes=modes, vA=0.01, u_gas=(0.0, 0.01, 0.0))
    dF = np.random.default_rng(2).standard_normal(F.shape)
    L, dL = oracle.tangent(p, F, dF, oracle.Particles(parts), steps=6)
    fd = _fd(p, parts, F, dF, 6, 1e-7)
    # CIC weights have kinks at the nodes: a packet crossing one inside +-h is
    # improbable at h = 1e-7 and would show as an O(1) mismatch
    assert abs(dL - fd) <= 1e-5 * max(abs(fd), 1e-3 * L), (dL, fd)


def _amp_sequence(modes, amp, steps, dt, vA, u_gas):
    m = dict(modes)
    m["amp"] = amp
    return np.stack([ri.field_grid(GRID, t=n * dt, modes=m, vA=vA, u_gas=u_gas)
                     for n in range(steps)])


def test_tangent_fd_amplitudes_time_dependent(steps=10):
    """Per-step fields F^n(A) from the Alfven source: dF^n/dA by central
    differences of the generator (exact: F is at most quadratic in A)."""
    p, parts, modes = _case(seed=8, c_tilde=0.5)
    vA, u_gas = 0.05, (0.0, 0.01, 0.0)
    A = modes["amp"].copy()
    dA = np.random.default_rng(3).standard_normal(A.shape)
    dA /= np.linalg.norm(dA)
    F = _amp_sequence(modes, A, steps, p.dt, vA, u_gas)
    e = 1e-3
    dF = (_amp_sequence(modes, A + e * dA, steps, p.dt, vA, u_gas)
          - _amp_sequence(modes, A - e * dA, steps, p.dt, vA, u_gas)) / (2 * e)
    L, dL = oracle.tangent(p, F, dF, oracle.Particles(parts))
    h = 1e-6
    Lp = oracle.momentum_source_loss(p, _amp_sequence(modes, A + h * dA, steps, p.dt, vA, u_gas),
                                     oracle.Particles(parts))
    Lm = oracle.momentum_source_loss(p, _amp_sequence(modes, A - h * dA, steps, p.dt, vA, u_gas),
                                     oracle.Particles(parts))
    fd = (Lp - Lm) / (2 * h)
    assert abs(dL - fd) <= 1e-6 * abs(fd), (dL, fd)


def test_tangent_zero_direction_and_scaling():
    p, parts, modes = _case(n=64)
    F = ri.field_grid(GRID, modes=modes, vA=0.01)
    L0, d0 = oracle.tangent(p, F, np.zeros_like(F), oracle.Particles(parts), steps=4)
    assert d0 == 0.0
    # L is positively homogeneous of degree one in the packet weights
    parts2 = dict(parts)
    parts2["w"] = 3.0 * parts["w"]
    dF = np.random.default_rng(4).standard_normal(F.shape)
    L1, d1 = oracle.tangent(p, F, dF, oracle.Particles(parts), steps=4)
    L3, d3 = oracle.tangent(p, F, dF, oracle.Particles(parts2), steps=4)
    assert abs(L3 - 3 * L1) <= 1e-13 * L3 and abs(d3 - 3 * d1) <= 1e-12 * abs(d3)
