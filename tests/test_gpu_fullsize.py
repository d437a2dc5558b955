"""Parity at the full workload sizes, in the configuration bench.py times.

128^3 grid, 2^24 packets, TSC, FP32, c/c~ = 10, after rsol_sort (binned kernel):
per-packet results for a random sample are recomputed by the oracle one by
one; the feedback at sampled nodes is recomputed by the oracle from every
packet whose stencil covers the node; the totals obey the paper's exchange
identities.  256^3, 2^27 packets with a streaming beam (deterministic
deposits, sort every 4 steps) must reproduce bit for bit across runs.
"""
from __future__ import annotations

import hashlib

import numpy as np
import pytest

import oracle
import paper_2111_14704_gb300 as rs
import rsol_inputs as ri

pytestmark = pytest.mark.gpu

GRID2 = (128, 128, 128)
N2 = 1 << 24


@pytest.fixture(scope="module")
def workload2():
    parts = ri.make_particles(N2, GRID2, 2)
    modes = ri.alfven_modes(64, 2, L=(128.0,) * 3, kmax=16, dB_rms=0.1)
    planes = ri.field_grid(GRID2, modes=modes, vA=1e-4).astype(np.float32).astype(np.float64)
    return parts, planes


def test_fullsize_sampled_packets_and_nodes(workload2):
    import torch
    parts, planes = workload2
    params = rs.Params(*GRID2, shape=2, precision=32, c=1.0, c_tilde=0.1)
    dt = 0.2 / params.c_tilde
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, 32)
    Q = rs.Particles.empty(N2, 32)
    ctx.sort(P, Q)
    torch.cuda.synchronize()
    before = Q.to_numpy()
    del P
    F = rs.fields_to_device(planes, 32)
    fb = ctx.grid_tensor()
    T0 = ctx.moments(Q)
    ctx.push_gather(Q, F, dt, fb)
    T1 = ctx.moments(Q, fb)
    ctx.check()
    after = Q.to_numpy()
    G = rs.grid_to_planes(fb)
    op = oracle.params(GRID2, shape=2, dt=dt, c=1.0, c_tilde=0.1)

    # per-packet: a random sample, each recomputed by the oracle on its own
    rng = np.random.default_rng(0)
    idx = rng.choice(N2, 3000, replace=False)
    sub = {k: (v[:, idx] if v.ndim == 2 else v[idx]) for k, v in before.items()}
    OP = oracle.Particles(sub)
    oracle.step(op, planes, OP, deposit=False)
    n = np.array(GRID2)[:, None]
    d = (after["cell"][:, idx] + after["off"][:, idx]) - (OP.cell + OP.off)
    assert np.abs((d + n / 2) % n - n / 2).max() < 1e-5
    np.testing.assert_allclose(after["u"][:, idx], OP.u, rtol=2e-6, atol=2e-6)

    # sampled nodes: the oracle deposits every packet whose TSC stencil covers the node
    X = before["cell"] + before["off"]
    near = np.floor(X + 0.5).astype(np.int64) % n  # TSC anchor: nearest node
    for node in rng.integers(0, 128, size=(12, 3)):
        dist = (near - node[:, None] + n // 2) % n - n // 2
        sel = np.nonzero(np.all(np.abs(dist) <= 1, axis=0))[0]
        S = {k: (v[:, sel] if v.ndim == 2 else v[sel]) for k, v in before.items()}
        OG = oracle.step(op, planes, oracle.Particles(S))
        ref = OG[:, node[2], node[1], node[0]]
        got = G[:, node[2], node[1], node[0]]
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 2e-5 * scale, (node, got, ref)

    # totals: charge, current, and the (c/c~) momentum exchange.  (The energy
    # exchange is ~1e-9 of the total energy per step here: FP32 rounding of gamma
    # over 2^24 packets is larger, so it is checked in FP64 below.)
    assert abs(T1[8] - N2) < 1e-6 * N2
    np.testing.assert_allclose(T1[9:12], T1[5:8], rtol=1e-5, atol=1e-3 * np.abs(T1[5:8]).max())
    r = params.c / params.c_tilde
    dP = r * (T1[1:4] - T0[1:4]) / dt
    assert np.all(np.abs(T1[12:15] + dP) <= 1e-4 * np.abs(dP).max())


def test_fullsize_fp64_exchange_identities(workload2):
    """Same workload in the FP64 build: sum S dV = -(c/c~) dP/dt and
    sum H dV = -(c/c~) dE/dt (Sec. 2) to FP64 round-off, charge = sum N q."""
    import torch
    parts, planes = workload2
    params = rs.Params(*GRID2, shape=2, precision=64, c=1.0, c_tilde=0.1)
    dt = 0.2 / params.c_tilde
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, 64)
    Q = rs.Particles.empty(N2, 64)
    ctx.sort(P, Q)
    del P
    F = rs.fields_to_device(planes, 64)
    fb = ctx.grid_tensor()
    T0 = ctx.moments(Q)
    ctx.push_gather(Q, F, dt, fb)
    T1 = ctx.moments(Q, fb)
    ctx.check()
    torch.cuda.synchronize()
    r = params.c / params.c_tilde
    dP = r * (T1[1:4] - T0[1:4]) / dt
    dE = r * (T1[4] - T0[4]) / dt
    assert abs(T1[8] - N2) < 1e-9 * N2
    assert np.all(np.abs(T1[12:15] + dP) <= 1e-7 * np.abs(dP).max())
    assert abs(T1[15] + dE) <= 1e-6 * abs(dE)


def _digest(arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(a.detach().cpu().numpy().tobytes())
    return h.hexdigest()


def test_config3_beam_bitwise_reproducible():
    """256^3, 2^27 packets with a 0.3 c~ beam along B0, p in [1, 1000], c/c~ = 30,
    TSC, FP32, deterministic deposits, sort every 4 steps: two runs agree bit for bit."""
    import torch
    grid = (256, 256, 256)
    n = 1 << 27
    parts = ri.make_particles(n, grid, 3, p_range=(1.0, 1000.0), beam_beta=0.3)
    modes = ri.alfven_modes(64, 3, L=(256.0,) * 3, kmax=16, dB_rms=0.1)
    params = rs.Params(*grid, shape=2, precision=32, deterministic=1, c=1.0, c_tilde=1.0 / 30)
    dt = 0.2 / params.c_tilde
    digests = []
    for _run in range(2):
        ctx = rs.Context(params)
        P = rs.Particles.from_numpy(parts, 32)
        Q = rs.Particles.empty(n, 32)
        F = ctx.grid_tensor()
        fb = ctx.grid_tensor()
        for k in range(8):
            if k % 4 == 0:
                ctx.sort(P, Q)
                P, Q = Q, P
            ctx.alfven_fields(modes, k * dt, 1.0, 1e-4, (0.0, 0.0, 0.0), F)
            fb.zero_()
            ctx.push_gather(P, F, dt, fb)
        torch.cuda.synchronize()
        ctx.check()
        tot = ctx.moments(P, fb)
        digests.append((_digest([fb]), _digest(P.tensors()), tot.tobytes()))
        del P, Q, F, fb, ctx
        torch.cuda.empty_cache()
    assert digests[0] == digests[1]
    assert np.isfinite(np.frombuffer(digests[0][2])).all()
