"""Per-packet adaptive timestep with sub-cycling (Sec. 3, timestep
constraints) through the C ABI, against the FP64 oracle.

Levels are integers decided by floating point.  Packets whose limit ratio
dt / dt_j lies within a small band of a power of two (where the two sides could
round to different levels) are left out of the parity inputs; that band is
chosen from the oracle's own limits.  Everything else must agree exactly
(levels) or within the precision's tolerance (states, time-averaged densities).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import paper_2111_14704_gb300 as rs
import rsol_inputs as ri
from tests.gpu_helpers import periodic_diff, positions, rel_l2

pytestmark = pytest.mark.gpu


def _case(grid, n, seed, precision, shape=2, c_tilde=0.1, adv=1.0, courant=0.2, sigma_nn=0.0,
          max_level=8, band=None):
    parts = ri.make_particles(n, grid, seed, p_range=(0.2, 100.0), fp32=(precision == 32))
    modes = ri.alfven_modes(8, seed, L=tuple(float(g) for g in grid), kmax=2, dB_rms=0.5)
    planes = ri.field_grid(grid, modes=modes, vA=0.02, u_gas=(0.0, 0.01, 0.0))
    if precision == 32:
        planes = planes.astype(np.float32).astype(np.float64)
    dt = adv / c_tilde
    op = oracle.params(grid, shape=shape, dt=dt, c=1.0, c_tilde=c_tilde)
    lim = oracle.dt_limits(op, planes, oracle.Particles(parts), courant, sigma_nn)
    r = np.log2(dt / lim)
    band = band if band is not None else (1e-9 if precision == 64 else 1e-3)
    keep = np.abs(r - np.round(r)) > band
    parts = {k: (v[:, keep] if v.ndim == 2 else v[keep]) for k, v in parts.items()}
    params = rs.Params(*grid, shape=shape, precision=precision, c=1.0, c_tilde=c_tilde)
    return params, parts, planes, op


def _gpu(params, parts, planes, dt, courant, steps=1, sigma_nn=0.0, max_level=8, ctx=None):
    import torch
    ctx = ctx or rs.Context(params)
    P = rs.Particles.from_numpy(parts, params.precision)
    F = rs.fields_to_device(planes, params.precision)
    fbs, levs = [], []
    for _ in range(steps):
        fb = ctx.grid_tensor()
        lev = torch.zeros(P.n, dtype=torch.uint8, device="cuda")
        ctx.push_subcycled(P, F, dt, courant, fb, lev, sigma_nn=sigma_nn, max_level=max_level)
        fbs.append(rs.grid_to_planes(fb))
        levs.append(lev.cpu().numpy().astype(np.int32))
    torch.cuda.synchronize()
    ctx.check()
    return P.to_numpy(), fbs, levs


def _oracle(op, parts, planes, courant, steps=1, sigma_nn=0.0, max_level=8):
    P = oracle.Particles(parts)
    fbs, levs = [], []
    for _ in range(steps):
        G, lev = oracle.step_subcycled(op, planes, P, courant, sigma_nn, max_level)
        fbs.append(G)
        levs.append(lev)
    return P.as_dict(), fbs, levs


@pytest.mark.parametrize("shape", [1, 2])
def test_fp64_matches_oracle(shape):
    grid = (12, 12, 12)
    params, parts, planes, op = _case(grid, 3000, 31, 64, shape=shape)
    g, gf, gl = _gpu(params, parts, planes, op.dt, 0.2, steps=3)
    o, of, ol = _oracle(op, parts, planes, 0.2, steps=3)
    for a, b in zip(gl, ol):
        assert np.array_equal(a, b)
    assert len(np.unique(ol[0])) >= 2
    d = periodic_diff(positions(g), positions(o), grid)
    assert np.abs(d).max() <= 1e-12 * 12
    np.testing.assert_allclose(g["u"], o["u"], rtol=1e-12, atol=1e-12)
    for a, b in zip(gf, of):
        assert rel_l2(a, b) <= 1e-12


def test_fp32_matches_oracle():
    grid = (12, 12, 12)
    params, parts, planes, op = _case(grid, 3000, 32, 32)
    g, gf, gl = _gpu(params, parts, planes, op.dt, 0.2)
    o, of, ol = _oracle(op, parts, planes, 0.2)
    assert np.array_equal(gl[0], ol[0])
    d = periodic_diff(positions(g), positions(o), grid)
    assert np.abs(d).max() <= 2e-5
    np.testing.assert_allclose(g["u"], o["u"], rtol=2e-5, atol=2e-5)
    assert rel_l2(gf[0], of[0]) <= 1e-5


def test_loss_limit_levels():
    grid = (8, 8, 8)
    params, parts, planes, op = _case(grid, 1500, 33, 64, sigma_nn=2.0, adv=0.5)
    g, gf, gl = _gpu(params, parts, planes, op.dt, 0.5, sigma_nn=2.0)
    o, of, ol = _oracle(op, parts, planes, 0.5, sigma_nn=2.0)
    assert np.array_equal(gl[0], ol[0])
    assert rel_l2(gf[0], of[0]) <= 1e-12


def test_max_level_zero_is_the_plain_step():
    """max_level = 0: the same arithmetic as rsol_push_gather's order-free kernel."""
    import torch
    grid = (12, 12, 12)
    params, parts, planes, op = _case(grid, 4000, 34, 64, adv=0.2, band=0.0)
    ctx = rs.Context(params)
    A = rs.Particles.from_numpy(parts, 64)
    B = rs.Particles.from_numpy(parts, 64)
    F = rs.fields_to_device(planes, 64)
    fa, fb = ctx.grid_tensor(), ctx.grid_tensor()
    ctx.push_gather(A, F, op.dt, fa)            # unsorted set: order-free kernel
    lev = torch.ones(A.n, dtype=torch.uint8, device="cuda")
    ctx.push_subcycled(B, F, op.dt, 0.2, fb, lev, max_level=0)
    torch.cuda.synchronize()
    ctx.check()
    assert int(lev.max()) == 0
    for a, b in zip(A.tensors(), B.tensors()):
        assert torch.equal(a, b)
    assert torch.allclose(fa, fb, rtol=1e-13, atol=1e-13 * float(fa.abs().max()))


def test_deterministic_bitwise_and_exchange_identity():
    """Deterministic deposits: two runs agree bit for bit; the time-averaged
    momentum source equals -(c/c~) dP/dt of the whole step."""
    import torch
    grid = (16, 16, 16)
    parts = ri.make_particles(20000, grid, 35, p_range=(0.2, 100.0), fp32=True)
    modes = ri.alfven_modes(8, 35, L=(16.0,) * 3, kmax=3, dB_rms=0.5)
    planes = ri.field_grid(grid, modes=modes, vA=0.02).astype(np.float32).astype(np.float64)
    params = rs.Params(*grid, shape=2, precision=32, deterministic=1, c=1.0, c_tilde=0.1)
    dt = 10.0
    outs = []
    for _ in range(2):
        ctx = rs.Context(params)
        P = rs.Particles.from_numpy(parts, 32)
        F = rs.fields_to_device(planes, 32)
        fb = ctx.grid_tensor()
        T0 = ctx.moments(P)
        ctx.push_subcycled(P, F, dt, 0.2, fb)
        T1 = ctx.moments(P, fb)
        ctx.check()
        outs.append((fb.cpu().numpy().tobytes(), b"".join(t.cpu().numpy().tobytes() for t in P.tensors()), T0, T1))
    assert outs[0][0] == outs[1][0] and outs[0][1] == outs[1][1]
    T0, T1 = outs[0][2], outs[0][3]
    dP = 10.0 * (T1[1:4] - T0[1:4]) / dt
    assert np.all(np.abs(T1[12:15] + dP) <= 2e-4 * np.abs(dP).max())
    assert abs(T1[8] - 20000) <= 1e-4 * 20000


def test_argument_errors():
    params = rs.Params(8, 8, 8, shape=2, precision=32, c=1.0, c_tilde=0.1)
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(ri.make_particles(64, (8, 8, 8), 1, fp32=True), 32)
    F = ctx.grid_tensor()
    for kw in (dict(courant=0.0), dict(courant=1.5), dict(courant=0.2, max_level=17),
               dict(courant=0.2, sigma_nn=-1.0)):
        with pytest.raises(rs.RsolError):
            ctx.push_subcycled(P, F, 10.0, **kw)
    with pytest.raises(rs.RsolError) as e:
        ctx.push_subcycled(P, F, 40.0, 0.2, max_level=1)   # c~ dt / dx / 2 = 2 > 1
    assert e.value.status == 5
    ctx.push_subcycled(P, F, 40.0, 0.2, max_level=2)       # 4 / 4 = 1: allowed
    ctx.check()


def test_fullsize_sampled_packets():
    """128^3, 2^24 packets, c~ dt = dx (five times the bench's step), C = 0.2:
    sampled packets recomputed one by one by the oracle."""
    import torch
    grid = (128, 128, 128)
    n = 1 << 24
    parts = ri.make_particles(n, grid, 2, fp32=True)
    modes = ri.alfven_modes(64, 2, L=(128.0,) * 3, kmax=16, dB_rms=0.1)
    planes = ri.field_grid(grid, modes=modes, vA=1e-4).astype(np.float32).astype(np.float64)
    params = rs.Params(*grid, shape=2, precision=32, c=1.0, c_tilde=0.1)
    dt = 10.0
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, 32)
    F = rs.fields_to_device(planes, 32)
    fb = ctx.grid_tensor()
    lev = torch.zeros(n, dtype=torch.uint8, device="cuda")
    T0 = ctx.moments(P)
    ctx.push_subcycled(P, F, dt, 0.2, fb, lev)
    T1 = ctx.moments(P, fb)
    ctx.check()
    after = P.to_numpy()
    levs = lev.cpu().numpy()
    assert len(np.unique(levs)) >= 2
    op = oracle.params(grid, shape=2, dt=dt, c=1.0, c_tilde=0.1)
    rng = np.random.default_rng(3)
    idx = rng.choice(n, 4000, replace=False)
    sub = {k: (v[:, idx] if v.ndim == 2 else v[idx]) for k, v in parts.items()}
    lim = oracle.dt_limits(op, planes, oracle.Particles(sub), 0.2)
    r = np.log2(dt / lim)
    ok = np.abs(r - np.round(r)) > 1e-3
    O = oracle.Particles(sub)
    _, ol = oracle.step_subcycled(op, planes, O, 0.2, deposit=False)
    assert np.array_equal(levs[idx][ok], ol[ok])
    d = periodic_diff(after["cell"][:, idx] + after["off"][:, idx], O.cell + O.off, grid)
    assert np.abs(d[:, ok]).max() < 2e-5
    np.testing.assert_allclose(after["u"][:, idx][:, ok], O.u[:, ok], rtol=2e-5, atol=2e-5)
    dP = 10.0 * (T1[1:4] - T0[1:4]) / dt
    assert np.all(np.abs(T1[12:15] + dP) <= 1e-4 * np.abs(dP).max())


def _tagged(parts, precision):
    """Unique weights 1 + j 2^-20 (exact in FP32) identify each packet after a sort."""
    p = dict(parts)
    p["w"] = 1.0 + np.arange(parts["w"].shape[0]) * 2.0 ** -20
    return p


@pytest.mark.parametrize("precision,shape", [(64, 2), (64, 1), (32, 2)])
def test_sorted_tiled_matches_oracle(precision, shape):
    """rsol_sort_push_subcycled: the same step on the tiled kernel, packets
    identified by their weights after the level sort."""
    import torch
    grid = (16, 16, 16)
    # 40000 packets: each level's bins hold more than the sparse-bin limit, so the
    # shared-memory tiles run
    params, parts, planes, op = _case(grid, 40000, 36, precision, shape=shape)
    parts = _tagged(parts, precision)
    ctx = rs.Context(params)
    A = rs.Particles.from_numpy(parts, precision)
    B = rs.Particles.empty(A.n, precision)
    F = rs.fields_to_device(planes, precision)
    fb = ctx.grid_tensor()
    counts = ctx.sort_push_subcycled(A, B, F, op.dt, 0.2, fb)
    torch.cuda.synchronize()
    ctx.check()
    g = B.to_numpy()
    o, of, ol = _oracle(op, parts, planes, 0.2)
    assert np.array_equal(counts[:9], np.bincount(ol[0], minlength=9)[:9])
    perm = np.rint((g["w"] - 1.0) * 2 ** 20).astype(np.int64)
    assert np.array_equal(np.sort(perm), np.arange(A.n))
    tol = 1e-12 if precision == 64 else 2e-5
    d = periodic_diff(positions(g), positions(o)[:, perm], grid)
    assert np.abs(d).max() <= tol * 16
    np.testing.assert_allclose(g["u"], o["u"][:, perm], rtol=tol, atol=tol)
    assert rel_l2(rs.grid_to_planes(fb), of[0]) <= (1e-12 if precision == 64 else 1e-5)


def test_sorted_tiled_deterministic_bitwise():
    import torch
    grid = (32, 32, 32)
    parts = ri.make_particles(60000, grid, 37, p_range=(0.2, 100.0), fp32=True)
    modes = ri.alfven_modes(8, 37, L=(32.0,) * 3, kmax=3, dB_rms=0.5)
    planes = ri.field_grid(grid, modes=modes, vA=0.02).astype(np.float32).astype(np.float64)
    params = rs.Params(*grid, shape=2, precision=32, deterministic=1, c=1.0, c_tilde=0.1)
    outs = []
    for _ in range(2):
        ctx = rs.Context(params)
        A = rs.Particles.from_numpy(parts, 32)
        B = rs.Particles.empty(A.n, 32)
        F = rs.fields_to_device(planes, 32)
        fb = ctx.grid_tensor()
        ctx.sort_push_subcycled(A, B, F, 10.0, 0.2, fb)
        torch.cuda.synchronize()
        ctx.check()
        outs.append((fb.cpu().numpy().tobytes(), b"".join(t.cpu().numpy().tobytes() for t in B.tensors())))
    assert outs[0] == outs[1]


def test_sorted_tiled_argument_errors():
    params = rs.Params(8, 8, 8, shape=2, precision=32, c=1.0, c_tilde=0.1)
    ctx = rs.Context(params)
    A = rs.Particles.from_numpy(ri.make_particles(64, (8, 8, 8), 1, fp32=True), 32)
    B = rs.Particles.empty(64, 32)
    F = ctx.grid_tensor()
    fb = ctx.grid_tensor()
    with pytest.raises(rs.RsolError):
        ctx.sort_push_subcycled(A, A, F, 10.0, 0.2, fb)          # in and out share arrays
    with pytest.raises(rs.RsolError) as e:
        ctx.sort_push_subcycled(A, B, F, 20.0, 0.2, fb)          # c~ dt / dx = 2 > 1
    assert e.value.status == 5
    counts = ctx.sort_push_subcycled(A, B, F, 10.0, 0.2, fb)
    assert counts.sum() == 64
    ctx.check()
