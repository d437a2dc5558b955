"""The binned shared-memory push (used after rsol_sort) against the FP64 oracle.

The oracle sorts the same packets with its own stable sort (the permutation
must agree bit for bit), then both advance several steps without re-sorting,
so packets drift towards and past the edges of their bin's tile and the
global fallback path runs too.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2111_14704_gb300 as rs
from tests.gpu_helpers import gpu_run, make_case, oracle_run, periodic_diff, positions, rel_l2

pytestmark = pytest.mark.gpu


def sorted_like_oracle(parts, grid, bin_, shape):
    keys = oracle.sort_keys(grid, bin_, shape, parts["cell"], parts["off"])
    perm = oracle.stable_sort(keys, oracle.n_keys(grid, bin_))
    return {k: (v[:, perm] if v.ndim == 2 else v[perm]) for k, v in parts.items()}


@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("bin_", [4, 8])
@pytest.mark.parametrize("grid,n", [((20, 16, 12), 20000), ((6, 5, 4), 3000)])
def test_binned_fp64_matches_oracle(shape, bin_, grid, n):
    params, parts, planes, _ = make_case(grid, n, seed=21, shape=shape, precision=64)
    params.bin = bin_
    dt = 0.2 / params.c_tilde
    steps = 8  # up to 1.6 cells of drift: some packets leave their tile
    g, gfb = gpu_run(params, parts, planes, dt, steps, sort_every=1000)
    o, ofb = oracle_run(params, sorted_like_oracle(parts, grid, bin_, shape), planes, dt, steps)
    np.testing.assert_array_equal(g["cell"], o["cell"])
    np.testing.assert_allclose(g["off"], o["off"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(g["u"], o["u"], rtol=1e-12, atol=1e-12)
    for k in range(steps):
        for q in range(8):
            assert rel_l2(gfb[k][q], ofb[k][q]) < 1e-12, (k, q)


@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("grid,n", [((32, 24, 16), 60000), ((32, 32, 32), 1 << 18)])
def test_binned_fp32_matches_oracle(shape, grid, n):
    """32^3: bins whose tile does not wrap around the grid take their fields
    with one bulk tensor copy (the others with ordinary loads)."""
    params, parts, planes, _ = make_case(grid, n, seed=22, shape=shape, precision=32)
    dt = 0.2 / params.c_tilde
    # sorted once, at step 0, where both sides hold identical packets (a later
    # re-sort could order FP32 and FP64 packets differently at a half-node)
    g, gfb = gpu_run(params, parts, planes, dt, 4, sort_every=1000)
    o_parts, ofb = oracle_run(params, sorted_like_oracle(parts, grid, 8, shape), planes, dt, 4)
    d = periodic_diff(positions(g), positions(o_parts), grid)
    assert np.abs(d).max() < 1e-5
    np.testing.assert_allclose(g["u"], o_parts["u"], rtol=1e-5, atol=1e-5)
    for k in range(4):
        for q in range(8):
            assert rel_l2(gfb[k][q], ofb[k][q]) <= 3e-6, (k, q, rel_l2(gfb[k][q], ofb[k][q]))


@pytest.mark.parametrize("shape", [1, 2])
def test_dense_bins_past_the_kept_key_capacity(shape):
    """Bins of ~12,000 packets (24 per cell): more than the 8192 origin keys the
    push and the state-moment deposit keep in shared memory, so the push's local
    sort recomputes them and the deposit visits its bins in sort order.  Four
    steps of drift without re-sorting, then the state moments, against the oracle.
    The feedback is held to the FP32 bar of 1e-5 relative L2: at three times the
    usual packets per node, the tile's fixed-point quantum (set by the node's
    packet count) is larger against the cancelling momentum source."""
    import torch
    grid = (16, 16, 16)
    params, parts, planes, _ = make_case(grid, 100000, seed=27, shape=shape, precision=32)
    params.bin = 8
    dt = 0.2 / params.c_tilde
    ctx = rs.Context(params)
    A = rs.Particles.from_numpy(parts, 32)
    B = rs.Particles.empty(A.n, 32)
    ctx.sort(A, B)
    F = rs.fields_to_device(planes, 32)
    gfb = []
    for _ in range(4):
        fb = ctx.grid_tensor()
        ctx.push_gather(B, F, dt, fb)
        gfb.append(rs.grid_to_planes(fb))
    M = ctx.grid_tensor()
    ctx.deposit(B, M)
    torch.cuda.synchronize()
    ctx.check()
    g = B.to_numpy()
    o_parts, ofb = oracle_run(params, sorted_like_oracle(parts, grid, 8, shape), planes, dt, 4)
    d = periodic_diff(positions(g), positions(o_parts), grid)
    assert np.abs(d).max() < 1e-5
    for k in range(4):
        for q in range(8):
            assert rel_l2(gfb[k][q], ofb[k][q]) <= 1e-5, (k, q, rel_l2(gfb[k][q], ofb[k][q]))
    op = oracle.params(grid, shape=shape, dt=dt, c=params.c, c_tilde=params.c_tilde,
                       q_over_m=params.q_over_m, q=params.q)
    G = oracle.state_moments(op, oracle.Particles(g))
    for q in range(8):
        assert rel_l2(rs.grid_to_planes(M)[q], G[q]) <= 2e-6, q


@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("precision", [32, 64])
def test_binned_deterministic_bitwise(shape, precision):
    grid = (24, 24, 24)
    params, parts, planes, _ = make_case(grid, 80000, seed=23, shape=shape, precision=precision)
    params.deterministic = 1
    dt = 0.2 / params.c_tilde
    a, fa = gpu_run(params, parts, planes, dt, 6, sort_every=3)
    b, fb = gpu_run(params, parts, planes, dt, 6, sort_every=3)
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)
    np.testing.assert_array_equal(a["cell"], b["cell"])
    assert np.array_equal(a["u"], b["u"])


def test_binned_equals_unbinned_fp64():
    """Same packets, same order: binned and order-free kernels agree to round-off."""
    import torch
    grid = (16, 16, 16)
    params, parts, planes, _ = make_case(grid, 40000, seed=24, precision=64)
    params.bin = 4  # the FP64 tile fits shared memory for 4^3 bins
    parts = sorted_like_oracle(parts, grid, 4, 2)
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, 64)
    Q = rs.Particles.empty(P.n, 64)
    ctx.sort(P, Q)                     # Q: binned path
    R = rs.Particles.from_numpy(parts, 64)  # R: same order, order-free path
    F = rs.fields_to_device(planes, 64)
    f1, f2 = ctx.grid_tensor(), ctx.grid_tensor()
    ctx.push_gather(Q, F, 2.0, f1)
    ctx.push_gather(R, F, 2.0, f2)
    torch.cuda.synchronize()
    a, b = Q.to_numpy(), R.to_numpy()
    np.testing.assert_array_equal(a["cell"], b["cell"])
    np.testing.assert_allclose(a["u"], b["u"], rtol=1e-15, atol=0)
    g1, g2 = rs.grid_to_planes(f1), rs.grid_to_planes(f2)
    for q in range(8):
        assert rel_l2(g1[q], g2[q]) < 1e-14


@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("precision", [32, 64])
def test_sparse_bins_match_oracle(shape, precision):
    """Bins holding few packets skip the shared tiles (global gathers and atomics):
    same results against the oracle, deterministic mode bitwise repeatable."""
    grid = (32, 32, 24)
    params, parts, planes, _ = make_case(grid, 2500, seed=26, shape=shape, precision=precision)
    dt = 0.2 / params.c_tilde
    bin_ = 8 if precision == 32 else 4
    g, gfb = gpu_run(params, parts, planes, dt, 3, sort_every=1000)
    o, ofb = oracle_run(params, sorted_like_oracle(parts, grid, bin_, shape), planes, dt, 3)
    tol = 1e-12 if precision == 64 else 3e-6
    for k in range(3):
        for q in range(8):
            assert rel_l2(gfb[k][q], ofb[k][q]) < tol, (k, q)
    params.deterministic = 1
    a, fa = gpu_run(params, parts, planes, dt, 2, sort_every=1000)
    b, fb = gpu_run(params, parts, planes, dt, 2, sort_every=1000)
    assert all(np.array_equal(x, y) for x, y in zip(fa, fb))


@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("precision,bin_", [(64, 4), (64, 8), (32, 8), (32, 4)])
def test_binned_state_moments_match_oracle(shape, precision, bin_):
    """rsol_deposit on the last sort's output (per-bin tiles) against the
    oracle's state moments, after pushes that move packets off their bins'
    cores and out of some tiles (global fallback)."""
    import torch
    grid = (20, 16, 12)
    params, parts, planes, _ = make_case(grid, 30000, 51, shape=shape, precision=precision,
                                         c=2.0, c_tilde=0.5, q_over_m=3.0, q=1.5)
    params.bin = bin_
    dt = 0.6 / params.c_tilde
    ctx = rs.Context(params)
    A = rs.Particles.from_numpy(parts, precision)
    B = rs.Particles.empty(A.n, precision)
    ctx.sort(A, B)
    F = rs.fields_to_device(planes, precision)
    for _ in range(4):                                  # 2.4 cells of drift at most
        ctx.push_gather(B, F, dt, ctx.grid_tensor())
    M = ctx.grid_tensor()
    ctx.deposit(B, M)                                   # binned: B is the sort's output
    M_free = ctx.grid_tensor()
    C_ = rs.Particles(B.cell.clone(), [t.clone() for t in B.off], [t.clone() for t in B.u], B.w.clone())
    ctx.deposit(C_, M_free)                             # order-free kernel on a copy
    torch.cuda.synchronize()
    ctx.check()
    op = oracle.params(grid, shape=shape, dt=dt, c=2.0, c_tilde=0.5, q_over_m=3.0, q=1.5)
    G = oracle.state_moments(op, oracle.Particles(B.to_numpy()))
    tol = 1e-12 if precision == 64 else 2e-6
    for q in range(8):
        assert rel_l2(rs.grid_to_planes(M)[q], G[q]) <= tol, q
        assert rel_l2(rs.grid_to_planes(M)[q], rs.grid_to_planes(M_free)[q]) <= tol, q


@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("precision,bin_", [(64, 4), (32, 8), (32, 4)])
def test_binned_losses_match_oracle(shape, precision, bin_):
    """rsol_losses with a gathered n_n on the last sort's output (per-bin n_n
    tiles), after pushes that move packets out of some tiles."""
    import torch
    grid = (20, 16, 12)
    params, parts, planes, _ = make_case(grid, 30000, 52, shape=shape, precision=precision)
    params.bin = bin_
    dt = 0.6 / params.c_tilde
    z, y, x = np.meshgrid(np.arange(12.0), np.arange(16.0), np.arange(20.0), indexing="ij")
    nn = 1.0 + 0.3 * np.sin(2 * np.pi * x / 20) * np.cos(2 * np.pi * z / 12)
    if precision == 32:
        nn = nn.astype(np.float32).astype(np.float64)
    ctx = rs.Context(params)
    A = rs.Particles.from_numpy(parts, precision)
    B = rs.Particles.empty(A.n, precision)
    ctx.sort(A, B)
    F = rs.fields_to_device(planes, precision)
    for _ in range(4):
        ctx.push_gather(B, F, dt, ctx.grid_tensor())
    before = B.to_numpy()
    dtype = torch.float32 if precision == 32 else torch.float64
    ctx.losses(B, sigma=0.07, dt=dt, nn=torch.from_numpy(nn).to("cuda", dtype))  # binned
    torch.cuda.synchronize()
    ctx.check()
    op = oracle.params(grid, shape=shape, dt=dt, c=params.c, c_tilde=params.c_tilde)
    OP = oracle.Particles(before)
    oracle.losses(op, OP, 0.07, nn=nn)
    tol = 1e-13 if precision == 64 else 2e-6
    np.testing.assert_allclose(B.to_numpy()["w"], OP.w, rtol=tol)
