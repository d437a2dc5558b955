"""GPU path (librsol through its C ABI) against the FP64 oracle.

Tolerances: FP64 build <= 1e-12 relative (positions, momenta, deposits);
FP32 build <= 1e-5 relative L2 on the deposited moments after 100 steps;
cell indices and sort order bit-exact given the same packet state.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import paper_2111_14704_gb300 as rs
import rsol_inputs as ri
from tests.gpu_helpers import gpu_run, make_case, oracle_run, periodic_diff, positions, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    rs.load_library()


# ------------------------------------------------------------------ one step, FP64, exact tolerance
@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("grid,n", [((12, 10, 8), 3001), ((5, 7, 9), 777)])
def test_fp64_one_step_matches_oracle(shape, grid, n):
    params, parts, planes, _ = make_case(grid, n, seed=41, shape=shape, precision=64)
    dt = 0.2 / params.c_tilde
    g, gfb = gpu_run(params, parts, planes, dt, 1)
    o, ofb = oracle_run(params, parts, planes, dt, 1)
    np.testing.assert_array_equal(g["cell"], o["cell"])
    np.testing.assert_allclose(g["off"], o["off"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(g["u"], o["u"], rtol=1e-12, atol=1e-12)
    scale = np.abs(ofb[0]).reshape(8, -1).max(1)[:, None, None, None]
    np.testing.assert_allclose(gfb[0] / scale, ofb[0] / scale, rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape", [1, 2])
def test_fp64_100_steps_matches_oracle(shape):
    grid = (16, 16, 16)
    params, parts, planes, _ = make_case(grid, 4096, seed=1, shape=shape, precision=64)
    dt = 0.2 / params.c_tilde
    g, gfb = gpu_run(params, parts, planes, dt, 100)
    o, ofb = oracle_run(params, parts, planes, dt, 100)
    np.testing.assert_array_equal(g["cell"], o["cell"])
    np.testing.assert_allclose(g["off"], o["off"], rtol=0, atol=1e-11)
    np.testing.assert_allclose(g["u"], o["u"], rtol=1e-12, atol=1e-12)
    for q in range(8):
        assert rel_l2(gfb[-1][q], ofb[-1][q]) < 1e-12, q


# ------------------------------------------------------------------ FP32 against the FP64 oracle
@pytest.mark.parametrize("shape", [1, 2])
def test_fp32_100_steps_moments_within_1e5(shape):
    grid = (16, 12, 20)
    params, parts, planes, _ = make_case(grid, 8000, seed=2, shape=shape, precision=32)
    dt = 0.2 / params.c_tilde
    g, gfb = gpu_run(params, parts, planes, dt, 100)
    o, ofb = oracle_run(params, parts, planes, dt, 100)
    for q in range(8):
        assert rel_l2(gfb[-1][q], ofb[-1][q]) <= 1e-5, (q, rel_l2(gfb[-1][q], ofb[-1][q]))
    d = periodic_diff(positions(g), positions(o), grid)
    assert np.abs(d).max() < 1e-3
    np.testing.assert_allclose(g["u"], o["u"], rtol=1e-3, atol=1e-4)


@pytest.mark.parametrize("shape", [1, 2])
def test_fp32_one_step_elementwise(shape):
    grid = (9, 8, 7)
    params, parts, planes, _ = make_case(grid, 2500, seed=3, shape=shape, precision=32)
    dt = 0.2 / params.c_tilde
    g, gfb = gpu_run(params, parts, planes, dt, 1)
    o, ofb = oracle_run(params, parts, planes, dt, 1)
    d = periodic_diff(positions(g), positions(o), grid)
    assert np.abs(d).max() < 1e-6
    np.testing.assert_allclose(g["u"], o["u"], rtol=2e-6, atol=2e-6)
    for q in range(8):
        assert rel_l2(gfb[0][q], ofb[0][q]) <= 2e-6, q


# ------------------------------------------------------------------ deterministic deposits
@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("precision", [32, 64])
def test_deterministic_mode_bitwise_reproducible(shape, precision):
    grid = (16, 16, 16)
    params, parts, planes, _ = make_case(grid, 20000, seed=5, shape=shape, precision=precision)
    params.deterministic = 1
    dt = 0.2 / params.c_tilde
    g1, f1 = gpu_run(params, parts, planes, dt, 3)
    g2, f2 = gpu_run(params, parts, planes, dt, 3)
    for a, b in zip(f1, f2):
        assert np.array_equal(a, b)
    o, ofb = oracle_run(params, parts, planes, dt, 3)
    tol = 1e-5 if precision == 32 else 1e-9
    for q in range(8):
        assert rel_l2(f1[-1][q], ofb[-1][q]) <= tol


# ------------------------------------------------------------------ sort: bit-exact vs stable sort
@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("grid,bin_,n", [((16, 16, 16), 8, 50000), ((13, 7, 11), 4, 12345),
                                         ((32, 32, 32), 1, 4097), ((20, 20, 20), 16, 1)])
def test_sort_bit_exact(grid, bin_, n, shape):
    import torch
    params, parts, planes, _ = make_case(grid, n, seed=7, precision=32, n_modes=0, shape=shape)
    params.bin = bin_
    parts["off"][:, ::7] = 0.5  # TSC anchor ties: f = 1/2 goes to the upper node
    # many ties: restrict cells to a few values on a sub-lattice
    parts["cell"][0] = (parts["cell"][0] // 3) * 3
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, 32)
    Q = rs.Particles.empty(n, 32)
    ctx.sort(P, Q)
    torch.cuda.synchronize()
    got = Q.to_numpy()
    keys = oracle.sort_keys(grid, bin_, shape, parts["cell"], parts["off"])
    perm = oracle.stable_sort(keys, oracle.n_keys(grid, bin_))
    np.testing.assert_array_equal(got["cell"], parts["cell"][:, perm])
    np.testing.assert_array_equal(got["off"], parts["off"][:, perm])
    np.testing.assert_array_equal(got["u"], parts["u"][:, perm])


def test_sort_then_push_equals_push_then_permute():
    grid = (16, 16, 16)
    params, parts, planes, _ = make_case(grid, 30000, seed=8, precision=64)
    dt = 0.2 / params.c_tilde
    g_sorted, f_sorted = gpu_run(params, parts, planes, dt, 4, sort_every=2)
    g_plain, f_plain = gpu_run(params, parts, planes, dt, 4)
    for q in range(8):
        assert rel_l2(f_sorted[-1][q], f_plain[-1][q]) < 1e-13
    # same multiset of packets (sorting only permutes)
    key = lambda d: np.lexsort(np.vstack([d["u"], d["off"], d["cell"]]))
    a, b = key(g_sorted), key(g_plain)
    np.testing.assert_array_equal(g_sorted["cell"][:, a], g_plain["cell"][:, b])
    np.testing.assert_allclose(g_sorted["u"][:, a], g_plain["u"][:, b], rtol=0, atol=0)


# ------------------------------------------------------------------ state moments and FP64 totals
@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("precision", [32, 64])
def test_state_moments_and_totals(shape, precision):
    import torch
    grid = (10, 12, 14)
    params, parts, planes, _ = make_case(grid, 5000, seed=9, shape=shape, precision=precision,
                                         c=2.0, c_tilde=0.5, q_over_m=3.0, q=1.5)
    parts["w"] = 0.5 + ri.uniform(9, 60, np.arange(5000, dtype=np.uint64))
    if precision == 32:
        parts["w"] = parts["w"].astype(np.float32).astype(np.float64)
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, precision)
    M = ctx.grid_tensor()
    ctx.deposit(P, M)
    T = ctx.moments(P)
    T2 = ctx.moments(P)
    torch.cuda.synchronize()
    op = oracle.params(grid, shape=shape, dt=1.0, c=2.0, c_tilde=0.5, q_over_m=3.0, q=1.5)
    OP = oracle.Particles(parts)
    G = oracle.state_moments(op, OP)
    OT = oracle.totals(op, OP)
    tol = 1e-12 if precision == 64 else 2e-6
    for q in range(8):
        assert rel_l2(rs.grid_to_planes(M)[q], G[q]) <= tol, q
    np.testing.assert_allclose(T[:8], OT, rtol=1e-12 if precision == 64 else 1e-7, atol=1e-9)
    assert np.array_equal(T, T2)


def test_totals_include_feedback_sums_and_conservation():
    """rho u + (c/c~) P conserved (Sec. 2): sum S dV + (c/c~) dP/dt = 0 on the GPU."""
    import torch
    grid = (16, 16, 16)
    params, parts, planes, _ = make_case(grid, 20000, seed=10, precision=64)
    dt = 0.2 / params.c_tilde
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, 64)
    F = rs.fields_to_device(planes, 64)
    T0 = ctx.moments(P)
    fb = ctx.grid_tensor()
    ctx.push_gather(P, F, dt, fb)
    T1 = ctx.moments(P, fb)
    torch.cuda.synchronize()
    r = params.c / params.c_tilde
    dP = r * (T1[1:4] - T0[1:4]) / dt
    dE = r * (T1[4] - T0[4]) / dt
    assert np.all(np.abs(T1[12:15] + dP) <= 1e-9 * np.abs(dP).max())
    assert abs(T1[15] + dE) <= 1e-9 * abs(dE)
    assert abs(T1[8] - parts["w"].sum() * params.q) < 1e-9


# ------------------------------------------------------------------ c~ independence on the GPU
def test_static_fields_c_tilde_independent_gpu():
    grid = (12, 12, 12)
    runs = []
    for ct in [1.0, 0.1, 0.01]:
        params, parts, planes, _ = make_case(grid, 3000, seed=11, precision=64, c_tilde=ct)
        g, f = gpu_run(params, parts, planes, 0.2 / ct, 20)
        runs.append((g, f))
    for g, f in runs[1:]:
        np.testing.assert_array_equal(g["cell"], runs[0][0]["cell"])
        np.testing.assert_allclose(g["off"], runs[0][0]["off"], rtol=0, atol=1e-12)
        for q in range(8):
            assert rel_l2(f[-1][q], runs[0][1][-1][q]) < 1e-12


# ------------------------------------------------------------------ field source
@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("grid", [(24, 20, 16), (100, 13, 6)])  # FP32 rows past 32 nodes rotate the x phase
def test_alfven_fields_match_input_module(precision, grid):
    import torch
    modes = ri.alfven_modes(64, 3, L=tuple(float(g) for g in grid), kmax=16, dB_rms=0.1)
    params = rs.Params(*grid, precision=precision, c=1.0, c_tilde=0.1)
    ctx = rs.Context(params)
    F = ctx.grid_tensor()
    for t in [0.0, 123.4]:
        ctx.alfven_fields(modes, t, 1.0, 1e-4, (0.0, 0.01, 0.0), F)
        torch.cuda.synchronize()
        got = rs.grid_to_planes(F)[:6]
        ref = ri.field_grid(grid, t=t, modes=modes, vA=1e-4, u_gas=(0.0, 0.01, 0.0))
        tol = 1e-12 if precision == 64 else 2e-6
        assert np.abs(got - ref).max() < tol
        assert np.all(rs.grid_to_planes(F)[6:] == 0)


# ------------------------------------------------------------------ edge cases
def test_empty_and_single_packet():
    import torch
    grid = (8, 8, 8)
    params, parts, planes, _ = make_case(grid, 1, seed=12, precision=64)
    ctx = rs.Context(params)
    F = rs.fields_to_device(planes, 64)
    E = rs.Particles.empty(0, 64)
    fb = ctx.grid_tensor()
    ctx.push_gather(E, F, 1.0, fb)
    ctx.sort(E, rs.Particles.empty(0, 64))
    assert np.all(ctx.moments(E) == 0)
    torch.cuda.synchronize()
    assert float(fb.abs().sum()) == 0.0
    g, gfb = gpu_run(params, parts, planes, 2.0, 3)
    o, ofb = oracle_run(params, parts, planes, 2.0, 3)
    np.testing.assert_array_equal(g["cell"], o["cell"])
    np.testing.assert_allclose(g["u"], o["u"], rtol=1e-12)


def test_boundary_offsets_and_wrap():
    """Packets at offset 0, at the TSC midpoint 1/2, just below 1, in the last cell."""
    grid = (6, 5, 4)
    n = 64
    params, parts, planes, _ = make_case(grid, n, seed=13, precision=64)
    special = np.array([0.0, 0.5, 1.0 - 2.0**-24, 2.0**-24, 0.25])
    parts["off"][:, :40] = special[np.arange(40) % 5][None, :]
    parts["cell"][0, :20] = grid[0] - 1
    parts["cell"][1, 10:30] = grid[1] - 1
    parts["cell"][2, ::3] = 0
    for shape in (1, 2):
        params.shape = shape
        g, gfb = gpu_run(params, parts, planes, 2.0, 2)
        o, ofb = oracle_run(params, parts, planes, 2.0, 2)
        np.testing.assert_array_equal(g["cell"], o["cell"])
        np.testing.assert_allclose(g["off"], o["off"], rtol=0, atol=1e-12)
        for q in range(8):
            assert rel_l2(gfb[-1][q], ofb[-1][q]) < 1e-12


def test_largest_axis_grid():
    """A 1024-node axis (the packed-cell limit) with a ragged packet count."""
    grid = (1024, 3, 2)
    params, parts, planes, _ = make_case(grid, 1001, seed=14, precision=64, n_modes=4, kmax=1)
    g, gfb = gpu_run(params, parts, planes, 2.0, 2)
    o, ofb = oracle_run(params, parts, planes, 2.0, 2)
    np.testing.assert_array_equal(g["cell"], o["cell"])
    for q in range(8):
        assert rel_l2(gfb[-1][q], ofb[-1][q]) < 1e-12


# ------------------------------------------------------------------ error reporting
def test_errors_reported_not_raised_on_device():
    import torch
    grid = (8, 8, 8)
    params, parts, planes, _ = make_case(grid, 100, seed=15, precision=32)
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, 32)
    F = rs.fields_to_device(planes, 32)
    with pytest.raises(rs.RsolError) as e:
        ctx.push_gather(P, F, 20.0)  # c~ dt / dx = 2 > 1
    assert e.value.status == 5
    with pytest.raises(rs.RsolError) as e:
        ctx.push_gather(P, F, -1.0)
    assert e.value.status == 1
    P.u[0][7] = float("nan")
    ctx.push_gather(P, F, 1.0)
    with pytest.raises(rs.RsolError) as e:
        ctx.check()
    assert e.value.status == 4
    ctx.check()  # the status word was cleared
    torch.cuda.synchronize()


# ------------------------------------------------------------------ catastrophic losses
@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("precision", [32, 64])
def test_losses_match_oracle(shape, precision):
    """Sec. 2 collisional terms on the GPU against the oracle (uniform and gathered n_n)."""
    import torch
    grid = (9, 10, 11)
    params, parts, planes, _ = make_case(grid, 3000, seed=19, shape=shape, precision=precision)
    z, y, x = np.meshgrid(np.arange(11.0), np.arange(10.0), np.arange(9.0), indexing="ij")
    nn = 1.0 + 0.3 * np.sin(2 * np.pi * x / 9) * np.cos(2 * np.pi * z / 11)
    if precision == 32:
        nn = nn.astype(np.float32).astype(np.float64)
    dt = 0.2 / params.c_tilde
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, precision)
    ctx.losses(P, sigma=0.07, dt=dt, nn_uniform=0.5)
    dtype = torch.float32 if precision == 32 else torch.float64
    ctx.losses(P, sigma=0.07, dt=dt, nn=torch.from_numpy(nn).to("cuda", dtype))
    torch.cuda.synchronize()
    ctx.check()
    op = oracle.params(grid, shape=shape, dt=dt, c=params.c, c_tilde=params.c_tilde)
    OP = oracle.Particles(parts)
    oracle.losses(op, OP, 0.07, nn_uniform=0.5)
    oracle.losses(op, OP, 0.07, nn=nn)
    tol = 1e-13 if precision == 64 else 2e-6
    np.testing.assert_allclose(P.to_numpy()["w"], OP.w, rtol=tol)
