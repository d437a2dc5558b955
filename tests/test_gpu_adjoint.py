"""Reverse-mode gradients of L = ||sum_n S^n||_2 (S the deposited momentum
source of Sec. 2) through the C ABI, against the oracle's forward-mode
tangent (an independent method) and against central differences of the
library's own FP64 forward run.

Small case: 8^3 grid, 256 packets, 16 random unit directions.  Full size:
64^3 grid, 2^20 packets, 64 steps with checkpoints every 8 steps, TSC.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2111_14704_gb300 as rs
import rsol_inputs as ri
from tests.gpu_helpers import anchor_nodes, bin_major_key, make_case, origin_order_breaks

pytestmark = pytest.mark.gpu


def _oparams(params, dt):
    return oracle.params(params.grid, shape=params.shape, dt=dt, c=params.c, c_tilde=params.c_tilde,
                         q_over_m=params.q_over_m, q=params.q, dx=params.dx)


def _sync(ctx):
    import torch
    torch.cuda.synchronize()
    ctx.check()


@pytest.mark.parametrize("precision,shape,tol", [(64, 2, 1e-9), (64, 1, 1e-9), (32, 2, 1e-4)])
def test_field_gradient_matches_oracle_tangent(precision, shape, tol):
    grid, n, steps, every = (8, 8, 8), 256, 12, 5   # segments 5, 5, 2
    params, parts, planes, _ = make_case(grid, n, 41, shape=shape, precision=precision,
                                         c_tilde=0.1, n_modes=16, kmax=3)
    dt = 0.2 / params.c_tilde
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, precision)
    F = rs.fields_to_device(planes, precision)
    o = ctx.gradient(P, steps, dt, checkpoint_every=every, fields=F)
    _sync(ctx)
    op = _oparams(params, dt)
    L = o["loss"][0].item()
    Lo = oracle.momentum_source_loss(op, planes, oracle.Particles(parts), steps)
    assert abs(L - Lo) <= (1e-12 if precision == 64 else 1e-5) * Lo
    assert abs(o["loss"][1].item() * L - 1.0) < 1e-15
    gb = rs.grid_to_planes(o["field_bar"])
    assert np.all(gb[6:] == 0)
    gb = gb[:6]
    scale = np.linalg.norm(gb) / np.sqrt(gb.size)
    rng = np.random.default_rng(7)
    for _ in range(16):
        dF = rng.standard_normal(planes.shape)
        dF /= np.linalg.norm(dF)
        _, dLo = oracle.tangent(op, planes, dF, oracle.Particles(parts), steps=steps)
        dLg = float((gb * dF).sum())
        assert abs(dLg - dLo) <= tol * max(abs(dLo), scale), (dLg, dLo)


def _amp_sequence(grid, modes, amp, steps, dt, vA, u_gas):
    m = dict(modes)
    m["amp"] = amp
    return np.stack([ri.field_grid(grid, t=k * dt, modes=m, vA=vA, u_gas=u_gas) for k in range(steps)])


@pytest.mark.parametrize("precision,tol", [(64, 1e-9), (32, 1e-4)])
def test_amplitude_gradient_matches_oracle_tangent(precision, tol):
    grid, n, steps, every = (8, 8, 8), 256, 10, 4   # segments 4, 4, 2
    parts = ri.make_particles(n, grid, 42, fp32=(precision == 32))
    modes = ri.alfven_modes(16, 42, L=(8.0,) * 3, kmax=3, dB_rms=0.3)
    vA, u_gas, c_tilde = 0.05, (0.0, 0.01, 0.0), 0.5
    dt = 0.2 / c_tilde
    params = rs.Params(*grid, shape=2, precision=precision, c=1.0, c_tilde=c_tilde)
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, precision)
    o = ctx.gradient(P, steps, dt, checkpoint_every=every, modes=modes, vA=vA, u_gas=u_gas)
    _sync(ctx)
    ab = o["amp_bar"].cpu().numpy()
    op = _oparams(params, dt)
    A = modes["amp"].copy()
    Fs = _amp_sequence(grid, modes, A, steps, dt, vA, u_gas)
    Lo = oracle.momentum_source_loss(op, Fs, oracle.Particles(parts))
    assert abs(o["loss"][0].item() - Lo) <= (1e-12 if precision == 64 else 1e-5) * Lo
    rng = np.random.default_rng(8)
    e = 1e-3
    for _ in range(16):
        dA = rng.standard_normal(A.shape)
        dA /= np.linalg.norm(dA)
        # F is at most quadratic in A: the central difference is exact
        dFs = (_amp_sequence(grid, modes, A + e * dA, steps, dt, vA, u_gas)
               - _amp_sequence(grid, modes, A - e * dA, steps, dt, vA, u_gas)) / (2 * e)
        _, dLo = oracle.tangent(op, Fs, dFs, oracle.Particles(parts))
        dLg = float(ab @ dA)
        assert abs(dLg - dLo) <= tol * max(abs(dLo), np.linalg.norm(ab) / np.sqrt(ab.size)), (dLg, dLo)


@pytest.mark.parametrize("precision", [32, 64])
def test_recompute_without_deposit_is_bitwise(precision):
    """The reverse sweep rebuilds states with the deposit-free step: it must
    reproduce the binned forward step's packet states bit for bit."""
    import torch
    grid = (32, 32, 32)
    params, parts, planes, _ = make_case(grid, 60000, 43, precision=precision, c_tilde=0.1,
                                         n_modes=16, kmax=4)
    dt = 0.2 / params.c_tilde
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, precision)
    A = rs.Particles.empty(P.n, precision)
    ctx.sort(P, A)
    B = rs.Particles(A.cell.clone(), [t.clone() for t in A.off], [t.clone() for t in A.u],
                     A.w.clone())
    F = rs.fields_to_device(planes, precision)
    fb = ctx.grid_tensor()
    for _ in range(8):
        ctx.push_gather(A, F, dt, fb)      # binned, with deposit
        ctx.push_gather(B, F, dt, None)    # order-free, no deposit
    _sync(ctx)
    for a, b in zip(A.tensors(), B.tensors()):
        assert torch.equal(a, b)


@pytest.mark.parametrize("precision,shape,tol", [(64, 2, 1e-12), (64, 1, 1e-12), (32, 2, 2e-5)])
def test_tiled_adjoint_equals_order_free(precision, shape, tol):
    """rsol_adjoint_step on the last sort's output (per-bin tiles; bins well above
    the sparse-bin limit) against the order-free kernel on a copy of the same
    packets, after pushes that move packets off their bins' cores."""
    import torch
    grid = (16, 16, 16)
    params, parts, planes, _ = make_case(grid, 1 << 17, 45, shape=shape, precision=precision,
                                         c_tilde=0.1, n_modes=16, kmax=4)
    dt = 0.2 / params.c_tilde
    ctx = rs.Context(params)
    A = rs.Particles.from_numpy(parts, precision)
    W = rs.Particles.empty(A.n, precision)
    ctx.sort(A, W)
    F = rs.fields_to_device(planes, precision)
    fb = ctx.grid_tensor()
    for _ in range(3):
        ctx.push_gather(W, F, dt, fb)
    loss = ctx.loss_norm(fb)
    C_ = rs.Particles(W.cell.clone(), [t.clone() for t in W.off], [t.clone() for t in W.u], W.w.clone())
    dtype = torch.float32 if precision == 32 else torch.float64
    g = torch.Generator(device="cuda").manual_seed(3)
    xb0 = torch.randn((3, A.n), generator=g, device="cuda", dtype=dtype)
    ub0 = torch.randn((3, A.n), generator=g, device="cuda", dtype=dtype)
    out = []
    for P in (W, C_):                    # W: tiled (sorted identity); C_: order-free
        xb, ub, fbar = xb0.clone(), ub0.clone(), ctx.grid_tensor()
        ctx.adjoint_step(P, F, dt, fb, loss, xb, ub, fbar)
        out.append((xb, ub, fbar))
    _sync(ctx)
    for a, b in zip(out[0], out[1]):
        a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)


def test_tiled_adjoint_local_sort_fp32():
    """FP32 tiled adjoint on bins below the 8192 packets whose visiting order it
    keeps in shared memory (32^3 grid, 2^17 packets: 64 bins of ~2048), after
    enough drift that more than 1 in 32 neighbours break the stencil-origin
    order in every bin, so every CTA sorts its bin locally before the run walk.
    That condition is checked on the host from the packets' anchors; the result
    must equal the order-free kernel's on a copy of the same packets."""
    import torch
    grid = (32, 32, 32)
    params, parts, planes, _ = make_case(grid, 1 << 17, 47, precision=32, c_tilde=0.1,
                                         n_modes=16, kmax=4)
    dt = 0.2 / params.c_tilde
    ctx = rs.Context(params)
    A = rs.Particles.from_numpy(parts, 32)
    W = rs.Particles.empty(A.n, 32)
    ctx.sort(A, W)
    F = rs.fields_to_device(planes, 32)
    fb = ctx.grid_tensor()
    for _ in range(3):
        ctx.push_gather(W, F, dt, fb)
    loss = ctx.loss_norm(fb)
    torch.cuda.synchronize()
    at0 = anchor_nodes(parts["cell"], parts["off"], grid)
    order = np.argsort(bin_major_key(at0, grid, 8), kind="stable")
    now = W.to_numpy()
    frac, counts, _ = origin_order_breaks(at0[:, order], anchor_nodes(now["cell"], now["off"], grid),
                                          grid, 8)
    assert 1024 < counts.min() and counts.max() <= 8192
    assert frac.min() > 1.0 / 32, frac.min()
    C_ = rs.Particles(W.cell.clone(), [t.clone() for t in W.off], [t.clone() for t in W.u], W.w.clone())
    g = torch.Generator(device="cuda").manual_seed(5)
    xb0 = torch.randn((3, A.n), generator=g, device="cuda", dtype=torch.float32)
    ub0 = torch.randn((3, A.n), generator=g, device="cuda", dtype=torch.float32)
    out = []
    for P in (W, C_):                    # W: tiled, sorted locally; C_: order-free
        xb, ub, fbar = xb0.clone(), ub0.clone(), ctx.grid_tensor()
        ctx.adjoint_step(P, F, dt, fb, loss, xb, ub, fbar)
        out.append((xb, ub, fbar))
    _sync(ctx)
    for a, b in zip(out[0], out[1]):
        a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
        assert np.linalg.norm(a - b) <= 2e-5 * np.linalg.norm(b)


def test_gradient_in_a_cuda_graph():
    """rsol_gradient captured once in a CUDA graph (after an eager call that sizes
    its scratch) and replayed: the same loss and gradients as the eager call."""
    import torch
    grid = (16, 16, 16)
    parts = ri.make_particles(1 << 16, grid, 46, fp32=True)
    modes = ri.alfven_modes(16, 46, L=(16.0,) * 3, kmax=4, dB_rms=0.2)
    params = rs.Params(*grid, shape=2, precision=32, c=1.0, c_tilde=0.1)
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, 32)
    kw = dict(checkpoint_every=4, modes=modes, vA=0.01, u_gas=(0.0, 0.01, 0.0))
    o = ctx.gradient(P, 12, 2.0, **kw)
    torch.cuda.synchronize()
    ref = {k: v.clone() for k, v in o.items()}
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        ctx.gradient(P, 12, 2.0, out=o, **kw)
    for k in o:
        o[k].zero_()
    g.replay()
    torch.cuda.synchronize()
    ctx.check()
    assert abs(o["loss"][0].item() - ref["loss"][0].item()) <= 1e-6 * ref["loss"][0].item()
    for k in ("field_bar", "amp_bar", "feedback"):
        a, b = o[k].double().cpu().numpy(), ref[k].double().cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b), k


def test_autograd_front_end():
    import torch
    from paper_2111_14704_gb300.autograd import (momentum_source_loss_amplitudes,
                                                 momentum_source_loss_fields)
    grid = (8, 8, 8)
    params, parts, planes, modes = make_case(grid, 256, 44, precision=64, c_tilde=0.5, n_modes=8)
    dt = 0.4
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, 64)
    F = rs.fields_to_device(planes, 64).requires_grad_(True)
    L = momentum_source_loss_fields(ctx, P, F, 6, dt, checkpoint_every=4)
    (2.0 * L).backward()
    ref = ctx.gradient(P, 6, dt, checkpoint_every=4, fields=F.detach())
    torch.cuda.synchronize()
    assert torch.allclose(F.grad[..., :6], 2.0 * ref["field_bar"][..., :6], rtol=1e-12, atol=0)
    amps = torch.tensor(modes["amp"], dtype=torch.float64, device="cuda", requires_grad=True)
    L2 = momentum_source_loss_amplitudes(ctx, P, amps, modes, 6, dt, vA=0.05)
    L2.backward()
    ref = ctx.gradient(P, 6, dt, modes=modes, vA=0.05)
    torch.cuda.synchronize()
    assert torch.allclose(amps.grad, ref["amp_bar"], rtol=1e-12, atol=0)
    ctx.check()


def test_gradient_argument_errors():
    params = rs.Params(8, 8, 8, shape=2, precision=32, c=1.0, c_tilde=0.5)
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(ri.make_particles(64, (8, 8, 8), 1, fp32=True), 32)
    F = ctx.grid_tensor()
    with pytest.raises(rs.RsolError):
        ctx.gradient(P, 0, 0.4, fields=F)          # steps >= 1
    with pytest.raises(rs.RsolError):
        ctx.gradient(P, 4, 0.4, checkpoint_every=0, fields=F)
    with pytest.raises(rs.RsolError):
        ctx.gradient(P, 4, 4.0, fields=F)          # c~ dt / dx > 1
    with pytest.raises(ValueError):
        ctx.gradient(P, 4, 0.4)                    # neither fields nor modes


# ---------------------------------------------------------------------------
# full size: 64^3, 2^20 packets, 64 steps, checkpoints every 8

GRID4, N4, STEPS4, EVERY4 = (64, 64, 64), 1 << 20, 64, 8
VA4, UG4 = 1e-4, (0.0, 0.0, 0.0)


@pytest.fixture(scope="module")
def config4():
    parts = ri.make_particles(N4, GRID4, 4, fp32=True)
    modes = ri.alfven_modes(64, 4, L=(64.0,) * 3, kmax=16, dB_rms=0.1)
    return parts, modes


def _forward_loss(ctx, P0, steps, dt, F=None, modes=None, A=None):
    """L of a forward-only run through the C ABI (sort once, then steps)."""
    W = rs.Particles.empty(P0.n, ctx.params.precision)
    ctx.sort(P0, W)
    fb = ctx.grid_tensor()
    Fd = F if F is not None else ctx.grid_tensor()
    m = None
    if modes is not None:
        m = dict(modes)
        m["amp"] = A
    for k in range(steps):
        if m is not None:
            ctx.alfven_fields(m, k * dt, 1.0, VA4, UG4, Fd)
        ctx.push_gather(W, Fd, dt, fb)
    return ctx.loss_norm(fb)[0].item()


def test_config4_field_gradient_fp64_central_differences(config4):
    import torch
    parts, modes = config4
    params = rs.Params(*GRID4, shape=2, precision=64, c=1.0, c_tilde=0.1)
    dt = 0.2 / params.c_tilde
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, 64)
    F = ctx.grid_tensor()
    ctx.alfven_fields(modes, 0.0, 1.0, VA4, UG4, F)
    o = ctx.gradient(P, STEPS4, dt, checkpoint_every=EVERY4, fields=F)
    _sync(ctx)
    gb = o["field_bar"][..., :6].clone()
    L = o["loss"][0].item()
    assert abs(_forward_loss(ctx, P, STEPS4, dt, F=F) - L) <= 1e-12 * L
    g = torch.Generator(device="cuda").manual_seed(9)
    h = 1e-6
    for _ in range(16):
        d = torch.randn(gb.shape, dtype=torch.float64, device="cuda", generator=g)
        d /= d.norm()
        dpad = torch.nn.functional.pad(d, (0, 2))
        Lp = _forward_loss(ctx, P, STEPS4, dt, F=F + h * dpad)
        Lm = _forward_loss(ctx, P, STEPS4, dt, F=F - h * dpad)
        fd = (Lp - Lm) / (2 * h)
        ad = float((gb * d).sum())
        assert abs(ad - fd) <= 1e-4 * abs(fd), (ad, fd)


def test_config4_amplitude_gradient_fp64_central_differences(config4):
    parts, modes = config4
    params = rs.Params(*GRID4, shape=2, precision=64, c=1.0, c_tilde=0.1)
    dt = 0.2 / params.c_tilde
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, 64)
    o = ctx.gradient(P, STEPS4, dt, checkpoint_every=EVERY4, modes=modes, vA=VA4, u_gas=UG4)
    _sync(ctx)
    ab = o["amp_bar"].cpu().numpy()
    A = modes["amp"].copy()
    rng = np.random.default_rng(10)
    h = 1e-6
    for _ in range(16):
        dA = rng.standard_normal(A.shape)
        dA /= np.linalg.norm(dA)
        fd = (_forward_loss(ctx, P, STEPS4, dt, modes=modes, A=A + h * dA)
              - _forward_loss(ctx, P, STEPS4, dt, modes=modes, A=A - h * dA)) / (2 * h)
        ad = float(ab @ dA)
        assert abs(ad - fd) <= 1e-4 * abs(fd), (ad, fd)


def test_config4_fp32_gradient_against_fp64(config4):
    """The FP32 run (the configuration the gradient benchmark times) against
    the FP64 run on the same FP32-rounded inputs."""
    import torch
    parts, modes = config4
    out = {}
    for prec in (32, 64):
        params = rs.Params(*GRID4, shape=2, precision=prec, c=1.0, c_tilde=0.1)
        dt = 0.2 / params.c_tilde
        ctx = rs.Context(params)
        P = rs.Particles.from_numpy(parts, prec)
        o = ctx.gradient(P, STEPS4, dt, checkpoint_every=EVERY4, modes=modes, vA=VA4, u_gas=UG4)
        _sync(ctx)
        out[prec] = (o["loss"][0].item(), o["field_bar"][..., :6].double().cpu().numpy(),
                     o["amp_bar"].cpu().numpy())
        del ctx, P, o
        torch.cuda.empty_cache()
    L32, g32, a32 = out[32]
    L64, g64, a64 = out[64]
    assert abs(L32 - L64) <= 1e-5 * L64
    rng = np.random.default_rng(11)
    for _ in range(16):
        d = rng.standard_normal(g64.shape)
        d /= np.linalg.norm(d)
        r64, r32 = float((g64 * d).sum()), float((g32 * d).sum())
        assert abs(r32 - r64) <= 1e-4 * max(abs(r64), np.linalg.norm(g64) / np.sqrt(g64.size))
        dA = rng.standard_normal(a64.shape)
        dA /= np.linalg.norm(dA)
        assert abs(a32 @ dA - a64 @ dA) <= 1e-4 * max(abs(a64 @ dA), np.linalg.norm(a64) / 8)
