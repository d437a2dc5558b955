"""Batched boxes (rsol_batch_*) against the single-box path and the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2111_14704_gb300 as rs
import rsol_inputs as ri
from tests.gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

# packets per 8^3 bin up to which a bin skips the shared-memory tiles
# (sparse_bin_limit in csrc/push_binned.cuh)
SPARSE_LIMIT_8 = 768


def _batch(n_boxes, seed, precision, shape=2, det=0, bin_=0, vA=0.01, n_lo=5, n_hi=20, p_lo=100,
           p_hi=3000):
    sh = ri.batch_boxes(n_boxes, seed, n_lo=n_lo, n_hi=n_hi, p_lo=p_lo, p_hi=p_hi)
    boxes, planes = [], []
    for b in range(n_boxes):
        e = int(sh["edge"][b])
        grid = (e, e + 1, e + 2)  # ragged, non-cubic
        parts = ri.make_particles(int(sh["count"][b]), grid, seed * 1000 + b, fp32=(precision == 32))
        modes = ri.alfven_modes(8, seed * 1000 + b, L=tuple(float(g) for g in grid), kmax=2,
                                dB_rms=float(sh["dB_rms"][b]))
        F = ri.field_grid(grid, modes=modes, vA=vA, u_gas=(0.0, 0.01, 0.0))
        if precision == 32:
            F = F.astype(np.float32).astype(np.float64)
        c_tilde = 1.0 / float(sh["c_over_c_tilde"][b])
        boxes.append((grid, parts, c_tilde, 0.2 / c_tilde))
        planes.append(F)
    common = rs.Params(2, 2, 2, shape=shape, precision=precision, deterministic=det, bin=bin_,
                       c=1.0, c_tilde=1.0)
    return common, boxes, planes


def _concat(boxes):
    keys = ("cell", "off", "u")
    out = {k: np.concatenate([b[1][k] for b in boxes], axis=1) for k in keys}
    out["w"] = np.concatenate([b[1]["w"] for b in boxes])
    offsets = np.concatenate([[0], np.cumsum([b[1]["w"].shape[0] for b in boxes])])
    return out, offsets


def _make_ctx(common, boxes, warps=0):
    _, offsets = _concat(boxes)
    return rs.BatchContext(common, [b[0] for b in boxes], [b[2] for b in boxes],
                           [b[3] for b in boxes], offsets, warps=warps)


def _fields_device(bctx, planes, precision):
    import torch
    F = bctx.grid_tensor()
    for b, pl in enumerate(planes):
        bctx.box_view(F, b).copy_(rs.fields_to_device(pl, precision))
    return F


def _slice(P: rs.Particles, lo: int, hi: int, precision: int) -> rs.Particles:
    Q = rs.Particles.empty(hi - lo, precision)
    for src, dst in zip(P.tensors(), Q.tensors()):
        dst.copy_(src[lo:hi])
    return Q


@pytest.mark.parametrize("precision,bin_,dense", [(32, 8, False), (32, 4, False), (64, 4, False),
                                                   (32, 8, True), (64, 4, True)])
def test_batch_sort_matches_per_box_sort(precision, bin_, dense):
    """Sparse batches take the radix sort, dense ones (at most two box-major keys per
    packet) the counting sort: both give every box the oracle's stable order."""
    import torch
    kw = dict(p_lo=2 ** 12, p_hi=2 ** 15) if dense else {}
    common, boxes, _ = _batch(9, 3, precision, bin_=bin_, **kw)
    b_ = bctx_bin(common, precision)
    nkeys = sum(oracle.n_keys(g, b_) for g, *_ in boxes)
    assert (nkeys <= 2 * sum(p["w"].shape[0] for _, p, *_ in boxes)) == dense
    bctx = _make_ctx(common, boxes)
    allp, offsets = _concat(boxes)
    P = rs.Particles.from_numpy(allp, precision)
    Q = rs.Particles.empty(P.n, precision)
    bctx.sort(P, Q)
    torch.cuda.synchronize()
    for b, (grid, parts, ct, dt) in enumerate(boxes):
        keys = oracle.sort_keys(grid, bctx_bin(common, precision), 2, parts["cell"], parts["off"])
        perm = oracle.stable_sort(keys, oracle.n_keys(grid, bctx_bin(common, precision)))
        got = _slice(Q, int(offsets[b]), int(offsets[b + 1]), precision).to_numpy()
        np.testing.assert_array_equal(got["cell"], parts["cell"][:, perm])
        np.testing.assert_array_equal(got["u"], parts["u"][:, perm])


def bctx_bin(common, precision):
    return common.bin if common.bin else (8 if precision == 32 else 4)


@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("warps", [8, 16])
def test_batch_push_deterministic_equals_per_box(shape, warps):
    """Deterministic deposits: the batched launch and one rsol_push_gather per box
    (same sort, same binned CTA body) give identical bits."""
    _det_batch_equals_per_box(_batch(7, 5, 32, shape=shape, det=1), shape, warps)


@pytest.mark.parametrize("shape", [1, 2])
def test_batch_dense_deterministic_equals_per_box(shape):
    """Boxes with both sparse bins (the warp-per-bin kernel) and dense ones (claimed
    from the list by the tiled kernel): bits equal to one rsol_push_gather per box."""
    b = _batch(6, 13, 32, shape=shape, det=1, n_lo=8, n_hi=20, p_lo=2 ** 11, p_hi=2 ** 15)
    common, boxes, _ = b
    counts = []
    for grid, parts, *_ in boxes:
        keys = oracle.sort_keys(grid, 8, shape, parts["cell"], parts["off"])
        counts.append(np.bincount(keys // 512, minlength=oracle.n_keys(grid, 8) // 512))
    counts = np.concatenate(counts)
    assert (counts > SPARSE_LIMIT_8).sum() >= 4 and ((counts > 0) & (counts <= SPARSE_LIMIT_8)).sum() >= 4
    _det_batch_equals_per_box(b, shape, 16)


def _det_batch_equals_per_box(batch, shape, warps):
    import torch
    common, boxes, planes = batch
    bctx = _make_ctx(common, boxes, warps=warps)
    allp, offsets = _concat(boxes)
    P = rs.Particles.from_numpy(allp, 32)
    Q = rs.Particles.empty(P.n, 32)
    bctx.sort(P, Q)
    F = _fields_device(bctx, planes, 32)
    fb = bctx.grid_tensor()
    bctx.push_gather(Q, F, fb)
    torch.cuda.synchronize()
    bctx.check()
    for b, (grid, parts, ct, dt) in enumerate(boxes):
        p = rs.Params(*grid, shape=shape, precision=32, deterministic=1, c=1.0, c_tilde=ct)
        ctx = rs.Context(p)
        A = rs.Particles.from_numpy(parts, 32)
        S = rs.Particles.empty(A.n, 32)
        ctx.sort(A, S)
        fb1 = ctx.grid_tensor()
        ctx.push_gather(S, rs.fields_to_device(planes[b], 32), dt, fb1)
        torch.cuda.synchronize()
        assert torch.equal(bctx.box_view(fb, b), fb1)
        got = _slice(Q, int(offsets[b]), int(offsets[b + 1]), 32)
        for x, y in zip(got.tensors(), S.tensors()):
            assert torch.equal(x, y)


@pytest.mark.parametrize("dense", [False, True])
def test_batch_fp64_matches_oracle(dense):
    """FP64 batch (4^3 bins) against the oracle at 1e-12: small boxes whose bins all
    take the sparse kernel, and boxes where most bins are dense (over 256 packets)
    and take the tiled kernel."""
    import torch
    if dense:
        common, boxes, planes = _batch(4, 17, 64, n_lo=8, n_hi=12, p_lo=2 ** 12, p_hi=2 ** 14)
    else:
        common, boxes, planes = _batch(6, 7, 64)
    counts = []
    for grid, parts, *_ in boxes:
        keys = oracle.sort_keys(grid, 4, 2, parts["cell"], parts["off"])
        counts.append(np.bincount(keys // 64, minlength=oracle.n_keys(grid, 4) // 64))
    assert ((np.concatenate(counts) > 256).sum() >= 40) == dense
    bctx = _make_ctx(common, boxes)
    allp, offsets = _concat(boxes)
    P = rs.Particles.from_numpy(allp, 64)
    Q = rs.Particles.empty(P.n, 64)
    bctx.sort(P, Q)
    F = _fields_device(bctx, planes, 64)
    fbs = []
    for _ in range(3):
        fb = bctx.grid_tensor()
        bctx.push_gather(Q, F, fb)
        fbs.append(fb)
    torch.cuda.synchronize()
    bctx.check()
    for b, (grid, parts, ct, dt) in enumerate(boxes):
        keys = oracle.sort_keys(grid, 4, 2, parts["cell"], parts["off"])
        perm = oracle.stable_sort(keys, oracle.n_keys(grid, 4))
        sp = {k: (v[:, perm] if v.ndim == 2 else v[perm]) for k, v in parts.items()}
        op = oracle.params(grid, shape=2, dt=dt, c=1.0, c_tilde=ct)
        OP = oracle.Particles(sp)
        for k in range(3):
            G = oracle.step(op, planes[b], OP)
            got = rs.grid_to_planes(bctx.box_view(fbs[k], b))
            for q in range(8):
                assert rel_l2(got[q], G[q]) < 1e-12, (b, k, q)
        out = _slice(Q, int(offsets[b]), int(offsets[b + 1]), 64).to_numpy()
        np.testing.assert_array_equal(out["cell"], OP.cell)
        np.testing.assert_allclose(out["u"], OP.u, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("warps", [8, 16])
def test_batch_fp32_matches_oracle(warps):
    """The FP32 batch as benched (32-bit fixed-point tiles, non-deterministic
    deposits): boxes dense enough that most bins take the tiles (2^12..2^15
    packets on 8..16 node edges) and a few sparse ones, 3 steps, every box's eight
    deposited grids against the FP64 oracle at 1e-5 relative L2 and the momenta
    at 1e-4."""
    import torch
    common, boxes, planes = _batch(6, 11, 32, n_lo=8, n_hi=16, p_lo=2 ** 12, p_hi=2 ** 15)
    bctx = _make_ctx(common, boxes, warps=warps)
    allp, offsets = _concat(boxes)
    P = rs.Particles.from_numpy(allp, 32)
    Q = rs.Particles.empty(P.n, 32)
    bctx.sort(P, Q)
    F = _fields_device(bctx, planes, 32)
    fbs = []
    for _ in range(3):
        fb = bctx.grid_tensor()
        bctx.push_gather(Q, F, fb)
        fbs.append(fb)
    torch.cuda.synchronize()
    bctx.check()
    tiled = 0
    for b, (grid, parts, ct, dt) in enumerate(boxes):
        keys = oracle.sort_keys(grid, 8, 2, parts["cell"], parts["off"])
        perm = oracle.stable_sort(keys, oracle.n_keys(grid, 8))
        bins = np.bincount(keys // 512, minlength=oracle.n_keys(grid, 8) // 512)
        tiled += int((bins > SPARSE_LIMIT_8).sum())
        sp = {k: (v[:, perm] if v.ndim == 2 else v[perm]) for k, v in parts.items()}
        op = oracle.params(grid, shape=2, dt=dt, c=1.0, c_tilde=ct)
        OP = oracle.Particles(sp)
        for k in range(3):
            G = oracle.step(op, planes[b], OP)
            got = rs.grid_to_planes(bctx.box_view(fbs[k], b))
            for q in range(8):
                assert rel_l2(got[q], G[q]) <= 1e-5, (b, k, q)
        out = _slice(Q, int(offsets[b]), int(offsets[b + 1]), 32).to_numpy()
        np.testing.assert_allclose(out["u"], OP.u, rtol=1e-4, atol=1e-6)
    assert tiled >= 6  # the tiled path ran


def test_batch_steps_in_a_cuda_graph():
    """Steps captured once in a CUDA graph and replayed give the bits of the same
    steps run eagerly (deterministic deposits)."""
    import torch
    common, boxes, planes = _batch(8, 9, 32, det=1)
    allp, _ = _concat(boxes)
    results = []
    for use_graph in (False, True):
        bctx = _make_ctx(common, boxes)
        P = rs.Particles.from_numpy(allp, 32)
        Q = rs.Particles.empty(P.n, 32)
        bctx.sort(P, Q)
        P, Q = Q, P
        F = _fields_device(bctx, planes, 32)
        fb = bctx.grid_tensor()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())

        def run_steps():
            for _ in range(4):
                fb.zero_()
                bctx.push_gather(P, F, fb)

        with torch.cuda.stream(s):
            run_steps()  # warm-up (kernel attributes, lazy loading) outside capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        if use_graph:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                run_steps()
            g.replay()
        else:
            run_steps()
        torch.cuda.synchronize()
        bctx.check()
        results.append((fb.clone(), [t.clone() for t in P.tensors()]))
    assert torch.equal(results[0][0], results[1][0])
    for x, y in zip(results[0][1], results[1][1]):
        assert torch.equal(x, y)


def test_batch_sorts_and_steps_in_a_cuda_graph():
    """A dense batch (the counting sort, its scratch from rsol_batch_init): sorts and
    steps captured in a CUDA graph and replayed give the bits of the same calls run
    eagerly (deterministic deposits)."""
    import torch
    common, boxes, planes = _batch(6, 12, 32, det=1, n_lo=8, n_hi=16, p_lo=2 ** 12, p_hi=2 ** 14)
    b_ = bctx_bin(common, 32)
    assert sum(oracle.n_keys(g, b_) for g, *_ in boxes) <= 2 * sum(p["w"].shape[0] for _, p, *_ in boxes)
    allp, _ = _concat(boxes)
    results = []
    for use_graph in (False, True):
        bctx = _make_ctx(common, boxes)
        A = rs.Particles.from_numpy(allp, 32)
        B = rs.Particles.empty(A.n, 32)
        bctx.sort(A, B)
        state = [B, A]
        F = _fields_device(bctx, planes, 32)
        fb = bctx.grid_tensor()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())

        def run_steps():
            for k in range(6):
                if k % 3 == 2:
                    bctx.sort(state[0], state[1])
                    state.reverse()
                fb.zero_()
                bctx.push_gather(state[0], F, fb)

        with torch.cuda.stream(s):
            run_steps()  # warm-up outside capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        if use_graph:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                run_steps()
            g.replay()
        else:
            run_steps()
        torch.cuda.synchronize()
        bctx.check()
        results.append((fb.clone(), [t.clone() for t in state[0].tensors()]))
    assert torch.equal(results[0][0], results[1][0])
    for x, y in zip(results[0][1], results[1][1]):
        assert torch.equal(x, y)
