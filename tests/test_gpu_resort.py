"""rsol_sort in the steady state of a run (the set its context sorted last,
after pushes) and on crowded keys: the result must be the oracle's stable
sort by anchor key bit for bit, whichever of the library's sorts runs (the
counting sort by key where there are at most two keys per packet, else the
radix sort).

The packets are read back from the GPU and sorted by the oracle (keys from
`oracle.sort_keys`, order from `oracle.stable_sort`); the library's sort must
return exactly those arrays in that order.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2111_14704_gb300 as rs
from tests.gpu_helpers import anchor_nodes, make_case

pytestmark = pytest.mark.gpu


def _oracle_sorted(parts, grid, bin_, shape):
    keys = oracle.sort_keys(grid, bin_, shape, parts["cell"], parts["off"])
    perm = oracle.stable_sort(keys, oracle.n_keys(grid, bin_))
    return {k: (v[:, perm] if v.ndim == 2 else v[perm]) for k, v in parts.items()}


def _sort_push_sort(params, parts, planes, pushes, edit=None):
    """Sort, push `pushes` times (the set stays the last sort's output), optionally
    edit the packets on the host, sort again.  Returns (input of the second
    sort, its output) as numpy dicts."""
    import torch
    ctx = rs.Context(params)
    A = rs.Particles.from_numpy(parts, params.precision)
    B = rs.Particles.empty(A.n, params.precision)
    ctx.sort(A, B)
    F = rs.fields_to_device(planes, params.precision)
    dt = 0.2 / params.c_tilde
    for _ in range(pushes):
        ctx.push_gather(B, F, dt, ctx.grid_tensor())
    if edit is not None:
        edit(B)
    torch.cuda.synchronize()
    before = B.to_numpy()
    ctx.sort(B, A)  # B is the set the last sort wrote
    torch.cuda.synchronize()
    ctx.check()
    return before, A.to_numpy()


def _assert_same(got, want):
    for k in ("cell", "off", "u", "w"):
        np.testing.assert_array_equal(got[k], want[k])


@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("precision,bin_,grid,n", [
    (32, 8, (32, 32, 32), 1 << 17), (32, 4, (20, 16, 12), 30000), (64, 4, (24, 16, 12), 20000),
    (32, 8, (24, 24, 24), 3 * 24 ** 3)])
def test_resort_after_pushes_is_the_stable_sort(shape, precision, bin_, grid, n):
    params, parts, planes, _ = make_case(grid, n, 91, shape=shape, precision=precision)
    params.bin = bin_
    parts["off"][:, ::11] = 0.5  # TSC anchor ties at the half-node
    before, got = _sort_push_sort(params, parts, planes, 4)
    # the pushes moved packets to new bins (so the second sort had work to do)
    at0 = anchor_nodes(parts["cell"], parts["off"], grid, shape) // bin_
    at1 = anchor_nodes(before["cell"], before["off"], grid, shape) // bin_
    keys0 = np.sort((at0[2] * 1000 + at0[1]) * 1000 + at0[0])
    keys1 = np.sort((at1[2] * 1000 + at1[1]) * 1000 + at1[0])
    assert not np.array_equal(keys0, keys1)
    _assert_same(got, _oracle_sorted(before, grid, bin_, shape))


def test_resort_when_packets_jump_bins():
    """Packets moved several bins (cells rewritten on the host between the sorts)."""
    import torch
    grid = (32, 32, 32)
    params, parts, planes, _ = make_case(grid, 50000, 92, precision=32)

    def jump(P):
        c = rs.unpack_cells(P.cell.cpu().numpy())
        c[0, ::97] = (c[0, ::97] + 13) % 32  # 13 cells: more than one 8-node bin
        c[1, ::89] = (c[1, ::89] + 21) % 32
        P.cell.copy_(torch.from_numpy(rs.pack_cells(c)).to(P.cell.device))

    before, got = _sort_push_sort(params, parts, planes, 2, edit=jump)
    _assert_same(got, _oracle_sorted(before, grid, 8, 2))


def test_resort_three_bins_per_axis_and_repeated():
    """Several sort-push cycles in a row on small grids (3 and 2 bins per axis),
    against the oracle each time."""
    import torch
    for grid, bin_ in (((24, 24, 24), 8), ((12, 12, 12), 4), ((16, 16, 16), 8)):
        params, parts, planes, _ = make_case(grid, 20000, 93, precision=32)
        params.bin = bin_
        ctx = rs.Context(params)
        A = rs.Particles.from_numpy(parts, 32)
        B = rs.Particles.empty(A.n, 32)
        F = rs.fields_to_device(planes, 32)
        ctx.sort(A, B)
        for cycle in range(3):
            for _ in range(3):
                ctx.push_gather(B, F, 0.2 / params.c_tilde, ctx.grid_tensor())
            torch.cuda.synchronize()
            before = B.to_numpy()
            ctx.sort(B, A)
            torch.cuda.synchronize()
            _assert_same(A.to_numpy(), _oracle_sorted(before, grid, bin_, 2))
            A, B = B, A
        ctx.check()


@pytest.mark.parametrize("precision", [32, 64])
def test_sort_crowded_keys(precision):
    """Keys shared by many packets, in random input order: one node holding
    20000 packets (sorted in runs and merged), one holding 3000 (one block
    sort), and nodes holding 9..40 packets (the per-thread networks and the
    block path just above them), among packets spread over the grid."""
    import torch
    grid = (16, 16, 16)
    rng = np.random.default_rng(94)
    params, parts, planes, _ = make_case(grid, 60000, 94, precision=precision)
    cells = parts["cell"]  # (3, n) integer cells
    sizes = [20000, 3000] + list(range(9, 41))
    at = 0
    for j, m in enumerate(sizes):
        cells[:, at:at + m] = np.array([j % 16, (5 * j + 1) % 16, 5 * (j // 16) + 3])[:, None]
        parts["off"][:, at:at + m] = 0.25  # one anchor node for CIC and TSC
        at += m
    order = rng.permutation(parts["w"].shape[0])
    parts = {k: v[..., order] for k, v in parts.items()}
    params.bin = 8
    for shape in (1, 2):
        params.shape = shape
        ctx = rs.Context(params)
        P = rs.Particles.from_numpy(parts, precision)
        Q = rs.Particles.empty(P.n, precision)
        ctx.sort(P, Q)
        torch.cuda.synchronize()
        ctx.check()
        _assert_same(Q.to_numpy(), _oracle_sorted(parts, grid, 8, shape))


@pytest.mark.parametrize("n", [30000, 1000])  # counting sort (3840 keys), radix sort
def test_sort_with_cells_off_the_grid(n):
    """Cells outside the grid are outside the contract of rsol_sort, but they must
    not be lost or break the bin ranges: the output is a permutation of the input,
    the packets with valid cells keep the oracle's stable order among themselves,
    and the push on the result reports the bad cells instead of faulting."""
    import torch
    grid = (20, 16, 12)
    params, parts, planes, _ = make_case(grid, n, 95, precision=32)
    params.bin = 4
    parts["w"] = 1.0 + np.arange(n) / 2.0 ** 20  # distinct weights identify the packets
    bad = np.zeros(n, bool)
    bad[7::97] = True
    cells = parts["cell"]
    cells[0, 7::194] = grid[0] + np.arange(cells[0, 7::194].shape[0]) % 5   # x past the grid
    cells[2, 104::194] = 1023                                               # z at the field's limit
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, 32)
    Q = rs.Particles.empty(n, 32)
    ctx.sort(P, Q)
    torch.cuda.synchronize()
    got = Q.to_numpy()
    # a permutation: match rows by weight (distinct draws)
    order_in = np.argsort(parts["w"], kind="stable")
    order_out = np.argsort(got["w"], kind="stable")
    for k in ("cell", "off", "u", "w"):
        np.testing.assert_array_equal(got[k][..., order_out], parts[k][..., order_in])
    src = order_in[np.argsort(order_out)]  # input index of each output packet
    valid_out = src[~bad[src]]
    good = {k: v[..., ~bad] for k, v in parts.items()}
    want = _oracle_sorted(good, grid, 4, 2)
    np.testing.assert_array_equal(parts["w"][valid_out], want["w"])
    F = rs.fields_to_device(planes, 32)
    ctx.push_gather(Q, F, 0.2 / params.c_tilde, ctx.grid_tensor())
    with pytest.raises(rs.RsolError, match="off the grid"):
        ctx.check()


@pytest.mark.parametrize("n,launches", [(1919, 10), (1920, 6), (30000, 6)])
def test_sort_choice_follows_key_space(n, launches):
    """The counting sort runs when the key space is at most two keys per packet
    (here 3840 keys: bins of 4^3 on 20 x 16 x 12), in six kernels; below that the
    radix sort runs, in 2 + 4 x passes kernels (12 key bits: 2 passes).  Both
    give the oracle's stable order."""
    import torch
    grid = (20, 16, 12)
    params, parts, planes, _ = make_case(grid, n, 96, precision=32)
    params.bin = 4
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, 32)
    Q = rs.Particles.empty(n, 32)
    before = ctx.kernel_launches()
    ctx.sort(P, Q)
    torch.cuda.synchronize()
    assert ctx.kernel_launches() - before == launches
    _assert_same(Q.to_numpy(), _oracle_sorted(parts, grid, 4, 2))
