"""rsol_sort of the set its context sorted last (after pushes): the re-sort by
neighbour bins must give the oracle's stable sort by anchor key bit for bit,
like the radix sort it replaces, and fall back to that radix sort on the
device when a packet moved further than one bin.

The packets after the pushes are read back from the GPU and sorted by the
oracle (keys from `oracle.sort_keys`, order from `oracle.stable_sort`); the
library's second sort must return exactly those arrays in that order.
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
    ctx.sort(B, A)  # B is the set the last sort wrote: the re-sort runs
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
    # the pushes moved packets to new bins (so the re-sort had work to do)
    at0 = anchor_nodes(parts["cell"], parts["off"], grid, shape) // bin_
    at1 = anchor_nodes(before["cell"], before["off"], grid, shape) // bin_
    keys0 = np.sort((at0[2] * 1000 + at0[1]) * 1000 + at0[0])
    keys1 = np.sort((at1[2] * 1000 + at1[1]) * 1000 + at1[0])
    assert not np.array_equal(keys0, keys1)
    _assert_same(got, _oracle_sorted(before, grid, bin_, shape))


def test_resort_falls_back_when_packets_jump_bins():
    """Packets moved several bins (cells rewritten on the host between the sorts):
    the re-sort notices on the device and the radix sort gives the result."""
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
    """The smallest grid the re-sort takes (3 bins per axis, every bin a neighbour
    of every other along an axis), several sort-push cycles in a row, against the
    oracle each time; and a grid of 2 bins per axis (the radix sort throughout)."""
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
