"""rsol_sort_static: the sort for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (their device memory belongs to another
component's allocator, or they must not stall on the synchronisation an
allocation can imply).  rsol_sort_static sorts with a static scratch array
inside the library instead; this file checks, through the C ABI, that it
returns exactly what rsol_sort returns, on two calls in a row, and that it
rejects problems too large for its scratch.  It is collected last on purpose.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import paper_2111_14704_gb300 as rs
from tests.gpu_helpers import make_case

pytestmark = pytest.mark.gpu


def _lib():
    L = rs.load_library()
    L.rsol_sort_static.argtypes = [C.POINTER(rs.CParams), C.POINTER(rs.CParticles),
                                   C.POINTER(rs.CParticles), C.c_void_p]
    L.rsol_sort_static.restype = C.c_int
    return L


def _stream():
    import torch
    return C.c_void_p(int(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("shape,precision", [(2, 32), (1, 64)])
def test_static_sort_matches_rsol_sort_twice(shape, precision):
    import torch
    L = _lib()
    grid = (20, 16, 12)
    for seed in (31, 32):  # two calls in a row share the static scratch
        params, parts, _, _ = make_case(grid, 100_000, seed, shape=shape, precision=precision,
                                        n_modes=0)
        cp = params.to_c()
        P = rs.Particles.from_numpy(parts, precision)
        A = rs.Particles.empty(P.n, precision)
        B = rs.Particles.empty(P.n, precision)
        sa, sb = P.c_struct(), A.c_struct()
        assert L.rsol_sort_static(C.byref(cp), C.byref(sa), C.byref(sb), _stream()) == 0
        rs.Context(params).sort(P, B)
        torch.cuda.synchronize()
        for x, y in zip(A.tensors(), B.tensors()):
            assert torch.equal(x, y)


def test_static_sort_rejects_problems_beyond_its_scratch():
    L = _lib()
    n = (1 << 20) + 1
    params = rs.Params(32, 32, 32, shape=2, precision=32)
    cp = params.to_c()
    P = rs.Particles.empty(n, 32)
    Q = rs.Particles.empty(n, 32)
    assert L.rsol_sort_static(C.byref(cp), C.byref(P.c_struct()), C.byref(Q.c_struct()),
                              _stream()) == 1


def test_static_sort_at_its_documented_limit_allocates_nothing():
    """The documented capacity: 262,144 packets on a grid of 65,536 bins
    (256 x 128 x 128 nodes in bins of 4^3) fits the static scratch and sorts
    exactly like rsol_sort.  After a first call (which loads the library's
    module on the device), two more calls leave the device's free memory
    unchanged: nothing is allocated."""
    import torch
    L = _lib()
    grid = (256, 128, 128)
    n = 262_144
    params, parts, _, _ = make_case(grid, n, 33, shape=2, precision=32, n_modes=0)
    params.bin = 4
    cp = params.to_c()
    P = rs.Particles.from_numpy(parts, 32)
    A = rs.Particles.empty(n, 32)
    B = rs.Particles.empty(n, 32)
    rs.Context(params).sort(P, B)
    sa, sb = P.c_struct(), A.c_struct()
    assert L.rsol_sort_static(C.byref(cp), C.byref(sa), C.byref(sb), _stream()) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        assert L.rsol_sort_static(C.byref(cp), C.byref(sa), C.byref(sb), _stream()) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for x, y in zip(A.tensors(), B.tensors()):
        assert torch.equal(x, y)
