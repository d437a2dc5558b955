"""Autotuner of the binned push (bin edge x CTA width, cached per GPU and
workload): the cache logic on the CPU, and on the GPU that the chosen
configuration gives the default configuration's results."""
from __future__ import annotations

import json

import numpy as np
import pytest

import paper_2111_14704_gb300 as rs
from paper_2111_14704_gb300 import autotune


def test_push_signature_separates_workloads():
    base = rs.Params(64, 64, 64, shape=2, precision=32)
    k = autotune.push_signature("GB300", base, 1 << 21)
    assert k == "GB300|push|p32|s2|d0|g64x64x64|ppc8.0"
    others = [autotune.push_signature("GB300", rs.Params(64, 64, 32), 1 << 21),
              autotune.push_signature("GB300", rs.Params(64, 64, 64, precision=64), 1 << 21),
              autotune.push_signature("GB300", rs.Params(64, 64, 64, shape=1), 1 << 21),
              autotune.push_signature("GB300", rs.Params(64, 64, 64, deterministic=1), 1 << 21),
              autotune.push_signature("GB300", base, 1 << 20),
              autotune.push_signature("B200", base, 1 << 21)]
    assert len({k, *others}) == 7


def test_best_of_and_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "cache.json"
    monkeypatch.setenv("RSOL_AUTOTUNE_CACHE", str(path))
    times = {"bin8_w16": 1.5, "bin8_w8": 1.7, "bin4_w16": 1.4, "bin4_w8": 2.0}
    best = autotune.best_of(times)
    assert (best["bin"], best["warps"]) == (4, 16) and best["ms"] == times
    autotune._store(autotune.cache_path(), "k1", best)
    autotune._store(autotune.cache_path(), "k2", {"bin": 8, "warps": 8, "ms": {}})
    got = json.loads(path.read_text())
    assert got["k1"] == best and got["k2"]["warps"] == 8


@pytest.mark.gpu
def test_tuned_push_matches_default(tmp_path, monkeypatch):
    """tune_push times the four candidates once, caches the choice (a second
    call reads it back), and the chosen bin edge and CTA width move packets
    exactly as the default does (the per-packet arithmetic is the same) and
    deposit the same feedback within FP32 round-off."""
    import torch
    from tests.gpu_helpers import make_case, rel_l2
    monkeypatch.setenv("RSOL_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    grid = (32, 32, 32)
    params, parts, planes, _ = make_case(grid, 1 << 18, 71, precision=32)
    dt = 0.2 / params.c_tilde
    F = rs.fields_to_device(planes, 32)
    P = rs.Particles.from_numpy(parts, 32)
    t1 = autotune.tune_push(params, P, F, dt)
    assert (t1["bin"], t1["warps"]) in autotune.CANDIDATES and len(t1["ms"]) == 4
    assert autotune.tune_push(params, P, F, dt) == t1
    out = []
    for bin_, warps in ((0, 0), (t1["bin"], t1["warps"])):
        p = rs.Params(**{**params.__dict__, "bin": bin_, "warps": warps})
        ctx = rs.Context(p)
        A = rs.Particles.from_numpy(parts, 32)
        Q = rs.Particles.empty(A.n, 32)
        ctx.sort(A, Q)
        fb = ctx.grid_tensor()
        ctx.push_gather(Q, F, dt, fb)
        torch.cuda.synchronize()
        ctx.check()
        g = Q.to_numpy()
        order = np.lexsort((g["w"], g["u"][2], g["u"][1], g["u"][0]))
        out.append(({k: (v[..., order]) for k, v in g.items()}, rs.grid_to_planes(fb)))
    (a, fa), (b, fbb) = out
    for k in ("cell", "off", "u", "w"):
        np.testing.assert_array_equal(a[k], b[k])
    for q in range(8):
        assert rel_l2(fbb[q], fa[q]) <= 3e-6, q
