"""Autotuners for the binned push: each picks the sort bin edge (4 or 8
anchors) and the CTA width (8 or 16 warps) by timing every candidate on the
caller's own packets, and caches the choice in a JSON file.

* tune_push: one box; keyed by GPU name, precision, shape, deterministic mode,
  grid and packets per cell.
* tune_batch: a batch of boxes; keyed by GPU name, precision, shape,
  deterministic mode and the batch's shape signature.

Cache file: $RSOL_AUTOTUNE_CACHE, else ~/.cache/rsol_gb300/autotune.json.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import BatchContext, Context, Params, Particles

CANDIDATES = ((8, 16), (8, 8), (4, 16), (4, 8))  # (bin edge, warps)


def cache_path() -> str:
    p = os.environ.get("RSOL_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "rsol_gb300", "autotune.json")


def signature(common: Params, dims, offsets) -> str:
    import torch
    h = hashlib.sha256()
    h.update(np.asarray(dims, dtype=np.int32).tobytes())
    h.update(np.diff(np.asarray(offsets, dtype=np.int64)).tobytes())
    name = torch.cuda.get_device_name()
    return f"{name}|p{common.precision}|s{common.shape}|d{common.deterministic}|{h.hexdigest()[:16]}"


def push_signature(device_name: str, params: Params, n_packets: int) -> str:
    """Cache key of a single-box push: GPU, precision, shape, mode, grid and
    packets per cell (to one decimal)."""
    ppc = n_packets / float(params.nx * params.ny * params.nz)
    return (f"{device_name}|push|p{params.precision}|s{params.shape}|d{params.deterministic}|"
            f"g{params.nx}x{params.ny}x{params.nz}|ppc{ppc:.1f}")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(path, key, result):
    cache = _load(path)
    cache[key] = result
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)


def best_of(times: dict) -> dict:
    """{"bin", "warps", "ms"} of the fastest candidate ("bin{b}_w{w}" keys)."""
    best = min(times, key=times.get)
    bin_, warps = (int(x) for x in best.replace("bin", "").split("_w"))
    return {"bin": bin_, "warps": warps, "ms": times}


def tune_push(params: Params, parts: Particles, fields, dt: float, steps: int = 3,
              use_cache: bool = True) -> dict:
    """Return {"bin": b, "warps": w, "ms": {...}} for this box: each candidate
    sorts a copy of the packets, then pushes it `steps` times (after one
    untimed push) with the fused deposit; from the cache when present."""
    import torch
    path = cache_path()
    key = push_signature(torch.cuda.get_device_name(), params, parts.n)
    if use_cache:
        cache = _load(path)
        if key in cache:
            return cache[key]
    times = {}
    s = torch.cuda.current_stream()
    for bin_, warps in CANDIDATES:
        p = Params(**{**params.__dict__, "bin": bin_, "warps": warps})
        ctx = Context(p)
        A = Particles(parts.cell.clone(), [t.clone() for t in parts.off],
                      [t.clone() for t in parts.u], parts.w.clone())
        Q = Particles.empty(parts.n, p.precision)
        ctx.sort(A, Q)
        fb = ctx.grid_tensor()
        ctx.push_gather(Q, fields, dt, fb)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            ctx.push_gather(Q, fields, dt, fb)
        e1.record(s)
        torch.cuda.synchronize()
        ctx.check()
        times[f"bin{bin_}_w{warps}"] = e0.elapsed_time(e1) / steps
        ctx.close()
        del A, Q, fb
    result = best_of(times)
    if use_cache:
        _store(path, key, result)
    return result


def tune_batch(common: Params, dims, c_tilde, dt, offsets, parts: Particles, fields,
               steps: int = 3, use_cache: bool = True) -> dict:
    """Return {"bin": b, "warps": w, "ms": {...}} for this batch (timing each
    candidate: sort once, then `steps` pushes), from the cache when present."""
    import torch
    path = cache_path()
    key = signature(common, dims, offsets)
    cache = _load(path) if use_cache else {}
    if key in cache:
        return cache[key]
    times = {}
    for bin_, warps in CANDIDATES:
        p = Params(**{**common.__dict__, "bin": bin_})
        bctx = BatchContext(p, dims, c_tilde, dt, offsets, warps=warps)
        Q = Particles.empty(parts.n, p.precision)
        bctx.sort(parts, Q)
        fb = bctx.grid_tensor()
        bctx.push_gather(Q, fields, fb)  # warm-up
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            bctx.push_gather(Q, fields, fb)
        e1.record(s)
        torch.cuda.synchronize()
        times[f"bin{bin_}_w{warps}"] = e0.elapsed_time(e1) / steps
        bctx.close()
        del Q, fb
    result = best_of(times)
    if use_cache:
        _store(path, key, result)
    return result
