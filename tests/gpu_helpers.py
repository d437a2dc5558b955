"""Shared drivers for the GPU parity tests: run the same seeded case through
librsol (via the C ABI binding) and through the FP64 oracle."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2111_14704_gb300 as rs
import rsol_inputs as ri


def make_case(grid, n, seed, *, shape=2, precision=32, c=1.0, c_tilde=0.1, q_over_m=1.0, q=1.0,
              n_modes=8, kmax=2, dB_rms=0.3, vA=0.01, u_gas=(0.0, 0.01, 0.0), p_range=(1.0, 100.0),
              beam_beta=0.0):
    parts = ri.make_particles(n, grid, seed, p_range=p_range, beam_beta=beam_beta,
                              fp32=(precision == 32))
    modes = ri.alfven_modes(n_modes, seed, L=tuple(float(g) for g in grid), kmax=kmax,
                            dB_rms=dB_rms) if n_modes else None
    planes = ri.field_grid(grid, modes=modes, vA=vA, u_gas=u_gas, c=c)
    if precision == 32:
        planes = planes.astype(np.float32).astype(np.float64)
    params = rs.Params(*grid, shape=shape, precision=precision, c=c, c_tilde=c_tilde,
                       q_over_m=q_over_m, q=q)
    return params, parts, planes, modes


def gpu_run(params, parts, planes, dt, steps, *, deposit=True, sort_every=0, ctx=None):
    """Returns (final particles as numpy dict, list of feedback planes per step)."""
    import torch
    ctx = ctx or rs.Context(params)
    P = rs.Particles.from_numpy(parts, params.precision)
    F = rs.fields_to_device(planes, params.precision)
    other = rs.Particles.empty(P.n, params.precision) if sort_every else None
    fbs = []
    for k in range(steps):
        if sort_every and k % sort_every == 0:
            ctx.sort(P, other)
            P, other = other, P
        fb = ctx.grid_tensor() if deposit else None
        ctx.push_gather(P, F, dt, fb)
        if deposit:
            fbs.append(rs.grid_to_planes(fb))
    torch.cuda.synchronize()
    ctx.check()
    return P.to_numpy(), fbs


def oracle_run(params, parts, planes, dt, steps, *, deposit=True):
    p = oracle.params(params.grid, shape=params.shape, dt=dt, c=params.c, c_tilde=params.c_tilde,
                      q_over_m=params.q_over_m, q=params.q, dx=params.dx)
    P = oracle.Particles(parts)
    fbs = []
    for _ in range(steps):
        G = oracle.step(p, planes, P, deposit=deposit)
        if deposit:
            fbs.append(G)
    return P.as_dict(), fbs


def positions(parts):
    return parts["cell"].astype(np.float64) + parts["off"]


def periodic_diff(a, b, grid):
    n = np.array(grid, dtype=np.float64)[:, None]
    return (a - b + 0.5 * n) % n - 0.5 * n


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def anchor_nodes(cell, off, grid, shape=2):
    """Anchor node of each packet per axis: its cell for CIC, the nearest node for
    TSC (x = i + f goes to i + 1 at f >= 1/2), wrapped on the periodic grid."""
    n = np.array(grid)[:, None]
    up = (off >= 0.5) if shape == 2 else 0
    return (cell.astype(np.int64) + up) % n


def bin_major_key(anchor, grid, bin_):
    """Bin-major linear key of anchor nodes (bins of bin_^3 nodes, x fastest)."""
    nb = [(g + bin_ - 1) // bin_ for g in grid]
    b, l = anchor // bin_, anchor % bin_
    return ((b[2] * nb[1] + b[1]) * nb[0] + b[0]) * bin_**3 + (l[2] * bin_ + l[1]) * bin_ + l[0]


def origin_order_breaks(anchor_at_sort, anchor_now, grid, bin_, shape=2):
    """Packets held in the order of a sort by anchor node (anchor_at_sort, already
    in that order) after drifting to anchor_now: per bin, the fraction of
    neighbours whose tile-local stencil origin decreases along the order (the
    binned kernels sort a bin locally past 1/32), and the number of packets
    whose stencil has left their bin's tile (the bin plus a 2-node halo)."""
    n = np.array(grid)[:, None]
    ns = 2 if shape == 1 else 3
    bins = anchor_at_sort // bin_
    first = 0 if shape == 1 else 1
    rel = (anchor_now - first - (bins * bin_ - 2)) % n
    out_of_tile = int((rel > bin_ + 4 - ns).any(0).sum())
    nb = [(g + bin_ - 1) // bin_ for g in grid]
    lin_bin = (bins[2] * nb[1] + bins[1]) * nb[0] + bins[0]
    lin_org = (rel[2] * 4096 + rel[1]) * 4096 + rel[0]
    desc = (lin_bin[1:] == lin_bin[:-1]) & (lin_org[1:] < lin_org[:-1])
    nbins = nb[0] * nb[1] * nb[2]
    breaks = np.bincount(lin_bin[1:][desc], minlength=nbins)
    counts = np.bincount(lin_bin, minlength=nbins)
    return breaks / np.maximum(counts, 1), counts, out_of_tile
