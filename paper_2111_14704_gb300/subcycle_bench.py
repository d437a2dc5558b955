"""Sub-cycling benchmark: one global step at the c~-Courant limit with
per-packet sub-steps, against plain steps covering the same time.

Workload (defaults): 128^3 periodic grid, 2^24 packets (power law on [1, 100]),
B0 along x plus 64 Alfven modes (dB/B0 = 0.1), c/c~ = 10, TSC, FP32.  The global
step is dt = 1.0 dx / c~; packets sub-cycle to C = 0.2 of their gyration and
crossing limits (max level 8).  The comparison runs the binned plain step five
times at dt = 0.2 dx / c~ (the same physical time, every packet at the finest
common step), sorting first.

    python -m paper_2111_14704_gb300.subcycle_bench [--reps 5]

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def run(argv=None) -> dict:
    """Run the benchmark (argv as on the command line); returns the JSON record."""
    import torch

    import paper_2111_14704_gb300 as rs
    import rsol_inputs as ri

    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--packets", type=int, default=1 << 24)
    ap.add_argument("--courant", type=float, default=0.2)
    ap.add_argument("--adv", type=float, default=1.0, help="c~ dt / dx of the global step")
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args(argv)
    rs.load_library()
    torch.cuda.set_device(0)
    g = (args.grid,) * 3
    parts = ri.make_particles(args.packets, g, 2, fp32=True)
    modes = ri.alfven_modes(64, 2, L=(float(args.grid),) * 3, kmax=min(16, args.grid // 2), dB_rms=0.1)
    params = rs.Params(*g, shape=2, precision=32, c=1.0, c_tilde=0.1)
    dt = args.adv / params.c_tilde
    ctx = rs.Context(params)
    P0 = rs.Particles.from_numpy(parts, 32)
    P = rs.Particles.empty(P0.n, 32)
    ctx.sort(P0, P)
    F = ctx.grid_tensor()
    ctx.alfven_fields(modes, 0.0, 1.0, 1e-4, (0.0, 0.0, 0.0), F)
    fb = ctx.grid_tensor()
    lev = torch.zeros(P.n, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    snap = [t.clone() for t in P.tensors()]

    def restore():
        for a, b in zip(P.tensors(), snap):
            a.copy_(b)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    # sub-cycled global step (the packet state is restored between repetitions)
    ctx.push_subcycled(P, F, dt, args.courant, fb, lev)
    torch.cuda.synchronize()
    ctx.check()
    hist = np.bincount(lev.cpu().numpy(), minlength=9)[:9]
    ts = []
    for _ in range(args.reps):
        restore()
        fb.zero_()
        a, b = ev(), ev()
        a.record(s)
        ctx.push_subcycled(P, F, dt, args.courant, fb, lev)
        b.record(s)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ctx.check()
    t_sub = float(np.median(ts))
    substeps = float((hist * (2.0 ** np.arange(9))).sum())

    # the same step on the tiled kernel: level sort into a second set, then
    # one launch per finest sub-step
    ts = []
    for _ in range(args.reps):
        restore()
        Q = rs.Particles.empty(P.n, 32)
        fb.zero_()
        a, b = ev(), ev()
        a.record(s)
        ctx.sort_push_subcycled(P, Q, F, dt, args.courant, fb)
        b.record(s)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
        del Q
    ctx.check()
    t_tiled = float(np.median(ts))

    # plain binned steps over the same time: sort, then round(adv / 0.2) steps
    n_plain = max(1, int(round(args.adv / 0.2)))
    ts = []
    for _ in range(args.reps):
        restore()
        Q = rs.Particles.empty(P.n, 32)
        fb.zero_()
        a, b = ev(), ev()
        a.record(s)
        ctx.sort(P, Q)
        for _k in range(n_plain):
            ctx.push_gather(Q, F, dt / n_plain, fb)
        b.record(s)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
        del Q
    ctx.check()
    t_plain = float(np.median(ts))
    n = P.n
    out = {
        "workload": f"{args.grid}^3 grid, {n} packets, 64 Alfven modes, c/c~ = 10, TSC, FP32, "
                    f"global step c~ dt = {args.adv} dx, C = {args.courant}, max level 8",
        "levels": {str(k): int(hist[k]) for k in range(9) if hist[k]},
        "mean_substeps_per_packet": substeps / n,
        "subcycled_ms_per_global_step": t_sub,
        "tiled_subcycled_ms_per_global_step": t_tiled,
        "tiled_packet_substeps_per_s": substeps / (t_tiled * 1e-3),
        "packet_steps_per_s": n / (t_sub * 1e-3),
        "packet_substeps_per_s": substeps / (t_sub * 1e-3),
        "plain_steps_same_time": n_plain,
        "plain_ms_same_time": t_plain,
        "plain_packet_steps_per_s": n * n_plain / (t_plain * 1e-3),
    }
    return out


def main():
    print(json.dumps(run()), flush=True)


if __name__ == "__main__":
    main()
