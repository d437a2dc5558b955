"""Sort benchmark: the steady-state cell sort (rsol_sort) of the step.

Workload (defaults): the headline step's packets (128^3 periodic grid, 2^24
packets, power law on [1, 100], B0 along x plus 64 Alfven modes, dB/B0 = 0.1,
c/c~ = 10, TSC, FP32), sorted once; then each repetition pushes the sorted set
--drift steps at c~ dt = 0.2 dx (untimed) and sorts it into the other buffer
(timed with CUDA events), so every timed sort meets the order it meets every
4th step of the bench: the set the context sorted last, drifted.  At this size
(2^21 keys for 2^24 packets) the library sorts by counting.

Bytes one counting sort moves, per packet:
- the count kernel reads cell and offsets (16 B) and writes a key (4 B);
- the placement reads the key (4 B) and writes the source index at the
  packet's position (4 B);
- the in-key fix-up reads and writes the index (8 B) and records the bin
  ranges from the counters;
- the payload gather reads the index (4 B) and reads and writes the packet
  (32 + 32 B);
and per key: the counter is zeroed (4 B), summed (4 B), scanned in place
(8 B) and read by the fix-up (4 B).  72 B per packet (the packet read and
written once, plus an index and a key) is the floor of a sort that moves the
packets; the record gives the achieved rate against both.

    python -m paper_2111_14704_gb300.sort_bench [--grid 128] [--packets 16777216]

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

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
    ap.add_argument("--drift", type=int, default=4, help="pushes between the two sorts")
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args(argv)
    rs.load_library()
    torch.cuda.set_device(0)
    g = (args.grid,) * 3
    parts = ri.make_particles(args.packets, g, 2, fp32=True)
    modes = ri.alfven_modes(64, 2, L=(float(args.grid),) * 3, kmax=min(16, args.grid // 2), dB_rms=0.1)
    params = rs.Params(*g, shape=2, precision=32, c=1.0, c_tilde=0.1)
    ctx = rs.Context(params)
    A = rs.Particles.from_numpy(parts, 32)
    B = rs.Particles.empty(A.n, 32)
    ctx.sort(A, B)
    F = ctx.grid_tensor()
    ctx.alfven_fields(modes, 0.0, 1.0, 1e-4, (0.0, 0.0, 0.0), F)
    fb = ctx.grid_tensor()
    s = torch.cuda.current_stream()
    ms = []
    for rep in range(args.reps + 1):  # the first sort is a warm-up
        for _ in range(args.drift):
            fb.zero_()
            ctx.push_gather(B, F, 0.2 / params.c_tilde, fb)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        ctx.sort(B, A)
        e1.record(s)
        torch.cuda.synchronize()
        if rep > 0:
            ms.append(e0.elapsed_time(e1))
        A, B = B, A
    ctx.check()
    n = args.packets
    nkeys = 1
    for d in g:  # bins per axis x bin edge: the key space the library sorts over (bin 8 in FP32)
        nkeys *= -(-d // 8) * 8
    alg_bytes = n * (20 + 8 + 8 + 68) + nkeys * 20
    floor_bytes = n * 72
    best = min(ms)
    return {"workload": f"{args.grid}^3 grid, {n} packets, TSC FP32, sorted after {args.drift} "
                        f"pushes of c~ dt = 0.2 dx",
            "packets": n, "keys": nkeys, "ms": ms, "best_ms": best,
            "packets_per_s": n / (best * 1e-3), "alg_bytes": alg_bytes,
            "alg_gb_per_s": alg_bytes / (best * 1e-3) / 1e9,
            "floor_72b_gb_per_s": floor_bytes / (best * 1e-3) / 1e9}


def main():
    print(json.dumps(run()), flush=True)


if __name__ == "__main__":
    main()
