"""Batched-box benchmark: many independent periodic boxes advanced together.

Workload (defaults): 512 boxes with cubic grids of edge log-uniform in
[16, 64] and packet counts log-uniform in [2^12, 2^18] (seeded), c/c~
log-uniform in [1, 100] (dt = 0.2 dx / c~ per box), each with its own
64-mode Alfven spectrum (rms dB/B0 uniform in [0.01, 0.3]) evaluated at t = 0,
FP32 TSC, 50 steps with a sort every 4 steps.  Three ways to run the same
steps: the batched push (its sparse-bin and dense-bin kernels) in a CUDA graph
captured once and replayed, the same launched eagerly, and one rsol_push_gather
(and rsol_sort) per box per step.  The autotuner picks the bin edge and CTA width first.

    python -m paper_2111_14704_gb300.batch_bench [--boxes 512] [--steps 50]

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def run(argv=None) -> dict:
    """Run the benchmark (argv as on the command line); returns the JSON record."""
    import torch

    import paper_2111_14704_gb300 as rs
    import rsol_inputs as ri
    from paper_2111_14704_gb300.autotune import tune_batch

    ap = argparse.ArgumentParser()
    ap.add_argument("--boxes", type=int, default=512)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--sort-every", type=int, default=4)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--loop", type=int, default=1, help="also time the per-box launch loop")
    args = ap.parse_args(argv)
    rs.load_library()
    torch.cuda.set_device(0)

    sh = ri.batch_boxes(args.boxes, args.seed)
    dims, cts, dts, parts = [], [], [], []
    for b in range(args.boxes):
        e = int(sh["edge"][b])
        dims.append((e, e, e))
        ct = 1.0 / float(sh["c_over_c_tilde"][b])
        cts.append(ct)
        dts.append(0.2 / ct)
        parts.append(ri.make_particles(int(sh["count"][b]), (e, e, e), args.seed + b))
    offsets = np.concatenate([[0], np.cumsum([p["w"].shape[0] for p in parts])])
    allp = {k: np.concatenate([p[k] for p in parts], axis=1) for k in ("cell", "off", "u")}
    allp["w"] = np.concatenate([p["w"] for p in parts])
    n_total = int(offsets[-1])
    common = rs.Params(2, 2, 2, shape=2, precision=32, c=1.0, c_tilde=1.0)

    # fields: each box's own spectrum at t = 0, written by the batch field source
    probe = rs.BatchContext(common, dims, cts, dts, offsets)
    F = probe.grid_tensor()
    for b in range(args.boxes):
        e = dims[b][0]
        modes = ri.alfven_modes(64, args.seed + b, L=(float(e),) * 3, kmax=min(16, e // 2),
                                dB_rms=float(sh["dB_rms"][b]))
        probe.alfven_fields(b, modes, 0.0, 1.0, 1e-4, (0.0, 0.0, 0.0), F)
    node_offsets = probe.node_offsets
    probe.close()

    P0 = rs.Particles.from_numpy(allp, 32)
    tune = tune_batch(common, dims, cts, dts, offsets, P0, F)
    common.bin = tune["bin"]

    def batched(use_graph: bool):
        bctx = rs.BatchContext(common, dims, cts, dts, offsets, warps=tune["warps"])
        A = rs.Particles.empty(n_total, 32)
        B = rs.Particles.empty(n_total, 32)
        for s_, d_ in zip(P0.tensors(), A.tensors()):
            d_.copy_(s_)
        fb = bctx.grid_tensor()
        bctx.sort(A, B)
        state = [B, A]

        def steps():
            for k in range(args.steps):
                if k > 0 and k % args.sort_every == 0:
                    bctx.sort(state[0], state[1])
                    state.reverse()
                fb.zero_()
                bctx.push_gather(state[0], F, fb)

        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            bctx.push_gather(state[0], F, fb)  # warm-up outside any capture
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = None
        if use_graph:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                steps()
            torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        if use_graph:
            g.replay()
        else:
            steps()
        e1.record(s)
        torch.cuda.synchronize()
        bctx.check()
        return e0.elapsed_time(e1)

    ms_graph = batched(True)
    ms_eager = batched(False)

    ms_loop = None
    if args.loop:
        ctxs, sets, views_f, views_b = [], [], [], []
        fb_all = torch.zeros_like(F)
        for b in range(args.boxes):
            p = rs.Params(*dims[b], shape=2, precision=32, c=1.0, c_tilde=cts[b], bin=common.bin)
            ctx = rs.Context(p)
            lo, hi = int(offsets[b]), int(offsets[b + 1])
            A = rs.Particles.empty(hi - lo, 32)
            Bq = rs.Particles.empty(hi - lo, 32)
            for s_, d_ in zip(P0.tensors(), A.tensors()):
                d_.copy_(s_[lo:hi])
            ctx.sort(A, Bq)
            ctxs.append(ctx)
            sets.append([Bq, A])
            n0, n1 = int(node_offsets[b]), int(node_offsets[b + 1])
            views_f.append(F[n0:n1])
            views_b.append(fb_all[n0:n1])
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        e0.record(s)
        for k in range(args.steps):
            fb_all.zero_()
            for b in range(args.boxes):
                if k > 0 and k % args.sort_every == 0:
                    ctxs[b].sort(sets[b][0], sets[b][1])
                    sets[b].reverse()
                ctxs[b].push_gather(sets[b][0], views_f[b], dts[b], views_b[b])
        e1.record(s)
        torch.cuda.synchronize()
        ms_loop = e0.elapsed_time(e1)
        wall_loop = (time.perf_counter() - w0) * 1e3
        for c in ctxs:
            c.check()

    out = {
        "workload": f"{args.boxes} boxes, edge log-U[16,64], packets log-U[2^12,2^18], "
                    f"c/c~ log-U[1,100], own 64-mode spectra, TSC FP32, {args.steps} steps, "
                    f"sort every {args.sort_every}",
        "packets": n_total, "nodes": int(node_offsets[-1]),
        "autotune": tune,
        "graph_ms_per_step": ms_graph / args.steps,
        "eager_batched_ms_per_step": ms_eager / args.steps,
        "per_box_loop_ms_per_step": None if ms_loop is None else ms_loop / args.steps,
        "per_box_loop_wall_ms_per_step": None if ms_loop is None else wall_loop / args.steps,
        "graph_packet_steps_per_s": n_total * args.steps / (ms_graph * 1e-3),
        "speedup_graph_vs_loop": None if ms_loop is None else ms_loop / ms_graph,
    }
    return out


def main():
    print(json.dumps(run()), flush=True)


if __name__ == "__main__":
    main()
