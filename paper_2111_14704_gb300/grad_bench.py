"""Differentiable-run benchmark: gradients of L = ||sum_n S^n||_2 with respect
to the E,B grid and the Alfven amplitudes.

Workload (defaults): 64^3 periodic grid, 2^20 packets (power-law momenta on
[1, 100], slope 4.5, isotropic), B0 along x plus 64 Alfven modes (|n| <= 16,
rms dB/B0 = 0.1, vA = 1e-4 c) evaluated every step, c/c~ = 10,
dt = 0.2 dx / c~, TSC, FP32, 64 steps with packet checkpoints every 8 steps.
One rsol_gradient call (forward sweep, loss, reverse sweep with recompute) is
timed with CUDA events, then each of its kernels on its own.

    python -m paper_2111_14704_gb300.grad_bench [--precision 32] [--reps 3]

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

# algorithmic bytes of one adjoint step per packet: state read (cell 4, offsets
# and momenta 6 elements, weight 1 element), adjoints read and written
# (6 elements each way); per node: fields and feedback read (8 + 8 elements),
# field adjoint read-modify-write (2 x 8 elements)
def adjoint_bytes(n, nodes, es):
    return n * (4 + 7 * es + 12 * es) + nodes * (32 * es)


def run(argv=None) -> dict:
    """Run the benchmark (argv as on the command line); returns the JSON record."""
    import torch

    import paper_2111_14704_gb300 as rs
    import rsol_inputs as ri

    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=64)
    ap.add_argument("--packets", type=int, default=1 << 20)
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--every", type=int, default=8)
    ap.add_argument("--precision", type=int, default=32)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--graph", type=int, default=1, help="also time a CUDA-graph replay of the call")
    args = ap.parse_args(argv)
    rs.load_library()
    torch.cuda.set_device(0)
    g = (args.grid,) * 3
    prec = args.precision
    es = 4 if prec == 32 else 8
    parts = ri.make_particles(args.packets, g, 4, fp32=(prec == 32))
    modes = ri.alfven_modes(64, 4, L=(float(args.grid),) * 3, kmax=min(16, args.grid // 2), dB_rms=0.1)
    vA, ug = 1e-4, (0.0, 0.0, 0.0)
    params = rs.Params(*g, shape=2, precision=prec, c=1.0, c_tilde=0.1)
    dt = 0.2 / params.c_tilde
    ctx = rs.Context(params)
    P = rs.Particles.from_numpy(parts, prec)
    s = torch.cuda.current_stream()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    o = ctx.gradient(P, args.steps, dt, checkpoint_every=args.every, modes=modes, vA=vA, u_gas=ug)
    torch.cuda.synchronize()
    ctx.check()
    times = []
    for _ in range(args.reps):
        e0, e1 = ev(), ev()
        e0.record(s)
        ctx.gradient(P, args.steps, dt, checkpoint_every=args.every, modes=modes, vA=vA, u_gas=ug, out=o)
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ctx.check()
    total_ms = float(np.median(times))

    # the same call captured once in a CUDA graph and replayed (the scratch it
    # needs exists after the calls above; nothing in it synchronises the host)
    graph_ms = None
    if args.graph:
        side = torch.cuda.Stream()
        side.wait_stream(s)
        torch.cuda.synchronize()
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, stream=side):
            ctx.gradient(P, args.steps, dt, checkpoint_every=args.every, modes=modes, vA=vA, u_gas=ug,
                         out=o, stream=side)
        torch.cuda.synchronize()
        gt = []
        for _ in range(args.reps):
            e0, e1 = ev(), ev()
            e0.record(s)
            gr.replay()
            e1.record(s)
            torch.cuda.synchronize()
            gt.append(e0.elapsed_time(e1))
        ctx.check()
        graph_ms = float(np.median(gt))

    # the parts on their own, on a sorted set at t = 0
    W = rs.Particles.empty(P.n, prec)
    ctx.sort(P, W)
    F = ctx.grid_tensor()
    fb = ctx.grid_tensor()
    ctx.alfven_fields(modes, 0.0, 1.0, vA, ug, F)

    def timed(fn, reps=10):
        fn()
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(s)
        for _ in range(reps):
            fn()
        b.record(s)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    Wc = rs.Particles(W.cell.clone(), [t.clone() for t in W.off], [t.clone() for t in W.u], W.w.clone())
    t_fields = timed(lambda: ctx.alfven_fields(modes, 0.0, 1.0, vA, ug, F))
    # the forward step on the sorted set (binned); restore the state after timing
    t_push = timed(lambda: ctx.push_gather(W, F, dt, fb), reps=1)
    for a, b in zip(W.tensors(), Wc.tensors()):
        a.copy_(b)
    Q = rs.Particles(Wc.cell.clone(), [t.clone() for t in Wc.off], [t.clone() for t in Wc.u], Wc.w)
    t_recompute = timed(lambda: ctx.push_gather(Q, F, dt, None), reps=1)
    dt_ = torch.float32 if prec == 32 else torch.float64
    xb = torch.zeros((3, P.n), dtype=dt_, device="cuda")
    ub = torch.zeros((3, P.n), dtype=dt_, device="cuda")
    fbar = ctx.grid_tensor()
    for a_, b_ in zip(W.tensors(), Wc.tensors()):
        a_.copy_(b_)
    # W is the context's last sort output: the tiled kernel; Wc: the order-free one
    t_adj = timed(lambda: ctx.adjoint_step(W, F, dt, o["feedback"], o["loss"], xb, ub, fbar))
    t_adj_free = timed(lambda: ctx.adjoint_step(Wc, F, dt, o["feedback"], o["loss"], xb, ub, fbar))
    amp = torch.zeros(64, dtype=torch.float64, device="cuda")
    fbt = ctx.grid_tensor()
    t_amp = timed(lambda: ctx.alfven_adjoint(modes, 0.0, 1.0, vA, ug, fbar, amp, field_bar_total=fbt))
    torch.cuda.synchronize()
    ctx.check()

    nodes = args.grid ** 3
    ab = adjoint_bytes(P.n, nodes, es)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs")
    nseg = -(-args.steps // args.every)
    out = {
        "workload": f"{args.grid}^3 grid, {P.n} packets, 64 Alfven modes evaluated each step, "
                    f"c/c~ = 10, TSC, FP{prec}, {args.steps} steps, checkpoints every {args.every}",
        "metric": "differentiable run: packet-steps per second (forward steps / whole gradient time)",
        "gradient_ms": total_ms,
        "gradient_graph_ms": graph_ms,
        "graph_packet_steps_per_s": None if graph_ms is None else P.n * args.steps / (graph_ms * 1e-3),
        "packet_steps_per_s": P.n * args.steps / (total_ms * 1e-3),
        "loss": float(o["loss"][0].item()),
        "parts_ms": {"alfven_fields": t_fields, "push_gather_binned": t_push,
                     "push_no_deposit": t_recompute, "adjoint_step_tiled": t_adj,
                     "adjoint_step_order_free": t_adj_free, "alfven_adjoint": t_amp},
        # the forward sweep keeps every step's mode fields (they fit), so the
        # field source runs once per step
        "launch_counts": {"alfven_fields": args.steps,
                          "push_gather_binned": args.steps, "push_no_deposit": args.steps - nseg,
                          "adjoint_step_tiled": args.steps, "alfven_adjoint": args.steps,
                          "sort": nseg},
        "adjoint_roofline": {"bound": "hbm", "algorithmic_bytes": ab,
                             "achieved_gbs": ab / (t_adj * 1e-3) / 1e9,
                             "peak_gbs": hbm, "peak_source": "measured" if hbm else None,
                             "frac": (ab / (t_adj * 1e-3) / 1e9) / hbm if hbm else None},
    }
    return out


def main():
    print(json.dumps(run()), flush=True)


if __name__ == "__main__":
    main()
