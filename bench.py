"""Benchmark of the RSOL cosmic-ray packet step on GB300.

Workload (one GPU): 3D periodic 128^3 grid, B0 x-hat plus 64 seeded Alfven
modes (|n| <= 16, dB/B0 = 0.1 rms, vA = 1e-4 c) re-evaluated every step,
2^24 packets with |u| from dN/dp ~ p^-4.5 on [1, 100], isotropic, c/c~ = 10,
TSC gather and deposit, FP32 packets (cell index + FP32 offset).

One step = field source at t^n (stand-in for the MHD solver), zeroing of the
feedback grid, the fused push (gather, Boris, feedback deposit, drift); every
4th step also the stable cell sort; every 10th step also the state-moment grid
and the FP64 totals.  Metric: packet-steps per second including gather and
deposit.  Packet arrays (2 x 512 MB) exceed the 129 MB L2, so no flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl rsol|reference]

With N > 1 (torchrun), every rank advances an independent replica box (its
own seed): weak scaling, no data-path collective.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CR particle-steps/s incl. gather+deposit; % of HBM roofline; FP32 vs FP64"
UNIT = "particle-steps/s"
GRID = (128, 128, 128)
N_PARTICLES = 1 << 24
N_MODES = 64
KMAX = 16
DB_RMS = 0.1
VA = 1e-4
C = 1.0
C_TILDE = 0.1
SORT_EVERY = 4
MOMENTS_EVERY = 10
SEED = 2
# Algorithmic bytes of one fused push launch (FP32): per packet read cell 4 +
# off 12 + u 12 + w 4, write cell 4 + off 12 + u 12 = 60 B; per node read the
# six field components 24 B and write eight feedback components 32 B = 56 B.
BYTES_PER_PACKET = 60
BYTES_PER_NODE = 56
# catastrophic losses: read cell 4 + offsets 12 + momenta 12 + weight 4, write weight 4
# (plus the n_n grid, 4 B per node, once)
LOSS_BYTES_PER_PACKET = 36
# DRAM traffic (read + write) of the binned push kernel per packet from an ncu
# capture of the same workload at half size (128 x 128 x 64 nodes, 2^23 packets:
# the same packets per cell, so the same bytes per packet), and the hash of the
# kernel sources it was taken on: the bench reports traffic only while the
# sources still match.
NCU_TRAFFIC_PER_PACKET = (342.832128e6 + 214.017536e6) / (1 << 23)
# warp instructions the same capture counted per packet (smsp__inst_executed.sum / packets)
NCU_INST_PER_PACKET = 420734654 / (1 << 23)
NCU_SOURCE_HASH = "1f1204edc712330c"
# instruction issue peak: 152 SMs x 4 schedulers x one warp instruction per clock
ISSUE_SCHEDULERS = 152 * 4


def kernel_source_hash() -> str:
    """Hash of the binned push kernel's code: its sources with comments and
    blank lines removed, so that editing a comment keeps the ncu figures."""
    h = hashlib.sha256()
    for f in ("push_binned.cuh", "rsol_device.cuh"):
        with open(os.path.join(ROOT, "paper_2111_14704_gb300", "csrc", f)) as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in text.splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str | None):
        self.samples = []
        self.proc = None
        self.device_id = device_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if self.device_id:
            cmd += ["-i", self.device_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append((time.perf_counter(), parts))

    def stop(self, window=None) -> dict:
        """Median SM clock and the throttle reasons of the samples taken inside
        `window` (host perf_counter start, end), else of all samples."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        chosen = [p for t, p in self.samples if window is None or window[0] <= t <= window[1]]
        if window is not None and not chosen:  # region shorter than the sampling period
            chosen = [p for t, p in self.samples if t >= window[0]][:1]
        for p in chosen:
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for name, v in zip(names, p[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def device_uuid(torch, dev: int):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def build_workload(rank: int, precision: int = 32):
    import rsol_inputs as ri
    from paper_2111_14704_gb300.replicas import replica_seed
    seed = replica_seed(SEED, rank)
    parts = ri.make_particles(N_PARTICLES, GRID, seed, p_range=(1.0, 100.0), fp32=(precision == 32))
    modes = ri.alfven_modes(N_MODES, seed, L=tuple(float(g) for g in GRID), kmax=KMAX,
                            dB_rms=DB_RMS)
    return parts, modes


def run_gpu(args, rank, world):
    import torch
    import torch.distributed as dist
    import paper_2111_14704_gb300 as rs

    from paper_2111_14704_gb300.autotune import tune_push
    dev = torch.cuda.current_device()
    parts_np, modes = build_workload(rank)
    dt = 0.2 / C_TILDE  # c~ dt = 0.2 dx
    P = rs.Particles.from_numpy(parts_np, 32)
    # sort bin edge and CTA width of the binned push: the autotuner's choice for
    # this GPU and workload (timed on these packets, cached)
    params = rs.Params(*GRID, shape=2, precision=32, c=C, c_tilde=C_TILDE)
    probe = rs.Context(params)
    F0 = probe.grid_tensor()
    probe.alfven_fields(modes, 0.0, 1.0, VA, (0.0, 0.0, 0.0), F0)
    tune = tune_push(params, P, F0, dt)
    probe.close()
    del F0
    params = rs.Params(*GRID, shape=2, precision=32, c=C, c_tilde=C_TILDE, bin=tune["bin"],
                       warps=tune["warps"])
    ctx = rs.Context(params)
    Q = rs.Particles.empty(P.n, 32)
    F = ctx.grid_tensor()
    fb = ctx.grid_tensor()
    M = ctx.grid_tensor()
    stream = torch.cuda.current_stream()
    ctx.sort(P, Q)
    P, Q = Q, P
    state = {"P": P, "Q": Q, "t": 0.0, "k": 0}
    events = {"field_source": [], "push": [], "sort": [], "moments": []}

    def part(name, record, fn):
        if not record:
            fn()
            return
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        events[name].append((e0, e1))

    def sort_swap():
        ctx.sort(state["P"], state["Q"])
        state["P"], state["Q"] = state["Q"], state["P"]

    dep_ev = []

    def state_moments():
        M.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record(stream)
        ctx.deposit(state["P"], M)
        e[1].record(stream)
        dep_ev.append(e)
        ctx.moments(state["P"], fb)  # FP64 totals read back to the host

    def step(record=False):
        k = state["k"]
        part("field_source", record, lambda: (ctx.alfven_fields(modes, state["t"], 1.0, VA, (0.0, 0.0, 0.0), F),
                                              fb.zero_()))
        part("push", record, lambda: ctx.push_gather(state["P"], F, dt, fb))
        if (k + 1) % SORT_EVERY == 0:
            part("sort", record, sort_swap)
        if (k + 1) % MOMENTS_EVERY == 0:
            part("moments", record, state_moments)
        state["t"] += dt
        state["k"] = k + 1

    for _ in range(args.warmup):
        step()
    ctx.check()
    sampler = ClockSampler(device_uuid(torch, dev))
    launches0 = ctx.kernel_launches()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    w_start = time.perf_counter()
    t0.record(stream)
    for _ in range(args.steps):
        step(record=True)
    t1.record(stream)
    torch.cuda.synchronize()
    w_end = time.perf_counter()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop(window=(w_start, w_end))
    launches = ctx.kernel_launches() - launches0
    ms = t0.elapsed_time(t1)
    push_ms = [a.elapsed_time(b) for a, b in events["push"]]
    # per-step device time of each part of the step (sort and moments amortised)
    breakdown = {name: sum(a.elapsed_time(b) for a, b in ev) / args.steps for name, ev in events.items()}
    ctx.check()
    deposit_ms = statistics.mean(a.elapsed_time(b) for a, b in dep_ev) if dep_ev else None
    # physics sanity of the run: totals finite, packet count conserved
    tot = ctx.moments(state["P"])
    assert math.isfinite(tot[4]) and abs(tot[0] - N_PARTICLES) < 1e-6 * N_PARTICLES

    # ---------------- end to end through host buffers (fields in, feedback out)
    # The same step as above, with the field source replaced by the host: every
    # step copies its fields in from pinned host memory and its feedback grid out
    # to pinned host memory.  The copies run on their own streams, double
    # buffered, so step k's push overlaps the copy-in of step k+1's fields and the
    # copy-out of step k-1's feedback.
    F_host = torch.empty_like(F, device="cpu").pin_memory()
    F_host.copy_(F)
    Fd = [F, torch.empty_like(F)]
    fbd = [fb, torch.empty_like(fb)]
    fb_host = [torch.empty_like(fb, device="cpu").pin_memory() for _ in range(2)]
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
    ev = {name: [torch.cuda.Event(), torch.cuda.Event()] for name in ("in", "push", "out")}
    for name in ev:  # recorded once so the first waits are satisfied
        for e in ev[name]:
            e.record(stream)
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for k in range(e2e_steps):
        i = k & 1
        with torch.cuda.stream(h2d):
            h2d.wait_event(ev["push"][i])  # step k-2 has finished reading Fd[i]
            Fd[i].copy_(F_host, non_blocking=True)
            ev["in"][i].record(h2d)
        stream.wait_event(ev["in"][i])
        stream.wait_event(ev["out"][i])  # step k-2's feedback has left fbd[i]
        fbd[i].zero_()
        ctx.push_gather(state["P"], Fd[i], dt, fbd[i])
        if (k + 1) % SORT_EVERY == 0:
            ctx.sort(state["P"], state["Q"])
            state["P"], state["Q"] = state["Q"], state["P"]
        if (k + 1) % MOMENTS_EVERY == 0:
            M.zero_()
            ctx.deposit(state["P"], M)
            ctx.moments(state["P"], fbd[i])  # FP64 totals read back to the host
        ev["push"][i].record(stream)
        with torch.cuda.stream(d2h):
            d2h.wait_event(ev["push"][i])
            fb_host[i].copy_(fbd[i], non_blocking=True)
            ev["out"][i].record(d2h)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - w0

    # ---------------- catastrophic losses (rsol_losses) on the same packets:
    # HBM-bound, 36 B per packet (cell, offsets, momenta, weight read; weight written)
    losses = None
    if args.loss_reps > 0:
        nn = torch.ones(GRID[::-1], dtype=torch.float32, device="cuda")  # n_n gathered with W
        ctx.losses(state["P"], 1e-3, dt, nn=nn)
        torch.cuda.synchronize()
        l0 = torch.cuda.Event(enable_timing=True)
        l1 = torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        for _ in range(args.loss_reps):
            ctx.losses(state["P"], 1e-3, dt, nn=nn)
        l1.record(stream)
        torch.cuda.synchronize()
        ctx.check()
        lms = l0.elapsed_time(l1) / args.loss_reps
        lbytes = LOSS_BYTES_PER_PACKET * N_PARTICLES + 4 * GRID[0] * GRID[1] * GRID[2]
        lpeak, lkind = measured_peaks()
        losses = {"ms": lms, "packets_per_s": N_PARTICLES / (lms * 1e-3),
                  "roofline": {"bound": "hbm", "achieved": lbytes / (lms * 1e-3) / 1e9, "peak": lpeak,
                               "unit": "GB/s", "frac": lbytes / (lms * 1e-3) / 1e9 / lpeak,
                               "alg_bytes_per_launch": lbytes, "peak_source": f"{lkind} hbm_gbs"},
                  "note": "n_n = 1 per node gathered with W (TSC), sigma = 1e-3: "
                          "w *= exp(-(c~/c) sigma c beta n_n dt) per launch"}

    # ---------------- the same workload at c/c~ = 1 and 100 (c~ dt = 0.2 dx each)
    sweep = None
    if args.sweep_steps > 0:
        sweep = {}
        for ratio in (1.0, 100.0):
            sweep[f"c_over_c_tilde_{ratio:g}"] = timed_steps(
                rs, parts_np, modes, 1.0 / ratio, args.sweep_steps, 3, stream)
    del parts_np

    # ---------------- the FP64 GPU build on the same workload (few steps)
    fp64 = None
    if args.fp64_steps > 0:
        del state, P, Q, F_host, fb_host
        torch.cuda.empty_cache()
        parts64, _ = build_workload(rank, precision=64)
        p64 = rs.Params(*GRID, shape=2, precision=64, c=C, c_tilde=C_TILDE)
        ctx64 = rs.Context(p64)
        A = rs.Particles.from_numpy(parts64, 64)
        B = rs.Particles.empty(A.n, 64)
        del parts64
        ctx64.sort(A, B)
        A, B = B, A
        F64 = ctx64.grid_tensor()
        fb64 = ctx64.grid_tensor()
        ctx64.alfven_fields(modes, 0.0, 1.0, VA, (0.0, 0.0, 0.0), F64)
        ctx64.push_gather(A, F64, dt, fb64)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for k in range(args.fp64_steps):
            ctx64.alfven_fields(modes, (k + 1) * dt, 1.0, VA, (0.0, 0.0, 0.0), F64)
            fb64.zero_()
            ctx64.push_gather(A, F64, dt, fb64)
        a1.record(stream)
        torch.cuda.synchronize()
        ms64 = a0.elapsed_time(a1) / args.fp64_steps
        fp64 = {"value": N_PARTICLES / (ms64 * 1e-3), "ms_per_step": ms64,
                "steps": args.fp64_steps, "note": "FP64 build, field source + push per step"}
        ctx64.check()

    return {"deposit_ms": deposit_ms, "autotune": tune, "sweep": sweep, "ms": ms, "push_ms": push_ms, "breakdown": breakdown, "clocks": clocks, "launches": launches,
            "e2e_s": e2e_s, "e2e_steps": e2e_steps, "field_bytes": F.numel() * F.element_size(),
            "fb_bytes": fb.numel() * fb.element_size(), "fp64": fp64, "losses": losses}


def push_roofline(push_ms: float, n: int, nodes: int, extra_bytes_per_packet: float = 0.0,
                  extra_ms: float = 0.0) -> dict:
    """Algorithmic bytes of a fused push (plus, optionally, an amortised sort)
    over its time, against the measured HBM peak."""
    peak, kind = measured_peaks()
    b = BYTES_PER_PACKET * n + BYTES_PER_NODE * nodes + extra_bytes_per_packet * n
    achieved = b / ((push_ms + extra_ms) * 1e-3) / 1e9
    return {"bytes_per_packet_step": round(b / n, 2), "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "peak_source": f"{kind} hbm_gbs"}


def timed_steps(rs, parts_np, modes, c_tilde, steps, warmup, stream, grid=None,
                sort_every=SORT_EVERY, P=None):
    """The benchmark step (field source, zeroing, fused push, a sort every
    sort_every steps) on a fresh context: device time per step and per part."""
    import torch
    grid = grid or GRID
    params = rs.Params(*grid, shape=2, precision=32, c=C, c_tilde=c_tilde)
    ctx = rs.Context(params)
    dt = 0.2 / c_tilde
    if P is None:
        P = rs.Particles.from_numpy(parts_np, 32)
    n = P.n
    Q = rs.Particles.empty(n, 32)
    F, fb = ctx.grid_tensor(), ctx.grid_tensor()
    ctx.sort(P, Q)
    P, Q = Q, P
    ev = {"push": [], "sort": []}
    t = 0.0
    for k in range(warmup + steps):
        rec = k >= warmup
        ctx.alfven_fields(modes, t, 1.0, VA, (0.0, 0.0, 0.0), F)
        fb.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        if rec:
            e[0].record(stream)
        ctx.push_gather(P, F, dt, fb)
        if rec:
            e[1].record(stream)
            ev["push"].append((e[0], e[1]))
        if (k + 1) % sort_every == 0:
            if rec:
                e[2].record(stream)
            ctx.sort(P, Q)
            P, Q = Q, P
            if rec:
                e[3].record(stream)
                ev["sort"].append((e[2], e[3]))
        if k == warmup - 1:
            t0 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
        t += dt
    t1 = torch.cuda.Event(enable_timing=True)
    t1.record(stream)
    torch.cuda.synchronize()
    ctx.check()
    ms = t0.elapsed_time(t1) / steps
    push = statistics.mean(a.elapsed_time(b) for a, b in ev["push"])
    sort = statistics.mean(a.elapsed_time(b) for a, b in ev["sort"]) if ev["sort"] else 0.0
    nodes = grid[0] * grid[1] * grid[2]
    out = {"value": n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "push_ms": push,
           "sort_ms_per_call": sort, "steps": steps, "warmup": warmup,
           "roofline_push": push_roofline(push, n, nodes)}
    del P, Q, F, fb, ctx
    torch.cuda.empty_cache()
    return out


def _packet_chunk(task):
    """Packets first .. first+n-1 of a seeded set in the device's FP32 layout
    (one worker of the parallel generation of a large workload)."""
    n, grid, seed, first, p_range, beam = task
    import numpy as np
    import rsol_inputs as ri
    from paper_2111_14704_gb300 import pack_cells
    parts = ri.make_particles(n, grid, seed, p_range=p_range, beam_beta=beam, first=first)
    return (pack_cells(parts["cell"]), parts["off"].astype(np.float32),
            parts["u"].astype(np.float32), parts["w"].astype(np.float32))


def device_particles(rs, n, grid, seed, p_range, beam, chunk=1 << 22):
    """A large seeded packet set generated on every host core (spawned workers,
    rsol_inputs unchanged: packet j is the same draw however the set is split)
    and copied to the device chunk by chunk."""
    import multiprocessing as mp
    import torch
    P = rs.Particles.empty(n, 32)
    tasks = [(min(chunk, n - f), grid, seed, f, p_range, beam) for f in range(0, n, chunk)]
    with mp.get_context("spawn").Pool(max(1, min(os.cpu_count() or 1, 16))) as pool:
        for task, (cell, off, u, w) in zip(tasks, pool.imap(_packet_chunk, tasks)):
            lo = task[3]
            hi = lo + cell.shape[0]
            P.cell[lo:hi].copy_(torch.from_numpy(cell))
            for a in range(3):
                P.off[a][lo:hi].copy_(torch.from_numpy(off[a]))
                P.u[a][lo:hi].copy_(torch.from_numpy(u[a]))
            P.w[lo:hi].copy_(torch.from_numpy(w))
    return P


CONFIG3 = {"grid": (256, 256, 256), "particles": 1 << 27, "c_over_c_tilde": 30.0, "seed": 3,
           "p_range": (1.0, 1000.0), "beam_beta": 0.3, "sort_every": 4}


def run_config3(args):
    """The 256^3, 2^27-packet beam workload (c/c~ = 30, a sort every 4 steps):
    ms per step, packet-steps/s and the HBM fraction at 67 B per packet-step
    (push) and at 85 B (push plus the sort amortised over 4 steps)."""
    import torch
    import rsol_inputs as ri
    import paper_2111_14704_gb300 as rs
    c3 = CONFIG3
    grid, n = c3["grid"], c3["particles"]
    t0 = time.perf_counter()
    P = device_particles(rs, n, grid, c3["seed"], c3["p_range"], c3["beam_beta"])
    gen_s = time.perf_counter() - t0
    modes = ri.alfven_modes(N_MODES, c3["seed"], L=tuple(float(g) for g in grid), kmax=KMAX,
                            dB_rms=DB_RMS)
    r = timed_steps(rs, None, modes, 1.0 / c3["c_over_c_tilde"], args.config3_steps, 4,
                    torch.cuda.current_stream(), grid=grid, sort_every=c3["sort_every"], P=P)
    nodes = grid[0] * grid[1] * grid[2]
    r["roofline_push_and_sort"] = push_roofline(r["push_ms"], n, nodes, 72.0 / c3["sort_every"],
                                                r["sort_ms_per_call"] / c3["sort_every"])
    r["workload"] = ("256^3 periodic grid, 64 Alfven modes (dB/B0=0.1, |n|<=16, vA=1e-4c), 2^27 "
                     "packets, power-law |u| in [1,1000] boosted by 0.3 along B0 (beam), c/c~=30, "
                     "TSC, FP32, sort every 4 steps")
    r["input_generation_s"] = gen_s
    return r


def cpu_baseline(sample_particles: int, steps: int):
    """The FP64 oracle, as it stands, on a bounded sample of the workload (one
    core).  Returns (packet-steps/s, seconds, the field planes it used)."""
    import oracle
    import rsol_inputs as ri
    parts = ri.make_particles(sample_particles, GRID, SEED)
    modes = ri.alfven_modes(N_MODES, SEED, L=tuple(float(g) for g in GRID), kmax=KMAX,
                            dB_rms=DB_RMS)
    planes = ri.field_grid(GRID, modes=modes, vA=VA, c=C)
    dt = 0.2 / C_TILDE
    p = oracle.params(GRID, shape=2, dt=dt, c=C, c_tilde=C_TILDE)
    P = oracle.Particles(parts)
    oracle.step(p, planes, P)  # warm
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.step(p, planes, P)
    el = time.perf_counter() - t0
    return sample_particles * steps / el, el, planes


def _oracle_worker(planes_path, sample, lo, hi, steps, barrier, out):
    """One process of the all-cores baseline: packets [lo, hi) of the sample."""
    import numpy as np
    import oracle
    import rsol_inputs as ri
    planes = np.load(planes_path, mmap_mode="r")
    parts = ri.make_particles(sample, GRID, SEED)
    parts = {k: np.ascontiguousarray(v[..., lo:hi]) for k, v in parts.items()}
    p = oracle.params(GRID, shape=2, dt=0.2 / C_TILDE, c=C, c_tilde=C_TILDE)
    P = oracle.Particles(parts)
    oracle.step(p, planes, P)  # warm
    barrier.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.step(p, planes, P)
    out.put((t0, time.perf_counter()))


def cpu_baseline_all_cores(per_core: int, steps: int, planes):
    """The same oracle on every host core: one spawned process per core, each
    stepping its own share of the sample (its own feedback grid); wall time from
    the first start to the last finish.  Returns (packet-steps/s, seconds, cores)."""
    import multiprocessing as mp
    import tempfile
    import numpy as np
    workers = os.cpu_count() or 1
    sample = per_core * workers
    ctx = mp.get_context("spawn")
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "planes.npy")
        np.save(path, planes)
        barrier, out = ctx.Barrier(workers), ctx.Queue()
        procs = [ctx.Process(target=_oracle_worker,
                             args=(path, sample, w * per_core, (w + 1) * per_core, steps, barrier, out))
                 for w in range(workers)]
        for pr in procs:
            pr.start()
        res = [out.get() for _ in procs]
        for pr in procs:
            pr.join()
    wall = max(t1 for _, t1 in res) - min(t0 for t0, _ in res)
    return sample * steps / wall, wall, workers


def row_bench(workload: str, args) -> dict:
    """One of the widened rows' benchmarks (GPU timing from the package's own
    benchmark module) with the oracle timed beside it on a bounded sample."""
    import numpy as np
    import oracle
    import rsol_inputs as ri
    oracle.build()
    if workload == "gradient":
        from paper_2111_14704_gb300 import grad_bench
        r = grad_bench.run(["--reps", "3"])
        g = (64, 64, 64)
        n, steps = 1 << 18, 32  # about 10 s of oracle work
        parts = ri.make_particles(n, g, 4)
        modes = ri.alfven_modes(64, 4, L=(64.0,) * 3, kmax=16, dB_rms=0.1)
        F = ri.field_grid(g, modes=modes, vA=1e-4)
        p = oracle.params(g, shape=2, dt=2.0, c=1.0, c_tilde=0.1)
        dF = np.random.default_rng(0).standard_normal(F.shape)
        t0 = time.perf_counter()
        oracle.tangent(p, F, dF, oracle.Particles(parts), steps=steps)
        el = time.perf_counter() - t0
        value, unit = r["graph_packet_steps_per_s"] or r["packet_steps_per_s"], "packet-steps/s"
        metric = ("differentiable run: packet-steps/s (64^3, 2^20 packets, 64 steps, gradient w.r.t. "
                  "fields and 64 amplitudes; the call replayed from a CUDA graph)")
        cpu = {"value": n * steps / el, "unit": unit, "cores": 1, "kind": "oracle",
               "sample": f"{n} packets x {steps} steps of the workload, forward-mode tangent along one "
                         f"field direction (static fields), {el:.1f} s"}
    elif workload == "subcycle":
        from paper_2111_14704_gb300 import subcycle_bench
        r = subcycle_bench.run(["--reps", "3"])
        n = 1 << 20  # about 10 s of oracle work
        parts = ri.make_particles(n, GRID, SEED)
        modes = ri.alfven_modes(N_MODES, SEED, L=tuple(float(x) for x in GRID), kmax=KMAX, dB_rms=DB_RMS)
        F = ri.field_grid(GRID, modes=modes, vA=VA)
        p = oracle.params(GRID, shape=2, dt=1.0 / C_TILDE, c=C, c_tilde=C_TILDE)
        t0 = time.perf_counter()
        oracle.step_subcycled(p, F, oracle.Particles(parts), 0.2)
        el = time.perf_counter() - t0
        value, unit = r["tiled_packet_substeps_per_s"] / r["mean_substeps_per_packet"], "packet-steps/s"
        metric = "sub-cycled global step (c~ dt = dx, C = 0.2): packet-steps/s, tiled kernel"
        cpu = {"value": n / el, "unit": unit, "cores": 1, "kind": "oracle",
               "sample": f"{n} packets x 1 sub-cycled global step of the workload, {el:.1f} s"}
    else:
        from paper_2111_14704_gb300 import batch_bench
        r = batch_bench.run(["--loop", "1"])
        nb, nsteps = 64, 4  # the first 64 boxes in full, about 10 s of oracle work
        sh = ri.batch_boxes(nb, 5)
        done, el = 0, 0.0
        for b in range(nb):
            e = int(sh["edge"][b])
            parts = ri.make_particles(int(sh["count"][b]), (e, e, e), 5 + b)
            modes = ri.alfven_modes(64, 5 + b, L=(float(e),) * 3, kmax=min(16, e // 2),
                                    dB_rms=float(sh["dB_rms"][b]))
            F = ri.field_grid((e, e, e), modes=modes, vA=1e-4)
            ct = 1.0 / float(sh["c_over_c_tilde"][b])
            p = oracle.params((e, e, e), shape=2, dt=0.2 / ct, c=1.0, c_tilde=ct)
            P = oracle.Particles(parts)
            t0 = time.perf_counter()
            for _ in range(nsteps):
                oracle.step(p, F, P)
            el += time.perf_counter() - t0
            done += parts["w"].shape[0] * nsteps
        value, unit = r["graph_packet_steps_per_s"], "packet-steps/s"
        metric = "batched boxes (512 boxes, steps replayed from a CUDA graph): packet-steps/s"
        cpu = {"value": done / el, "unit": unit, "cores": 1, "kind": "oracle",
               "sample": f"first {nb} boxes ({done // nsteps} packets) x {nsteps} steps, {el:.1f} s"}
    return {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic", "config": {"workload": r["workload"]},
            "cpu_baseline": cpu, "details": r}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rsol", choices=["rsol", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--cpu-sample", type=int, default=1 << 18)
    ap.add_argument("--cpu-steps", type=int, default=12)
    ap.add_argument("--cpu-per-core", type=int, default=1 << 16,
                    help="packets per host core for the all-cores oracle baseline (0: skip)")
    ap.add_argument("--loss-reps", type=int, default=10)
    ap.add_argument("--workload", default="push", choices=["push", "gradient", "subcycle", "batch"],
                    help="push: the headline fused step (default); the others time a widened "
                         "row with the oracle beside it and print their own JSON line")
    ap.add_argument("--sweep-steps", type=int, default=40,
                    help="timed steps of the same workload at c/c~ = 1 and 100 (0: skip)")
    ap.add_argument("--config3-steps", type=int, default=8,
                    help="timed steps of the 256^3, 2^27-packet beam workload (0: skip)")
    ap.add_argument("--grid", default=None,
                    help="nx,ny,nz of a smaller push workload (profiling captures); default 128^3")
    ap.add_argument("--particles", type=int, default=None,
                    help="packets of a smaller push workload (profiling captures); default 2^24")
    args = ap.parse_args()
    global GRID, N_PARTICLES
    if args.grid:
        GRID = tuple(int(v) for v in args.grid.split(","))
    if args.particles:
        N_PARTICLES = args.particles
    if args.workload != "push":
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(row_bench(args.workload, args)), flush=True)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    config = {"workload": f"{'x'.join(map(str, GRID))} periodic grid, 64 Alfven modes (dB/B0=0.1, "
                          f"|n|<=16, vA=1e-4c), {N_PARTICLES} packets, power-law |u| in [1,100] "
                          "(p^-4.5), c/c~=10, TSC, FP32",
              "grid": list(GRID), "particles": N_PARTICLES, "shape": "TSC", "c_over_c_tilde": 10,
              "sort_every": SORT_EVERY, "moments_every": MOMENTS_EVERY,
              "bin_and_warps": "autotuned (see the autotune key)",
              "l2": "inputs larger than L2 (packet arrays 2 x 512 MB), no flush",
              "parallelism": f"replicas x{args.gpus}"}

    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        oracle.build()
        import rsol_inputs as ri
        # size the per-step sample so that the K timed steps take about a minute
        probe = ri.make_particles(4096, GRID, SEED)
        modes_p = ri.alfven_modes(N_MODES, SEED, L=tuple(float(g) for g in GRID), kmax=KMAX,
                                  dB_rms=DB_RMS)
        planes_p = ri.field_grid(GRID, modes=modes_p, vA=VA, c=C)
        pp = oracle.params(GRID, shape=2, dt=0.2 / C_TILDE, c=C, c_tilde=C_TILDE)
        tp = time.perf_counter()
        oracle.step(pp, planes_p, oracle.Particles(probe))
        rate = 4096 / max(time.perf_counter() - tp, 1e-6)
        sample = int(min(args.cpu_sample, max(1024, rate * 60.0 / max(args.steps, 1))))
        parts = ri.make_particles(sample, GRID, SEED)
        planes = planes_p
        dt = 0.2 / C_TILDE
        p = pp
        P = oracle.Particles(parts)
        for _ in range(args.warmup):
            oracle.step(p, planes, P)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle.step(p, planes, P)
        el = time.perf_counter() - t0
        v = sample * args.steps / el
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": el * 1e3 / args.steps * (N_PARTICLES / sample),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"{sample} packets of the workload per step, fields held "
                                           "at t=0, single-threaded FP64 C oracle"},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2111_14704_gb300 as rs
    rs.load_library()

    from paper_2111_14704_gb300.replicas import job_throughput, reduce_max
    r = run_gpu(args, rank, world)
    ms_max, e2e_max = reduce_max([r["ms"], r["e2e_s"]], world, device="cuda")
    ms_per_step = ms_max / args.steps
    value = job_throughput(world, N_PARTICLES, args.steps, ms_max)
    push_avg = statistics.mean(r["push_ms"])
    n_nodes = GRID[0] * GRID[1] * GRID[2]
    alg_bytes = BYTES_PER_PACKET * N_PARTICLES + BYTES_PER_NODE * n_nodes
    achieved = alg_bytes / (push_avg * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = None
    issue = None
    if NCU_TRAFFIC_PER_PACKET is not None and NCU_SOURCE_HASH == kernel_source_hash():
        traffic = NCU_TRAFFIC_PER_PACKET * N_PARTICLES
        sm_mhz = r["clocks"].get("sm_mhz")
        if sm_mhz:
            # the kernel is bound by instruction issue, not HBM: the same launches
            # against the issue peak at the clock sampled during the timed steps
            inst_rate = NCU_INST_PER_PACKET * N_PARTICLES / (push_avg * 1e-3)
            issue_peak = ISSUE_SCHEDULERS * sm_mhz * 1e6
            issue = {"achieved": inst_rate, "peak": issue_peak, "unit": "warp-instructions/s",
                     "frac": inst_rate / issue_peak,
                     "note": "ncu warp instructions per packet of the first push after a sort "
                             f"({NCU_INST_PER_PACKET:.1f}) x packets / mean push time; peak = "
                             "152 SMs x 4 schedulers x sampled SM clock"}
    e2e_value = job_throughput(world, N_PARTICLES, r["e2e_steps"], e2e_max * 1e3)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "rsol_push_gather (fused gather+Boris+deposit+drift)",
                         "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": push_avg,
                         "peak_source": f"{peak_kind} hbm_gbs", "issue": issue},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": r["field_bytes"],
                    "d2h_bytes_per_step": r["fb_bytes"],
                    "note": "fields copied in from pinned host memory and the feedback grid "
                            "copied out to pinned host memory every step, on copy streams "
                            "overlapping the push (double-buffered); packets stay resident"},
            "gpu_launches": r["launches"], "clocks": r["clocks"],
            "push_only": {"value": N_PARTICLES / (push_avg * 1e-3), "ms": push_avg},
            "state_moment_deposit_ms": r["deposit_ms"],
            "step_breakdown_ms": {**{k: round(v, 4) for k, v in r["breakdown"].items()},
                                  "note": f"device time per step: field source + feedback zeroing, "
                                          f"fused push, sort every {SORT_EVERY} steps, state "
                                          f"moments + FP64 totals every {MOMENTS_EVERY} steps "
                                          f"(amortised)"},
            "fp64": r["fp64"], "losses": r["losses"], "c_sweep": r["sweep"],
            "autotune": r["autotune"]}
    if args.config3_steps > 0 and world == 1:
        line["config3"] = run_config3(args)
    if rank == 0 and world == 1:
        v, el, planes = cpu_baseline(args.cpu_sample, args.cpu_steps)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{args.cpu_sample} packets x {args.cpu_steps} steps of "
                                          f"the workload (fields at t=0), {el:.1f} s"}
        if args.cpu_per_core > 0:
            va, ela, cores = cpu_baseline_all_cores(args.cpu_per_core, args.cpu_steps, planes)
            line["cpu_baseline_all_cores"] = {
                "value": va, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"{args.cpu_per_core} packets per core x {args.cpu_steps} steps of the "
                          f"workload (fields at t=0), one process per core, {ela:.1f} s wall"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
