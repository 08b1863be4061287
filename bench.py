#!/usr/bin/env python
"""Benchmark of the signature-kernel Gram workload on GB300.

Workload (one step): the Gram matrices of B = 64 Brownian paths with 1024
segments in R^16, increments N(0, sigma^2/1024), for sigma = 1 and sigma = 4
(seeds 2001 / 2004) -- 2 x 2080 unique pairs x 1024^2 tiles.  Metric: tile
cells per second, cells = sum over computed pairs of L1*L2 (the lower
triangle is mirrored, not recomputed, and is not counted).

Output: one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload instead (the reference arm of this
build; there is no other implementation of the method to run).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_PATHS, N_SEG, DIM = 64, 1024, 16
SIGMAS = ((1.0, 2001, 8, 4), (4.0, 2004, 16, 6))   # sigma, seed, order P, rings
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x FMA x max clock
L2_FLUSH_BYTES = 512 << 20
ORACLE_SAMPLE_PAIRS = 16


METRIC = ("fwd & fwd+bwd sig-kernel cells/s (pairs*L1*L2/s), Gram B=64 L=1024 d=16 "
          "sigma in {1,4}")


def tile_flops(P: int, nr: int, d: int) -> int:
    """FP32 operations per tile of the solver (FMA = 2), as executed: the
    increment inner product (2d), the ring powers, the Hankel sums of both
    edges, the edge evaluation, the convolutions and the float-float corner."""
    nrm = min(P, 8)
    nr = min(nr, nrm)
    f = 2 * (nr - 1)
    f += sum(2 * (1 + 2 * (P - p)) for p in range(1, nr + 1))
    f += 2 * P
    for p in range(1, P + 1):
        f += 4 * min(p - 1, nr) + (4 if p <= nr else 0)
    f += 10 + 18  # float-float corner; compensated first-order coefficients
    return f + 2 * d


def adjoint_tile_flops(P: int, nr: int, d: int, replay: bool = True) -> int:
    """FP32 operations per tile of the adjoint kernel (FMA = 2): in pass B the
    increment dot, the inverse bottom-edge update, the tile adjoint and the
    two gradient FMAs; with `replay`, also pass A's forward replay
    (tile_flops), which is skipped when the forward stored the tile records."""
    nrm = min(P, 8)
    nr = min(nr, nrm)
    inv = 2 * (nr - 1) + sum(2 * (1 + 2 * (P - p)) for p in range(1, nr + 1))
    inv += sum(2 * min(p - 1, nr) + (2 if p <= nr else 0) for p in range(1, P + 1))
    adj = 2 * (nr - 1) + sum(2 * (1 + 2 * (P - p)) for p in range(1, nr + 1))  # hb
    adj += sum(4 * (P - m) + 6 for m in range(1, nr + 1))                     # chb, cbar
    adj += 2 * nr                                                              # hab, hbb
    for s_ in range(1, P + 1):
        adj += 4 * min(nr, P - s_) + 2 + 4 * min(nr, P - s_)                   # conv^T, S, Hankel^T
    adj += 2 * nr
    return (tile_flops(P, nr, d) if replay else 0) + 2 * d + inv + adj + 4 * d


def rank_workloads(rank: int, n_paths: int):
    """The batches rank `rank` solves: the Gram workload with per-rank seeds
    (independent problems per GPU: weak scaling, no data-path collective)."""
    from paper_2502_20392_gb300 import synth
    return [synth.workload_gram_1024(s, seed + 1000 * rank, n_paths=n_paths) for s, seed, _, _ in SIGMAS]


def max_over_ranks(x: float, device, dist) -> float:
    """Max of a per-rank time over the process group (the job's time is the
    slowest rank's)."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def pairs_of_gram(n):
    return n * (n + 1) // 2


def cells_per_step():
    return len(SIGMAS) * pairs_of_gram(N_PATHS) * N_SEG * N_SEG


BWD_SIGMA = 0  # index into SIGMAS of the Gram whose adjoint is part of the step


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in rows for k in range(4) if r[2 + k] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


def oracle_sample(pts_lens, n_pairs):
    """FP64 oracle on the first n_pairs upper-triangle pairs (a, b) of each
    Gram; returns (values per sigma, seconds, threads)."""
    import numpy as np

    import oracle
    from paper_2502_20392_gb300 import synth
    oracle.build()
    out, t0 = [], time.perf_counter()
    for pts, lens in pts_lens:
        inc = [np.diff(p.astype(np.float64), axis=0) for p in synth.split(pts, lens)]
        idx = [(a, b) for a in range(N_PATHS) for b in range(a, N_PATHS)][:n_pairs]
        xs = [inc[a] for a, _ in idx]
        ys = [inc[b] for _, b in idx]
        out.append((idx, oracle.series_pairs(xs, ys)))
    return out, time.perf_counter() - t0, oracle.num_threads()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", default="full", choices=["full", "small"],
                    help="small: 16 paths per Gram (for ncu captures; not a bench line)")
    ap.add_argument("--sweep", default=None, choices=["roughness", "dimension", "length", "configs"],
                    help="print one JSON line per point of a sweep instead of the bench line")
    args = ap.parse_args()
    if args.sweep:
        return run_sweep(args)
    if args.case == "small":
        global N_PATHS
        N_PATHS = 16

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2502_20392_gb300 import build, sigk, synth
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    sigk.load()

    # each rank solves its own batch (independent problems: weak scaling)
    host = rank_workloads(rank, N_PATHS)
    X = [torch.from_numpy(p).to(dev) for p, _ in host]
    L = [torch.from_numpy(l).to(dev) for _, l in host]
    opts = [sigk.Opts(order=P, rings=nr, max_len=N_SEG) for _, _, P, nr in SIGMAS]
    wss = [sigk.Workspace() for _ in SIGMAS]
    G = [torch.empty((N_PATHS, N_PATHS), dtype=torch.float64, device=dev) for _ in SIGMAS]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # upstream gradient of the Gram in the adjoint (a fixed dense weighting)
    W = torch.from_numpy(np.random.default_rng(7).standard_normal((N_PATHS, N_PATHS))).to(dev)
    bws = sigk.Workspace()

    def step(ev_pairs=None, pts=X, lens=L):
        # the Gram whose gradient is taken runs as a training forward (it keeps
        # its seams and tile records for the adjoint, as an autograd forward
        # does); the other as an inference forward; then the adjoint
        state = None
        for k in range(len(SIGMAS)):
            if ev_pairs is not None:
                sigk.profile_events(*ev_pairs[k])
            if k == BWD_SIGMA:
                _, state = sigk.forward_train(sigk.OP_GRAM, pts[k], lens[k], None, None, opts[k],
                                              ws=bws, out=G[k], check=False)
            else:
                sigk.gram(pts[k], lens[k], opts=opts[k], out=G[k], ws=wss[k], check=False)
        if ev_pairs is not None:
            sigk.profile_events(*ev_pairs[len(SIGMAS)])
        gX, _ = sigk.adjoint(state, W, need_y=False, check=False)
        if ev_pairs is not None:
            sigk.profile_events(None, None)
        return gX

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for ws in wss:
        sigk.sync_status(ws)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(len(SIGMAS) + 1)] for _ in range(args.steps)]
    for row in kev:  # torch creates an event on first record: do it before handing out handles
        for a, b in row:
            a.record()
            b.record()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))  # evict the inputs from L2 (outside the timed span)
            starts[i].record()
            step(kev[i])
            ends[i].record()
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    for ws in wss + [bws]:
        sigk.sync_status(ws)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    kern_ms = [[a.elapsed_time(b) for a, b in row] for row in kev]
    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        ms = max_over_ranks(ms, dev, dist)

    cells = cells_per_step()
    value = cells * world / (ms * 1e-3)

    # counters of the last launch of each sigma (tiles actually solved)
    bcnt = sigk.counters(bws)
    tiles = [bcnt[0] if k == BWD_SIGMA else sigk.counters(wss[k])[0] for k in range(len(SIGMAS))]

    # roofline of the solver kernel (dominant: the sigma = 4, P = 16 launch)
    roof = []
    for k, (sg, _, P, nr) in enumerate(SIGMAS):
        kms = statistics.mean(r[k] for r in kern_ms)
        flops = tiles[k] * tile_flops(P, nr, DIM)
        ach = flops / (kms * 1e-3) / 1e12
        roof.append({"sigma": sg, "order": P, "rings": nr, "kernel_ms": round(kms, 4),
                     "kernel": (f"fwd_kernel<P={P},D=16> (training: stores the tile records)"
                                if k == BWD_SIGMA else f"fwd_kernel<P={P},D=16>"),
                     "flops_per_launch": flops, "achieved": round(ach, 3)})
    sg, _, P, nr = SIGMAS[BWD_SIGMA]
    kms = statistics.mean(r[len(SIGMAS)] for r in kern_ms)
    # pass B over every tile, pass A over the replayed ones (none when the
    # training forward stored the tile records)
    flops = bcnt[2] * adjoint_tile_flops(P, nr, DIM, replay=False) + bcnt[3] * tile_flops(P, nr, DIM)
    roof.append({"sigma": sg, "order": P, "rings": nr, "kernel": "bwd_kernel (adjoint)",
                 "kernel_ms": round(kms, 4), "flops_per_launch": flops,
                 "achieved": round(flops / (kms * 1e-3) / 1e12, 3)})
    dom = max(range(len(roof)), key=lambda k: roof[k]["kernel_ms"])
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(tpath) as f:
            tj = json.load(f)
        with open(os.path.join(ROOT, "paper_2502_20392_gb300", "_build", "libsigk.sha256")) as f:
            digest = f.read().strip()
        if tj.get("digest") == digest:
            traffic = tj.get("bytes_per_launch")
    except (OSError, ValueError):
        traffic = None
    roofline = {"bound": "alu", "achieved": roof[dom]["achieved"], "peak": round(FP32_PEAK_TFLOPS, 2),
                "unit": "TFLOP/s", "frac": round(roof[dom]["achieved"] / FP32_PEAK_TFLOPS, 4),
                "traffic": traffic,
                "kernel": roof[dom].get("kernel", f"fwd_kernel<P={roof[dom]['order']},D=16>"),
                "per_launch": roof}
    fwd_ms = sum(statistics.mean(r[k] for r in kern_ms) for k in range(len(SIGMAS)))

    # end-to-end through the public API: pinned host inputs -> device, both
    # Gram calls, Gram matrices -> pinned host, every step
    h_pts = [torch.from_numpy(p).pin_memory() for p, _ in host]
    h_len = [torch.from_numpy(l).pin_memory() for _, l in host]
    h_out = [torch.empty((N_PATHS, N_PATHS), dtype=torch.float64).pin_memory() for _ in SIGMAS]
    d_pts = [torch.empty_like(x) for x in X]
    d_len = [torch.empty_like(x) for x in L]
    h_grad = torch.empty_like(h_pts[BWD_SIGMA]).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in h_pts + h_len)
    d2h = sum(t.numel() * t.element_size() for t in h_out + [h_grad])
    e_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        e_s[i].record()
        for k in range(len(SIGMAS)):
            d_pts[k].copy_(h_pts[k], non_blocking=True)
            d_len[k].copy_(h_len[k], non_blocking=True)
        gX = step(pts=d_pts, lens=d_len)
        for k in range(len(SIGMAS)):
            h_out[k].copy_(G[k], non_blocking=True)
        h_grad.copy_(gX, non_blocking=True)
        e_e[i].record()
    torch.cuda.synchronize()
    for ws in wss + [bws]:
        sigk.sync_status(ws)
    e2e_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(e_s, e_e))
    if world > 1:
        e2e_ms = max_over_ranks(e2e_ms, dev, dist)

    line = {
        "metric": METRIC,
        "value": value,
        "fwd_only": {"value": cells * world / (fwd_ms * 1e-3), "unit": "cells/s",
                     "ms": fwd_ms, "note": "forward solver kernels of both Grams alone"}, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (float-float corner, f64 reductions)",
        "data": "synthetic (seeded Brownian, PCG64)",
        "config": {"workload": "gram_B64_L1024_d16_sigma1+4", "paths": N_PATHS, "segments": N_SEG,
                   "d": DIM, "sigmas": [s for s, *_ in SIGMAS],
                   "order_rings": [[P, nr] for _, _, P, nr in SIGMAS],
                   "unique_pairs_per_gram": pairs_of_gram(N_PATHS), "l2": "flushed between steps",
                   "step": "forward Gram (sigma 1 and 4; sigma 1 as the training forward "
                           "that keeps the adjoint's state) + adjoint of the sigma=1 Gram "
                           "(upstream: fixed dense weights)",
                   "parallelism": f"independent batch per rank x{world}"},
        # per step: planner + solver for each Gram, adjoint set-up + adjoint
        "gpu_launches": (2 * len(SIGMAS) + 2) * args.steps,
        "clocks": clk.summary(),
        "e2e": {"value": cells * world / (e2e_ms * 1e-3), "unit": "cells/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "roofline": roofline,
        "wall_s": t_wall,
    }

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        host_G = [g.cpu().numpy() for g in G]
        vals, secs, thr = oracle_sample(host, ORACLE_SAMPLE_PAIRS)
        errs = []
        for (idx, ref), Gk in zip(vals, host_G):
            for (a, b), r in zip(idx, ref):
                e = abs(Gk[a, b] - r) / max(abs(r), 1e-300)
                cs_scale = (abs(Gk[a, a] * Gk[b, b])) ** 0.5
                if abs(r) < 1e-2 * cs_scale:  # near-zero cross entry: Cauchy-Schwarz scale
                    e = min(e, abs(Gk[a, b] - r) / cs_scale)
                errs.append(e)
        n_cells = sum(len(idx) for idx, _ in vals) * N_SEG * N_SEG
        line["cpu_baseline"] = {"value": n_cells / secs, "unit": "cells/s", "cores": thr,
                                "kind": "oracle",
                                "sample": f"first {ORACLE_SAMPLE_PAIRS} upper-triangle pairs of each "
                                          f"Gram ({n_cells:.3e} cells), FP64 tile series N=24, "
                                          f"OpenMP over pairs, {secs:.1f} s"}
        line["rel_err_vs_oracle_sample"] = max(errs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_sweep(args):
    """Throughput over the sweeps that widen the tested range (one GPU, forward
    solve with the plan's options; CUDA events around the solve, after
    warm-up).  roughness: 4096 pairs of 2-D fBM paths of 51 points, H from 0.4
    down to 0.005, FP32 and FP64; dimension: a Gram of 16 Brownian paths of
    512 segments, d = 2 .. 8192; length: one 2-D Brownian self-kernel of
    2^k + 1 points (k = 10 .. 19), with the workspace bytes (O(L))."""
    import json

    import numpy as np
    import torch

    from paper_2502_20392_gb300 import build, sigk, synth
    build.build()
    sigk.load()
    dev = torch.device("cuda", 0)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def emit(**kw):
        print(json.dumps(kw), flush=True)

    if args.sweep == "roughness":
        for H in (0.4, 0.2, 0.1, 0.05, 0.01, 0.005):
            X, lx = synth.fbm(4096, 50, 2, H, seed=6000 + int(H * 1000))
            Y, ly = synth.fbm(4096, 50, 2, H, seed=7000 + int(H * 1000))
            a = [torch.from_numpy(v).to(dev) for v in (X, lx, Y, ly)]
            for flags in (0, sigk.FLAG_FP64):
                o = sigk.plan(sigk.OP_PAIRS, *a, tol=1e-5, opts=sigk.Opts(max_len=4096, flags=flags))
                ws = sigk.Workspace()
                ms = timed(lambda: sigk.pairs(*a, opts=o, ws=ws, check=False))
                emit(sweep="roughness", hurst=H, precision="fp64" if flags else "fp32",
                     metric="cells/s", value=4096 * 2500 / (ms * 1e-3), ms=ms,
                     opts=dict(order=o.order, rings=o.rings, refine_c=o.refine_c, max_len=o.max_len))
    elif args.sweep == "dimension":
        for d in (2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192):
            pts, lens = synth.brownian(16, 512, d, 1.0, seed=8000 + d)
            X, L = torch.from_numpy(pts).to(dev), torch.from_numpy(lens).to(dev)
            o = sigk.plan(sigk.OP_GRAM, X, L, None, None, tol=1e-6, opts=sigk.Opts(max_len=513))
            ws = sigk.Workspace()
            ms = timed(lambda: sigk.gram(X, L, opts=o, ws=ws, check=False))
            cells = 136 * 512 * 512
            emit(sweep="dimension", d=d, metric="cells/s", value=cells / (ms * 1e-3), ms=ms,
                 kernel="register" if d <= 16 else "two-phase",
                 opts=dict(order=o.order, rings=o.rings, refine_c=o.refine_c))
    elif args.sweep == "configs":
        run_configs(timed, emit, dev)
    else:
        for k in range(10, 20):
            n = 2 ** k
            pts, lens = synth.brownian(1, n, 2, 1.0, seed=9000 + k)
            X, L = torch.from_numpy(pts).to(dev), torch.from_numpy(lens).to(dev)
            o = sigk.Opts(order=8, rings=4, max_len=n + 1)
            ws = sigk.Workspace()
            ms = timed(lambda: sigk.pairs(X, L, X, L, opts=o, ws=ws, check=False), reps=1)
            emit(sweep="length", points=n + 1, metric="cells/s", value=n * n / (ms * 1e-3), ms=ms,
                 workspace_bytes=int(sigk.workspace_size(sigk.OP_PAIRS, 1, 1, 2, o)),
                 opts=dict(order=8, rings=4))
    return 0


def run_configs(timed, emit, dev):
    """Throughput (and the accuracy checks that are cheap on the host) for the
    five workloads: a 256-segment pair (d=4), the Gram B=64 (both sigmas), a
    pair of 10^6-segment paths (collinear, against I0(2 sqrt(<X,Y>)), and
    Brownian), 512 ragged pairs with d=256 (FP32 and FP64), and the MMD of
    2 x 32 paths of 2048 segments with its gradient."""
    import math

    import numpy as np
    import torch
    from scipy.special import i0

    import oracle
    from paper_2502_20392_gb300 import sigk, synth

    def t(a):
        return torch.from_numpy(a).to(dev)

    def oracle_rate(xs, ys, N=24):
        """FP64 oracle (series, OpenMP over pairs) on a bounded sample: cells/s."""
        t0 = time.perf_counter()
        oracle.series_pairs(xs, ys, N=N)
        secs = time.perf_counter() - t0
        cells = float(sum(len(x) * len(y) for x, y in zip(xs, ys)))
        return {"value": cells / secs, "unit": "cells/s", "cores": oracle.num_threads(),
                "kind": "oracle", "sample_cells": cells, "seconds": secs}

    def incs(pts, lens):
        return [np.diff(p.astype(np.float64), axis=0) for p in synth.split(pts, lens)]

    oracle.build()

    # pair 256, d=4
    pts, lens = synth.workload_pair_256()  # two packed paths: x, y
    xs = synth.split(pts, lens)
    X, lx = synth.pack(xs[:1])
    Y, ly = synth.pack(xs[1:])
    a = [t(v) for v in (X, lx, Y, ly)]
    o = sigk.plan(sigk.OP_PAIRS, *a, tol=1e-6, opts=sigk.Opts(max_len=257))
    ws = sigk.Workspace()
    ms = timed(lambda: sigk.pairs(*a, opts=o, ws=ws, check=False))
    k = sigk.pairs(*a, opts=o, ws=ws).item()
    r = oracle.series_pair(np.diff(X.astype(np.float64), axis=0), np.diff(Y.astype(np.float64), axis=0))
    # the same call captured in a CUDA graph (no host work per replay)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    sigk.pairs(*a, opts=o, out=out, ws=ws)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            sigk.pairs(*a, opts=o, out=out, ws=ws, check=False)
    torch.cuda.current_stream().wait_stream(side)
    ms_g = timed(graph.replay, reps=20)
    emit(config="pair_L256_d4", metric="cells/s", value=256 * 256 / (ms * 1e-3), ms=ms,
         graph={"value": 256 * 256 / (ms_g * 1e-3), "ms": ms_g},
         rel_err_vs_oracle=abs(k - r) / abs(r),
         cpu_baseline=oracle_rate(incs(X, lx) * 32, incs(Y, ly) * 32))
    # Gram B=64 L=1024 d=16, sigma 1 and 4 (forward)
    for sg in (1.0, 4.0):
        pts, lens = synth.workload_gram_1024(sg)
        Xd, Ld = t(pts), t(lens)
        o = sigk.plan(sigk.OP_GRAM, Xd, Ld, None, None, tol=1e-5, opts=sigk.Opts(max_len=1025))
        ws = sigk.Workspace()
        ms = timed(lambda: sigk.gram(Xd, Ld, opts=o, ws=ws, check=False))
        zs = incs(pts, lens)
        emit(config=f"gram_B64_L1024_d16_sigma{sg:g}", metric="cells/s",
             value=2080 * 1024 * 1024 / (ms * 1e-3), ms=ms, opts=dict(order=o.order, rings=o.rings),
             cpu_baseline=oracle_rate([zs[0]] * 16, zs[:16]))
    # 10^6-segment pairs (increments), collinear against the closed form
    inc, segs, u, tot = synth.collinear_increments(1_000_000, 8, seed=3002, n_paths=2)
    Xd, Ld = t(inc), t(segs)
    o = sigk.Opts(order=4, rings=2, flags=sigk.FLAG_INCREMENTS, max_len=1_000_000)
    ws = sigk.Workspace()
    n = 1_000_000
    ms = timed(lambda: sigk.pairs(Xd[:n], Ld[:1], Xd[n:], Ld[1:], opts=o, ws=ws, check=False), reps=1)
    k = sigk.pairs(Xd[:n], Ld[:1], Xd[n:], Ld[1:], opts=o, ws=ws).item()
    ref = i0(2 * math.sqrt(float(u @ u) * tot[0] * tot[1]))
    emit(config="long_pair_1e6_d8_collinear", metric="cells/s", value=1e12 / (ms * 1e-3), ms=ms,
         rel_err_vs_closed_form=abs(k - ref) / ref, workspace_bytes=int(ws.buf.numel()))
    inc, segs = synth.workload_long_pair()
    Xd, Ld = t(inc), t(segs)
    o = sigk.Opts(order=8, rings=4, flags=sigk.FLAG_INCREMENTS, max_len=1_000_000)
    ws = sigk.Workspace()
    ms = timed(lambda: sigk.pairs(Xd[:n], Ld[:1], Xd[n:], Ld[1:], opts=o, ws=ws, check=False), reps=1)
    pre = [inc[:3000].astype(np.float64), inc[n:n + 3000].astype(np.float64)]
    emit(config="long_pair_1e6_d8_brownian", metric="cells/s", value=1e12 / (ms * 1e-3), ms=ms,
         workspace_bytes=int(ws.buf.numel()),
         cpu_baseline=dict(oracle_rate([pre[0]], [pre[1]], N=8), sample="3000-segment prefix pair (one thread: the oracle parallelises over pairs)"))
    # 512 ragged pairs, d=256
    (X, lx), (Y, ly) = synth.workload_ragged_512()
    a = [t(v) for v in (X, lx, Y, ly)]
    cells = float(((lx - 1) * (ly - 1)).sum())
    short = [p for p in np.argsort((lx - 1) * (ly - 1))[:8]]
    xs4, ys4 = incs(X, lx), incs(Y, ly)
    cpu4 = oracle_rate([xs4[p] for p in short], [ys4[p] for p in short])
    for flags, name in ((0, "fp32"), (sigk.FLAG_FP64, "fp64")):
        o = sigk.plan(sigk.OP_PAIRS, *a, tol=1e-5, opts=sigk.Opts(max_len=8193, flags=flags))
        ws = sigk.Workspace()
        ms = timed(lambda: sigk.pairs(*a, opts=o, ws=ws, check=False), reps=1)
        emit(config=f"ragged_512_d256_{name}", metric="cells/s", value=cells / (ms * 1e-3), ms=ms,
             opts=dict(order=o.order, rings=o.rings, refine_c=o.refine_c, max_len=o.max_len),
             cpu_baseline=dict(cpu4, sample="the 8 pairs of fewest cells"))
    # MMD 2 x 32 x 2048, d=8: value, then value + gradient
    (X, lx), (Y, ly) = synth.workload_mmd_2048()
    a = [t(v) for v in (X, lx, Y, ly)]
    o = sigk.Opts(order=6, rings=4, max_len=2048)
    ws, bws = sigk.Workspace(), sigk.Workspace()
    cells = 64 * 65 / 2 * 2048 * 2048
    one = torch.ones(1, dtype=torch.float64)
    ms_f = timed(lambda: sigk.mmd(*a, opts=o, ws=ws, check=False))
    ms_b = timed(lambda: sigk.backward(sigk.OP_MMD, *a, one, o, ws=bws, check=False))
    zx, zy = incs(X, lx), incs(Y, ly)
    emit(config="mmd_2x32_L2048_d8", metric="cells/s", value=cells / (ms_f * 1e-3), ms=ms_f,
         fwd_bwd={"value": cells / (ms_b * 1e-3), "ms": ms_b},
         cpu_baseline=dict(oracle_rate(zx[:16], zy[:16], N=12), sample="16 cross pairs"))


def run_reference(args, world, rank):
    """Reference arm: the FP64 oracle, timed as it stands on the host cores, on
    a bounded sample of the workload per step (rank 0 only)."""
    if rank != 0:
        return
    from paper_2502_20392_gb300 import synth
    host = [synth.workload_gram_1024(s, seed) for s, seed, _, _ in SIGMAS]
    per_step = max(1, ORACLE_SAMPLE_PAIRS // 4)
    for _ in range(args.warmup):
        oracle_sample(host, 1)
    times = []
    thr = 1
    for _ in range(args.steps):
        _, secs, thr = oracle_sample(host, per_step)
        times.append(secs)
    n_cells = len(SIGMAS) * per_step * N_SEG * N_SEG
    v = n_cells / statistics.mean(times)
    line = {"impl": "reference",
            "metric": METRIC,
            "value": v, "unit": "cells/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(times) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Brownian, PCG64)",
            "config": {"workload": "gram_B64_L1024_d16_sigma1+4",
                       "sample": f"{per_step} pairs per sigma per step",
                       "step": "forward only: the FP64 oracle has no adjoint (its gradient is by "
                               "finite differences), so every sampled cell is a forward cell"},
            "cpu_baseline": {"value": v, "unit": "cells/s", "cores": thr, "kind": "oracle",
                             "sample": f"{per_step} upper-triangle pairs per sigma per step, FP64 "
                                       f"tile series N=24, OpenMP over pairs"},
            "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
