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
SIGMAS = ((1.0, 2001, 6, 3), (4.0, 2004, 12, 6))   # sigma, seed, order P, rings (as planned and launched)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x FMA x max clock
L2_FLUSH_BYTES = 512 << 20
ORACLE_SAMPLE_PAIRS = 80   # per sigma: ~10-15 s of FP64 oracle work on 16 host cores
REF_PAIRS_PER_STEP = 16    # reference arm, per sigma and step (at least one per oracle thread)


METRIC = ("fwd & fwd+bwd sig-kernel cells/s (pairs*L1*L2/s), Gram B=64 L=1024 d=16 "
          "sigma in {1,4}")


def launch_order(P: int, nr: int) -> int:
    """Edge degree the FP32 solvers launch with: the truncation keeps entries
    of weighted degree 2m + k <= 2 nr + 1, which reach no degree above 2 nr,
    so a larger order is clamped (the results are the same)."""
    return min(P, 2 * nr)


def keep_entry(P: int, nt: int, nr: int, m: int, k: int) -> bool:
    """The tile-matrix entries the FP32 solvers keep (ring m, offset k)."""
    return 1 <= m <= nr and k >= 0 and m + k <= P and 2 * m + k <= 2 * nt + 1


def kept_entries(P: int, nt: int, nr: int) -> int:
    return sum((1 if k == 0 else 2) for m in range(1, P + 1) for k in range(P + 1)
               if keep_entry(P, nt, nr, m, k))


def useful_tile_fma(P: int, nr: int, d: int) -> int:
    """Algorithmic FMAs of one tile by the work model of the method: the
    increment inner product (d), ring m = 1..n adding 2(P - m) + 1
    multiply-adds into the two outgoing edges (every entry of the square
    truncation of order P), and the 2P additions of the exact transport
    (ring 0).  P is the order the kernel runs with."""
    nr = min(nr, P, 8)
    return d + sum(2 * (P - m) + 1 for m in range(1, nr + 1)) + 2 * P


def kept_tile_fma(P: int, nr: int, d: int) -> int:
    """The same model counting only the entries the truncation keeps."""
    nr = min(nr, P, 8)
    return d + kept_entries(P, nr, nr) + 2 * P


def useful_tile_flops(P: int, nr: int, d: int, adjoint: bool = False) -> int:
    """2 flops per algorithmic FMA; the adjoint counts twice the forward's
    work (recomputation is overhead, not useful work)."""
    return (4 if adjoint else 2) * useful_tile_fma(P, nr, d)


def tile_flops(P: int, nr: int, d: int) -> int:
    """FP32 operations per tile of the solver kernel as executed (FMA = 2): the
    increment inner product (2d), the ring powers, two FMAs per kept entry of
    the tile matrix (one into each outgoing edge) plus one multiply per ring
    for the corner's term, the edge evaluation, the float-float corner and
    the compensated first-order terms (tile_flops in sigk_device.cuh)."""
    nr = min(nr, P, 8)
    f = 2 * (nr - 1) + 2 * nr + 4 * kept_entries(P, nr, nr) + 2 * P + 10 + 18
    return f + 2 * d


def adjoint_tile_flops(P: int, nr: int, d: int, replay: bool = True) -> int:
    """FP32 operations per tile of the adjoint kernel as executed (FMA = 2): the
    coefficient (phase 0, 2d), the inverse bottom-edge update and the tile
    adjoint (pass B), the two contractions of the chain to the increments
    (phase C, 4d); with `replay`, also pass A's forward replay (tile_flops),
    which is skipped when the forward stored the tile records.  K1 counts the
    kept off-diagonal entries on one side of the diagonal."""
    nr = min(nr, P, 8)
    k1 = (kept_entries(P, nr, nr) - nr) // 2
    inv = 2 * (nr - 1) + 3 * nr + 4 * k1
    adj = 2 * (nr - 1) + 14 * nr + 14 * k1 + 2 * P
    return (tile_flops(P, nr, d) if replay else 0) + 2 * d + inv + adj + 4 * d


def sources_digest(files) -> str:
    """SHA-256 over the given source files (paths relative to the repository
    root, each hashed with its path): the identity of the build of a kernel
    whose ncu counters are recorded in profiles/traffic.json."""
    import hashlib
    h = hashlib.sha256()
    for rel in files:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(rel.encode() + b"\0" + f.read())
    return h.hexdigest() if files else ""


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


def sample_pairs(n_pairs, seed):
    """n_pairs distinct upper-triangle entries (a, b), a <= b, of the Gram,
    drawn uniformly over the whole matrix (seeded): a quarter of them on the
    diagonal (the self-kernels, the largest values), the rest off it (cross
    kernels, often a large cancellation measured on the Cauchy-Schwarz
    scale)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    n_diag = min(n_pairs // 4, N_PATHS)
    off = [(a, b) for a in range(N_PATHS) for b in range(a + 1, N_PATHS)]
    pick = rng.choice(len(off), size=min(n_pairs - n_diag, len(off)), replace=False)
    diag = rng.choice(N_PATHS, size=n_diag, replace=False)
    return sorted([off[i] for i in pick] + [(int(a), int(a)) for a in diag])


def oracle_sample(pts_lens, n_pairs, seed=0):
    """FP64 oracle on n_pairs random upper-triangle pairs (a, b) of each Gram;
    returns (values per sigma, seconds, threads)."""
    import numpy as np

    import oracle
    from paper_2502_20392_gb300 import synth
    oracle.build()
    out, t0 = [], time.perf_counter()
    for k, (pts, lens) in enumerate(pts_lens):
        inc = [np.diff(p.astype(np.float64), axis=0) for p in synth.split(pts, lens)]
        idx = sample_pairs(n_pairs, seed + k)
        xs = [inc[a] for a, _ in idx]
        ys = [inc[b] for _, b in idx]
        out.append((idx, oracle.series_pairs(xs, ys)))
    return out, time.perf_counter() - t0, oracle.num_threads()


def rel_err_entry(G, a, b, r):
    """Relative error of Gram entry (a, b) against the reference r; a near-zero
    cross entry (|r| below 1e-2 of sqrt(G_aa G_bb)) is measured on that
    Cauchy-Schwarz scale."""
    e = abs(G[a, b] - r) / max(abs(r), 1e-300)
    cs_scale = (abs(G[a, a] * G[b, b])) ** 0.5
    if abs(r) < 1e-2 * cs_scale:
        e = min(e, abs(G[a, b] - r) / cs_scale)
    return e


def timed_loop(step, n_kernels, steps, flush):
    """Runs `steps` timed steps, L2 flushed before each (outside the timed
    span); CUDA events around each step and, through the library's profiling
    hook, around each solver kernel (on the launching stream).  Returns
    (per-step ms, per-step list of per-kernel ms)."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    kev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(n_kernels)] for _ in range(steps)]
    for row in kev:  # torch creates an event on first record: do it before handing out handles
        for a, b in row:
            a.record()
            b.record()
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(float(i))
        starts[i].record()
        step(kev[i])
        ends[i].record()
    torch.cuda.synchronize()
    return ([a.elapsed_time(b) for a, b in zip(starts, ends)],
            [[a.elapsed_time(b) for a, b in row] for row in kev])


def e2e_loop(step, h_in, d_in, outs, h_outs, steps, flush):
    """End to end through the public API: pinned host inputs -> device, the
    step, results -> pinned host, every step; CUDA events around it."""
    import torch
    e_s = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e_e = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        e_s[i].record()
        for h, d in zip(h_in, d_in):
            d.copy_(h, non_blocking=True)
        res = step(None, d_in)
        for o, h in zip(outs(res), h_outs):
            h.copy_(o, non_blocking=True)
        e_e[i].record()
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in zip(e_s, e_e))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", default="full", choices=["full", "medium", "small", "large_d"],
                    help="small / medium: 16 / 32 paths per Gram (for ncu captures; not a bench "
                         "line; medium gives the forward several waves of work items); "
                         "large_d: two launches of 64 ragged pairs with d = 256 (the two-phase "
                         "kernel, for ncu captures)")
    ap.add_argument("--sweep", default=None, choices=["roughness", "dimension", "length", "configs"],
                    help="print one JSON line per point of a sweep instead of the bench line")
    ap.add_argument("--no-tensor", action="store_true",
                    help="large_d: the FMA micro-GEMM for the increment Gram instead of the tensor cores")
    args = ap.parse_args()
    if args.sweep:
        return run_sweep(args)
    if args.case == "large_d":
        return run_large_d(args.no_tensor)
    if args.case in ("small", "medium"):
        global N_PATHS
        N_PATHS = 16 if args.case == "small" else 32

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2502_20392_gb300 import build, sigk
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
    # training forward of the Gram whose gradient is taken: only the seams of
    # the 32-row strips are kept (checkpointed wavefront boundaries); the
    # adjoint recomputes each strip from its seam
    _, _, Pb, nrb = SIGMAS[BWD_SIGMA]
    bopts = sigk.Opts(order=Pb, rings=nrb, max_len=N_SEG, flags=sigk.FLAG_REPLAY)
    wss = [sigk.Workspace() for _ in SIGMAS]
    bws = sigk.Workspace()
    G = [torch.empty((N_PATHS, N_PATHS), dtype=torch.float64, device=dev) for _ in SIGMAS]
    Gb = torch.empty((N_PATHS, N_PATHS), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    # upstream gradient of the Gram in the adjoint (a fixed dense weighting)
    W = torch.from_numpy(np.random.default_rng(7).standard_normal((N_PATHS, N_PATHS))).to(dev)

    def fwd_step(ev=None, inp=None):
        # forward: both Grams (inference)
        inp = inp or (X + L)
        for k in range(len(SIGMAS)):
            if ev is not None:
                sigk.profile_events(*ev[k])
            sigk.gram(inp[k], inp[len(SIGMAS) + k], opts=opts[k], out=G[k], ws=wss[k], check=False)
        if ev is not None:
            sigk.profile_events(None, None)
        return G

    def fb_step(ev=None, inp=None):
        # forward + backward of the sigma = 1 Gram: training forward (keeps
        # the strip seams), then the adjoint from that state
        pts, lens = inp if inp else (X[BWD_SIGMA], L[BWD_SIGMA])
        if ev is not None:
            sigk.profile_events(*ev[0])
        _, state = sigk.forward_train(sigk.OP_GRAM, pts, lens, None, None, bopts, ws=bws, out=Gb,
                                      check=False)
        if ev is not None:
            sigk.profile_events(*ev[1])
        gX, _ = sigk.adjoint(state, W, need_y=False, check=False)
        if ev is not None:
            sigk.profile_events(None, None)
        return Gb, gX

    for _ in range(args.warmup):
        fwd_step()
        fb_step()
    torch.cuda.synchronize()
    for ws in wss + [bws]:
        sigk.sync_status(ws)

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        f_ms, f_kern = timed_loop(fwd_step, len(SIGMAS), args.steps, flush)
        b_ms, b_kern = timed_loop(fb_step, 2, args.steps, flush)
        t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    for ws in wss + [bws]:
        sigk.sync_status(ws)
    ms = statistics.mean(f_ms)
    ms_fb = statistics.mean(b_ms)
    if world > 1:
        ms = max_over_ranks(ms, dev, dist)
        ms_fb = max_over_ranks(ms_fb, dev, dist)

    cells = cells_per_step()                        # both Grams' cells
    cells_fb = pairs_of_gram(N_PATHS) * N_SEG * N_SEG  # the sigma = 1 Gram's cells
    value = cells * world / (ms * 1e-3)

    # per-kernel rooflines: useful work (the algorithmic model) and the
    # executed operation count, both over the kernel's CUDA-event time
    tiles = [sigk.counters(wss[k])[0] for k in range(len(SIGMAS))]
    bcnt = sigk.counters(bws)
    roof = []

    def entry(name, kms, useful, executed, sg, P, nr, extra=None, kept=None):
        e = {"kernel": name, "sigma": sg, "order": P, "rings": nr, "kernel_ms": round(kms, 4),
             "useful_flops": useful, "achieved": round(useful / (kms * 1e-3) / 1e12, 3),
             "frac": round(useful / (kms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS, 4),
             "executed_flops": executed,
             "executed_tflops": round(executed / (kms * 1e-3) / 1e12, 3)}
        if kept is not None:  # the model over the kept entries of the truncation only
            e["kept_entry_flops"] = kept
            e["kept_entry_frac"] = round(kept / (kms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS, 4)
        if extra:
            e.update(extra)
        roof.append(e)

    for k, (sg, _, Pk, nr) in enumerate(SIGMAS):
        P = launch_order(Pk, nr)
        kms = statistics.mean(r[k] for r in f_kern)
        # compulsory increment reads: each pair's two paths once (points, FP32)
        inc_bytes = pairs_of_gram(N_PATHS) * 2 * (N_SEG + 1) * DIM * 4
        useful, executed = tiles[k] * useful_tile_flops(P, nr, DIM), tiles[k] * tile_flops(P, nr, DIM)
        entry(f"fwd_kernel<P={P},D=16> (inference)", kms, useful, executed, sg, P, nr,
              {"increment_read_gbs": round(inc_bytes / (kms * 1e-3) / 1e9, 1),
               "launch": sigk.launch_info(sigk.OP_GRAM, N_PATHS, 0, DIM, opts[k])},
              kept=tiles[k] * 2 * kept_tile_fma(P, nr, DIM))
    sg, _, Pk, nr = SIGMAS[BWD_SIGMA]
    P = launch_order(Pk, nr)
    kms = statistics.mean(r[0] for r in b_kern)
    entry(f"fwd_kernel<P={P},D=16> (training: keeps the strip seams)", kms,
          bcnt[0] * useful_tile_flops(P, nr, DIM), bcnt[0] * tile_flops(P, nr, DIM), sg, P, nr,
          kept=bcnt[0] * 2 * kept_tile_fma(P, nr, DIM))
    roof[-1]["launch"] = sigk.launch_info(sigk.OP_GRAM, N_PATHS, 0, DIM, bopts)
    kms = statistics.mean(r[1] for r in b_kern)
    # pass B over every tile (useful: twice the forward's work); pass A's
    # replay of the forward is recomputation (executed, not useful)
    entry(f"bwd2_kernel<P={P},NR={nr}> (adjoint, recomputes each strip from its seam)", kms,
          bcnt[2] * useful_tile_flops(P, nr, DIM, adjoint=True),
          bcnt[2] * adjoint_tile_flops(P, nr, DIM, replay=False) + bcnt[3] * tile_flops(P, nr, DIM),
          sg, P, nr, {"replayed_tiles": bcnt[3],
                      "launch": sigk.launch_info(sigk.OP_GRAM, N_PATHS, 0, DIM, bopts, train=True)},
          kept=bcnt[2] * 4 * kept_tile_fma(P, nr, DIM))
    dom = max(range(len(roof)), key=lambda k: roof[k]["kernel_ms"])
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(tpath) as f:
            tj = json.load(f)
        # the counters hold while the measured kernel's sources are unchanged
        if (tj.get("kernel") == roof[dom]["kernel"] and
                tj.get("digest") == sources_digest(tj.get("sources", []))):
            traffic = tj.get("bytes_per_launch")
    except (OSError, ValueError):
        traffic = None
    roofline = {"bound": "alu", "achieved": roof[dom]["achieved"], "peak": round(FP32_PEAK_TFLOPS, 2),
                "unit": "TFLOP/s", "frac": roof[dom]["frac"], "traffic": traffic,
                "kernel": roof[dom]["kernel"],
                "work_model": "useful flops = 2 x (d + sum_{m=1..n} (2(P-m)+1) + 2P) per tile at the "
                              "launched order P; adjoint 2x the forward; peak = 152 SMs x 128 FP32 "
                              "lanes x 2 x 2.07 GHz; kept_entry_frac: the same model over the "
                              "tile-matrix entries the truncation keeps (2m + k <= 2n + 1)",
                "kept_entry_frac": roof[dom].get("kept_entry_frac"),
                "executed_tflops": roof[dom]["executed_tflops"], "per_launch": roof}

    # end to end through the public API: pinned host inputs -> device, the
    # calls, results -> pinned host, every step
    h_in = [torch.from_numpy(p).pin_memory() for p, _ in host] + \
           [torch.from_numpy(l).pin_memory() for _, l in host]
    d_in = [torch.empty_like(x) for x in X] + [torch.empty_like(x) for x in L]
    h_G = [torch.empty((N_PATHS, N_PATHS), dtype=torch.float64).pin_memory() for _ in SIGMAS]
    e2e_ms = e2e_loop(fwd_step, h_in, d_in, lambda res: res, h_G, args.steps, flush)
    h_inb = [h_in[BWD_SIGMA], h_in[len(SIGMAS) + BWD_SIGMA]]
    d_inb = [d_in[BWD_SIGMA], d_in[len(SIGMAS) + BWD_SIGMA]]
    h_Gb = torch.empty((N_PATHS, N_PATHS), dtype=torch.float64).pin_memory()
    h_grad = torch.empty_like(h_inb[0]).pin_memory()
    e2e_fb_ms = e2e_loop(fb_step, h_inb, d_inb, lambda res: res, [h_Gb, h_grad], args.steps, flush)
    for ws in wss + [bws]:
        sigk.sync_status(ws)
    if world > 1:
        e2e_ms = max_over_ranks(e2e_ms, dev, dist)
        e2e_fb_ms = max_over_ranks(e2e_fb_ms, dev, dist)
    h2d = sum(t.numel() * t.element_size() for t in h_in)
    d2h = sum(t.numel() * t.element_size() for t in h_G)
    h2d_fb = sum(t.numel() * t.element_size() for t in h_inb)
    d2h_fb = h_Gb.numel() * h_Gb.element_size() + h_grad.numel() * h_grad.element_size()
    ws_fb = sigk.backward_workspace_size(sigk.OP_GRAM, N_PATHS, 0, DIM, bopts)
    ws_rec = sigk.backward_workspace_size(
        sigk.OP_GRAM, N_PATHS, 0, DIM, sigk.Opts(order=Pb, rings=nrb, max_len=N_SEG))

    line = {
        "metric": METRIC,
        "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (float-float corner, f64 reductions)",
        "data": "synthetic (seeded Brownian, PCG64)",
        "config": {"workload": "gram_B64_L1024_d16_sigma1+4", "paths": N_PATHS, "segments": N_SEG,
                   "d": DIM, "sigmas": [s_ for s_, *_ in SIGMAS],
                   "order_rings": [[launch_order(P_, nr_), nr_] for _, _, P_, nr_ in SIGMAS],
                   "unique_pairs_per_gram": pairs_of_gram(N_PATHS), "l2": "flushed between steps",
                   "step": "forward: the Grams for sigma = 1 and sigma = 4 (inference); "
                           "fwd_bwd: training forward + adjoint of the sigma = 1 Gram "
                           "(upstream: fixed dense weights)",
                   "parallelism": f"independent batch per rank x{world}"},
        "fwd_bwd": {"value": cells_fb * world / (ms_fb * 1e-3), "unit": "cells/s", "ms_per_step": ms_fb,
                    "cells_per_step": cells_fb,
                    "note": "training forward keeps only the 32-row strip seams (checkpointed "
                            "wavefront boundaries); the adjoint recomputes each strip from its seam",
                    "workspace_bytes": ws_fb, "workspace_bytes_with_stored_tile_records": ws_rec,
                    "e2e": {"value": cells_fb * world / (e2e_fb_ms * 1e-3), "unit": "cells/s",
                            "h2d_bytes_per_step": h2d_fb, "d2h_bytes_per_step": d2h_fb,
                            "ms_per_step": e2e_fb_ms}},
        # per forward step: planner + solver per Gram; per fwd_bwd step:
        # planner, training forward, adjoint set-up, adjoint
        "gpu_launches": 2 * len(SIGMAS) * args.steps + 4 * args.steps,
        "clocks": clk.summary(),
        "e2e": {"value": cells * world / (e2e_ms * 1e-3), "unit": "cells/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "roofline": roofline,
        "wall_s": t_wall,
    }

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        host_G = [g.cpu().numpy() for g in G]
        vals, secs, thr = oracle_sample(host, ORACLE_SAMPLE_PAIRS, seed=11)
        errs = [rel_err_entry(Gk, a, b, r) for (idx, ref), Gk in zip(vals, host_G)
                for (a, b), r in zip(idx, ref)]
        n_cells = sum(len(idx) for idx, _ in vals) * N_SEG * N_SEG
        line["cpu_baseline"] = {"value": n_cells / secs, "unit": "cells/s", "cores": thr,
                                "kind": "oracle",
                                "sample": f"{ORACLE_SAMPLE_PAIRS} random upper-triangle pairs of each "
                                          f"Gram ({n_cells:.3e} cells), FP64 tile series N=24, "
                                          f"OpenMP over pairs, {secs:.1f} s"}
        line["rel_err_vs_oracle_sample"] = max(errs)
        gb = Gb.cpu().numpy()
        line["fwd_bwd"]["rel_err_vs_oracle_sample"] = max(
            rel_err_entry(gb, a, b, r) for (a, b), r in zip(*vals[BWD_SIGMA]))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_large_d(no_tensor=False):
    """64 ragged pairs of 1500-2048 segments, d = 256, sigma in [0.5, 1.5]:
    the large-d solver (increment Gram on the tensor cores, or with
    no_tensor the FMA micro-GEMM; then the sweep), one warm-up call and one
    measured call.  The inputs exceed the 129 MB L2 while the device footprint
    stays at a few GB (for profiler captures of that kernel)."""
    import torch

    from paper_2502_20392_gb300 import build, sigk, synth
    build.build()
    sigk.load()
    (X, lx), (Y, ly) = synth.ragged_pairs(64, 1500, 2048, 256, 0.5, 1.5, seed=4401)
    a = [torch.from_numpy(v).cuda() for v in (X, lx, Y, ly)]
    o = sigk.Opts(order=12, rings=6, max_len=2048, flags=sigk.FLAG_NO_TENSOR if no_tensor else 0)
    ws = sigk.Workspace()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for _ in range(2):
        ev[0].record()
        k = sigk.pairs(*a, opts=o, ws=ws)
        ev[1].record()
    torch.cuda.synchronize()
    print(json.dumps({"case": "large_d", "no_tensor": no_tensor, "ms": ev[0].elapsed_time(ev[1])}))
    torch.cuda.synchronize()
    assert torch.isfinite(k).all()
    return 0


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
            cells = 136 * 512 * 512
            variants = [(0, "register" if d <= 16 else ("tensor-core" if d <= 1024 else "fma-gemm"))]
            if 16 < d <= 1024:
                variants.append((sigk.FLAG_NO_TENSOR, "fma-gemm"))
            for flag, name in variants:
                oo = sigk.Opts(order=o.order, rings=o.rings, refine_c=o.refine_c, max_len=o.max_len,
                               flags=o.flags | flag)
                ws = sigk.Workspace()
                ms = timed(lambda: sigk.gram(X, L, opts=oo, ws=ws, check=False))
                emit(sweep="dimension", d=d, metric="cells/s", value=cells / (ms * 1e-3), ms=ms,
                     kernel=name, opts=dict(order=o.order, rings=o.rings, refine_c=o.refine_c))
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
    a bounded sample of the workload per step (rank 0 only): per step and
    sigma, as many random pairs of the Gram as the oracle has threads (it
    parallelises over pairs), so that every host core works."""
    if rank != 0:
        return
    import oracle
    from paper_2502_20392_gb300 import synth
    oracle.build()
    host = [synth.workload_gram_1024(s_, seed) for s_, seed, _, _ in SIGMAS]
    per_step = max(REF_PAIRS_PER_STEP, oracle.num_threads())
    for w in range(args.warmup):
        oracle_sample(host, 1, seed=1000 + w)
    times = []
    thr = 1
    for i in range(args.steps):
        _, secs, thr = oracle_sample(host, per_step, seed=2000 + i)
        times.append(secs)
    n_cells = len(SIGMAS) * per_step * N_SEG * N_SEG
    v = n_cells / statistics.mean(times)
    line = {"impl": "reference",
            "metric": METRIC,
            "value": v, "unit": "cells/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(times) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Brownian, PCG64)",
            "config": {"workload": "gram_B64_L1024_d16_sigma1+4",
                       "sample": f"{per_step} random pairs per sigma per step",
                       "step": "forward only: the FP64 oracle has no adjoint (its gradient is by "
                               "finite differences), so every sampled cell is a forward cell"},
            "cpu_baseline": {"value": v, "unit": "cells/s", "cores": thr, "kind": "oracle",
                             "sample": f"{per_step} random upper-triangle pairs per sigma per step, "
                                       f"FP64 tile series N=24, OpenMP over pairs"},
            "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
