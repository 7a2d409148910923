#!/usr/bin/env python3
"""Benchmark: exact multiplication of two 2^24-digit decimal integers on one GB300.

One step = one product of two seeded random 2^24-digit operands (1,864,136 base-10^9 limbs each)
through the full path: forward column pass, fused row pass, inverse column pass with CRT, carry
scan.  Operands are resident in HBM before the timed region; L2 is flushed (a 512 MiB write)
between timed steps, outside the per-step events.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the paper has no runnable code) on host cores on the
same workload.  Under torchrun (N > 1) every rank runs an independent replica (the path does
not shard), value = all ranks' digits / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "product digits/s"
WORKLOAD = "2^24 x 2^24-digit random multiplication (base-10^9 uint32 limbs)"
DIGITS = 1 << 24


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------------
# work model (algorithmic modular multiplications and bytes per kernel launch)
# ----------------------------------------------------------------------------------------------
def _dft_mults(R: int) -> int:
    """Nontrivial constant multiplications of one in-register R-point DFT (radix-2 DIF network
    with the factor-1 butterflies peeled, Sec. 5.6; radix 3: one)."""
    if R == 3:
        return 1
    if R == 5:
        return 6
    n, h, total = R, R // 2, 0
    while h >= 1:
        total += (n // (2 * h)) * (h - 1)
        h //= 2
    return total


def _transform_mults(n: int, radices: list[int]) -> float:
    """Constant multiplications of one length-n transform with the given stage radices
    (DFT constants + inter-stage twiddles of every stage with m > R)."""
    m, tot = n, 0.0
    for R in radices:
        tot += (n // R) * _dft_mults(R)
        if m > R:
            tot += n * (R - 1) / R
        m //= R
    return tot


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of each stage's kernel on the
# 2^24 x 2^24-digit workload, from one ncu --set full capture of the current kernels (cold L2;
# summarized under profiles/).  Keyed by (stage, N, N1, N2, half-width column tiles); a stage whose
# kernel changes after the capture must be dropped from this table until it is captured again.
NCU_TRAFFIC = {
    ("col_fwd", 4194304, 1024, 4096, 1): 23.665920e6 + 46.631936e6,
    ("row_mul", 4194304, 1024, 4096, 1): 100.954624e6 + 8.025856e6,
    ("col_inv_crt", 4194304, 1024, 4096, 1): 58.211584e6 + 0.839936e6,
    ("carry_scan", 4194304, 1024, 4096, 1): 15.895040e6 + 0.000000e6,
}


def work_model(info, nx: int, ny: int, square: bool) -> dict:
    N, N1, N2 = info.N, info.N1, info.N2
    cr = [r for r in info.col_radix if r]
    rr = [r for r in info.row_radix if r]
    L = nx + ny
    ops = 1 if square else 2
    Rs = cr[-1]
    col = (N2 * _transform_mults(N1, cr) + N * (2 - 1 / Rs))  # + four-step twiddles
    row_t = N1 * _transform_mults(N2, rr)
    k = {}
    # Shoup products: 3 IMAD each; Montgomery products: 4 IMAD each
    k["col_fwd"] = {"imad": 3 * 3 * ops * col, "bytes": 4 * (nx + (0 if square else ny)) + 4 * 3 * N * ops}
    k["row_mul"] = {"imad": 3 * (3 * (ops + 1) * row_t) + 4 * 3 * N,
                    "bytes": 4 * 3 * N * (ops + 1)}
    k["col_inv_crt"] = {"imad": 3 * 3 * col + L * (3 * 4 + 2 * 6), "bytes": 4 * 3 * N + 4 * L + 8 * (L // 32)}
    k["carry_scan"] = {"imad": 0.0, "bytes": 8 * L + 8 * (L // 32)}
    return k


# ----------------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------------
def aggregate(total_ms_local: float, digits_per_step: int, steps: int, world: int, device=None):
    """Replicas: every rank ran `steps` independent products.  Whole-job value = all ranks'
    digits / the slowest rank's time (max over ranks).  Returns (value, max_total_ms)."""
    total_ms = total_ms_local
    if world > 1:
        import torch
        t = torch.tensor([total_ms_local], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    return digits_per_step * steps * world / (total_ms * 1e-3), total_ms


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_11524_gb300 import dmul as d
    from paper_2011_11524_gb300 import workloads as wl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    digits = args.digits
    x_np, y_np = wl.c2_random_pair(digits)
    nx, ny = len(x_np), len(y_np)
    L = nx + ny
    ctx = d.Context(local)
    stream = torch.cuda.Stream(device=dev)
    x = d.to_device(x_np, dev)
    y = d.to_device(y_np, dev)
    z = torch.empty(L, dtype=torch.int32, device=dev)
    nz = torch.zeros(1, dtype=torch.int64, device=dev)
    flush = torch.empty(max(1, args.flush_mb) << 20, dtype=torch.uint8, device=dev)
    sptr = stream.cuda_stream

    def step():
        rc = d.dmul_mul(ctx.handle, x, nx, y, ny, z, L, nz, sptr)
        if rc:
            raise d.DmulError(rc, "dmul_mul")

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            step()
        torch.cuda.synchronize()
        rc = d.dmul_sync(ctx.handle, sptr)
        if rc:
            raise d.DmulError(rc, "warmup")
        if world > 1:
            torch.distributed.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        torch.cuda.nvtx.range_push("timed")  # ncu --nvtx-include "timed/" captures only these
        for i in range(args.steps):
            flush.zero_()
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ms = [a.elapsed_time(b) for a, b in evs]
        clk = clocks.stop()
    rc = d.dmul_sync(ctx.handle, sptr)
    if rc:
        raise d.DmulError(rc, "timed region")
    # per-stage device times in a separate pass (the events between stages would otherwise sit
    # inside the timed steps and serialize the kernels' launch overlap)
    stage_steps = min(args.steps, 100)
    ctx.stage_timing(True)
    with torch.cuda.stream(stream):
        for _ in range(stage_steps):
            flush.zero_()
            step()
        torch.cuda.synchronize()
    stages = ctx.stage_times()
    ctx.stage_timing(False)
    digits_per_step = 2 * digits
    value, total_ms = aggregate(sum(ms), digits_per_step, args.steps, world, dev)
    ms_per_step = total_ms / args.steps

    # ---- end to end through the host-buffer entry point (pinned host memory) ----
    e2e_out = None
    if not args.no_e2e:
        hx = torch.from_numpy(x_np.view(np.int32).copy()).pin_memory()
        hy = torch.from_numpy(y_np.view(np.int32).copy()).pin_memory()
        hz = torch.empty(L, dtype=torch.int32).pin_memory()

        def e2e_seconds(c):
            for _ in range(max(3, args.warmup // 2)):
                rc, _ = d.dmul_mul_host(c.handle, hx, nx, hy, ny, hz, L)
            e2e = []
            for _ in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, nzh = d.dmul_mul_host(c.handle, hx, nx, hy, ny, hz, L)
                e2e.append(time.perf_counter() - t0)
                if rc:
                    raise d.DmulError(rc, "dmul_mul_host")
            # the host product is the device product, limb for limb
            if not torch.equal(hz, z.cpu()):
                raise RuntimeError("dmul_mul_host result differs from dmul_mul")
            return sum(e2e) / len(e2e)

        # page-locked buffers: the carry scan writes z in place; the forward pass reads x and y in
        # place for short products only (longer ones are copied: every prime reads the tile again)
        z_in_place = d.dmul_host_direct(ctx.handle, hz)
        xy_in_place = d.dmul_host_direct(ctx.handle, hx) and L <= d.DMUL_HOST_IN_PLACE_LIMBS
        e2e_s = e2e_seconds(ctx)
        # the same calls through device staging buffers and copy-engine transfers, for comparison
        cst = d.Context(local, flags=d.DMUL_FLAG_HOST_STAGED_IN | d.DMUL_FLAG_HOST_STAGED_OUT)
        staged_s = e2e_seconds(cst)
        cst.close()
        e2e_out = {"value": digits_per_step / e2e_s * world, "unit": "digits/s",
                   "h2d_bytes_per_step": 4 * (nx + ny), "d2h_bytes_per_step": 4 * L + 12,
                   "ms_per_step": e2e_s * 1e3,
                   "host_path": {"operands": "read in place" if xy_in_place else "copied (cudaMemcpyAsync)",
                                 "product": "written in place by the carry scan" if z_in_place
                                 else "copied (cudaMemcpyAsync)"},
                   "staged_copies_ms_per_step": staged_s * 1e3}

    # ---- roofline of the dominant kernel ----
    info = d.dmul_get_plan(ctx.handle, L)
    model = work_model(info, nx, ny, False)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    imad_peak_t = n_sm * 64 * sm_max * 1e6 / 1e12  # T IMAD/s at the maximum SM clock
    dom = max((k for k in stages if k in model), key=lambda k: stages[k][0])
    dms = stages[dom][0] / max(1, stages[dom][1])
    imad_t = model[dom]["imad"] / (dms * 1e-3) / 1e12
    gbs = model[dom]["bytes"] / (dms * 1e-3) / 1e9
    if imad_t / imad_peak_t >= gbs / hbm_peak:
        roof = {"bound": "alu", "achieved": round(imad_t, 3), "peak": round(imad_peak_t, 3),
                "unit": "TIMAD/s", "frac": round(imad_t / imad_peak_t, 4), "traffic": None,
                "kernel": dom, "peak_source": f"{n_sm} SMs x 64 IMAD/clk x {sm_max:.0f} MHz (derived)",
                "hbm_gbs": round(gbs, 1), "hbm_frac_of_measured": round(gbs / hbm_peak, 4)}
    else:
        roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(gbs / hbm_peak, 4), "traffic": None, "kernel": dom,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                "imad_tps": round(imad_t, 3), "imad_frac": round(imad_t / imad_peak_t, 4)}
    roof["traffic"] = NCU_TRAFFIC.get((dom, int(info.N), int(info.N1), int(info.N2), int(info.col_half)))
    launches = sum(v[1] for v in stages.values()) // max(1, stage_steps)

    out = {
        "metric": METRIC, "value": value, "unit": "digits/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD if digits == DIGITS else f"{digits} x {digits}-digit random multiplication",
                   "digits_x": digits, "digits_y": digits, "limbs": [nx, ny],
                   "N": int(info.N), "split": [int(info.N1), int(info.N2)], "primes": 3,
                   "col_radix": [r for r in info.col_radix if r], "row_radix": [r for r in info.row_radix if r],
                   "col_threads": int(info.col_threads), "row_threads": int(info.row_threads),
                   "col_tile": [int(info.N1), 16 if info.col_half else 32],
                   "row_pass": (f"persistent TMA-fed, {int(info.row_grid)} CTAs/prime" if info.row_tma
                                else "one CTA per row"),
                   "l2": f"flushed between timed steps ({args.flush_mb} MiB write)", "parallelism": "replicas"},
        "e2e": e2e_out,
        "gpu_launches": int(launches) * args.steps,
        "stages_ms_per_step": {k: round(v[0] / stage_steps, 4) for k, v in stages.items()},
        "roofline": roof,
        "clocks": clk,
    }
    if rank == 0 and not args.no_forms:
        out["other_configs"] = run_other_configs(d, torch, dev, flush, stream)
        out["batched"] = run_batched(d, torch, dev)
        out["served"] = run_served(d, torch, dev)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(x_np, y_np, d.to_host(z), budget_s=args.cpu_seconds,
                                           digits=digits)
    ctx.close()
    return out


def _upload_jobs(d, torch, jobs, dev):
    """Operands of a job list on the device (squarings share x), outputs allocated."""
    import numpy as np
    out = []
    for j in jobs:
        tx = torch.from_numpy(j.x.view(np.int32)).to(dev)
        ty = tx if j.square else torch.from_numpy(j.y.view(np.int32)).to(dev)
        L = len(j.x) + len(j.y)
        out.append((tx, len(j.x), ty, len(j.y), torch.empty(L, dtype=torch.int32, device=dev), L,
                    torch.zeros(1, dtype=torch.int64, device=dev)))
    return out


def time_product(d, torch, dev, ctx, x_np, y_np, reps, flush, stream, square=False):
    """Median device time (ms) of one product through dmul_mul, L2 flushed before each run."""
    import numpy as np
    x = d.to_device(x_np, dev)
    y = x if square else d.to_device(y_np, dev)
    L = len(x_np) + len(y_np)
    z = torch.empty(L, dtype=torch.int32, device=dev)
    nz = torch.zeros(1, dtype=torch.int64, device=dev)
    sp = stream.cuda_stream
    ts = []
    with torch.cuda.stream(stream):
        for i in range(reps + 2):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = d.dmul_mul(ctx.handle, x, len(x_np), y, len(y_np), z, L, nz, sp)
            e1.record(stream)
            assert rc == 0
            torch.cuda.synchronize()
            if i >= 2:
                ts.append(e0.elapsed_time(e1))
    assert d.dmul_sync(ctx.handle, sp) == 0
    return float(np.median(ts))


def run_other_configs(d, torch, dev, flush, stream) -> dict:
    """The other workload configurations, one product each (median of several runs)."""
    import numpy as np
    from paper_2011_11524_gb300 import workloads as wl
    out = {}
    with d.Context(dev.index or 0) as ctx:
        x, y = wl.c1_pair()
        ms = time_product(d, torch, dev, ctx, x, y, 50, flush, stream)
        out["c1_100k_x_100k"] = {"ms": ms, "digits_per_s": 200_000 / (ms * 1e-3)}
        x, y = wl.c2_random_pair()
        ms = time_product(d, torch, dev, ctx, x, x, 10, flush, stream, square=True)
        out["c2_2e24_sqr"] = {"ms": ms, "digits_per_s": 2 * DIGITS / (ms * 1e-3)}
        xn, yn = wl.c2_nines_pair()
        ms = time_product(d, torch, dev, ctx, xn, yn, 10, flush, stream)
        out["c2_2e24_nines_mul"] = {"ms": ms, "digits_per_s": 2 * DIGITS / (ms * 1e-3)}
        for name, (a, b), nd in zip(("c3a_64M_x_1M", "c3b_32M_x_16M"), wl.c3_pairs(),
                                    (65_000_000, 48_000_000)):
            ms = time_product(d, torch, dev, ctx, a, b, 10, flush, stream)
            out[name] = {"ms": ms, "digits_per_s": nd / (ms * 1e-3)}
        # a length in (2^22, 5 2^20]: N = 5 2^20 (radix-5 first column stage) instead of 3 2^21
        rng = np.random.Generator(np.random.PCG64(6))
        a5, b5 = wl.random_operand(19_000_000, rng), wl.random_operand(19_000_000, rng)
        ms = time_product(d, torch, dev, ctx, a5, b5, 10, flush, stream)
        out["len5_19M_x_19M"] = {"ms": ms, "digits_per_s": 38_000_000 / (ms * 1e-3),
                                 "N": int(d.dmul_get_plan(ctx.handle, len(a5) + len(b5)).N)}
    with d.Context(dev.index or 0, flags=d.DMUL_FLAG_NO_RADIX5) as ctx23:
        ms = time_product(d, torch, dev, ctx23, a5, b5, 10, flush, stream)
        out["len5_19M_x_19M_without_5x2k"] = {
            "ms": ms, "digits_per_s": 38_000_000 / (ms * 1e-3),
            "N": int(d.dmul_get_plan(ctx23.handle, len(a5) + len(b5)).N),
            "note": "same product with lengths from {2^k, 3 2^k} only"}
    with d.Context(dev.index or 0, flags=d.DMUL_FLAG_SIXSTEP) as ctx6:
        x, y = wl.c2_random_pair()
        ms = time_product(d, torch, dev, ctx6, x, y, 5, flush, stream)
        out["c2_2e24_mul_sixstep"] = {"ms": ms, "digits_per_s": 2 * DIGITS / (ms * 1e-3),
                                      "note": "six-step form with the in-place transposes (Sec. 7.2, 7.6)"}
        a, b = wl.c3_pairs()[0]
        ms = time_product(d, torch, dev, ctx6, a, b, 5, flush, stream)
        out["c3a_64M_x_1M_sixstep"] = {"ms": ms, "digits_per_s": 65_000_000 / (ms * 1e-3),
                                       "N": int(d.dmul_get_plan(ctx6.handle, len(a) + len(b)).N),
                                       "note": "six-step form at N = 2^23 (odd power: n x 2n transposes)"}
    return out


def run_batched(d, torch, dev, reps=3, count=4096):
    """4096 independent products, operand sizes log-uniform over 10^3..10^6 digits, 20% squarings:
    one dmul_batch call (grouped launches, replayed CUDA graph) against the same jobs issued one
    at a time through dmul_mul."""
    from paper_2011_11524_gb300 import workloads as wl
    jobs = wl.c4_jobs(count)
    dj = _upload_jobs(d, torch, jobs, dev)
    arr = d.make_jobs(dj)
    digits = sum(len(j.x) + len(j.y) for j in jobs) * 9
    ctx = d.Context(dev.index or 0)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    for _ in range(2):  # plans, autotuning, graph capture
        assert d.dmul_batch(ctx.handle, arr, len(dj), sp) == 0
    assert d.dmul_sync(ctx.handle, sp) == 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for _ in range(reps):
        torch.cuda.synchronize()
        e0.record(stream)
        assert d.dmul_batch(ctx.handle, arr, len(dj), sp) == 0
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    assert d.dmul_sync(ctx.handle, sp) == 0
    # the plain form, one product at a time on the same stream
    for (tx, nx, ty, ny, z, L, nz) in dj[:64]:
        d.dmul_mul(ctx.handle, tx, nx, ty, ny, z, L, nz, sp)
    torch.cuda.synchronize()
    e0.record(stream)
    t0 = time.perf_counter()
    for (tx, nx, ty, ny, z, L, nz) in dj:
        rc = d.dmul_mul(ctx.handle, tx, nx, ty, ny, z, L, nz, sp)
        assert rc == 0
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = max(e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3)
    assert d.dmul_sync(ctx.handle, sp) == 0
    ctx.close()
    return {"workload": f"{count} jobs, digits log-uniform 10^3..10^6 per operand, 20% squarings",
            "mults_per_s": count / (best * 1e-3), "digits_per_s": digits / (best * 1e-3),
            "ms_per_batch": best, "plain_mults_per_s": count / (plain_ms * 1e-3),
            "plain_ms_for_same_jobs": plain_ms, "speedup_vs_plain": plain_ms / best}


def run_served(d, torch, dev, count=2000, load=0.7, budget_gib=8, loads=(0.1, 0.3, 0.5, 0.9)):
    """Poisson stream of requests (digits log-uniform 10^2..10^7, 30% squarings) into the serving
    loop at a sweep of arrival rates (fractions `loads` and `load` of its measured saturated rate);
    p50/p99 latency from arrival to completion at each.  The headline point is `load`."""
    from paper_2011_11524_gb300 import workloads as wl
    _, jobs = wl.c5_stream(1.0, count)
    dj = _upload_jobs(d, torch, jobs, dev)
    arr = d.make_jobs(dj)
    budget = budget_gib << 30
    # one request of every transform length the stream uses: plans (twiddle tables, autotuned
    # splits) are built before the measurement and stay resident, as in a running server
    def tlen(n):  # the transform length classes: the one-cluster path's and the four-step plan's
        best, p = None, 1
        while best is None or p <= best:
            for c in (p, 3 * p):
                if c >= max(n, 64) and (best is None or c < best):
                    best = c
            p *= 2
        return best, int(d.dmul_get_plan(None, n).N)
    warm, seen = [], set()
    for i, j in enumerate(jobs):
        nlen = tlen(len(j.x) + len(j.y))
        if nlen not in seen:
            seen.add(nlen)
            warm.append(i)
    # saturated rate: everything submitted at once
    with d.Context(dev.index or 0, hbm_budget_bytes=budget) as srv:
        for i in warm + list(range(min(64, count))):
            d.dmul_wait(srv.handle, d.dmul_submit(srv.handle, arr[i])[1])
        t0 = time.perf_counter()
        tk = [d.dmul_submit(srv.handle, arr[i])[1] for i in range(count)]
        for t in tk:
            assert d.dmul_wait(srv.handle, t) == 0
        sat = count / (time.perf_counter() - t0)
        sweep = []
        for ld in sorted(set(list(loads) + [load])):
            rate = ld * sat
            arrivals, _ = wl.c5_stream(rate, count)
            # one thread: submit at each arrival time, and in between poll every outstanding
            # ticket, oldest first, so that each request's completion is seen when it happens, not
            # when the requests before it complete
            tickets = [0] * count
            done_t = [0.0] * count
            start = time.perf_counter() + 0.05
            i = ndone = 0
            pending = []
            while ndone < count:
                now = time.perf_counter()
                if i < count and now >= start + float(arrivals[i]):
                    rc, tickets[i] = d.dmul_submit(srv.handle, arr[i])
                    assert rc == 0
                    pending.append(i)
                    i += 1
                    continue
                still = []
                for k in pending:
                    rc, done = d.dmul_poll(srv.handle, tickets[k])
                    assert rc == 0
                    if done:
                        done_t[k] = time.perf_counter()
                        ndone += 1
                    else:
                        still.append(k)
                pending = still
            lat = sorted((done_t[i] - (start + float(arrivals[i]))) * 1e3 for i in range(count))
            wall = max(done_t) - start
            sweep.append({"load": ld, "offered_rate_per_s": rate, "mults_per_s": count / wall,
                          "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))]})
        head_pt = next(p for p in sweep if p["load"] == load)
    # the same requests one at a time through the plain form, back to back
    with d.Context(dev.index or 0) as plain:
        stream = torch.cuda.Stream(device=dev)
        sp = stream.cuda_stream
        for (tx, nx, ty, ny, z, L, nz) in [dj[i] for i in warm] + dj[:64]:
            d.dmul_mul(plain.handle, tx, nx, ty, ny, z, L, nz, sp)
        assert d.dmul_sync(plain.handle, sp) == 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for (tx, nx, ty, ny, z, L, nz) in dj:
            assert d.dmul_mul(plain.handle, tx, nx, ty, ny, z, L, nz, sp) == 0
        assert d.dmul_sync(plain.handle, sp) == 0
        plain_rate = count / (time.perf_counter() - t0)
    digits = sum(len(j.x) + len(j.y) for j in jobs) * 9
    return {"workload": f"{count} Poisson requests, digits log-uniform 10^2..10^7, 30% squarings",
            "plain_mults_per_s_same_requests": plain_rate,
            "hbm_budget_gib": budget_gib, "saturated_mults_per_s": sat,
            "offered_rate_per_s": head_pt["offered_rate_per_s"], "mults_per_s": head_pt["mults_per_s"],
            "digits_per_s": digits / count * head_pt["mults_per_s"],
            "p50_ms": head_pt["p50_ms"], "p99_ms": head_pt["p99_ms"], "load": load,
            "sweep": sweep}


def cpu_baseline(x, y, z_gpu=None, budget_s=10.0, digits=DIGITS) -> dict:
    """The CPU oracle (slow two-prime NTT route, as it stands) on the same 2^24-digit product,
    repeated until about budget_s seconds of CPU work.  Its product also checks, limb by limb, the
    GPU's result of the last timed step."""
    import numpy as np

    import oracle
    reps, t0 = 0, time.perf_counter()
    while True:
        ref = oracle.mul_ntt(x, y)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 8:
            break
    out = {"value": 2 * digits * reps / el, "unit": "digits/s", "cores": 1, "kind": "oracle",
           "sample": f"{reps} full {digits} x {digits}-digit products by the oracle's two-prime NTT route "
                     f"({el:.1f} s, single thread)"}
    if z_gpu is not None:
        out["gpu_result_matches_oracle"] = bool(np.array_equal(np.asarray(z_gpu), ref))
    return out


def run_reference(args, rank, world, local):
    """The reference arm: the paper ships no runnable code, so its stand-in is the CPU oracle,
    timed as it stands on the host cores, on this arm's workload and metric."""
    if rank != 0:
        return None
    import numpy as np  # noqa: F401

    from paper_2011_11524_gb300 import workloads as wl
    import oracle
    oracle.build()
    x, y = wl.c2_random_pair(DIGITS)
    for _ in range(min(args.warmup, 1)):
        oracle.mul_ntt(x, y)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.mul_ntt(x, y)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = 2 * DIGITS * len(times) / tot
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "digits/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / len(times) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "parallelism": "none (host CPU)"},
        "cpu_baseline": {"value": value, "unit": "digits/s", "cores": 1, "kind": "oracle",
                         "sample": f"{len(times)} full products, single thread"},
        "e2e": {"value": value, "unit": "digits/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batched (4096 jobs) and served (Poisson stream) measurements")
    ap.add_argument("--flush-mb", type=int, default=512,
                    help="L2 flush buffer written between timed steps (MiB); profiling runs use 1")
    ap.add_argument("--digits", type=int, default=DIGITS,
                    help="operand size in decimal digits (profiling of smaller cases only)")
    args = ap.parse_args()
    rank, world, local = _dist()
    if args.impl == "reference":
        out = run_reference(args, rank, world, local)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world, local)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
