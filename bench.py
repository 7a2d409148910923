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

    def wait_samples(self, n: int, timeout: float = 2.0) -> None:
        """Block until at least n samples have arrived (or timeout), so that a short timed region
        is bracketed by a sample just before it and one just after it."""
        if self.proc is None:
            return
        t_end = time.perf_counter() + timeout
        while len(self.lines) < n and time.perf_counter() < t_end:
            time.sleep(0.005)

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
    ("col_fwd", 4194304, 1024, 4096, 1): 23.667968e6 + 46.707456e6,
    ("row_mul", 4194304, 1024, 4096, 1): 100.974848e6 + 7.706624e6,
    ("col_inv_crt", 4194304, 1024, 4096, 1): 58.211584e6 + 1.039360e6,
    ("carry_scan", 4194304, 1024, 4096, 1): 15.895808e6 + 0.000000e6,
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


def _butterfly_mults(n: int) -> float:
    """Modular products of the butterflies of one length-n transform in the scope table's count:
    (n/2) log2 n for n = 2^a; a radix-3 first pass (n = 3 2^a) adds 2n, a radix-5 one 1.2 n."""
    odd = 1
    while n % 2 == 0 and n > 1:
        n //= 2
        odd *= 2
    a, m = odd.bit_length() - 1, n * odd
    extra = {1: 0.0, 3: 2.0, 5: 1.2}[n]
    return m / 2 * a + extra * m


def scope_model(info, nx: int, ny: int, square: bool) -> dict:
    """Algorithmic work per kernel launch by the hot-path scope table's count: modular products of
    the transforms ((n/2) log2 n butterflies per length-n transform, N four-step twiddles per
    column pass), N pointwise Montgomery products, and the CRT's three products per coefficient;
    a Shoup product counts 3 IMAD, a Montgomery product 4.  Bytes: each pass's residues once in
    and once out, limbs once (the two-pass HBM model)."""
    N, N1, N2 = int(info.N), int(info.N1), int(info.N2)
    L = nx + ny
    ops = 1 if square else 2
    l = 3
    col = N2 * _butterfly_mults(N1) + N
    k = {
        "col_fwd": {"modmuls": l * ops * col, "imad": 3 * l * ops * col,
                    "bytes": 4 * (nx + (0 if square else ny)) + 4 * l * N * ops},
        "row_mul": {"modmuls": l * ((ops + 1) * N1 * _butterfly_mults(N2) + N),
                    "imad": 3 * l * (ops + 1) * N1 * _butterfly_mults(N2) + 4 * l * N,
                    "bytes": 4 * l * N * (ops + 1)},
        "col_inv_crt": {"modmuls": l * col + l * L, "imad": 3 * l * col + 3 * l * L,
                        "bytes": 4 * l * N + 4 * L + 8 * (L // 32)},
        "carry_scan": {"modmuls": 0, "imad": 0.0, "bytes": 8 * L + 8 * (L // 32)},
    }
    k["total"] = {"modmuls": sum(v["modmuls"] for v in k.values()), "imad": sum(v["imad"] for v in k.values()),
                  "bytes": (6 if not square else 4) * l * 4 * N + (8 * L if not square else 4 * nx + 4 * L)}
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
        clocks.wait_samples(1)  # sampling runs before the first timed step ...
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
        clocks.wait_samples(len(clocks.lines) + 1)  # ... and one more lands after the last
        clk = clocks.stop()
        clk["window"] = "every 50 ms sample from the last one before the timed region to the first after it"
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
        z_in_place = d.dmul_host_direct(ctx.handle, hz) and L <= d.DMUL_HOST_IN_PLACE_LIMBS
        xy_in_place = d.dmul_host_direct(ctx.handle, hx) and L <= d.DMUL_HOST_IN_PLACE_LIMBS
        e2e_s = e2e_seconds(ctx)
        # for comparison: every buffer through device staging and copy-engine transfers, and the
        # product written into host memory by the carry scan whatever its length
        cst = d.Context(local, flags=d.DMUL_FLAG_HOST_STAGED_IN | d.DMUL_FLAG_HOST_STAGED_OUT)
        staged_s = e2e_seconds(cst)
        cst.close()
        cdo = d.Context(local, flags=d.DMUL_FLAG_HOST_DIRECT_OUT)
        direct_out_s = e2e_seconds(cdo)
        cdo.close()
        e2e_out = {"value": digits_per_step / e2e_s * world, "unit": "digits/s",
                   "h2d_bytes_per_step": 4 * (nx + ny), "d2h_bytes_per_step": 4 * L + 12,
                   "ms_per_step": e2e_s * 1e3,
                   "host_path": {"operands": "read in place" if xy_in_place else "copied (cudaMemcpyAsync)",
                                 "product": "written in place by the carry scan" if z_in_place
                                 else "copied (cudaMemcpyAsync)"},
                   "staged_copies_ms_per_step": staged_s * 1e3,
                   "product_in_place_ms_per_step": direct_out_s * 1e3}

    # ---- roofline of the dominant kernel and of the whole product ----
    info = d.dmul_get_plan(ctx.handle, L)
    model = work_model(info, nx, ny, False)
    smodel = scope_model(info, nx, ny, False)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    imad_derived_t = n_sm * 64 * sm_max * 1e6 / 1e12  # T IMAD/s at the maximum SM clock
    # the integer-pipe peak, measured: independent IMAD chains on every SM (dmul_probe_imad), with
    # the SM clock sampled while the probe runs
    probe_clk = ClockSampler(local)
    probe_clk.start()
    probes = []
    t_end = time.perf_counter() + 0.6
    while time.perf_counter() < t_end:
        probes.append(ctx.probe_imad())
    pclk = probe_clk.stop()
    imad_peak_t = max(probes) / 1e12
    # the dominant pipeline kernel; a short product that took a one-launch path (the one-cluster or
    # the cooperative kernel) does the whole product's work in that one kernel
    piped = [k for k in stages if k in model]
    if piped:
        dom = max(piped, key=lambda k: stages[k][0])
        k_imad, k_r16, k_bytes = smodel[dom]["imad"], model[dom]["imad"], smodel[dom]["bytes"]
    else:
        dom = max(stages, key=lambda k: stages[k][0])
        k_imad, k_bytes = smodel["total"]["imad"], smodel["total"]["bytes"]
        k_r16 = sum(v["imad"] for v in model.values())
    dms = stages[dom][0] / max(1, stages[dom][1])
    imad_t = k_imad / (dms * 1e-3) / 1e12
    imad_r16_t = k_r16 / (dms * 1e-3) / 1e12
    gbs = k_bytes / (dms * 1e-3) / 1e9
    t_int_us = smodel["total"]["imad"] / (imad_peak_t * 1e12) * 1e6
    t_hbm_us = smodel["total"]["bytes"] / (hbm_peak * 1e9) * 1e6
    roof = {"bound": "alu", "achieved": round(imad_t, 3), "peak": round(imad_peak_t, 3),
            "unit": "TIMAD/s", "frac": round(imad_t / imad_peak_t, 4), "traffic": None, "kernel": dom,
            "peak_source": "measured (dmul_probe_imad): independent 32-bit IMAD chains on every SM, "
                           f"best of {len(probes)}, SM clock median {pclk.get('sm_mhz')} MHz during the probe",
            "count_model": "hot-path scope table: butterfly modmuls (n/2) log2 n per length-n transform + N "
                           "twiddles (four-step) + N pointwise + 3 L CRT; Shoup = 3 IMAD, Montgomery = 4",
            "frac_per_survey_model": round(imad_t / imad_peak_t, 4),
            "kernel_imad_per_launch": k_imad,
            "kernel_ms": round(dms, 5),
            "frac_radix16_count": round(imad_r16_t / imad_peak_t, 4),
            "radix16_count_imad_per_launch": k_r16,
            "peak_derived": round(imad_derived_t, 3),
            "peak_derived_source": f"{n_sm} SMs x 64 IMAD/clk x {sm_max:.0f} MHz",
            "frac_of_derived": round(imad_t / imad_derived_t, 4),
            "hbm_gbs": round(gbs, 1), "hbm_frac_of_measured": round(gbs / hbm_peak, 4),
            "whole_product": {"imad": smodel["total"]["imad"], "bytes": smodel["total"]["bytes"],
                              "T_int_us": round(t_int_us, 2), "T_hbm_us": round(t_hbm_us, 2),
                              "bound": "alu" if t_int_us >= t_hbm_us else "hbm",
                              "ms_per_step": ms_per_step},
            "whole_product_frac": round(max(t_int_us, t_hbm_us) * 1e-3 / ms_per_step, 4)}
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
        # the prime width chosen by measurement (Sec. 4.2's two 64-bit primes against the three
        # 30-bit primes): the same fused row pass over this product's transform length
        ms64, ms32 = d.dmul_probe_prime_width(ctx.handle, int(info.N))
        out["prime_width_probe"] = {
            "N": int(info.N), "row_pass_ms_two_62bit_primes": ms64, "row_pass_ms_three_30bit_primes": ms32,
            "ratio": ms64 / ms32,
            "what": "fused row pass (forward row DFTs of x and y, pointwise Montgomery, inverse) on resident "
                    "operands, rows of 4096; 64-bit words with Shoup and R = 2^64 Montgomery for the two "
                    "primes c 3 2^n + 1 < 2^62, the library's specialized pass for the three primes < 2^30"}
        out["other_configs"] = run_other_configs(d, torch, dev, flush, stream)
        out["batched"] = run_batched(d, torch, dev, check=not args.no_cpu_baseline)
        out["served"] = run_served(d, torch, dev, check=not args.no_cpu_baseline)
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


def stage_ms(d, torch, dev, ctx, x_np, y_np, flush, stream, reps=20) -> dict:
    """Per-stage device times (ms, mean of reps) of one product, events between the stages."""
    x, y = d.to_device(x_np, dev), d.to_device(y_np, dev)
    L = len(x_np) + len(y_np)
    z = torch.empty(L, dtype=torch.int32, device=dev)
    nz = torch.zeros(1, dtype=torch.int64, device=dev)
    sp = stream.cuda_stream
    with torch.cuda.stream(stream):
        for _ in range(3):
            d.dmul_mul(ctx.handle, x, len(x_np), y, len(y_np), z, L, nz, sp)
        torch.cuda.synchronize()
        ctx.stage_times()
        ctx.stage_timing(True)
        for _ in range(reps):
            flush.zero_()
            d.dmul_mul(ctx.handle, x, len(x_np), y, len(y_np), z, L, nz, sp)
        torch.cuda.synchronize()
        st = ctx.stage_times()
        ctx.stage_timing(False)
    assert d.dmul_sync(ctx.handle, sp) == 0
    return {k: round(v[0] / reps, 5) for k, v in st.items()}


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
        # An internal base of 10^18 (two I/O limbs per coefficient, Sec. 4.2-4.3) halves the transform
        # length but needs five primes below 2^30 (B^2 min(n, m) ~ 2^140 for 2^24 digits).  Its
        # transform stages are the same per-prime kernels at N / 2: time them on a product of half
        # the limbs (2^23 digits per operand, N = 2^21) and scale the three primes to five.
        xs, ys = wl.c2_random_pair(DIGITS // 2)
        full = stage_ms(d, torch, dev, ctx, *wl.c2_random_pair(), flush, stream)
        half = stage_ms(d, torch, dev, ctx, xs, ys, flush, stream)
        tf = lambda st: st.get("col_fwd", 0) + st.get("row_mul", 0) + st.get("col_inv_crt", 0)
        out["base_1e18_estimate"] = {
            "transform_ms_base_1e9_3_primes_N": tf(full), "transform_ms_3_primes_half_N": tf(half),
            "transform_ms_base_1e18_5_primes_half_N": tf(half) * 5 / 3,
            "stages_full": full, "stages_half": half,
            "note": "col_inv_crt includes the CRT; a five-prime CRT would cost more per coefficient"}
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


def _fp_moduli(count=4):
    """The first `count` primes of the seeded stream of 61-bit candidates (the fingerprint moduli
    of the tests)."""
    import oracle
    from paper_2011_11524_gb300 import workloads as wl
    out = []
    for q in wl.fingerprint_candidates():
        if oracle.is_prime_mr(q):
            out.append(q)
            if len(out) == count:
                return out


def check_products(d, xs, ys, zs, nzs, full_sample=8, seed=0):
    """Oracle check of a list of GPU products (host arrays): x*y = z (mod q) for four seeded 61-bit
    primes q on every product (fingerprints by Horner's rule, Sec. 3.2's value of a limb vector),
    every normalized length, and a sample checked limb for limb against the oracle's product.
    Runs outside every timed region."""
    import numpy as np

    import oracle
    qs = _fp_moduli()
    t0 = time.perf_counter()
    fx = oracle.fingerprint_many(xs, qs)
    fy = oracle.fingerprint_many(ys, qs)
    fz = oracle.fingerprint_many(zs, qs)
    bad = 0
    for i in range(len(zs)):
        ok = all(int(fz[i, j]) == int(fx[i, j]) * int(fy[i, j]) % q for j, q in enumerate(qs))
        nzv = np.flatnonzero(zs[i])
        ok = ok and int(nzs[i]) == (int(nzv[-1]) + 1 if nzv.size else 1)
        bad += not ok
    rng = np.random.Generator(np.random.PCG64(seed))
    small = [i for i in range(len(zs)) if len(xs[i]) * len(ys[i]) <= 2 * 10**9]
    sample = sorted(rng.choice(small, size=min(full_sample, len(small)), replace=False).tolist()) if small else []
    full_bad = sum(not np.array_equal(zs[i], oracle.mul(xs[i], ys[i])) for i in sample)
    return {"products": len(zs), "fingerprint_moduli": len(qs), "mismatches": bad,
            "all_fingerprints_match": bad == 0, "full_oracle_sample": len(sample),
            "full_oracle_mismatches": full_bad, "check_s": round(time.perf_counter() - t0, 2)}


def run_batched(d, torch, dev, reps=5, count=4096, check=True):
    """4096 independent products, operand sizes log-uniform over 10^3..10^6 digits, 20% squarings:
    one dmul_batch call (grouped launches, replayed CUDA graph) against the same jobs issued one
    at a time through dmul_mul.  Every product is then checked against the oracle (fingerprints,
    and a sample in full)."""
    import numpy as np
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
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0.record(stream)
        assert d.dmul_batch(ctx.handle, arr, len(dj), sp) == 0
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    assert d.dmul_sync(ctx.handle, sp) == 0
    statuses = d.job_statuses(arr, len(dj))
    med = float(np.median(times))
    verdict = None
    if check:
        zs = [d.to_host(z) for (_, _, _, _, z, _, _) in dj]
        nzs = [int(nz.item()) for (_, _, _, _, _, _, nz) in dj]
        verdict = check_products(d, [j.x for j in jobs], [j.y for j in jobs], zs, nzs, seed=4)
        verdict["job_statuses_ok"] = all(v == d.DMUL_OK for v in statuses)
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
    out = {"workload": f"{count} jobs, digits log-uniform 10^3..10^6 per operand, 20% squarings",
           "mults_per_s": count / (med * 1e-3), "digits_per_s": digits / (med * 1e-3),
           "ms_per_batch": med, "ms_per_batch_runs": [round(t, 4) for t in times],
           "ms_per_batch_stat": f"median of {reps}",
           "plain_mults_per_s": count / (plain_ms * 1e-3),
           "plain_ms_for_same_jobs": plain_ms, "speedup_vs_plain": plain_ms / med}
    if verdict is not None:
        out["check"] = verdict
        out["all_fingerprints_match"] = verdict["all_fingerprints_match"] and verdict["full_oracle_mismatches"] == 0
    return out


def run_served(d, torch, dev, distinct=2000, repeat=10, load=0.75, budget_gib=8,
               loads=(0.1, 0.25, 0.5, 0.9, 1.0, 1.2), check=True):
    """Poisson stream of requests (digits log-uniform 10^2..10^7, 30% squarings) into the serving
    loop at a sweep of arrival rates (fractions `loads` and `load` of its measured saturated rate);
    p50/p99 latency from arrival to completion at each.  The headline point is `load`.

    Each rate point submits distinct * repeat requests (20,000 by default): `distinct` seeded
    operand pairs, each submitted `repeat` times at its own Poisson arrival time and written to its
    own output.  Every product is checked: the first copy of each pair against the oracle
    (fingerprints, and a sample in full), every other copy, and every later rate point's outputs,
    bit for bit against it on the device."""
    import numpy as np
    from paper_2011_11524_gb300 import workloads as wl
    jp = wl.c5_pool(distinct)
    count = distinct * repeat
    dpool = torch.from_numpy(jp.pool.view(np.int32)).to(dev)
    base = dpool.data_ptr()
    Ls = np.array([len(j.x) + len(j.y) for j in jp.jobs], dtype=np.int64)
    zoff = np.zeros(count + 1, dtype=np.int64)
    zoff[1:] = np.cumsum(np.tile(Ls, repeat))
    zbig = torch.full((int(zoff[-1]),), -1, dtype=torch.int32, device=dev)
    nzs = torch.zeros(count, dtype=torch.int64, device=dev)
    zb, nzb = zbig.data_ptr(), nzs.data_ptr()
    rows = []
    for r in range(count):
        k = r % distinct
        j = jp.jobs[k]
        rows.append((base + 4 * int(jp.offsets[k, 0]), len(j.x), base + 4 * int(jp.offsets[k, 1]), len(j.y),
                     zb + 4 * int(zoff[r]), int(Ls[k]), nzb + 8 * r))
    arr = d.make_jobs(rows)
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
    for i in range(distinct):
        nlen = tlen(int(Ls[i]))
        if nlen not in seen:
            seen.add(nlen)
            warm.append(i)
    verdict = None
    with d.Context(dev.index or 0, hbm_budget_bytes=budget) as srv:
        for i in warm + list(range(min(64, count))):
            assert d.dmul_wait(srv.handle, d.dmul_submit(srv.handle, arr[i])[1]) == 0
        # saturated rate: everything submitted at once
        t0 = time.perf_counter()
        tk = [d.dmul_submit(srv.handle, arr[i])[1] for i in range(count)]
        for t in tk:
            assert d.dmul_wait(srv.handle, t) == 0
        sat = count / (time.perf_counter() - t0)
        torch.cuda.synchronize()
        # every copy of a pair equals the first; the first copies go to the oracle
        zs = [zbig[int(zoff[r]):int(zoff[r + 1])] for r in range(count)]
        copies_equal = all(torch.equal(zs[r], zs[r % distinct]) for r in range(distinct, count)) and \
            torch.equal(nzs.view(repeat, distinct), nzs[:distinct].expand(repeat, distinct))
        ref = zbig.clone()
        ref_nz = nzs.clone()
        if check:
            zh = d.to_host(zbig[:int(zoff[distinct])])
            verdict = check_products(d, [j.x for j in jp.jobs], [j.y for j in jp.jobs],
                                     [zh[int(zoff[r]):int(zoff[r + 1])] for r in range(distinct)],
                                     nzs[:distinct].cpu().tolist(), seed=5)
            del zh
        sweep = []
        later_equal = True
        for ld in sorted(set(list(loads) + [load])):
            rate = ld * sat
            arrivals = wl.c5_arrivals(rate, count)
            zbig.fill_(-1)
            nzs.zero_()
            torch.cuda.synchronize()
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
                    if done:
                        assert rc == 0
                        done_t[k] = time.perf_counter()
                        ndone += 1
                    else:
                        assert rc == 0
                        still.append(k)
                pending = still
            lat = sorted((done_t[i] - (start + float(arrivals[i]))) * 1e3 for i in range(count))
            wall = max(done_t) - start
            torch.cuda.synchronize()
            later_equal = later_equal and torch.equal(zbig, ref) and torch.equal(nzs, ref_nz)
            sweep.append({"load": ld, "offered_rate_per_s": rate, "mults_per_s": count / wall,
                          "requests": count, "p50_ms": lat[len(lat) // 2],
                          "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))]})
        head_pt = next(p for p in sweep if p["load"] == load)
        stats = d.dmul_serve_stats(srv.handle)
    # the same requests one at a time through the plain form, back to back
    with d.Context(dev.index or 0) as plain:
        stream = torch.cuda.Stream(device=dev)
        sp = stream.cuda_stream
        for r in warm + list(range(64)):
            x, nx, y, ny, z, L, nz = rows[r]
            d.dmul_mul(plain.handle, x, nx, y, ny, z, L, nz, sp)
        assert d.dmul_sync(plain.handle, sp) == 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for (x, nx, y, ny, z, L, nz) in rows:
            assert d.dmul_mul(plain.handle, x, nx, y, ny, z, L, nz, sp) == 0
        assert d.dmul_sync(plain.handle, sp) == 0
        plain_rate = count / (time.perf_counter() - t0)
        torch.cuda.synchronize()
        plain_equal = torch.equal(zbig, ref) and torch.equal(nzs, ref_nz)
    digits = int(np.tile(Ls, repeat).sum()) * 9
    out = {"workload": f"{count} Poisson requests per rate point ({distinct} seeded operand pairs x {repeat}), "
                       f"digits log-uniform 10^2..10^7, 30% squarings",
           "plain_mults_per_s_same_requests": plain_rate,
           "hbm_budget_gib": budget_gib, "saturated_mults_per_s": sat,
           "offered_rate_per_s": head_pt["offered_rate_per_s"], "mults_per_s": head_pt["mults_per_s"],
           "digits_per_s": digits / count * head_pt["mults_per_s"],
           "p50_ms": head_pt["p50_ms"], "p99_ms": head_pt["p99_ms"], "load": load,
           "requests_per_point": count, "sweep": sweep, "peak_running": stats["peak_running"],
           "tickets_held_after": stats["held"],
           "copies_bit_identical": bool(copies_equal), "rate_points_bit_identical": bool(later_equal),
           "plain_form_bit_identical": bool(plain_equal)}
    if verdict is not None:
        out["check"] = verdict
        out["all_fingerprints_match"] = (verdict["all_fingerprints_match"] and verdict["full_oracle_mismatches"] == 0
                                         and bool(copies_equal) and bool(later_equal) and bool(plain_equal))
    return out


def host_cpu() -> dict:
    """The host's core count and CPU model (lscpu where it names one, else the kernel's own)."""
    import platform
    fields = {}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            fields.setdefault(k.strip(), v.strip())
    except Exception:
        pass
    model = fields.get("Model name") or fields.get("Vendor ID") or platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "model": model, "machine": platform.machine()}


def libmpdec_context(sizes=(100_000, 1_000_000, DIGITS), budget_s=3.0) -> dict:
    """CPython's decimal (libmpdec, the paper's comparison library, Sec. 10) multiplying random
    operands of the same digit counts, single thread, operands built before timing, up to
    floor(8 10^7 / n) repetitions per size as in the paper (capped by a time budget).  Context only:
    a third-party library, not this project's oracle."""
    import decimal

    import numpy as np
    from paper_2011_11524_gb300 import workloads as wl
    if hasattr(sys, "set_int_max_str_digits"):
        sys.set_int_max_str_digits(0)
    ctx = decimal.Context(prec=decimal.MAX_PREC, Emax=decimal.MAX_EMAX, Emin=decimal.MIN_EMIN)
    out = {"library": f"libmpdec {decimal.__libmpdec_version__} via CPython decimal", "threads": 1, "points": []}
    for nd in sizes:
        rng = np.random.Generator(np.random.PCG64(10 + nd % 97))
        x, y = wl.random_operand(nd, rng), wl.random_operand(nd, rng)
        dx = ctx.create_decimal("".join(f"{int(v):09d}" for v in x[::-1]))
        dy = ctx.create_decimal("".join(f"{int(v):09d}" for v in y[::-1]))
        reps, t0 = 0, time.perf_counter()
        while reps < max(1, 80_000_000 // nd):
            ctx.multiply(dx, dy)
            reps += 1
            if time.perf_counter() - t0 >= budget_s:
                break
        el = time.perf_counter() - t0
        out["points"].append({"digits": nd, "reps": reps, "ms_per_mult": el / reps * 1e3,
                              "digits_per_s": 2 * nd * reps / el})
    return out


def cpu_baseline(x, y, z_gpu=None, budget_s=10.0, digits=DIGITS, all_cores=True, mpdec=True) -> dict:
    """The CPU oracle (slow two-prime NTT route, as it stands) on the same 2^24-digit product,
    repeated until about budget_s seconds of CPU work, on one thread; then the same on every core
    (independent products, one per thread).  Its product also checks, limb by limb, the GPU's
    result of the last timed step.  libmpdec's timings are added as context."""
    import concurrent.futures as cf

    import numpy as np

    import oracle
    reps, t0 = 0, time.perf_counter()
    while True:
        ref = oracle.mul_ntt(x, y)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 8:
            break
    cpu = host_cpu()
    out = {"value": 2 * digits * reps / el, "unit": "digits/s", "cores": 1, "kind": "oracle",
           "sample": f"{reps} full {digits} x {digits}-digit products by the oracle's two-prime NTT route "
                     f"({el:.1f} s, single thread)",
           "host": cpu}
    if z_gpu is not None:
        out["gpu_result_matches_oracle"] = bool(np.array_equal(np.asarray(z_gpu), ref))
    if all_cores and (cpu["nproc"] or 1) > 1:
        n = int(cpu["nproc"])
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=n) as ex:  # the oracle's C call releases the GIL
            res = list(ex.map(lambda _: oracle.mul_ntt(x, y), range(n)))
        el_all = time.perf_counter() - t0
        out["all_cores"] = {"value": 2 * digits * n / el_all, "unit": "digits/s", "cores": n,
                            "sample": f"{n} independent full products, one per thread ({el_all:.1f} s)",
                            "all_equal": all(np.array_equal(r, ref) for r in res)}
    if mpdec:
        out["libmpdec_context"] = libmpdec_context()
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
