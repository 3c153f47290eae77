#!/usr/bin/env python3
"""Benchmark: SCA+Adam steps/s on the 40x40 ionic Hubbard workload (U=4, Delta=1, T=0.1,
128 Matsubara frequencies x 2 spins = 256 complex 1600x1600 blocks per step).

A step is one full pass of the hot path over every block: assemble, blocked pivoted
Gauss-Jordan inversion (log-det from the pivots), adjoint diag(G) with float64 refinement,
fixed-order gradient reduction and the fused Adam update.  The mixed-precision path is the
headline; the float64 path is timed beside it for the ratio.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica (the path shards by
problem; no data-path collective) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SCA+Adam steps/s at L=40 (mixed precision; FP64 path timed beside it)"
UNIT = "steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ionic_40x40")
    ap.add_argument("--prec", default=None,
                    help="fp32 | 3xtf32 | bf16x3 (default: bf16x3)")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed FP64 steps (0 = skip)")
    ap.add_argument("--repeats", type=int, default=5,
                    help="extra timings of the same K-step region (best / median reported)")
    ap.add_argument("--c1-steps", type=int, default=500,
                    help="timed steps of the 4x4 Hubbard case (0: skip)")
    ap.add_argument("--variant-steps", type=int, default=10,
                    help="timed steps of the no-pivoting variant (0 = skip)")
    ap.add_argument("--dos-points", type=int, default=128,
                    help="real frequencies of the timed density of states (0 = skip)")
    ap.add_argument("--sm-partition", type=int, default=DEFAULT_SM_PARTITION,
                    help="SMs kept free of the dominant group's launches (0 = none, "
                         "-1 = the library's default for the problem)")
    ap.add_argument("--sm-partition-mode", default="dominant",
                    choices=["dominant", "both", "alternate"],
                    help="partition mode when --sm-partition > 0")
    ap.add_argument("--metro-steps", type=int, default=10,
                    help="timed Metropolis steps (0 = skip)")
    ap.add_argument("--cpu-blocks", type=int, default=0, help="oracle sample size (0 = #cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve", type=int, default=512,
                    help="serving sweep beside the step timing: replay this many requests of "
                         "the seeded trace (0 = skip)")
    ap.add_argument("--serve-only", action="store_true",
                    help="print only the serving sweep's own JSON line")
    ap.add_argument("--serve-rate", type=float, default=20.0, help="Poisson arrivals per second")
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--serve-steps", type=int, default=5000)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [l.strip().split(",") for l in self.file.read().splitlines() if l.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# Nominal dense ratios (tf32 1.1 PF vs bf16 2.25 PF per GPU) and the CUDA-core rates measured
# on this GB300 with an FMA-chain probe (FP32 75.0 TF/s, FP64 1.20 TF/s).
TF32_OVER_BF16 = 1.1 / 2.25
DEFAULT_PREC = "bf16x3"
DEFAULT_SM_PARTITION = -1  # the library's default (16 SMs in mode 1 for 1024 <= N <= 2048, >= 64 dominant blocks)
# DRAM traffic of the dominant group's update launches, per block: ncu dram__bytes_read.sum +
# dram__bytes_write.sum of the 7 update launches of one step of the 16-block workload
# ionic_40x40_w8 (6 merged pairs at 400.1 MB, one single last step at 344.6 MB per 16-block
# launch), averaged and divided by 16 (traffic grows with the blocks; profiles/).
UPDATE_BYTES_PER_BLOCK_N1600 = {"bf16x3": 392.2e6 / 16}
# sha256 (first 16 hex digits) of csrc/sca_tc.cu when those counters were taken: the traffic
# is reported only while the update kernel's source is unchanged, else null.
UPDATE_TRAFFIC_SOURCE_SHA16 = "f56c4bc0089e0c21"


def tc_source_sha16():
    import hashlib
    path = os.path.join(ROOT, "paper_2311_04435_gb300", "csrc", "sca_tc.cu")
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


FP32_SIMT_TFLOPS = 75.0
FP64_SIMT_TFLOPS = 1.20


def dominant_update_launches(prec: str, N: int, nb: int, sym: bool, paired: bool):
    """Algorithmic flops and bytes, per dominant block, of every update launch of one gradient
    evaluation, in launch order: a list of (kind, flops, bytes).  Flops: 8 per complex
    multiply-add, K = the step widths, over the lower triangle (diagonal included) when the
    block is updated symmetrically, else the full block.  Bytes: the updated tiles of M read and
    written once (complex64) plus the F and W split planes of the launch's steps read once
    (4 + 4 planes of N x nb, bf16 or float32 elements).  With paired steps a pair is one update
    of the second step's cross (its tile row and column, K = the first step) and one merged
    update of every other lower tile (K = both steps) and of the cross (K = the second step)."""
    es = 2 if prec == "bf16x3" else 4
    T = (N + 127) // 128
    rows = [min(128, N - 128 * t) for t in range(T)]
    tiles = [(a, b) for a in range(T) for b in range(T) if b <= a or not sym]

    def area(ts):
        return sum(rows[a] * rows[b] for a, b in ts)

    def entries(ts):  # algorithmic entries: the diagonal tiles' lower triangles when symmetric
        return sum(rows[a] * (rows[a] + 1) / 2 if (sym and a == b) else rows[a] * rows[b]
                   for a, b in ts)

    planes = 8.0 * N * nb * es
    out, k0 = [], 0
    while k0 < N:
        kb = min(nb, N - k0)
        if paired and k0 + kb < N:
            k2 = k0 + kb
            kb2 = min(nb, N - k2)
            t2 = k2 // 128
            cross = [(t2, j) for j in range(t2 + 1)] + [(i, t2) for i in range(t2 + 1, T)]
            out.append(("update_cross", 8.0 * kb * entries(cross), 16.0 * area(cross) + planes))
            out.append(("update", 8.0 * (kb + kb2) * entries(tiles) - 8.0 * kb * entries(cross),
                        16.0 * area(tiles) + 2 * planes))
            k0 = k2 + kb2
        else:
            out.append(("update", 8.0 * kb * entries(tiles), 16.0 * area(tiles) + planes))
            k0 += kb
    return out


def roofline_for(prec: str, flops: float, bytes_: float, seconds: float, traffic):
    """The dominant kernel against the roofline: its bound is the lower of the tensor peak for
    its arithmetic and the HBM bandwidth times its algorithmic intensity."""
    pk, src = peaks()
    hbm = pk["hbm_gbs"]
    if prec == "3xtf32":
        tf32 = pk["bf16_tflops_sustained"] * TF32_OVER_BF16
        peak = tf32 / 3.0  # three TF32 products per complex-split product
        bound, note = "tensor", f"tf32 = {src} sustained bf16 x 1.1/2.25, / 3 for the split"
    elif prec == "bf16x3":
        peak = pk["bf16_tflops_sustained"] / 3.0  # three bf16 products per split product
        bound, note = "tensor", f"{src} sustained bf16, / 3 for the split"
    elif prec == "fp32":
        peak, bound, note = FP32_SIMT_TFLOPS, "alu", "FP32 CUDA-core FMA rate measured on GB300"
    else:
        peak, bound, note = FP64_SIMT_TFLOPS, "alu", "FP64 FMA rate measured on GB300"
    tflops = flops / seconds / 1e12 if seconds > 0 else 0.0
    gbs = bytes_ / seconds / 1e9 if seconds > 0 else 0.0
    intensity = flops / bytes_
    out = {"kernel": "update (merged pairs of rank-128 Gauss-Jordan steps: one K = 256 contraction per pair)",
           "intensity_flop_per_byte": round(intensity, 2),
           "tensor_tflops": round(tflops, 3), "tensor_peak": round(peak, 3)}
    if bound == "tensor" and intensity * hbm / 1e3 < peak:
        out.update({"bound": "hbm", "achieved": round(gbs, 1), "peak": round(hbm, 1),
                    "unit": "GB/s", "frac": round(gbs / hbm, 4), "traffic": traffic,
                    "peak_source": f"{src} HBM copy bandwidth (intensity {intensity:.1f} flop/B "
                                   f"is below the ridge {peak * 1e3 / hbm:.1f} of {note})"})
    else:
        out.update({"bound": bound, "achieved": round(tflops, 3), "peak": round(peak, 3),
                    "unit": "TFLOP/s", "frac": round(tflops / peak, 4), "traffic": traffic,
                    "peak_source": note})
    return out


def aggregate_replicas(ms_local: float, steps: int, world: int):
    """Max of the timed region over ranks and the job-wide throughput (replicas: every rank
    processes `steps` steps of its own problem)."""
    ms = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * steps / (ms / 1e3)


def run_ours(args):
    import numpy as np
    import torch

    from paper_2311_04435_gb300 import api, inputs

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    wl = inputs.WORKLOADS[args.workload]
    prec = args.prec or DEFAULT_PREC
    params = api.Params(wl.L, wl.n_omega, U=wl.U, T=wl.T, delta=wl.delta, t=wl.t, mu=wl.mu,
                        prec=prec)
    adam = api.AdamConfig(lr=wl.lr, seed=wl.seed)
    stream = torch.cuda.Stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---------------- device-resident timing (inputs resident in HBM)
    ctx = api.Context(params)
    ctx.set_stream(stream)
    partition = list(ctx.set_sm_partition(args.sm_partition, args.sm_partition_mode)
                     if args.sm_partition >= 0 else ctx.sm_partition())
    ctx.adam_init(adam)
    ctx.adam_step(args.warmup)
    l0 = api.kernel_launches()
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    om, gm = ctx.adam_step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    launches = api.kernel_launches() - l0
    ms, value = aggregate_replicas(e0.elapsed_time(e1), args.steps, world)
    ms_per_step = ms / args.steps

    # ---------------- the same K-step region timed again, for its spread (best / median of 5);
    # the line's value stays the single region above
    repeats = None
    if rank == 0 and args.repeats > 0:
        per = []
        for _ in range(args.repeats):
            torch.cuda.synchronize()
            r0e, r1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            r0e.record(stream)
            ctx.adam_step(args.steps)
            r1e.record(stream)
            torch.cuda.synchronize()
            per.append(r0e.elapsed_time(r1e) / args.steps)
        repeats = {"n": args.repeats, "steps_each": args.steps,
                   "best_ms_per_step": round(min(per), 3),
                   "median_ms_per_step": round(statistics.median(per), 3),
                   "worst_ms_per_step": round(max(per), 3)}

    # ---------------- per-kernel durations (CUDA events on the launching stream)
    ctx.profile(True)
    ctx.adam_step(1)
    prof = ctx.profile_read()
    ctx.profile(False)
    # dominant kernel: the rank-nb update of the diagonally dominant blocks.  On the tensor
    # cores those blocks are updated symmetrically (they are complex symmetric and never
    # pivoted): the algorithmic flops are 8 kb per lower-triangle entry per elimination step,
    # 4 N^2 (N + 1) per block; the full update (CUDA cores, or SCA_SYM=0) needs 8 N^3.
    upd_ms, upd_n = prof["update"]
    n_dom = 2 * wl.n_omega - api.pivoted_blocks(params)
    tcp = prec in ("3xtf32", "bf16x3")
    sym = tcp and os.environ.get("SCA_SYM", "1") != "0"
    paired = sym and os.environ.get("SCA_PAIR", "1") != "0"
    sched = dominant_update_launches(prec, params.N, 128 if tcp else 64, sym, paired)
    upd = [(f, b) for k, f, b in sched if k == "update"]
    assert len(upd) == upd_n, (len(upd), upd_n)
    # per launch (averaged over the step's update launches): flops and bytes of all dominant
    # blocks, and the average duration
    fl_blk = sum(f for f, _ in upd) / len(upd)
    by_blk = sum(b for _, b in upd) / len(upd)
    launch_s = (upd_ms / 1e3) / max(upd_n, 1)  # average duration of one update launch
    traffic = None
    per_block = UPDATE_BYTES_PER_BLOCK_N1600.get(prec)
    src_sha = tc_source_sha16()
    if sym and params.N == 1600 and per_block and src_sha == UPDATE_TRAFFIC_SOURCE_SHA16:
        traffic = round(per_block * n_dom, 0)  # bytes per launch
    traffic_note = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the 16-block capture "
                    "(workload ionic_40x40_w8), mean over the step's update launches, per "
                    "block, times the dominant blocks; reported "
                    f"only for the kernel source it was taken on (sca_tc.cu sha16 "
                    f"{UPDATE_TRAFFIC_SOURCE_SHA16}; this run {src_sha})")
    per_kernel = {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in prof.items()}
    # per-block log-dets and sigma Re G_ii of the seeded start field, for the error against
    # the oracle on the blocks the CPU baseline samples
    phi_s = inputs.seed_phi(wl.seed, params.N)
    blk_gpu = ctx.blocks(phi_s, grad=True) if rank == 0 and not args.no_cpu_baseline else None
    ctx.close()

    # ---------------- end to end through the public API with host buffers
    phi0 = np.ascontiguousarray(inputs.seed_phi(wl.seed, params.N))
    ctx2 = api.Context(params)
    ctx2.set_stream(stream)
    if args.sm_partition >= 0:
        ctx2.set_sm_partition(args.sm_partition, args.sm_partition_mode)
    ctx2.adam_init(adam, phi0)
    ctx2.adam_step(max(1, args.warmup))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx2.adam_init(adam, phi0)                    # H2D of the start field
    for _ in range(args.steps):
        ctx2.adam_step(1)                         # D2H of Omega / max|g| every step
    phi_end = ctx2.phi()                          # D2H of the final field
    e2e_s = time.perf_counter() - t0
    ctx2.close()
    e2e = {"value": round(world * args.steps / e2e_s, 4), "unit": UNIT,
           "h2d_bytes_per_step": round(8 * params.N / args.steps, 1),
           "d2h_bytes_per_step": round(64 + 8 * params.N / args.steps, 1)}

    # ---------------- FP64 path beside it
    fp64 = None
    blk_64 = None
    if args.fp64_steps > 0 and rank == 0:
        p64 = api.Params(wl.L, wl.n_omega, U=wl.U, T=wl.T, delta=wl.delta, prec="fp64")
        c64 = api.Context(p64)
        c64.set_stream(stream)
        c64.adam_init(adam)
        c64.adam_step(1)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        c64.adam_step(args.fp64_steps)
        a1.record(stream)
        torch.cuda.synchronize()
        ms64 = a0.elapsed_time(a1) / args.fp64_steps
        blk_64 = c64.blocks(phi_s, grad=True) if blk_gpu is not None else None
        c64.close()
        fp64 = {"steps_per_s": round(1e3 / ms64, 5), "ms_per_step": round(ms64, 2),
                "timed_steps": args.fp64_steps, "warmup": 1,
                "mixed_over_fp64": round(ms64 / ms_per_step, 2)}

    # ---------------- the same step without interchanges in any block (complex-symmetric
    # elimination throughout; a variant beside the paper's pivoted LU, not the headline)
    nopiv = None
    if args.variant_steps > 0 and rank == 0 and api.pivoted_blocks(params) > 0:
        cn = api.Context(params)
        cn.set_stream(stream)
        cn.set_pivoting("none")
        cn.adam_init(adam)
        cn.adam_step(1)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        omn, gmn = cn.adam_step(args.variant_steps)
        a1.record(stream)
        torch.cuda.synchronize()
        msn = a0.elapsed_time(a1) / args.variant_steps
        cn.close()
        nopiv = {"steps_per_s": round(1e3 / msn, 4), "ms_per_step": round(msn, 3),
                 "timed_steps": args.variant_steps, "warmup": 1, "final_omega": omn,
                 "final_gmax": gmn}

    # ---------------- the other split precision beside it (same workload, same path)
    other = None
    if args.variant_steps > 0 and rank == 0 and prec in ("3xtf32", "bf16x3"):
        oprec = "3xtf32" if prec == "bf16x3" else "bf16x3"
        po = api.Params(wl.L, wl.n_omega, U=wl.U, T=wl.T, delta=wl.delta, t=wl.t, mu=wl.mu,
                        prec=oprec)
        co = api.Context(po)
        co.set_stream(stream)
        co.adam_init(adam)
        co.adam_step(1)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        omo, gmo = co.adam_step(args.variant_steps)
        a1.record(stream)
        torch.cuda.synchronize()
        mso = a0.elapsed_time(a1) / args.variant_steps
        co.close()
        other = {"prec": oprec, "steps_per_s": round(1e3 / mso, 4), "ms_per_step": round(mso, 3),
                 "timed_steps": args.variant_steps, "warmup": 1, "final_omega": omo,
                 "final_gmax": gmo}

    # ---------------- density of states at the final field (Sec. II): one batch of n_omega
    # real frequencies per spin, every resolvent pivoted (eta < 4t)
    dos = None
    if args.dos_points > 0 and rank == 0:
        cd = api.Context(params)
        cd.set_stream(stream)
        wgrid = np.linspace(-6.0, 6.0, args.dos_points)
        phi_dos = inputs.seed_phi(wl.seed, params.N)
        cd.dos(phi_dos, wgrid, 0.05)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rho = cd.dos(phi_dos, wgrid, 0.05)
        dos_s = time.perf_counter() - t0
        cd.close()
        dos = {"points": int(args.dos_points), "eta": 0.05, "ms": round(dos_s * 1e3, 2),
               "resolvents_per_s": round(2 * args.dos_points / dos_s, 2),
               "rho_max": round(float(rho.max()), 6)}

    # ---------------- Metropolis sampling of exp(-Omega/T) (Sec. II): LU-only elimination per
    # step, decisions on the device
    metro = None
    if args.metro_steps > 0 and rank == 0:
        cm = api.Context(params)
        cm.set_stream(stream)
        cm.metropolis_init(0.01, seed=wl.seed)
        cm.metropolis_step(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, acc, _, _ = cm.metropolis_step(args.metro_steps)
        mt_s = time.perf_counter() - t0
        cm.close()
        metro = {"steps_per_s": round(args.metro_steps / mt_s, 3),
                 "ms_per_step": round(mt_s * 1e3 / args.metro_steps, 3), "delta": 0.01,
                 "acceptance": round(float(acc.mean()), 3), "timed_steps": args.metro_steps}

    # ---------------- the pivoted blocks' panel factorisation in float64 (same workload)
    panel64, blk_p64 = None, None
    if args.variant_steps > 0 and rank == 0 and prec in ("3xtf32", "bf16x3") and \
            api.pivoted_blocks(params) > 0:
        cq = api.Context(params)
        cq.set_stream(stream)
        cq.set_panel_precision("fp64")
        cq.adam_init(adam)
        cq.adam_step(1)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        omq, gmq = cq.adam_step(args.variant_steps)
        a1.record(stream)
        torch.cuda.synchronize()
        msq = a0.elapsed_time(a1) / args.variant_steps
        if not args.no_cpu_baseline:
            blk_p64 = cq.blocks(phi_s, grad=True)
        cq.close()
        panel64 = {"steps_per_s": round(1e3 / msq, 4), "ms_per_step": round(msq, 3),
                   "timed_steps": args.variant_steps, "warmup": 1, "final_omega": omq,
                   "over_fp32_panel": round(msq / ms_per_step, 3)}

    cpu = None
    mixed_vs_oracle = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, sample, o_ld, o_gd = cpu_baseline(args, wl, with_blocks=True)
        npb = api.pivoted_blocks(params)
        mixed_vs_oracle = {"blocks": [int(b) for b in sample],
                           prec: block_errors(blk_gpu, sample, o_ld, o_gd, npb)}
        if blk_p64 is not None:
            mixed_vs_oracle[prec + "_fp64_panel"] = block_errors(blk_p64, sample, o_ld, o_gd, npb)
        if blk_64 is not None:
            mixed_vs_oracle["fp64"] = block_errors(blk_64, sample, o_ld, o_gd, npb)
        mixed_vs_oracle["note"] = ("per-block ln|det A_b| and sigma Re G_b,ii at the seeded "
                                   "start field against the FP64 oracle on the CPU baseline's "
                                   "sample of blocks")

    serve = None
    if rank == 0 and args.serve > 0 and world == 1:
        serve = serve_sweep(args)

    # ---------------- the 4x4 Hubbard case (latency-bound: microseconds per step), FP64
    c1 = None
    if rank == 0 and args.c1_steps > 0:
        w1 = inputs.WORKLOADS["hubbard_4x4"]
        p1 = api.Params(w1.L, w1.n_omega, U=w1.U, T=w1.T, delta=w1.delta, t=w1.t, mu=w1.mu,
                        prec="fp64")
        cc = api.Context(p1)
        cc.set_stream(stream)
        cc.adam_init(api.AdamConfig(lr=w1.lr, seed=w1.seed))
        cc.adam_step(16)
        torch.cuda.synchronize()
        c0e, c1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0e.record(stream)
        om1, gm1 = cc.adam_step(args.c1_steps)
        c1e.record(stream)
        torch.cuda.synchronize()
        us1 = 1e3 * c0e.elapsed_time(c1e) / args.c1_steps
        cc.close()
        c1 = {"workload": "hubbard_4x4: L=4, U=6, Delta=0, T=0.1, 128 blocks of 16x16, FP64",
              "us_per_step": round(us1, 2), "timed_steps": args.c1_steps, "warmup": 16,
              "omega": om1, "gmax": gm1}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": f"f32 storage, {prec} contractions, f64 log-det and diag(G) refinement"
            if prec in ("3xtf32", "bf16x3") else "f32" if prec == "fp32" else "f64",
            "data": "synthetic (seeded SplitMix64 start field, no dataset)",
            "config": {"workload": f"{args.workload}: L={wl.L} (N={params.N}), U={wl.U}, "
                                   f"Delta={wl.delta}, T={wl.T}, n_omega={wl.n_omega}, "
                                   f"{2 * wl.n_omega} complex {params.N}x{params.N} blocks",
                       "prec": prec, "parallelism": f"replicas x{world}",
                       "sm_partition": partition,
                       "sm_partition_mode": (args.sm_partition_mode if args.sm_partition > 0
                                             else "library default"),
                       "l2": "inputs larger than L2 (blocks resident in HBM, "
                             f"{api.workspace_bytes(params) / 1e9:.1f} GB)",
                       "final_omega": om, "final_gmax": gm},
            "e2e": e2e,
            "gpu_launches": int(launches),
            "roofline": dict(roofline_for(prec, fl_blk * n_dom, by_blk * n_dom, launch_s, traffic),
                             traffic_source=traffic_note),
            "kernels_ms_one_step": per_kernel,
            "repeats": repeats,
            "hubbard_4x4": c1,
            "fp64_path": fp64,
            "no_pivoting_variant": nopiv,
            "other_precision": other,
            "fp64_panel_variant": panel64,
            "dos": dos,
            "metropolis": metro,
            "clocks": clk,
            "cpu_baseline": cpu,
            "mixed_vs_oracle": mixed_vs_oracle,
            "serve": serve,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def block_errors(blk, sample, o_ld, o_gd, n_piv=0):
    """Largest errors of the GPU's per-block ld and sigma Re G_ii on the sampled blocks, and on
    the sampled pivoted ones (blocks b < n_piv) alone."""
    import numpy as np
    ld, gd = blk
    sample = np.asarray(sample)

    def errs(sel):
        d_ld = np.abs(ld[sample[sel]] - o_ld[sel])
        d_gd = np.abs(gd[sample[sel]] - o_gd[sel])
        return {"ld_max_abs_err": float(d_ld.max()),
                "ld_max_rel_err": float((d_ld / np.maximum(1.0, np.abs(o_ld[sel]))).max()),
                "gdiag_max_abs_err": float(d_gd.max()),
                "gdiag_scale": float(max(1.0, np.abs(o_gd[sel]).max()))}
    out = errs(np.ones(len(sample), bool))
    piv = sample < n_piv
    if piv.any():
        out["pivoted"] = errs(piv)
    return out


def cpu_baseline(args, wl, steps_timed=1, with_blocks=False):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload: as many blocks
    as host threads (LU + inverse columns each), scaled to a full step."""
    import numpy as np

    import oracle
    from paper_2311_04435_gb300 import inputs

    cores = oracle.num_threads()
    nblk = args.cpu_blocks or cores
    B = 2 * wl.n_omega
    nblk = min(nblk, B)
    p = oracle.make_params(wl.L, wl.n_omega, U=wl.U, T=wl.T, delta=wl.delta, t=wl.t, mu=wl.mu)
    phi = inputs.seed_phi(wl.seed, wl.L * wl.L)
    # the pivoted blocks (lowest frequencies, omega_n <= 4|t|: 2 per frequency) first, up to
    # three quarters of the sample, then dominant blocks spread over the rest
    n_piv = 0
    while n_piv < wl.n_omega and (2 * n_piv + 1) * math.pi * wl.T <= 4.0 * abs(wl.t) * (1 + 1e-3):
        n_piv += 1
    take = min(2 * n_piv, (3 * nblk) // 4)
    rest = np.linspace(2 * n_piv, B - 1, nblk - take) if nblk > take else np.zeros(0)
    blocks = np.concatenate([np.arange(take), rest]).astype(np.int32)
    t0 = time.perf_counter()
    o_ld, o_gd = oracle.blocks_sample(p, phi, blocks)
    dt = time.perf_counter() - t0
    per_step = dt * B / nblk
    out = {"value": round(1.0 / per_step, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{nblk} of {B} blocks (dense LU + inverse columns, FP64), "
                     f"{dt:.1f} s, scaled to a full step",
           "sample_s": round(dt, 3), "sample_blocks": int(nblk)}
    if with_blocks:
        return out, blocks, o_ld, o_gd
    return out


def run_reference(args):
    """The oracle as the reference arm: each step a bounded sample of the workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2311_04435_gb300 import inputs

    wl = inputs.WORKLOADS[args.workload]
    import oracle
    cores = oracle.num_threads()
    per, wall = [], []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(argparse.Namespace(cpu_blocks=args.cpu_blocks or cores), wl)
        if k >= args.warmup:
            per.append(1.0 / r["value"])
            wall.append(r["sample_s"])
    total = sum(per)
    value = args.steps / total
    # each timed step is a bounded sample of the workload's blocks: ms_per_step is the measured
    # time of one sample, value the full-step rate extrapolated from it (blocks are independent)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * sum(wall) / args.steps, 1),
            "ms_per_full_step_extrapolated": round(1e3 * total / args.steps, 1),
            "value_basis": "full steps/s extrapolated from the timed sample of each step "
                           f"({r['sample_blocks']} of {2 * wl.n_omega} blocks)",
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 start field)",
            "config": {"workload": args.workload, "impl": "FP64 CPU oracle (C, OpenMP)"},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": r["sample"]},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """--serve-only: the serving sweep's own JSON line."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    line = serve_sweep(args)
    print(json.dumps(line), flush=True)


def serve_sweep(args):
    """Serving sweep: the seeded mixed-size Poisson trace replayed in real time through
    sca_submit / sca_poll; solves/s and p50/p99 latency (submit -> finish)."""
    import numpy as np

    from paper_2311_04435_gb300 import api, inputs

    rank, world, local = dist_env()
    trace = inputs.serving_trace(args.serve, rate_per_s=args.serve_rate)
    prec = args.prec or DEFAULT_PREC
    reqs = [(api.Params(r.L, r.n_omega, U=r.U, T=r.T, delta=r.delta, prec=prec),
             api.AdamConfig(lr=0.01, grad_tol=1e-6, max_steps=args.serve_steps, seed=r.seed))
            for r in trace]
    l0 = api.kernel_launches()
    t_start = time.perf_counter()
    ids = []
    with api.Server(hbm_budget_bytes=120 << 30, max_slots=args.serve_slots) as srv:
        for r, (p, a) in zip(trace, reqs):
            delay = r.arrival_s - (time.perf_counter() - t_start)
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(p, a))
        results, lat, steps, conv = [], [], [], 0
        for rid, (p, a) in zip(ids, reqs):
            while True:
                res = srv.poll(rid, p.N)
                if res is not None:
                    break
                time.sleep(0.002)
            t = srv.times(rid)
            lat.append(t[3] - t[0])
            steps.append(res.steps)
            conv += int(res.gmax < a.grad_tol)
        wall = time.perf_counter() - t_start
    launches = api.kernel_launches() - l0
    lat = np.array(lat)
    line = {
        "metric": "SCA solves/s, serving sweep (mixed L, U, Delta, T; continuous batching)",
        "value": round(len(ids) / wall, 4), "unit": "solves/s", "n_gpus": world,
        "steps": len(ids), "warmup": 0, "ms_per_step": round(1e3 * wall / len(ids), 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": f"f32 storage, {prec} contractions (f32 below 128 x 128), f64 refinement"
        if prec != "fp64" else "f64",
        "data": "synthetic (seeded Poisson trace, SplitMix64 start fields)",
        "config": {"workload": f"{len(ids)} requests, L in {{8..32}}, Poisson {args.serve_rate}/s, "
                               f"max|g| < 1e-6 or {args.serve_steps} steps, 120 GB budget, "
                               f"{args.serve_slots} slots", "prec": prec},
        "latency_s": {"p50": round(float(np.percentile(lat, 50)), 3),
                      "p99": round(float(np.percentile(lat, 99)), 3),
                      "max": round(float(lat.max()), 3)},
        "converged": conv, "mean_steps": round(float(np.mean(steps)), 1),
        "wall_s": round(wall, 2), "gpu_launches": int(launches),
    }
    return line


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.serve_only:
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
