#!/usr/bin/env python3
"""Benchmark of libpcal on its headline workload.

Workload (one step = one pass of the whole hot path over one batch): a
single 2-bit channel, fs 64 MHz, f_comb 1 MHz (N = 64), f_offset 10 kHz
(L = 6400), 512M samples (8 s, 128 MB packed), tone amplitude 0.01 sigma,
t_d = 12.5 ns; accumulate the 512M samples, then finalize (rotate the L
bins, fold to N, DFT, amplitude/phase/unwrap/delay fit).  Inputs are
synthetic (seeded Philox generator), generated on the host and copied once
to 8 device buffers (1 GB) that the steps rotate through, so every step
reads its 128 MB from HBM rather than from the 126 MB L2.

Arms:
  --impl gb300      (default) libpcal on the GPU, device-resident inputs;
                    plus an end-to-end pass from pinned host memory.
  --impl reference  the FP64 CPU oracle (the method's direct definition) on
                    the host cores, on a bounded sample of the same stream.

Multi-GPU (torchrun): every rank runs its own independent channel on its own
GPU (replicas, weak scaling); ranks only meet at the timing barriers.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FS, FC, FO, N_TONES = 64_000_000, 1_000_000, 10_000, 64
AMP, TD = 0.01, 12.5e-9
M = 512_000_000
N_BUFFERS = 8
SEED = 2501059932
WORKLOAD = "2-bit single channel, fs=64 MHz, f_comb=1 MHz (N=64), f_offset=10 kHz (L=6400), 512M samples (128 MB)"
METRIC = "PCal Gsamples/s (2-bit single-stream extraction: accumulate + finalize)"
UNIT = "Gsamples/s"


def rank_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def reduce_max(x: float, dist, device: str) -> float:
    """Maximum of a per-rank scalar over all ranks (identity without dist)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(world: int, samples_per_rank_step: int, steps: int, total_ms: float) -> float:
    """Whole-job throughput in Gsamples/s: every rank's samples over the
    slowest rank's time."""
    return world * samples_per_rank_step * steps / (total_ms / 1e3) / 1e9


def shard_range(n_total: int, world: int, rank: int, quantum: int = 4):
    """Contiguous share [start, start+count) of a stream of n_total samples for
    `rank`, in whole quanta (4 samples = one 2-bit byte).  A rank folds its
    share starting at absolute index `start`; the exact integer bins of all
    shares add up to those of the whole stream."""
    units = n_total // quantum
    lo = units * rank // world
    hi = units * (rank + 1) // world
    start = lo * quantum
    count = (hi - lo) * quantum + (n_total - units * quantum if rank == world - 1 else 0)
    return start, count


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def read_traffic(kernel_file: str):
    """Per-launch DRAM bytes of the fold kernel from the committed ncu
    summary, or None when the kernel source changed since the capture."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "fold2bit_c2_dram.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    kv = dict(l.split("=", 1) for l in lines if "=" in l and not l.startswith("#"))
    try:
        src = open(os.path.join(ROOT, "paper_2501_05993_gb300", "csrc", kernel_file), "rb").read()
        if kv.get("source_sha256", "").strip() != hashlib.sha256(src).hexdigest():
            return None
        return int(kv["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the GPU is under load."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path).read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(sample_samples: int):
    """The FP64 oracle's direct definition on a bounded prefix of the stream,
    single-threaded on this host; returns (Gsamples/s, seconds)."""
    import oracle
    import synth

    s = synth.Stream(fs=FS, fc=FC, fo=FO, amp=AMP, td=TD, seed=SEED)
    host = s.bits2(0, sample_samples)
    t0 = time.perf_counter()
    oracle.direct(host, "2bit", 0, FS, FC, FO)
    dt = time.perf_counter() - t0
    return sample_samples / dt / 1e9, dt


def run_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return
    # size each step so that the whole run stays within about two minutes
    rate, _ = cpu_oracle_rate(1_000_000)
    budget = 120.0 / (args.warmup + args.steps)
    sample = int(min(args.ref_sample, max(65_536, rate * 1e9 * budget))) // 64 * 64
    vals = []
    for i in range(args.warmup + args.steps):
        v, dt = cpu_oracle_rate(sample)
        if i >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    ms = sample / (value * 1e9) * 1e3
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_per_step": f"first {sample} samples of the stream"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"direct FP64 definition over the first {sample} samples"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def run_gpu(args):
    import torch

    import paper_2501_05993_gb300 as pcal
    import synth
    from paper_2501_05993_gb300 import build as libbuild

    rank, world, local = rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    libbuild.build()
    pcal.load()

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- inputs: one seeded channel per rank, copied to N_BUFFERS buffers
    s = synth.Stream(fs=FS, fc=FC, fo=FO, amp=AMP, td=TD, seed=SEED, stream=rank)
    host = s.bits2(0, M)
    nbytes = host.size
    bufs = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(N_BUFFERS)]
    src = torch.from_numpy(host)
    for b in bufs:
        b.copy_(src)
    torch.cuda.synchronize()

    plan = pcal.Plan(FS, FC, FO, "2bit")
    stream = torch.cuda.current_stream()
    h = plan.handle

    def step(i):
        pcal.pcal_accumulate(h, bufs[i % N_BUFFERS], M, stream)
        pcal.pcal_finalize_device(h, stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    barrier()

    # clocks: sampled through a short untimed soak plus the timed region
    clocks = ClockSampler(dev)
    clocks.start()
    t_soak = time.perf_counter()
    i = 0
    while time.perf_counter() - t_soak < args.soak_s:
        step(i)
        i += 1
        if i % 64 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    barrier()

    launches0 = plan.stats()["kernel_launches"]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    # timed region: K whole steps; events only at its ends, so that each
    # kernel can launch as a programmatic dependent of the one before it
    t_start.record(stream)
    for k in range(args.steps):
        pcal.pcal_accumulate(h, bufs[k % N_BUFFERS], M, stream)
        pcal.pcal_finalize_device(h, stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = plan.stats()["kernel_launches"] - launches0
    total_ms = t_start.elapsed_time(t_end)
    res = plan.results()  # the last timed step's phasors and delay
    # the dominant kernel alone: K back-to-back fold launches on the same
    # stream (CUDA events around them), then K finalize launches
    f0, f1, f2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    launches_f = plan.stats()["kernel_launches"]
    f0.record(stream)
    for k in range(args.steps):
        pcal.pcal_accumulate(h, bufs[k % N_BUFFERS], M, stream)
    f1.record(stream)
    for k in range(args.steps):
        pcal.pcal_finalize_device(h, stream)
    f2.record(stream)
    torch.cuda.synchronize()
    fold_launches = plan.stats()["kernel_launches"] - launches_f - args.steps
    fold_ms = f0.elapsed_time(f1) / args.steps
    fin_ms = f1.elapsed_time(f2) / args.steps
    total_ms = reduce_max(total_ms, dist, "cuda")
    value = aggregate_value(world, M, args.steps, total_ms)

    # ---- end to end through the C ABI from pinned host memory
    e2e = None
    if not args.no_e2e:
        pinned = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
        pinned.copy_(src)
        ph = pinned.numpy()
        for _ in range(2):
            plan.accumulate_host(ph, M, stream)
            plan.finalize()
        k_e2e = max(3, min(args.steps, 20))
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            plan.accumulate_host(ph, M, stream)
            plan.finalize()  # device -> host read of the phasors, synchronising
        torch.cuda.synchronize()
        dt = reduce_max(time.perf_counter() - t0, dist, "cuda")
        e2e = {"value": aggregate_value(world, M, k_e2e, dt * 1e3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": (5 * N_TONES + 3) * 8, "steps": k_e2e}

    peak, peak_kind = read_peaks()
    achieved = nbytes / (fold_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": read_traffic("fold_bulk.cu"), "peak_kind": f"{peak_kind} (copy bandwidth)",
                "kernel": "bulk_fold_kernel<2-bit>", "algorithmic_bytes_per_launch": nbytes}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, dt = cpu_oracle_rate(args.cpu_sample)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"direct FP64 definition over the first {args.cpu_sample} samples ({dt:.1f} s)"}

    plan.close()
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": f"inputs rotate over {N_BUFFERS} device buffers ({N_BUFFERS * nbytes >> 20} MB) > L2",
                       "fold_ms": fold_ms, "finalize_ms": fin_ms, "fold_launches_per_step": fold_launches / args.steps,
                       "kernel_timing": "fold and finalize each timed over K back-to-back launches after the timed region", "td_s": res["td"], "sigma_td_s": res["sigma_td"],
                       "td_injected_s": TD},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": launches,
        }
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--soak-s", type=float, default=1.5, help="untimed load before timing (clock sampling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=64_000_000)
    ap.add_argument("--ref-sample", type=int, default=8_000_000)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
