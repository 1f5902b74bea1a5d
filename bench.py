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
KERNEL_LAUNCHES = 100  # back-to-back launches of the dominant kernel timed alone
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


def read_tensor_peak():
    """Measured dense bf16 tensor throughput (burst, TFLOP/s), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def read_batch_traffic_ratio():
    """DRAM bytes per sample byte of the batched fold from its committed ncu
    summary (captured on a reduced batch), or None when batch.cu changed."""
    import hashlib

    try:
        lines = open(os.path.join(ROOT, "profiles", "batch_fold_mixed.txt")).read().splitlines()
        kv = dict(l.split("=", 1) for l in lines if "=" in l and not l.startswith("#") and " = " not in l)
        src = open(os.path.join(ROOT, "paper_2501_05993_gb300", "csrc", "batch.cu"), "rb").read()
        if kv.get("source_sha256", "").strip() != hashlib.sha256(src).hexdigest():
            return None
        return float(kv["traffic_per_algorithmic_byte"])
    except Exception:
        return None


def read_traffic(kernel_file: str, summary: str = "fold2bit_c2_dram.txt"):
    """Per-launch DRAM bytes of a fold kernel from its committed ncu
    summary, or None when the kernel source changed since the capture."""
    import hashlib

    path = os.path.join(ROOT, "profiles", summary)
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
        text = open(self.path).read()
        os.unlink(self.path)
        return self.parse(text)

    @staticmethod
    def parse(text: str) -> dict:
        """Median SM clock, highest max clock and the throttle reasons seen
        active, from nvidia-smi's csv rows in FIELDS order (malformed rows
        skipped)."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in text.splitlines():
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


_SLICES: dict = {}


def _direct_slice(job):
    """One worker of the all-core direct oracle: the FP64 tone sums of its slice (phases referenced to the
    slice's absolute start, so the slices' phasors add)."""
    import oracle
    import synth

    n0, count = job
    host = _SLICES.get(job)
    if host is None:  # a worker generates its slice once and keeps it for the next steps
        host = synth.Stream(fs=FS, fc=FC, fo=FO, amp=AMP, td=TD, seed=SEED).bits2(n0, count)
        _SLICES.clear()
        _SLICES[job] = host
    t0 = time.perf_counter()
    T = oracle.direct(host, "2bit", n0, FS, FC, FO)
    return T, time.perf_counter() - t0


def cpu_oracle_allcore_rate(sample: int):
    """The oracle's direct definition on every core: one spawned process per core sums its own slice of the
    bounded prefix, the phasors add.  Returns (Gsamples/s, cores, seconds)."""
    import multiprocessing as mp

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    per = sample // cores // 64 * 64
    jobs = [(k * per, per) for k in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_direct_slice, [(0, 64)] * cores)  # workers import and warm up
        parts = pool.map(_direct_slice, jobs)
    t0 = time.perf_counter()
    sum(T for T, _ in parts)
    dt = max(d for _, d in parts) + (time.perf_counter() - t0)
    return per * cores / dt / 1e9, cores, dt


def _fold_counts_slice(job):
    """One worker of the all-core CPU fold: exact per-code counts of its slice."""
    import oracle
    import synth

    n0, count, L = job
    s = synth.Stream(fs=FS, fc=FC, fo=FO, amp=AMP, td=TD, seed=SEED)
    host = s.bits2(n0, count)
    t0 = time.perf_counter()
    c = oracle.counts_2bit(host, n0, L)
    return c, time.perf_counter() - t0


def cpu_fold_rates(sample: int):
    """The oracle's fold-first route on the host (exact per-code counts, FP64
    decode and tones): single-threaded, and on every core with one spawned
    process per core folding its own slice (the slices' counts add exactly).
    Returns (single-core Gsamples/s, all-core Gsamples/s, cores)."""
    import multiprocessing as mp

    import oracle

    L = oracle.plan(FS, FC, FO)["L"]
    sample = sample // 64 * 64
    c1, dt1 = _fold_counts_slice((0, sample, L))
    t0 = time.perf_counter()
    oracle.tones_from_bins(oracle.decode_counts(c1), FS, FC, FO)
    dt1 += time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    per = sample // cores // 64 * 64
    jobs = [(k * per, per, L) for k in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_fold_counts_slice, [(0, 64, L)] * cores)  # workers import and warm up
        parts = pool.map(_fold_counts_slice, jobs)
    # the slices fold at the same time: the slowest fold, then the combine
    t0 = time.perf_counter()
    total = sum(c for c, _ in parts)
    oracle.tones_from_bins(oracle.decode_counts(total), FS, FC, FO)
    dtn = max(dt for _, dt in parts) + (time.perf_counter() - t0)
    return sample / dt1 / 1e9, per * cores / dtn / 1e9, cores


def run_reference(args):
    """The reference arm: the FP64 oracle's direct definition, as it stands, on every host core (one spawned
    process per core sums its slice of the step's bounded sample; the phasors add)."""
    import multiprocessing as mp

    rank, world, _ = rank_env()
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    # size each step so that the whole run stays within about two minutes
    rate, _ = cpu_oracle_rate(1_000_000)
    budget = 120.0 / (args.warmup + args.steps)
    sample = int(min(args.ref_sample * cores, max(65_536 * cores, rate * cores * 1e9 * budget)))
    per = sample // cores // 64 * 64
    sample = per * cores
    vals = []
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_direct_slice, [(0, 64)] * cores)  # workers import and warm up
        for i in range(args.warmup + args.steps):
            parts = pool.map(_direct_slice, [(k * per, per) for k in range(cores)])
            t0 = time.perf_counter()
            sum(T for T, _ in parts)
            dt = max(d for _, d in parts) + (time.perf_counter() - t0)
            if i >= args.warmup:
                vals.append(sample / dt / 1e9)
    value = statistics.mean(vals)
    ms = sample / (value * 1e9) * 1e3
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_per_step": f"first {sample} samples of the stream"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"direct FP64 definition over the first {sample} samples, one spawned process "
                                   f"per core summing its slice (time = slowest slice + the sum)"},
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
    # host work before the bracket: an idle GPU's first kernel runs slower (a C2 fold after 1 ms idle took
    # 13-17 us longer, after 100 ms 40 us longer), so the first launch follows the synchronisation at once
    launches0 = plan.stats()["kernel_launches"]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
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
    # (at least KERNEL_LAUNCHES of each: a loop pays ~40 us once to fill and drain, 2 us per launch at K = 20)
    f0, f1, f2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    nk = max(args.steps, KERNEL_LAUNCHES)
    launches_f = plan.stats()["kernel_launches"]
    f0.record(stream)
    for k in range(nk):
        pcal.pcal_accumulate(h, bufs[k % N_BUFFERS], M, stream)
    f1.record(stream)
    for k in range(nk):
        pcal.pcal_finalize_device(h, stream)
    f2.record(stream)
    torch.cuda.synchronize()
    fold_launches = plan.stats()["kernel_launches"] - launches_f - nk
    fold_ms = f0.elapsed_time(f1) / nk
    fin_ms = f1.elapsed_time(f2) / nk
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
        # Pipelined like a streaming client: step k queues its copies and its finalize (whose results
        # copy back into a pinned ring) and then reads step k-1's results, so the host link never waits
        # for the host; every step's inputs cross the link and every step's results are read back
        # inside the timed region.
        t0 = time.perf_counter()
        td_e2e = []
        for k in range(k_e2e):
            plan.accumulate_host_async(ph, M, stream)
            plan.finalize_async(stream)
            if k:
                td_e2e.append(plan.read_async(age=1)["td"])
        td_e2e.append(plan.read_async(age=0)["td"])
        torch.cuda.synchronize()
        dt = reduce_max(time.perf_counter() - t0, dist, "cuda")
        e2e = {"value": aggregate_value(world, M, k_e2e, dt * 1e3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": (5 * N_TONES + 3) * 8 + 4, "steps": k_e2e,
               "results_read": len(td_e2e), "td_spread_s": float(np.ptp(td_e2e))}

    peak, peak_kind = read_peaks()
    achieved = nbytes / (fold_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": read_traffic("fold_bulk.cu"), "peak_kind": f"{peak_kind} (copy bandwidth)",
                "kernel": "bulk_fold_kernel<2-bit>", "algorithmic_bytes_per_launch": nbytes}

    cpu = None
    cpu_fold = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:  # the host baseline: N = 1 only
        v, dt = cpu_oracle_rate(args.cpu_sample)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"direct FP64 definition over the first {args.cpu_sample} samples ({dt:.1f} s)"}
        try:
            va, ca, dta = cpu_oracle_allcore_rate(4 * args.cpu_sample)
            cpu.update({"value_allcore": va, "cores_allcore": ca,
                        "sample_allcore": f"the same definition over the first {4 * args.cpu_sample} samples, one "
                                          f"spawned process per core summing its slice ({dta:.1f} s, slowest slice "
                                          f"+ the sum)"})
        except Exception as e:
            cpu["allcore_error"] = f"{type(e).__name__}: {e}"[:200]
        try:
            one, alln, cores = cpu_fold_rates(M)
            cpu_fold = {"value_1core": one, "value_allcore": alln, "unit": UNIT, "cores": cores, "kind": "oracle fold",
                        "sample": f"the oracle's fold-first route (exact per-code counts, FP64 decode and tones) "
                                  f"over {M} samples; all cores: one spawned process per core folds its slice "
                                  f"(time = slowest slice + the combine)"}
        except Exception as e:
            cpu_fold = {"error": f"{type(e).__name__}: {e}"[:200]}

    plan.close()
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": f"inputs rotate over {N_BUFFERS} device buffers ({N_BUFFERS * nbytes >> 20} MB) > L2",
                       "fold_ms": fold_ms, "finalize_ms": fin_ms, "fold_launches_per_step": fold_launches / nk,
                       "kernel_timing": f"fold and finalize each timed over max(K, {KERNEL_LAUNCHES}) = {nk} back-to-back launches after the timed region", "td_s": res["td"], "sigma_td_s": res["sigma_td"],
                       "td_injected_s": TD},
            "roofline": roofline, "cpu_baseline": cpu, "cpu_fold_baseline": cpu_fold, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches,
        }
        if world == 1 and not args.no_extras:
            # the other parts of the headline metric: batched vs plain, serving latency
            del bufs
            torch.cuda.empty_cache()
            out["batched"] = summarize_extra(lambda: run_batch(extra_args(args, steps=10, warmup=3, no_e2e=False),
                                                               emit=False),
                                             ("value", "unit", "ms_per_step", "plain", "graph", "roofline", "e2e",
                                              "config"))
            torch.cuda.empty_cache()
            out["serving"] = summarize_extra(lambda: run_serve(extra_args(args), emit=False),
                                             ("p50_ms", "p99_ms", "periods", "lag", "realtime", "saturation", "config"))
            torch.cuda.empty_cache()
            out["tensor_dft"] = summarize_extra(lambda: run_tensor_dft(extra_args(args), emit=False),
                                                ("modes", "speedup_vs_fp32", "config"))
            torch.cuda.empty_cache()
            out["c1_f32"] = summarize_extra(lambda: run_c1(extra_args(args), emit=False),
                                            ("value", "unit", "ms_per_step", "step_frac", "roofline", "config"))
            torch.cuda.empty_cache()
            out["precision"] = summarize_extra(lambda: run_precision(extra_args(args), emit=False),
                                               ("value", "unit", "variants", "config"))
            torch.cuda.empty_cache()
            out["rotplan"] = summarize_extra(lambda: run_rotplan(extra_args(args), emit=False),
                                             ("value", "unit", "ms_per_step", "prefix_max_phasor_err_rel", "config"))
            # the driver keeps the end of the line: the metric's parts, compact, come last
            out["summary"] = compact_summary(out)
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def extra_args(args, **kw):
    a = argparse.Namespace(**vars(args))
    a.no_cpu_baseline, a.no_e2e = True, True
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def summarize_extra(fn, keys):
    """Run a secondary workload; keep the named keys of its line, or the error."""
    try:
        out = fn()
        return {k: out.get(k) for k in keys} if out else None
    except Exception as e:  # the headline number stands on its own
        return {"error": f"{type(e).__name__}: {e}"[:300]}


# ---- batched workload: 64 channels of mixed format, rate, offset and length ----------

BATCH_SEED = 2501059932 + 1
BATCH_WORKLOAD = ("64 channels, length U[0.5, 8] s in whole 10 ms, fs in {32, 64, 128, 256} MHz, f_comb 1 MHz, "
                  "f_offset 10 kHz x U{0..99}, even channels 2-bit, odd int8 (sigma 20), tone amplitude "
                  "U[0.005, 0.02] sigma, t_d U[0, 50] ns")
BATCH_METRIC = "PCal Gsamples/s, batched (one persistent fold launch + one finalize launch per step) vs plain"
BLOCK_SAMPLES = 32 * 1024 * 1024


def batch_channels(n_channels: int = 64):
    """The channels of the batched workload (parameters drawn from a seeded
    generator; sample values come from the synth module)."""
    rng = np.random.default_rng(BATCH_SEED)
    chans = []
    for i in range(n_channels):
        fs = int(rng.choice([32, 64, 128, 256])) * 1_000_000
        centis = int(rng.integers(50, 801))  # length in units of 10 ms
        fo = 10_000 * int(rng.integers(0, 100))
        chans.append({"fs": fs, "fc": 1_000_000, "fo": fo, "fmt": "2bit" if i % 2 == 0 else "i8",
                      "n": fs // 100 * centis, "amp": float(rng.uniform(0.005, 0.02)),
                      "td": float(rng.uniform(0.0, 50e-9)), "id": i})
    return chans


def batch_inputs(chans, geoms):
    """Device buffer per channel: a seeded block of whole periods L,
    repeated to the channel's length (the comb is L-periodic, so the stream
    stays a comb plus noise; the noise repeats every block).  Also returns
    the host blocks (for the end-to-end pass)."""
    import torch

    import synth

    bufs, blocks = [], []
    for ch, g in zip(chans, geoms):
        L = int(g.L)
        B = min(ch["n"], max(L, BLOCK_SAMPLES // L * L))
        B -= B % 4
        s = synth.Stream(fs=ch["fs"], fc=ch["fc"], fo=ch["fo"], amp=ch["amp"], td=ch["td"], seed=BATCH_SEED,
                         stream=1000 * ch["id"])
        blk = s.samples(ch["fmt"], 0, B).view(np.uint8)
        spb = 4 if ch["fmt"] == "2bit" else 1
        nbytes = ch["n"] // spb
        buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        dblk = torch.from_numpy(blk).cuda()
        for o in range(0, nbytes, blk.size):
            k = min(blk.size, nbytes - o)
            buf[o:o + k].copy_(dblk[:k])
        bufs.append(buf)
        blocks.append(blk)
    torch.cuda.synchronize()
    return bufs, blocks


def run_batch(args, emit=True):
    import torch

    import paper_2501_05993_gb300 as pcal
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
    chans = batch_channels(args.batch_channels)
    for c in chans:  # a smaller case of the same workload (profiling)
        c["n"] = max(4 * c["fs"] // 100, int(c["n"] * args.batch_scale) // (c["fs"] // 100) * (c["fs"] // 100))
    batch = pcal.Batch([(c["fs"], c["fc"], c["fo"], c["fmt"]) for c in chans])
    bufs, blocks = batch_inputs(chans, batch.geometry)
    ptrs = [b.data_ptr() for b in bufs]
    n = [c["n"] for c in chans]
    total_samples = sum(n)
    total_bytes = sum(b.numel() for b in bufs)
    stream = torch.cuda.current_stream()
    chosen = batch.autotune(ptrs, n, stream)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    for _ in range(args.warmup):
        batch.accumulate(ptrs, n, stream)
        batch.finalize_device(stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    launches0 = batch.stats()["kernel_launches"]
    t0, t1 = ev(), ev()
    t0.record(stream)
    for _ in range(args.steps):
        batch.accumulate(ptrs, n, stream)
        batch.finalize_device(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = batch.stats()["kernel_launches"] - launches0
    batched_ms = reduce_max(t0.elapsed_time(t1) / args.steps, dist, "cuda")
    res_batch = [batch.results(c) for c in range(len(chans))]

    # the same steps as one replayed CUDA graph each
    for _ in range(2):
        batch.step_graph(ptrs, n, stream)
    g0, g1 = ev(), ev()
    g0.record(stream)
    for _ in range(args.steps):
        batch.step_graph(ptrs, n, stream)
    g1.record(stream)
    torch.cuda.synchronize()
    graph_ms = g0.elapsed_time(g1) / args.steps

    # the persistent fold alone (roofline): accumulate-only steps
    f0, f1 = ev(), ev()
    f0.record(stream)
    for _ in range(args.steps):
        batch.accumulate(ptrs, n, stream)
    f1.record(stream)
    torch.cuda.synchronize()
    fold_ms = f0.elapsed_time(f1) / args.steps
    batch.finalize_device(stream)
    torch.cuda.synchronize()

    # plain: one plan per channel, its own accumulate + finalize launches
    plans = [pcal.Plan(c["fs"], c["fc"], c["fo"], c["fmt"]) for c in chans]
    k_plain = max(3, min(args.steps, 10))

    def plain_step():
        for p, b, m in zip(plans, bufs, n):
            pcal.pcal_accumulate(p.handle, b, m, stream)
            pcal.pcal_finalize_device(p.handle, stream)

    for _ in range(2):
        plain_step()
    p0, p1 = ev(), ev()
    p0.record(stream)
    for _ in range(k_plain):
        plain_step()
    p1.record(stream)
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1) / k_plain
    # agreement of the two paths on the last step's phasors
    worst = 0.0
    for c, p in enumerate(plans):
        T = p.results()["phasors"]
        scale = float(np.max(np.abs(T))) or 1.0
        worst = max(worst, float(np.max(np.abs(res_batch[c]["phasors"] - T))) / scale)
    for p in plans:
        p.close()

    # end to end: every step copies each channel's samples from pinned host
    # memory (its block, repeated to the channel's length) and reads back
    # every channel's results
    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(b).pin_memory() for b in blocks]

        def e2e_step():
            for buf, pb in zip(bufs, pinned):
                for o in range(0, buf.numel(), pb.numel()):
                    k = min(pb.numel(), buf.numel() - o)
                    buf[o:o + k].copy_(pb[:k], non_blocking=True)
            batch.accumulate(ptrs, n, stream)
            batch.finalize_device(stream)
            for c in range(len(chans)):
                batch.results(c)

        e2e_step()
        k_e2e = 3
        torch.cuda.synchronize()
        te = time.perf_counter()
        for _ in range(k_e2e):
            e2e_step()
        dt = reduce_max(time.perf_counter() - te, dist, "cuda")
        e2e = {"value": world * total_samples * k_e2e / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": total_bytes,
               "d2h_bytes_per_step": sum((5 * int(g.N) + 3) * 8 for g in batch.geometry), "steps": k_e2e}

    peak, peak_kind = read_peaks()
    achieved = total_bytes / (fold_ms / 1e3) / 1e9
    ratio = read_batch_traffic_ratio()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": int(ratio * total_bytes) if ratio else None,
                "traffic_note": "scaled from a reduced batch capture (profiles/batch_fold_mixed.txt)",
                "peak_kind": f"{peak_kind} (copy bandwidth)", "kernel": "batch_fold_kernel",
                "algorithmic_bytes_per_launch": total_bytes}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:  # the host baseline: N = 1 only
        v, dt = cpu_oracle_rate(args.cpu_sample)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"direct FP64 definition over the first {args.cpu_sample} samples of a 2-bit channel "
                         f"({dt:.1f} s)"}
    # the finalize alone with each tone DFT (fused CUDA-core FP32 vs one tensor-core contraction per N)
    fin_modes = {}
    for mode in ("fp32", "tf32x3", "bf16x6"):
        batch.set_dft(mode)
        batch.accumulate(ptrs, n, stream)
        for _ in range(3):
            batch.finalize_device(stream)
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        for _ in range(20):
            batch.finalize_device(stream)
        k1.record(stream)
        torch.cuda.synchronize()
        fin_modes[mode] = k0.elapsed_time(k1) / 20
    batch.set_dft("fp32")
    batch.close()
    value = world * total_samples / (batched_ms / 1e3) / 1e9
    if rank == 0:
        n2 = sum(1 for c in chans if c["fmt"] == "2bit")
        out = {
            "metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": batched_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "channels": len(chans), "two_bit_channels": n2,
                       "samples_per_step": total_samples, "bytes_per_step": total_bytes,
                       "max_L": max(int(g.L) for g in batch.geometry), "schedule": chosen,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": f"{total_bytes / 1e9:.2f} GB of inputs per step > L2",
                       "fold_ms": fold_ms, "batched_vs_plain_max_phasor_diff": worst,
                       "finalize_ms_by_dft": fin_modes},
            "plain": {"value": world * total_samples / (plain_ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": plain_ms,
                      "steps": k_plain, "launches": "per channel: fold + ragged + finalize"},
            "graph": {"value": world * total_samples / (graph_ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": graph_ms},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": launches,
        }
        if emit:
            print(json.dumps(out))
        return out
    return None


# ---- the small float32 configuration: launch-dominated ------------------------------------

C1_WORKLOAD = ("f32 single channel, fs=16 MHz, f_comb=1 MHz (N=16), f_offset=10 kHz (L=1600), 16M samples (1 s, "
               "64 MB), Gaussian sigma 1 + 16 tones of amplitude 0.02, t_d 3.7 ns")


def run_c1(args, emit=True, n_buffers=8):
    """C1 step (accumulate 16M float32 samples + finalize) with inputs rotating over 8 device buffers
    (512 MB > L2); the fold + partial reduction alone timed after it."""
    import torch

    import paper_2501_05993_gb300 as pcal
    import synth
    from paper_2501_05993_gb300 import build as libbuild

    libbuild.build()
    pcal.load()
    fs, fc, fo, m = 16_000_000, 1_000_000, 10_000, 16_000_000
    host = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.02, td=3.7e-9, seed=2501059930).f32(0, m)
    src = torch.from_numpy(host).cuda()
    bufs = [src.clone() for _ in range(n_buffers)]
    plan = pcal.Plan(fs, fc, fo, "f32")
    stream = torch.cuda.current_stream()
    h = plan.handle
    for i in range(max(args.warmup, 3)):
        pcal.pcal_accumulate(h, bufs[i % n_buffers], m, stream)
        pcal.pcal_finalize_device(h, stream)
    # an untimed soak, as for the headline workload, so the clocks have settled
    t_soak, i = time.perf_counter(), 0
    while time.perf_counter() - t_soak < min(args.soak_s, 1.0):
        pcal.pcal_accumulate(h, bufs[i % n_buffers], m, stream)
        pcal.pcal_finalize_device(h, stream)
        i += 1
        if i % 64 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    k = max(args.steps, KERNEL_LAUNCHES)  # an extra line: its own K, long enough that fill and drain do not count
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(stream)
    for i in range(k):
        pcal.pcal_accumulate(h, bufs[i % n_buffers], m, stream)
        pcal.pcal_finalize_device(h, stream)
    e[1].record(stream)
    for i in range(k):
        pcal.pcal_accumulate(h, bufs[i % n_buffers], m, stream)
    e[2].record(stream)
    torch.cuda.synchronize()
    step_ms, fold_ms = e[0].elapsed_time(e[1]) / k, e[1].elapsed_time(e[2]) / k
    res = plan.results()
    plan.close()
    peak, peak_kind = read_peaks()
    nbytes = 4 * m
    out = {"metric": "PCal Gsamples/s (f32 single-stream extraction: accumulate + finalize)",
           "value": m / (step_ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": step_ms, "steps": k,
           "step_frac": nbytes / (step_ms / 1e3) / 1e9 / peak,
           "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": C1_WORKLOAD, "fold_ms": fold_ms, "td_s": res["td"], "sigma_td_s": res["sigma_td"],
                      "l2": f"inputs rotate over {n_buffers} device buffers ({n_buffers * nbytes >> 20} MB) > L2"},
           "roofline": {"bound": "hbm", "achieved": nbytes / (fold_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": nbytes / (fold_ms / 1e3) / 1e9 / peak,
                        "traffic": read_traffic("fold_bulk.cu", "fold_f32_c1_dram.txt"),
                        "peak_kind": f"{peak_kind} (copy bandwidth)", "kernel": "bulk_fold_kernel<f32> (+ the partial reduction, one per four folds)",
                        "algorithmic_bytes_per_launch": nbytes}}
    if emit:
        print(json.dumps(out))
    return out


# ---- batched tone DFT on the tensor cores ------------------------------------------------

DFT_WORKLOAD = "batched tone DFT, 4096 channels x N 1024 (complex64 P -> T), seeded complex Gaussian P plus a pulse"


def run_tensor_dft(args, emit=True, C=4096, N=1024, reps=20):
    """pcal_dft_execute in every mode on one batch of P: time per launch (CUDA events over back-to-back
    launches), achieved TFLOP/s of the algorithmic contraction against the measured tensor peak, and the
    error against the DFT definition in FP64."""
    import torch

    import paper_2501_05993_gb300 as pcal
    from paper_2501_05993_gb300 import build as libbuild

    libbuild.build()
    pcal.load()
    rng = np.random.default_rng(2501059932 + 5)
    P = (rng.standard_normal((C, N)) + 1j * rng.standard_normal((C, N))).astype(np.complex64)
    P += (3 * np.sqrt(N) * np.exp(2j * np.pi * rng.integers(0, N, (C, 1)) * np.arange(N) / N)).astype(np.complex64)
    ref = np.fft.fft(P.astype(np.complex128), axis=1)
    dP = torch.from_numpy(P).cuda()
    dT = torch.empty((C, N), dtype=torch.complex64, device="cuda")
    peak_bf16, peak_kind = read_tensor_peak()
    modes = {}
    method_flops = 8.0 * C * N * N  # the DFT itself: C x N x N complex multiply-adds
    for mode in ("fp32", "tf32x3", "bf16x6"):
        with pcal.Dft(N, mode) as d:
            for _ in range(3):
                d.execute(dP, C, dT)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                d.execute(dP, C, dT)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            flags = d.check()
        T = dT.cpu().numpy()
        err = np.max(np.abs(T - ref), axis=1) / np.max(np.abs(ref), axis=1)
        roof = None
        executed = method_flops
        if mode != "fp32":
            # real C x 2N x 2N products: three (split TF32) or six (split BF16)
            executed = (3 if mode == "tf32x3" else 6) * 2.0 * C * (2 * N) * (2 * N)
            # TF32 from the measured bf16 peak and the nominal dense ratio (1.1 / 2.25 PFLOP/s)
            peak = peak_bf16 * (1.1 / 2.25) if mode == "tf32x3" else peak_bf16
            ach = method_flops / (ms / 1e3) / 1e12
            roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                    "traffic": None, "work": "method flops 8 C N^2 (the DFT itself)",
                    "executed_tflops": executed / (ms / 1e3) / 1e12,
                    "executed_frac": executed / (ms / 1e3) / 1e12 / peak,
                    "peak_kind": f"{peak_kind} bf16 burst" + (" x 1.1/2.25 (tf32)" if mode == "tf32x3" else "")}
        modes[mode] = {"ms": ms, "tflops": method_flops / (ms / 1e3) / 1e12, "max_rel_err": float(err.max()),
                       "median_rel_err": float(np.median(err)), "device_error_bits": flags, "roofline": roof}
    out = {"metric": "batched tone DFT time per launch", "value": modes["tf32x3"]["ms"], "unit": "ms",
           "higher_is_better": False, "data": "synthetic", "config": {"workload": DFT_WORKLOAD, "C": C, "N": N},
           "modes": modes,
           "speedup_vs_fp32": {m: modes["fp32"]["ms"] / modes[m]["ms"] for m in ("tf32x3", "bf16x6")}}
    if emit:
        print(json.dumps(out))
    return out


# ---- serving workload: 256 live streams, 10 ms chunks, Poisson arrivals ------------------

SERVE_SEED = 2501059932 + 3
SERVE_WORKLOAD = ("256 streams, fs in {32, 64, 128, 256, 512, 1024} MHz, f_comb 1 MHz, f_offset 10 kHz x U{0..99}, "
                  "even streams 2-bit, odd int8 (sigma 20), 10 ms chunks with Poisson arrivals (mean 10 ms per "
                  "stream), 40 GB HBM admission budget, phasors every 1 s")


def serve_streams(n_streams: int):
    rng = np.random.default_rng(SERVE_SEED)
    out = []
    for i in range(n_streams):
        fs = int(rng.choice([32, 64, 128, 256, 512, 1024])) * 1_000_000
        out.append({"fs": fs, "fc": 1_000_000, "fo": 10_000 * int(rng.integers(0, 100)),
                    "fmt": "2bit" if i % 2 == 0 else "i8", "amp": float(rng.uniform(0.005, 0.02)),
                    "td": float(rng.uniform(0.0, 50e-9)), "id": i})
    return out


def serve_chunks(st, k_chunks: int, chunk_s: float):
    """k distinct pinned chunks of chunk_s seconds (whole periods L: the comb stays coherent when they repeat)."""
    import torch

    import synth

    n = int(st["fs"] * chunk_s)
    s = synth.Stream(fs=st["fs"], fc=st["fc"], fo=st["fo"], amp=st["amp"], td=st["td"], seed=SERVE_SEED,
                     stream=1000 * st["id"])
    raw = s.samples(st["fmt"], 0, n * k_chunks).view(np.uint8)
    nb = raw.size // k_chunks
    out = []
    for k in range(k_chunks):
        t = torch.from_numpy(raw[k * nb:(k + 1) * nb].copy()).pin_memory()
        out.append((t, t.numpy(), n))
    return out


def run_serve(args, emit=True):
    import torch

    import paper_2501_05993_gb300 as pcal
    from paper_2501_05993_gb300 import build as libbuild

    rank, world, local = rank_env()
    if world > 1:
        torch.cuda.set_device(local)
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    libbuild.build()
    pcal.load()
    chunk_s, period_s = 0.01, 1.0
    streams = serve_streams(args.serve_streams)
    pools = [serve_chunks(st, 2, chunk_s) for st in streams]
    rate = sum(st["fs"] * (0.25 if st["fmt"] == "2bit" else 1.0) for st in streams)  # bytes/s offered
    srv = pcal.Server(args.serve_budget_gb << 30, len(streams), period_s, 0.1)
    ids = [srv.open(st["fs"], st["fc"], st["fo"], st["fmt"]) for st in streams]
    rng = np.random.default_rng(SERVE_SEED + 1)
    # the clock sampler starts here, so that nvidia-smi's own start-up is over before the real-time phase
    clocks = ClockSampler(dev)
    clocks.start()
    t_adm = time.perf_counter()  # every stream admitted (its memory carved) before the clock starts
    while srv.stats()["admitted"] < len(streams) and time.perf_counter() - t_adm < 30:
        time.sleep(0.001)
    # before the clock: the server's first iterations (first launches of its kernels), and a first GPU read of
    # every pinned chunk buffer (the first reads of a freshly pinned buffer over the host link ran at 8-16 GB/s,
    # the later ones at ~210 GB/s): each stream submits both of its chunks once
    for k in range(2):
        srv.submit_many(ids, [pools[i][k][1] for i in range(len(streams))],
                        [pools[i][k][2] for i in range(len(streams))])
    srv.drain(60)
    warm = 2

    # real time: each stream's chunks arrive as a Poisson process (mean chunk_s); due chunks are submitted
    # together every tick, each stamped with its scheduled arrival time, so a period's latency runs from
    # the arrival of its last chunk (through any submit lag, the copy, the fold and the finalize) to its
    # results on the host
    import gc

    gc.collect()
    gc.disable()  # a latency-sensitive client keeps the collector out of its real-time loop
    t0 = time.perf_counter()
    lib0 = pcal.clock_s() - (time.perf_counter() - t0)  # library clock at t0
    next_t = t0 + rng.exponential(chunk_s, len(streams))
    sent = np.zeros(len(streams), dtype=np.int64)
    lags = []
    worst = (0.0, 0.0)  # (lag, seconds into the real-time phase)
    slow_submits = []   # (seconds into the phase, submit duration) of submits longer than 5 ms
    duration = args.serve_seconds
    while True:
        now = time.perf_counter()
        if now - t0 >= duration:
            break
        due = np.nonzero(next_t <= now)[0]
        if due.size == 0:
            time.sleep(max(0.0, min(next_t.min() - now, 0.001)))
            continue
        arrivals = next_t[due]
        lags.extend((now - arrivals).tolist())
        lag_max = float(now - arrivals.min())
        if lag_max > worst[0]:
            worst = (lag_max, now - t0)
        srv.submit_many([ids[i] for i in due], [pools[i][(sent[i] + warm) % 2][1] for i in due],
                        [pools[i][(sent[i] + warm) % 2][2] for i in due], arrival_s=(lib0 + (arrivals - t0)).tolist())
        t_sub = time.perf_counter() - now
        if t_sub > 0.005 and len(slow_submits) < 8:
            slow_submits.append((round(now - t0, 4), round(t_sub * 1e3, 2)))
        sent[due] += 1
        next_t[due] += rng.exponential(chunk_s, due.size)
    t_rt = time.perf_counter() - t0
    gc.enable()
    srv.drain(120)
    clk = clocks.stop()
    rt = srv.stats()
    lat = []
    while True:
        r = srv.poll(0.0)
        if r is None:
            break
        lat.append(r["latency_s"])
    rt_samples = int(sum(sent[i] * pools[i][0][2] for i in range(len(streams))))
    lags.sort()

    # saturation: every stream submits its next second of chunks as fast as the
    # rings and the GPU take them
    s0 = srv.stats()
    t1 = time.perf_counter()
    per = int(period_s / chunk_s)
    for k in range(per * args.serve_sat_periods):
        srv.submit_many(ids, [pools[i][k % 2][1] for i in range(len(streams))],
                        [pools[i][k % 2][2] for i in range(len(streams))])
    srv.drain(300)
    t_sat = time.perf_counter() - t1
    s1 = srv.stats()
    sat_samples = s1["samples"] - s0["samples"]
    sat_bytes = s1["bytes_h2d"] - s0["bytes_h2d"]
    srv.close()
    lat.sort()
    p50 = lat[(len(lat) - 1) // 2] if lat else None
    p99 = lat[int((len(lat) - 1) * 0.99)] if lat else None
    if rank == 0:
        out = {
            "metric": "PCal serving p99 latency (arrival of the last chunk of a 1 s period -> phasors on the host)",
            "value": p99 * 1e3 if p99 is not None else None, "unit": "ms", "n_gpus": world, "steps": len(lat),
            "warmup": 0, "ms_per_step": None, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": SERVE_WORKLOAD, "streams": len(streams), "offered_GBps": rate / 1e9,
                       "realtime_seconds": t_rt, "hbm_budget_GB": args.serve_budget_gb,
                       "latency": "scheduled arrival of a period's last chunk -> phasors on the host",
                       "chunk_pool": "2 distinct seeded chunks per stream, repeated"},
            "p50_ms": p50 * 1e3 if p50 is not None else None, "p99_ms": p99 * 1e3 if p99 is not None else None,
            "periods": len(lat),
            "lag": {"p50_ms": lags[(len(lags) - 1) // 2] * 1e3 if lags else None,
                    "p99_ms": lags[int((len(lags) - 1) * 0.99)] * 1e3 if lags else None,
                    "max_ms": lags[-1] * 1e3 if lags else None, "chunks": len(lags),
                    "max_at_s": round(worst[1], 4), "slow_submits_s_ms": slow_submits,
                    "what": "scheduled arrival -> submit start"},
            "realtime": {"value": rt_samples / t_rt / 1e9, "unit": UNIT, "launches": rt["launches"],
                         "admitted": rt["admitted"], "hbm_in_use_GB": rt["hbm_in_use"] / 2**30},
            "saturation": {"value": sat_samples / t_sat / 1e9, "unit": UNIT, "h2d_GBps": sat_bytes / t_sat / 1e9,
                           "seconds": t_sat, "periods_per_stream": args.serve_sat_periods},
            "e2e": {"value": sat_samples / t_sat / 1e9, "unit": UNIT, "h2d_bytes_per_step": sat_bytes,
                    "d2h_bytes_per_step": sum((5 * int(round(st["fs"] / st["fc"])) + 3) * 8 for st in streams)},
            "clocks": clk,
        }
        if emit:
            print(json.dumps(out))
        return out
    return None


# ---- precision workload: one int8 channel, 16 s, every accumulation variant --------------

PREC_SEED = 2501059932 + 2
PREC_WORKLOAD = ("int8 (sigma 20), fs 1024 MHz, f_comb 1 MHz (N 1024), f_offset 10 kHz (L 102400), 16.384e9 "
                 "samples (16 s) streamed in 2^30-sample chunks (not L-aligned), tone amplitude 1e-3 sigma; the "
                 "stream repeats one seeded block of 256 periods L (26.2M samples), so the comb stays coherent")
PREC_BLOCK_PERIODS = 256


def run_precision(args, emit=True):
    """C4: every accumulation variant over the same 16.4G int8 samples, phase error per tone against the
    FP64 oracle's exact bins.  The stream is one seeded block of whole periods repeated, so the oracle's
    bins are (repeats) x (the block's bins) + (the bins of the last partial block), exactly."""
    import torch

    import oracle
    import paper_2501_05993_gb300 as pcal
    import synth
    from paper_2501_05993_gb300 import build as libbuild

    torch.cuda.set_device(0)
    libbuild.build()
    pcal.load()
    fs, fc, fo, N = 1_024_000_000, 1_000_000, 10_000, 1024
    total = int(16.384e9 * args.prec_scale) // 4 * 4
    chunk = 1 << 30
    plan_i8 = pcal.Plan(fs, fc, fo, "i8")
    plan_f32 = pcal.Plan(fs, fc, fo, "f32")
    rot = {v: pcal.RotFold(fs, fc, fo, "i8", v, lanes=args.prec_lanes) for v in ("table", "table_kahan", "dfr")}
    L = plan_i8.L
    B = L * PREC_BLOCK_PERIODS
    block = synth.Stream(fs=fs, fc=fc, fo=fo, amp=1e-3, td=12.5e-9, seed=PREC_SEED).samples("i8", 0, B)
    q, r = divmod(total, B)
    S = q * oracle.sums_i8(block, 0, L) + oracle.sums_i8(block[:r], 0, L)  # the oracle's exact bins
    dblk = torch.from_numpy(block).cuda()
    reps = (min(chunk, total) + B - 1) // B + 1
    R = dblk.repeat(reps)  # R[j] = block[j mod B] for every window of one chunk
    del dblk
    times = {k: 0.0 for k in ("fold-first int64", "fold-first fp32 compensated", "table", "table_kahan", "dfr")}
    s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream()

    def timed(name, fn):
        s_ev.record(cur)
        fn()
        e_ev.record(cur)
        torch.cuda.synchronize()
        times[name] += s_ev.elapsed_time(e_ev) / 1e3

    n0 = 0
    while n0 < total:
        n = min(chunk, total - n0)
        o = n0 % B
        d = R[o:o + n]
        timed("fold-first int64", lambda: plan_i8.accumulate(d, n))
        df32 = d.float()
        timed("fold-first fp32 compensated", lambda: plan_f32.accumulate(df32, n))
        del df32
        for v, rf in rot.items():
            timed(v, lambda rf=rf: rf.accumulate(d, n))
        n0 += n
    del R
    ref = oracle.tones_from_bins(S.astype(np.float64), fs, fc, fo)
    results = {"fold-first int64": plan_i8.finalize(), "fold-first fp32 compensated": plan_f32.finalize()}
    for v, rf in rot.items():
        results[v] = rf.finalize()
        rf.close()
    plan_i8.close()
    plan_f32.close()
    torch.cuda.empty_cache()
    scale = float(np.max(np.abs(ref)))
    sig = np.abs(ref) > 1e-3 * scale
    variants = {}
    for name, T in results.items():
        dphi = np.abs(oracle.wrap(np.angle(T[sig]) - np.angle(ref[sig])))
        variants[name] = {"max_phase_err_rad": float(dphi.max()), "median_phase_err_rad": float(np.median(dphi)),
                          "max_phasor_err_rel": float(np.max(np.abs(T - ref)) / scale),
                          "gsamples_per_s": total / times[name] / 1e9}
    out = {
        "metric": "PCal precision: max tone phase error vs the FP64 oracle, fold-first integer path (rad)",
        "value": variants["fold-first int64"]["max_phase_err_rad"], "unit": "rad", "n_gpus": 1, "steps": 1,
        "warmup": 0, "ms_per_step": times["fold-first int64"] * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "i64", "data": "synthetic",
        "config": {"workload": PREC_WORKLOAD, "samples": total, "chunk_samples": chunk, "lanes": args.prec_lanes,
                   "tones_compared": int(sig.sum())},
        "variants": variants,
    }
    if emit:
        print(json.dumps(out))
    return out


# ---- long-period plan: a prime comb offset, every sample rotated ----------------------------

ROT_WORKLOAD = ("int8 (sigma 20), fs 64 MHz, f_comb 1 MHz (N 64), f_offset 10007 Hz (prime: period 64e6 samples, "
                "no fold), 256M samples (4 s) per step, tone amplitude 0.01 sigma")


def run_rotplan(args, emit=True, m=256 << 20, k_steps=5):
    """Long-period plan throughput (accumulate + finalize per step, inputs rotating over two device buffers
    of 256 MB), and its phasors on a 4M-sample prefix against the oracle's direct definition."""
    import torch

    import oracle
    import paper_2501_05993_gb300 as pcal
    import synth
    from paper_2501_05993_gb300 import build as libbuild

    torch.cuda.set_device(0)
    libbuild.build()
    pcal.load()
    fs, fc, fo = 64_000_000, 1_000_000, 10_007.0
    s = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.01, td=12.5e-9, seed=2501059932 + 7)
    pre = 4_000_000
    head = s.samples("i8", 0, pre)
    with pcal.RotPlan(fs, fc, fo, "i8") as rp:
        rp.accumulate(torch.from_numpy(head).cuda(), pre)
        rp.finalize_device()
        T = rp.results()["phasors"]
    ref = oracle.direct_any(head, "i8", 0, fs, fc, fo)
    err = float(np.max(np.abs(T - ref)) / np.max(np.abs(ref)))
    base = torch.from_numpy(head).cuda()
    bufs = [base.repeat(m // pre + 1)[:m].contiguous() for _ in range(2)]
    stream = torch.cuda.current_stream()
    with pcal.RotPlan(fs, fc, fo, "i8") as rp:
        for i in range(2):
            rp.accumulate(bufs[i % 2], m, stream)
            rp.finalize_device(stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(k_steps):
            rp.accumulate(bufs[i % 2], m, stream)
            rp.finalize_device(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k_steps
    del bufs, base
    torch.cuda.empty_cache()
    out = {"metric": "PCal Gsamples/s, long-period plan (per-sample rotation)", "value": m / (ms / 1e3) / 1e9,
           "unit": UNIT, "ms_per_step": ms, "steps": k_steps, "higher_is_better": True, "dtype": "f32 (double-float)",
           "data": "synthetic", "config": {"workload": ROT_WORKLOAD, "samples_per_step": m},
           "prefix_max_phasor_err_rel": err}
    if emit:
        print(json.dumps(out))
    return out


def _sig(x, digits=4):
    """x rounded to `digits` significant digits (None and non-numbers pass through)."""
    if isinstance(x, bool) or not isinstance(x, (int, float)) or x == 0 or x != x:
        return x
    from math import floor, log10

    return round(float(x), -int(floor(log10(abs(x)))) + digits - 1)


def compact_summary(out: dict) -> dict:
    """The headline metric's parts in a few hundred characters, written last on the line."""

    def get(d, *path):
        for k in path:
            if not isinstance(d, dict):
                return None
            d = d.get(k)
        return d

    sm = {"c2": {"gs": _sig(out.get("value")), "step_us": _sig(out.get("ms_per_step", 0) * 1e3),
                 "fold_frac": _sig(get(out, "roofline", "frac"), 3), "e2e_gs": _sig(get(out, "e2e", "value"))}}
    c1 = out.get("c1_f32") or {}
    if "value" in c1:
        sm["c1_f32"] = {"gs": _sig(c1["value"]), "step_frac": _sig(c1.get("step_frac"), 3),
                        "fold_frac": _sig(get(c1, "roofline", "frac"), 3)}
    b = out.get("batched") or {}
    if "value" in b:
        pv = get(b, "plain", "value")
        sm["batched"] = {"gs": _sig(b["value"]), "plain_gs": _sig(pv), "graph_gs": _sig(get(b, "graph", "value")),
                         "x_plain": _sig(b["value"] / pv, 3) if pv else None,
                         "fold_frac": _sig(get(b, "roofline", "frac"), 3),
                         "e2e_gs": _sig(get(b, "e2e", "value")),
                         "phasor_diff": _sig(get(b, "config", "batched_vs_plain_max_phasor_diff"), 2)}
    sv = out.get("serving") or {}
    if "p99_ms" in sv:
        sm["serving"] = {"p50_ms": _sig(sv["p50_ms"], 3), "p99_ms": _sig(sv["p99_ms"], 3),
                         "lag_p99_ms": _sig(get(sv, "lag", "p99_ms"), 3), "lag_max_ms": _sig(get(sv, "lag", "max_ms"), 3),
                         "rt_gs": _sig(get(sv, "realtime", "value"), 3), "sat_gs": _sig(get(sv, "saturation", "value"), 3),
                         "periods": sv.get("periods")}
    pr = out.get("precision") or {}
    if "variants" in pr:
        short = {"fold-first int64": "int64", "fold-first fp32 compensated": "f32c", "table": "tab",
                 "table_kahan": "tab_kahan", "dfr": "dfr"}
        sm["precision"] = {short[k]: [_sig(v["gsamples_per_s"], 3), _sig(v["max_phase_err_rad"], 2)]
                           for k, v in pr["variants"].items()}
        sm["precision"]["fmt"] = "[Gs/s, max phase err rad]"
    rp = out.get("rotplan") or {}
    if "value" in rp:
        sm["rotplan"] = {"gs": _sig(rp["value"], 3), "err": _sig(rp.get("prefix_max_phasor_err_rel"), 2)}
    td = get(out, "tensor_dft", "modes") or {}
    if td:
        sm["dft"] = {m: [_sig(v["ms"], 3), _sig(v["max_rel_err"], 2), _sig(get(v, "roofline", "frac"), 3)]
                     for m, v in td.items()}
        sm["dft"]["fmt"] = "[ms, max err, method-work frac]"
    return sm


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
    ap.add_argument("--batch-channels", type=int, default=64)
    ap.add_argument("--batch-scale", type=float, default=1.0, help="batch workload: scale every channel's length")
    ap.add_argument("--serve-streams", type=int, default=256)
    ap.add_argument("--serve-seconds", type=float, default=4.0, help="serve workload: real-time phase, seconds")
    ap.add_argument("--serve-sat-periods", type=int, default=2)
    ap.add_argument("--serve-budget-gb", type=int, default=40)
    ap.add_argument("--no-extras", action="store_true", help="single workload: skip the batched and serving summaries")
    ap.add_argument("--prec-scale", type=float, default=1.0, help="precision workload: fraction of the 16 s")
    ap.add_argument("--prec-lanes", type=int, default=128)
    ap.add_argument("--workload", default="single", choices=["single", "batch", "serve", "precision", "dft", "c1", "rotplan"],
                    help="single: the 2-bit single-channel headline workload; batch: 64 mixed channels")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "rotplan":
        run_rotplan(args)
    elif args.workload == "dft":
        run_tensor_dft(args)
    elif args.workload == "c1":
        run_c1(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
