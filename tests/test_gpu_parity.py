"""GPU parity: libpcal through its C ABI against the FP64 CPU oracle.

Integer bins (2-bit per-code counts, int8 sums) must match bit for bit.
Floating point: phasors within 1e-5 of the oracle's largest phasor
(relative, infinity norm) and 1e-3 rad in phase; float32 bins within a
bound derived from FP32 compensated summation; the delay within 1e-3 of its
own 1-sigma.  Inputs come from the seeded generator only.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

PHASOR_RTOL = 1e-5
PHASE_ATOL = 1e-3


@pytest.fixture(scope="module")
def pcal():
    import torch

    from paper_2501_05993_gb300 import build as libbuild

    libbuild.build()
    import paper_2501_05993_gb300 as pkg

    pkg.load()
    torch.cuda.set_device(0)
    return pkg


def to_dev(host: np.ndarray, offset: int = 0):
    """Copy host bytes to the device so that element 0 sits `offset` bytes
    past a 256-byte boundary; returns (keepalive, device address)."""
    import torch

    raw = host.view(np.uint8)
    buf = torch.empty(raw.size + 512, dtype=torch.uint8, device="cuda")
    base = buf.data_ptr()
    start = ((base + 255) // 256 * 256 - base) + offset
    buf[start:start + raw.size].copy_(torch.from_numpy(raw))
    return buf, base + start


def n_samples(host, fmt):
    return host.size * 4 if fmt == "2bit" else host.size


def oracle_bins(host, fmt, n0, L):
    if fmt == "2bit":
        return oracle.counts_2bit(host, n0, L)
    if fmt == "i8":
        return oracle.sums_i8(host, n0, L)
    return oracle.sums_f32(host, n0, L)


def check_bins(gpu, ref, fmt, host=None, L=None, n0=0):
    if fmt in ("2bit", "i8"):
        assert gpu.dtype == np.int64 and np.array_equal(gpu, ref), \
            f"bins differ at {np.argwhere(gpu != ref)[:5].tolist()}"
    else:
        # FP32 compensated partial sums combined in FP64: error well below
        # 1e-6 of the sum of magnitudes per bin
        mag = oracle.fold_real(np.abs(host), "f32", n0, L)
        assert np.all(np.abs(gpu - ref) <= 1e-6 * mag + 1e-9)


def check_phasors(T, ref):
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(T - ref)) <= PHASOR_RTOL * scale, np.max(np.abs(T - ref)) / scale
    sig = np.abs(ref) > 1e-3 * scale
    dphi = np.abs(oracle.wrap(np.angle(T[sig]) - np.angle(ref[sig])))
    assert np.all(dphi <= PHASE_ATOL), dphi.max()


PLANS = {
    "c2": (64_000_000, 1_000_000, 10_000),       # L = 6400
    "c1": (16_000_000, 1_000_000, 10_000),       # L = 1600 (2-bit rows of 2 periods)
    "tiny": (16, 4, 1),                          # L = 16
    "image": (32_000_000, 1_000_000, 500_000),   # L = 64, f_offset = f_comb / 2
    "wide": (1_024_000_000, 1_000_000, 10_000),  # L = 102400, 25 column groups
    "odd": (48_000_000, 1_000_000, 30_000),      # L = 1600, N = 48
    "long": (256_000_000, 1_000_000, 1_000),     # L = 256000, N = 256: finalize by completion ticket
}


@pytest.mark.parametrize("fmt", ["2bit", "i8", "f32"])
@pytest.mark.parametrize("plan_name", list(PLANS))
@pytest.mark.parametrize("n_case", ["small", "bulk"])
def test_bins_and_phasors(pcal, fmt, plan_name, n_case):
    fs, fc, fo = PLANS[plan_name]
    if n_case == "small":
        n = 4 * 5003
    else:
        # several bulk tiles (>= 1 MB body) plus a ragged tail
        n = {"2bit": 4 * (1_600_000 + 4 * 1237), "i8": 3_000_000 + 1237, "f32": 900_000 + 1237}[fmt]
    s = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.05, td=7.1e-9 if fs > 1000 else 0.01, seed=17, stream=3)
    host = s.samples(fmt, 0, n)
    with pcal.Plan(fs, fc, fo, fmt) as p:
        keep, addr = to_dev(host, offset=4 if fmt == "f32" else 3)
        p.accumulate(addr, n)
        st = p.stats()
        if n_case == "bulk" and plan_name != "tiny":
            assert st["bulk_launches"] >= 1
        bins = p.bins()
        ref = oracle_bins(host, fmt, 0, p.L)
        check_bins(bins, ref, fmt, host, p.L)
        T = p.finalize()
        res = p.results()
    S = oracle.bins(host, fmt, 0, p.L)
    check_phasors(T, oracle.tones_from_bins(S, fs, fc, fo))
    assert np.allclose(res["amp"], 2 * np.abs(T) / n, rtol=1e-6)  # FP32 amplitudes


@pytest.mark.parametrize("fmt", ["2bit", "i8", "f32"])
def test_direct_definition_small(pcal, fmt):
    """Against the O(M*N) direct definition on a ragged, phase-shifted run."""
    fs, fc, fo = 64_000, 1000, 30
    n0, n = 4 * 321, 4 * 30011
    s = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.2, td=2.5e-6, seed=99)
    pre = s.samples(fmt, 0, n0)
    host = s.samples(fmt, n0, n)
    with pcal.Plan(fs, fc, fo, fmt) as p:
        k1, a1 = to_dev(pre, 1 if fmt != "f32" else 0)
        p.accumulate(a1, n0)
        p.finalize()  # first period ends; the absolute index keeps counting
        k2, a2 = to_dev(host, 7 if fmt != "f32" else 8)
        p.accumulate(a2, n)
        T = p.finalize()
    check_phasors(T, oracle.direct(host, fmt, n0, fs, fc, fo))


@pytest.mark.parametrize("fmt", ["2bit", "i8"])
def test_chunk_splits_are_invisible(pcal, fmt):
    fs, fc, fo = PLANS["c2"]
    n = 4 * 1_700_000
    host = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.01, td=1e-9, seed=5).samples(fmt, 0, n)
    cuts = [0, 4 * 3, 4 * 700_001, 4 * 700_013, 4 * 1_650_000, n]
    with pcal.Plan(fs, fc, fo, fmt) as p:
        keep = []
        for a, b in zip(cuts[:-1], cuts[1:]):
            per = 4 if fmt == "2bit" else 1
            part = host[a // per: b // per]
            kk, addr = to_dev(part, offset=(a // 4) % 13)
            keep.append(kk)
            p.accumulate(addr, b - a)
        bins = p.bins()
    assert np.array_equal(bins, oracle_bins(host, fmt, 0, p.L))


@pytest.mark.parametrize("fmt", ["2bit", "i8", "f32"])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_chunk_splits_and_offsets(pcal, fmt, seed):
    """Random cut points (whole bytes for 2-bit) and random byte offsets of
    each chunk's device buffer: the bins are those of the whole stream (exact
    for 2-bit and int8), whatever mix of ragged and bulk work each call gets."""
    rng = np.random.default_rng(100 + seed)
    fs, fc, fo = PLANS["odd"] if seed == 2 else PLANS["c2"]
    n = {"2bit": 4 * 1_500_000, "i8": 4_200_000, "f32": 2_000_000}[fmt]
    q = 4 if fmt == "2bit" else 1
    host = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.03, td=2e-9, seed=seed).samples(fmt, 0, n)
    cuts = sorted(set([0, n] + [int(c) // q * q for c in rng.integers(1, n, 6)]))
    with pcal.Plan(fs, fc, fo, fmt) as p:
        keep = []
        for a, b in zip(cuts[:-1], cuts[1:]):
            part = host[a // q: b // q]
            off = int(rng.integers(0, 16)) // (4 if fmt == "f32" else 1) * (4 if fmt == "f32" else 1)
            kk, addr = to_dev(part, offset=off)
            keep.append(kk)
            p.accumulate(addr, b - a)
        bins = p.bins()
    check_bins(bins, oracle_bins(host, fmt, 0, p.L), fmt, host, p.L)


def test_two_bit_levels_and_spill(pcal):
    """Small L forces the packed 21-bit fields to spill; custom levels."""
    fs, fc, fo = 16, 4, 1
    n = 4 * 9_000_000  # 36M samples > (2^21 - 2) * 16
    host = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.3, td=0.02, seed=8).bits2(0, n)
    lev = (-2.5, -0.75, 0.5, 4.0)
    with pcal.Plan(fs, fc, fo, "2bit") as p:
        p.set_levels(lev)
        keep, addr = to_dev(host)
        p.accumulate(addr, n)
        bins = p.bins()
        T = p.finalize()
    cnt = oracle.counts_2bit(host, 0, 16)
    assert np.array_equal(bins, cnt)
    check_phasors(T, oracle.tones_from_bins(oracle.decode_counts(cnt, lev), fs, fc, fo))


def test_products_and_delay(pcal):
    # A weak comb (0.005 sigma): 2-bit quantisation of a strong comb biases
    # the delay through intermodulation (about -49 ps at 0.01 sigma), which
    # is a property of the data, not of the extraction.
    fs, fc, fo, td = 64_000_000, 1_000_000, 10_000, 12.5e-9
    n = 4 * 16_000_000
    host = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.005, td=td, seed=21).bits2(0, n)
    with pcal.Plan(fs, fc, fo, "2bit") as p:
        keep, addr = to_dev(host)
        p.accumulate(addr, n)
        p.finalize()
        r = p.results()
    ref = oracle.products(oracle.fold(host, "2bit", 0, fs, fc, fo), n, fs, fc, fo)
    assert np.allclose(r["amp"], ref["amp"], rtol=1e-5)
    assert np.max(np.abs(oracle.wrap(r["phase"] - ref["phase"]))) < PHASE_ATOL
    assert np.max(np.abs(r["unwrapped"] - ref["unwrapped"])) < PHASE_ATOL
    assert abs(r["td"] - ref["td"]) <= 1e-3 * ref["sigma_td"]
    assert abs(r["sigma_td"] - ref["sigma_td"]) <= 1e-3 * ref["sigma_td"]
    assert abs(r["td"] - td) < 5 * ref["sigma_td"]  # physics: delay recovered


@pytest.mark.parametrize("plan_name", ["c2", "c1", "odd", "long", "wide"])
def test_peak_delay_and_bandpass(pcal, plan_name):
    """Post-processing (cluster and completion-ticket finalizes): the delay
    from the time-domain pulse and the delay-corrected bandpass phase against
    the oracle's, on a strong comb (float32, so no 2-bit intermodulation)."""
    fs, fc, fo = PLANS[plan_name]
    L = oracle.plan(fs, fc, fo)["L"]
    n = max(2 * L, 2_000_000) // L * L
    td = 17.3 / fs
    host = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.2, td=td, seed=5).f32(0, n)
    with pcal.Plan(fs, fc, fo, "f32") as p:
        keep, addr = to_dev(host, 4)
        p.accumulate(addr, n)
        T = p.finalize()
        post = p.post()
    ref = oracle.products(oracle.tones_from_bins(oracle.bins(host, "f32", 0, L), fs, fc, fo), n, fs, fc, fo)
    N = fs // fc
    assert abs(post["td_peak"] - ref["td_peak"]) <= 1e-3 / fs
    half = N / (2 * fs)
    assert abs(post["td_peak"] - ((td + half) % (2 * half) - half)) < 0.25 / fs  # the pulse is where td puts it
    ok = np.isfinite(ref["bandpass_phase"])
    assert ok.all()
    assert np.max(np.abs(post["bandpass_phase"] - ref["bandpass_phase"])) < PHASE_ATOL
    assert np.max(np.abs(post["bandpass_phase"])) < 0.05  # a flat band once the delay is removed


def test_empty_and_invalid(pcal):
    with pcal.Plan(64_000_000, 1_000_000, 10_000, "2bit") as p:
        p.accumulate(0, 0)  # no-op
        with pytest.raises(pcal.PcalError) as ei:
            p.accumulate(1, 6)  # 2-bit needs whole bytes
        assert ei.value.code == pcal.PCAL_EINVAL
        T = p.finalize()
        r = p.results()
        assert np.all(T == 0) and np.all(r["amp"] == 0) and np.isnan(r["td"])
    with pcal.Plan(16_000_000, 1_000_000, 10_000, "f32") as p:
        with pytest.raises(pcal.PcalError):
            p.accumulate(2, 16)  # misaligned float pointer


def test_host_accumulate_matches_device(pcal):
    fs, fc, fo = PLANS["c2"]
    n = 4 * 40_000_000  # 160 MB: three staging chunks
    host = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.01, td=1e-9, seed=6).bits2(0, n)
    with pcal.Plan(fs, fc, fo, "2bit") as p:
        p.accumulate_host(host)
        bins_h = p.bins()
    assert np.array_equal(bins_h, oracle.counts_2bit(host, 0, p.L))


def test_pipelined_host_periods(pcal):
    """accumulate_host_async + finalize_async over three periods, each period's results read one call later
    from the pinned ring (and the last at age 0): every period matches the oracle, and ages outside the ring
    are refused."""
    fs, fc, fo = PLANS["c2"]
    n = 4 * 17_000_003  # two staging chunks and a ragged tail
    hosts = [synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.02, td=2e-9, seed=60 + k).bits2(k * n, n) for k in range(3)]
    got = []
    with pcal.Plan(fs, fc, fo, "2bit") as p:
        with pytest.raises(pcal.PcalError):
            p.read_async(0)  # nothing finalized yet
        for k, h in enumerate(hosts):
            p.accumulate_host_async(h, n)
            p.finalize_async()
            if k:
                got.append(p.read_async(age=1))
        got.append(p.read_async(age=0))
        with pytest.raises(pcal.PcalError):
            p.read_async(2)
        L = p.L
    for k, (h, r) in enumerate(zip(hosts, got)):
        ref = oracle.tones_from_bins(oracle.bins(h, "2bit", k * n, L), fs, fc, fo)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(r["phasors"] - ref)) <= PHASOR_RTOL * scale, k
        pr = oracle.products(ref, n, fs, fc, fo)
        assert abs(r["td"] - pr["td"]) <= 1e-3 * pr["sigma_td"]


def test_f32_partial_slots_across_many_calls(pcal):
    """Float32 folds leave per-tile partials in a ring of slots that the
    finalize adds into the bins: seven calls of growing size in one period
    (the ring fills and is flushed, the slots are reallocated larger), a host
    read of the bins in the middle (which adds the pending slots first), then
    the finalize, against the oracle; a second period starts from empty bins."""
    fs, fc, fo = PLANS["c1"]
    sizes = [300_001, 1_200_000, 900_003, 2_500_000, 700_000, 1_800_017, 3_100_000]
    host = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.05, td=3.7e-9, seed=41).f32(0, sum(sizes) + 1_000_000)
    with pcal.Plan(fs, fc, fo, "f32") as p:
        keep, addr = to_dev(host)
        n0 = 0
        for i, n in enumerate(sizes):
            p.accumulate(addr + 4 * n0, n)
            n0 += n
            if i == 3:  # mid-period host read
                check_bins(p.bins(), oracle.sums_f32(host[:n0], 0, p.L), "f32", host[:n0], p.L)
        check_bins(p.bins(), oracle.sums_f32(host[:n0], 0, p.L), "f32", host[:n0], p.L)
        p.accumulate(addr + 4 * n0, 900_000)  # pending again when the period ends
        T = p.finalize()
        m = n0 + 900_000
        check_phasors(T, oracle.tones_from_bins(oracle.sums_f32(host[:m], 0, p.L), fs, fc, fo))
        p.accumulate(addr + 4 * m, 100_000)
        T2 = p.finalize()
    check_phasors(T2, oracle.direct(host[m:m + 100_000], "f32", m, fs, fc, fo))


def test_f32_is_deterministic(pcal):
    fs, fc, fo = PLANS["c1"]
    n = 4_000_000 + 17
    host = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.02, td=3.7e-9, seed=4).f32(0, n)
    out = []
    for _ in range(2):
        with pcal.Plan(fs, fc, fo, "f32") as p:
            keep, addr = to_dev(host)
            p.accumulate(addr, n)
            out.append(p.finalize())
    assert np.array_equal(out[0], out[1])


def test_full_size_two_bit_bench_workload(pcal):
    """The benchmark's workload: 2-bit, fs 64 MHz, N 64, L 6400, 512M samples
    in one accumulate call (the launch configuration bench.py times)."""
    fs, fc, fo, td, n = 64_000_000, 1_000_000, 10_000, 12.5e-9, 512_000_000
    host = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.01, td=td, seed=2501059932).bits2(0, n)
    with pcal.Plan(fs, fc, fo, "2bit") as p:
        keep, addr = to_dev(host)
        p.accumulate(addr, n)
        bins = p.bins()
        T = p.finalize()
        r = p.results()
    cnt = oracle.counts_2bit(host, 0, p.L)
    assert np.array_equal(bins, cnt)
    ref = oracle.tones_from_bins(oracle.decode_counts(cnt), fs, fc, fo)
    check_phasors(T, ref)
    pr = oracle.products(ref, n, fs, fc, fo)
    assert abs(r["td"] - pr["td"]) <= 1e-3 * pr["sigma_td"]
    assert abs(r["sigma_td"] - pr["sigma_td"]) <= 1e-3 * pr["sigma_td"]


def test_full_size_f32_c1(pcal):
    """Config 1 at full size against the direct definition."""
    fs, fc, fo, td, n = 16_000_000, 1_000_000, 10_000, 3.7e-9, 16_000_000
    host = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.02, td=td, seed=2501059931).f32(0, n)
    with pcal.Plan(fs, fc, fo, "f32") as p:
        keep, addr = to_dev(host)
        p.accumulate(addr, n)
        T = p.finalize()
        r = p.results()
    ref = oracle.direct(host, "f32", 0, fs, fc, fo)
    check_phasors(T, ref)
    pr = oracle.products(ref, n, fs, fc, fo)
    assert abs(r["td"] - pr["td"]) <= 1e-3 * pr["sigma_td"]
    assert abs(r["td"] - td) < 5 * pr["sigma_td"]  # unquantised data: no bias


def test_bounded_wait_runs_out_and_the_context_survives(pcal):
    """A wait on a phase nothing completes gives up after its limit, the
    kernel reports it through the error bits and returns, and the device
    keeps working (a plan runs right after)."""
    import time

    t0 = time.perf_counter()
    rc, flags = pcal.pcal_selftest_wait_timeout(0.05)
    dt = time.perf_counter() - t0
    assert rc == pcal.PCAL_ETIMEOUT and flags & 1
    assert dt < 5.0
    fs, fc, fo = PLANS["c1"]
    host = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.1, td=1e-9, seed=2).bits2(0, 4 * 40_000)
    with pcal.Plan(fs, fc, fo, "2bit") as p:
        keep, addr = to_dev(host, 1)
        p.accumulate(addr, 4 * 40_000)
        assert np.array_equal(p.bins(), oracle.counts_2bit(host, 0, p.L))
