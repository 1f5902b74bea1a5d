"""Batched extraction (pcal_batch_*) against the FP64 CPU oracle.

Every channel of a batch -- mixed 2-bit and int8, different fs, f_offset,
period L and length, misaligned device buffers, channels too short for a
bulk row and empty channels -- must give exactly the oracle's integer bins
and phasors within the stated tolerance, whatever the launch schedule, and
the same through a replayed CUDA graph.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

PHASOR_RTOL = 1e-5

# (fs, f_comb, f_offset, format, samples, byte offset of the device buffer)
CHANNELS = [
    (64_000_000, 1_000_000, 10_000, "2bit", 4 * 1_003_217, 3),   # L 6400
    (32_000_000, 1_000_000, 0, "i8", 1_500_011, 5),              # f_offset 0: L = N = 32
    (128_000_000, 1_000_000, 370_000, "2bit", 4 * 901_237, 0),   # L 12800
    (256_000_000, 1_000_000, 990_000, "i8", 2_600_003, 11),      # L 25600
    (32_000_000, 1_000_000, 500_000, "2bit", 4 * 500_001, 7),    # f_offset = f_comb/2: L 64
    (16, 4, 1, "i8", 40_000, 1),                                 # L 16, N 4
    (64_000_000, 1_000_000, 20_000, "2bit", 4 * 1_000, 2),       # too short for one bulk row
    (128_000_000, 1_000_000, 50_000, "i8", 0, 0),                # empty this period
    (1_024_000_000, 1_000_000, 10_000, "i8", 1_500_007, 9),      # N 1024, L 102400: DFT over the cluster
    (512_000_000, 1_000_000, 30_000, "2bit", 4 * 700_001, 4),    # N 512, L 51200
]


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
    import torch

    raw = host.view(np.uint8)
    buf = torch.zeros(raw.size + 512, dtype=torch.uint8, device="cuda")
    base = buf.data_ptr()
    start = ((base + 255) // 256 * 256 - base) + offset
    if raw.size:
        buf[start:start + raw.size].copy_(torch.from_numpy(raw))
    return buf, base + start


def make_inputs(channels, seed=5, n0=None):
    hosts = []
    for i, (fs, fc, fo, fmt, n, _) in enumerate(channels):
        s = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.05, td=3e-9 * (i + 1) if fs > 1000 else 0.01, seed=seed,
                         stream=i)
        hosts.append(s.samples(fmt, 0 if n0 is None else n0[i], n))
    return hosts


def upload(channels, hosts):
    keep, ptrs = [], []
    for (fs, fc, fo, fmt, n, off), h in zip(channels, hosts):
        k, a = to_dev(h, off)
        keep.append(k)
        ptrs.append(a)
    return keep, ptrs


def check_channel(batch, c, ch, host, n0=0):
    fs, fc, fo, fmt, n, _ = ch
    L = int(batch.geometry[c].L)
    bins = batch.bins(c)
    if fmt == "2bit":
        ref = oracle.counts_2bit(host, n0, L)
    else:
        ref = oracle.sums_i8(host, n0, L)
    assert np.array_equal(bins, ref), f"channel {c}: bins differ at {np.argwhere(bins != ref)[:4].tolist()}"
    return bins


def check_results(batch, c, ch, host, n0=0):
    fs, fc, fo, fmt, n, _ = ch
    res = batch.results(c)
    if n == 0:
        return res  # no samples this period: nothing to compare
    L = int(batch.geometry[c].L)
    S = oracle.bins(host, fmt, n0, L)
    ref = oracle.tones_from_bins(S, fs, fc, fo)
    T = res["phasors"]
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(T - ref)) <= PHASOR_RTOL * scale, (c, np.max(np.abs(T - ref)) / scale)
    assert np.allclose(res["amp"], 2 * np.abs(T) / n, rtol=1e-6)
    post = batch.post(c)
    pref = oracle.products(ref, n, fs, fc, fo)
    assert abs(post["td_peak"] - pref["td_peak"]) <= 1e-3 / fs
    mag = np.abs(ref)
    if np.all(np.isfinite(pref["bandpass_phase"])) and mag.min() > 0.05 * mag.max():  # unwrapping well defined
        assert np.max(np.abs(post["bandpass_phase"] - pref["bandpass_phase"])) < 1e-3
    return res


def test_batch_bins_and_phasors(pcal):
    hosts = make_inputs(CHANNELS)
    keep, ptrs = upload(CHANNELS, hosts)
    with pcal.Batch([c[:4] for c in CHANNELS]) as b:
        b.accumulate(ptrs, [c[4] for c in CHANNELS])
        st = b.stats()
        assert st["bulk_launches"] == 1  # one persistent launch for every channel
        for c, (ch, h) in enumerate(zip(CHANNELS, hosts)):
            check_channel(b, c, ch, h)
        b.finalize_device()
        for c, (ch, h) in enumerate(zip(CHANNELS, hosts)):
            check_results(b, c, ch, h)


@pytest.mark.parametrize("mode", ["tf32x3", "bf16x6"])
def test_batch_tensor_core_dft(pcal, mode):
    """The finalize with the tone DFT as one tensor-core contraction per N: every channel's phasors and
    post-processing within the stated tolerance of the oracle, and the delay within 1e-3 sigma_td, the bound
    of the CUDA-core paths (on the strongest combs here sigma_td ~ 7e-13 s)."""
    hosts = make_inputs(CHANNELS, seed=9)
    keep, ptrs = upload(CHANNELS, hosts)
    with pcal.Batch([c[:4] for c in CHANNELS]) as b:
        b.set_dft(mode)
        b.accumulate(ptrs, [c[4] for c in CHANNELS])
        b.finalize_device()
        assert b.stats()["kernel_launches"] >= 3  # clusters up to P, one DFT per N, products
        for c, (ch, h) in enumerate(zip(CHANNELS, hosts)):
            res = check_results(b, c, ch, h)
            if ch[4]:
                pr = oracle.products(oracle.tones_from_bins(oracle.bins(h, ch[3], 0, int(b.geometry[c].L)),
                                                            *ch[:3]), ch[4], *ch[:3])
                assert abs(res["td"] - pr["td"]) <= 1e-3 * pr["sigma_td"], (c, abs(res["td"] - pr["td"]) / pr["sigma_td"])
        # a second period in the same mode, then back to the CUDA-core DFT
        hosts2 = make_inputs(CHANNELS, seed=10, n0=[c[4] for c in CHANNELS])
        keep2, ptrs2 = upload(CHANNELS, hosts2)
        b.accumulate(ptrs2, [c[4] for c in CHANNELS])
        b.finalize_device()
        for c, (ch, h) in enumerate(zip(CHANNELS, hosts2)):
            check_results(b, c, ch, h, n0=ch[4])
        b.set_dft("fp32")
        hosts3 = make_inputs(CHANNELS, seed=11, n0=[2 * c[4] for c in CHANNELS])
        keep3, ptrs3 = upload(CHANNELS, hosts3)
        b.accumulate(ptrs3, [c[4] for c in CHANNELS])
        b.finalize_device()
        for c, (ch, h) in enumerate(zip(CHANNELS, hosts3)):
            check_results(b, c, ch, h, n0=2 * ch[4])


@pytest.mark.parametrize("sched", [
    dict(ctas=152, box_rows=32, static_pct=0, min_chunk=1, col_cap=224),
    dict(ctas=37, box_rows=64, static_pct=100, min_chunk=8, col_cap=128),
    dict(ctas=300, box_rows=32, static_pct=60, min_chunk=3, col_cap=128, stages=3),
    dict(ctas=136, box_rows=64, static_pct=90, min_chunk=16, col_cap=224, col_cap_bucket=[64, 128, 64, 0, 224, 64, 128, 64]),
])
def test_batch_schedule_does_not_change_bins(pcal, sched):
    hosts = make_inputs(CHANNELS, seed=9)
    keep, ptrs = upload(CHANNELS, hosts)
    with pcal.Batch([c[:4] for c in CHANNELS]) as b:
        b.set_schedule(**sched)
        b.accumulate(ptrs, [c[4] for c in CHANNELS])
        for c, (ch, h) in enumerate(zip(CHANNELS, hosts)):
            check_channel(b, c, ch, h)


def test_batch_matches_single_channel_plans(pcal):
    """The same channels one plan at a time give the same exact bins and
    phasors within the tolerance."""
    hosts = make_inputs(CHANNELS[:4], seed=21)
    keep, ptrs = upload(CHANNELS[:4], hosts)
    with pcal.Batch([c[:4] for c in CHANNELS[:4]]) as b:
        b.accumulate(ptrs, [c[4] for c in CHANNELS[:4]])
        bb = [b.bins(c) for c in range(4)]
        b.finalize_device()
        rb = [b.results(c) for c in range(4)]
    for c, (fs, fc, fo, fmt, n, off) in enumerate(CHANNELS[:4]):
        with pcal.Plan(fs, fc, fo, fmt) as p:
            p.accumulate(ptrs[c], n)
            assert np.array_equal(p.bins(), bb[c])
            T = p.finalize()
        scale = np.max(np.abs(T))
        assert np.max(np.abs(rb[c]["phasors"] - T)) <= PHASOR_RTOL * scale


def test_batch_two_calls_and_two_periods(pcal):
    """Chunks continue each channel's sample index; a finalize starts the
    next period with empty bins."""
    chans = CHANNELS[:6]
    hosts = make_inputs(chans, seed=33)
    cut = [((ch[4] // 3) // 4) * 4 for ch in chans]
    first = [h[:c // 4] if ch[3] == "2bit" else h[:c] for h, c, ch in zip(hosts, cut, chans)]
    second = [h[c // 4:] if ch[3] == "2bit" else h[c:] for h, c, ch in zip(hosts, cut, chans)]
    with pcal.Batch([c[:4] for c in chans]) as b:
        k1, p1 = upload(chans, first)
        b.accumulate(p1, cut)
        k2, p2 = upload([(c[0], c[1], c[2], c[3], c[4], (c[5] + 6) % 16) for c in chans], second)
        b.accumulate(p2, [ch[4] - c for ch, c in zip(chans, cut)])
        for c, (ch, h) in enumerate(zip(chans, hosts)):
            check_channel(b, c, ch, h)
        b.finalize_device()
        for c, (ch, h) in enumerate(zip(chans, hosts)):
            check_results(b, c, ch, h)
        # period 2 starts at each channel's absolute index n
        hosts2 = make_inputs(chans, seed=34, n0=[ch[4] for ch in chans])
        k3, p3 = upload(chans, hosts2)
        b.accumulate(p3, [ch[4] for ch in chans])
        for c, (ch, h) in enumerate(zip(chans, hosts2)):
            check_channel(b, c, ch, h, n0=ch[4])
        b.finalize_device()
        for c, (ch, h) in enumerate(zip(chans, hosts2)):
            check_results(b, c, ch, h, n0=ch[4])


def test_batch_repeated_call_on_the_same_buffers(pcal):
    """A call that repeats the previous call's buffers and lengths reuses its device descriptors: the samples are
    read again and continue each channel's index (bins = the oracle over the stream twice over)."""
    chans = CHANNELS
    hosts = make_inputs(chans, seed=51)
    keep, ptrs = upload(chans, hosts)
    n = [ch[4] for ch in chans]
    with pcal.Batch([c[:4] for c in chans]) as b:
        for _ in range(3):
            b.accumulate(ptrs, n)
        for c, (ch, h) in enumerate(zip(chans, hosts)):
            L = int(b.geometry[c].L)
            count = oracle.counts_2bit if ch[3] == "2bit" else oracle.sums_i8
            ref = sum(count(h, k * ch[4], L) for k in range(3))
            bins = b.bins(c)
            assert np.array_equal(bins, ref), f"channel {c}: bins differ at {np.argwhere(bins != ref)[:4].tolist()}"
        b.finalize_device()
        for c, (ch, h) in enumerate(zip(chans, hosts)):
            if ch[4] == 0:
                continue
            fs, fc, fo, fmt = ch[:4]
            L = int(b.geometry[c].L)
            S = sum(oracle.bins(h, fmt, k * ch[4], L) for k in range(3))
            ref = oracle.tones_from_bins(S, fs, fc, fo)
            T = b.results(c)["phasors"]
            assert np.max(np.abs(T - ref)) <= PHASOR_RTOL * np.max(np.abs(ref)), c


@pytest.mark.parametrize("mode", ["fp32", "tf32x3"])
def test_batch_graph_replay(pcal, mode):
    """A captured step replayed on refilled buffers gives each period's
    oracle results (with either DFT of the finalize)."""
    import torch

    chans = CHANNELS[:6]
    with pcal.Batch([c[:4] for c in chans]) as b:
        b.set_dft(mode)
        hosts = make_inputs(chans, seed=40)
        keep, ptrs = upload(chans, hosts)
        n = [ch[4] for ch in chans]
        for period in range(3):
            if period:
                n0 = [period * ch[4] for ch in chans]
                hosts = make_inputs(chans, seed=40 + period, n0=n0)
                for k, h, ch in zip(keep, hosts, chans):
                    raw = torch.from_numpy(h.view(np.uint8))
                    base = k.data_ptr()
                    start = ((base + 255) // 256 * 256 - base) + ch[5]
                    if raw.numel():
                        k[start:start + raw.numel()].copy_(raw)
            b.step_graph(ptrs, n)
            for c, (ch, h) in enumerate(zip(chans, hosts)):
                check_results(b, c, ch, h, n0=period * ch[4])


def expected_tiling(cols: int, cap: int):
    """Column groups of a row of `cols` words under a width cap: as few groups as the cap allows, of equal width
    rounded up to 8 words."""
    gc = -(-cols // cap)
    cw = min(cap, -(-(-(-cols // gc)) // 8) * 8)
    return cw, -(-cols // cw)


def test_batch_bucket_caps_cut_each_channel(pcal):
    """Every channel's rows are cut by its own bucket's cap (format x row width), else by col_cap; a cap
    outside {0, 64, 128, 224} is refused."""
    with pcal.Batch([c[:4] for c in CHANNELS]) as b:
        caps = [64, 128, 224, 64, 128, 64, 0, 224]
        b.set_schedule(col_cap=128, col_cap_bucket=caps)
        assert b.schedule["col_cap_bucket"] == caps
        for c in range(len(CHANNELS)):
            t = b.channel_tiling(c)
            g = b.geometry[c]
            cols = int(g.row_samples) // (16 if CHANNELS[c][3] == "2bit" else 4)
            cls = 0 if cols <= 256 else 1 if cols <= 1024 else 2 if cols <= 4096 else 3
            assert t["bucket"] == (4 if CHANNELS[c][3] == "i8" else 0) + cls
            cap = caps[t["bucket"]] or 128
            assert (t["col_width"], t["col_groups"]) == expected_tiling(cols, cap), (c, t, cols, cap)
        with pytest.raises(pcal.PcalError):
            b.set_schedule(col_cap_bucket=[0, 0, 0, 96, 0, 0, 0, 0])
        assert b.schedule["col_cap_bucket"] == caps


def test_batch_autotune_keeps_results(pcal):
    hosts = make_inputs(CHANNELS, seed=50)
    keep, ptrs = upload(CHANNELS, hosts)
    n = [c[4] for c in CHANNELS]
    with pcal.Batch([c[:4] for c in CHANNELS]) as b:
        chosen = b.autotune(ptrs, n)
        assert chosen["box_rows"] in (32, 64) and chosen["col_cap"] in (128, 224)
        import torch

        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert chosen["ctas"] == 0 or sms - chosen["ctas"] in (8, 16)
        assert all(v in (0, 64, 128, 224) for v in chosen["col_cap_bucket"])
        assert b.schedule == chosen
        for c in range(len(CHANNELS)):  # the chosen caps are the ones the channels are cut by
            t = b.channel_tiling(c)
            cols = int(b.geometry[c].row_samples) // (16 if CHANNELS[c][3] == "2bit" else 4)
            cap = chosen["col_cap_bucket"][t["bucket"]] or chosen["col_cap"]
            assert (t["col_width"], t["col_groups"]) == expected_tiling(cols, cap)
        for c in range(len(CHANNELS)):  # bins emptied again
            assert not np.any(b.bins(c)[:, 1:] if CHANNELS[c][3] == "2bit" else b.bins(c))
        b.accumulate(ptrs, n)
        for c, (ch, h) in enumerate(zip(CHANNELS, hosts)):
            check_channel(b, c, ch, h)
