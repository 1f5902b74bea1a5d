"""Serving (pcal_server_*): continuous batching of live streams.

Each stream's per-period phasors must match the FP64 oracle within the
stated tolerance and be the same whether the stream runs alone or mixed with
others that arrive in interleaved chunks; streams beyond the HBM budget wait
and are admitted when a closed stream returns its memory.
"""
import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

PHASOR_RTOL = 1e-5
PERIOD_S = 0.02   # integration period of these tests (the workload uses 1 s)
CHUNK_S = 0.002   # chunk length (the workload uses 10 ms)
RING_S = 0.01

# (fs, f_comb, f_offset, format)
STREAMS = [
    (32_000_000, 1_000_000, 10_000, "2bit"),
    (64_000_000, 1_000_000, 370_000, "i8"),
    (16_000_000, 1_000_000, 0, "2bit"),
    (128_000_000, 1_000_000, 990_000, "i8"),
    (32_000_000, 1_000_000, 500_000, "i8"),
    (256_000_000, 1_000_000, 20_000, "2bit"),
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


def stream_samples(i, st, periods):
    fs, fc, fo, fmt = st
    n = int(fs * PERIOD_S) * periods
    s = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.05, td=2e-9 * (i + 1), seed=77, stream=100 + i)
    return s.samples(fmt, 0, n)


def chunks(host, st):
    """Host chunk views of CHUNK_S seconds (pinned copies)."""
    import torch

    fs, _, _, fmt = st
    spb = 4 if fmt == "2bit" else 1
    nb = int(fs * CHUNK_S) // spb
    out = []
    raw = host.view(np.uint8)
    for o in range(0, raw.size, nb):
        part = torch.from_numpy(raw[o:o + nb].copy()).pin_memory()
        out.append((part, part.numpy(), part.numel() * spb))
    return out


def run(pcal, ids_hosts, budget=1 << 30, order="round_robin"):
    """Submit every stream's chunks (interleaved), drain, return results by (stream index, period)."""
    with pcal.Server(budget, 16, PERIOD_S, RING_S) as srv:
        sid = {}
        for i, st, host in ids_hosts:
            sid[srv.open(*st)] = i
        queues = {s: chunks(h, st) for s, (i, st, h) in zip(sid, ids_hosts)}
        rng = np.random.default_rng(3)
        pending = {s: 0 for s in queues}
        while pending:
            live = sorted(pending)
            if order == "random":
                rng.shuffle(live)
            for s in live:
                _, arr, n = queues[s][pending[s]]
                srv.submit(s, arr, n)
                pending[s] += 1
                if pending[s] == len(queues[s]):
                    del pending[s]
        srv.drain(60)
        out = {}
        while True:
            r = srv.poll(0.0)
            if r is None:
                break
            out[(sid[r["stream"]], r["period"])] = r
        stats = srv.stats()
    return out, stats


def check_oracle(res, i, st, host, periods):
    fs, fc, fo, fmt = st
    per = int(fs * PERIOD_S)
    spb = 4 if fmt == "2bit" else 1
    L = int(pcal_geometry_L(st))
    for p in range(periods):
        part = host[p * per // spb:(p + 1) * per // spb]
        ref = oracle.tones_from_bins(oracle.bins(part, fmt, p * per, L), fs, fc, fo)
        T = res[(i, p)]["phasors"]
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(T - ref)) <= PHASOR_RTOL * scale, (i, p, np.max(np.abs(T - ref)) / scale)
        assert res[(i, p)]["n_samples"] == per


def pcal_geometry_L(st):
    import paper_2501_05993_gb300 as pkg

    fs, fc, fo, fmt = st
    return pkg.pcal_plan_geometry(fs, fc, fo, round(fs / fc), pkg.FORMATS[fmt]).L


def test_serve_alone_and_in_the_mix(pcal):
    periods = 2
    hosts = [stream_samples(i, st, periods) for i, st in enumerate(STREAMS)]
    mix, stats = run(pcal, [(i, st, h) for i, st, h in zip(range(len(STREAMS)), STREAMS, hosts)], order="random")
    assert stats["periods"] == periods * len(STREAMS)
    assert stats["p50_latency_s"] <= stats["p99_latency_s"] <= stats["max_latency_s"]
    for i, st in enumerate(STREAMS):
        check_oracle(mix, i, st, hosts[i], periods)
    for i in (0, 3):
        alone, _ = run(pcal, [(i, STREAMS[i], hosts[i])])
        for p in range(periods):
            a, m = alone[(i, p)]["phasors"], mix[(i, p)]["phasors"]
            assert np.max(np.abs(a - m)) <= PHASOR_RTOL * np.max(np.abs(a)), (i, p)


def test_serve_admission_by_budget(pcal):
    st = STREAMS[0]
    need = pcal.pcal_server_stream_bytes(*st, period_s=PERIOD_S, ring_s=RING_S)
    periods = 1
    hosts = [stream_samples(10 + k, st, periods) for k in range(3)]
    with pcal.Server(int(need * 2.5), 16, PERIOD_S, RING_S) as srv:
        a, b, c = (srv.open(*st) for _ in range(3))
        s0 = srv.stats()
        assert s0["admitted"] + s0["queued"] == 3 and s0["queued"] >= 1
        done = {}

        def feed(sid, host):
            for _, arr, n in chunks(host, st):
                srv.submit(sid, arr, n)
            done[sid] = True

        tc = threading.Thread(target=feed, args=(c, hosts[2]))  # blocks until admitted
        tc.start()
        feed(a, hosts[0])
        feed(b, hosts[1])
        srv.drain(60)
        assert c not in done  # still queued: the budget holds two streams
        srv.close_stream(a)
        tc.join(60)
        assert done.get(c)
        srv.drain(60)
        got = {}
        while True:
            r = srv.poll(0.0)
            if r is None:
                break
            got[r["stream"]] = r
        s1 = srv.stats()
        assert s1["admitted"] == 3 and s1["hbm_in_use"] <= s1["hbm_budget"]
    L = pcal_geometry_L(st)
    for sid, host in ((b, hosts[1]), (c, hosts[2])):
        ref = oracle.tones_from_bins(oracle.bins(host, st[3], 0, L), *st[:3])
        T = got[sid]["phasors"]
        assert np.max(np.abs(T - ref)) <= PHASOR_RTOL * np.max(np.abs(ref))


def test_serve_rejects_bad_streams(pcal):
    with pcal.Server(1 << 26, 4, PERIOD_S, RING_S) as srv:
        with pytest.raises(pcal.PcalError) as ei:
            srv.open(16_000_000, 1_000_000, 0, "f32")
        assert ei.value.code == pcal.PCAL_EINVAL
        with pytest.raises(pcal.PcalError) as ei:
            srv.open(2_048_000_000, 1_000_000, 10_000, "i8")
        assert ei.value.code == pcal.PCAL_ETOOLARGE
        sid = srv.open(*STREAMS[0])
        srv.close_stream(sid)
        srv.drain(10)
        with pytest.raises(pcal.PcalError):
            srv.submit(sid, np.zeros(16, np.uint8), 64)


def test_serve_latency_counts_from_the_chunk_arrival(pcal):
    """A period's latency runs from the arrival the client stamps on the chunk
    that completes it to its results on the host: a chunk stamped as having
    arrived 0.25 s before its submit reports at least 0.25 s more than the
    same chunk stamped at its submit, and an unstamped chunk counts from the
    submit's return."""
    st = STREAMS[0]
    host = stream_samples(0, st, 3)
    parts = chunks(host, st)
    per = len(parts) // 3
    with pcal.Server(1 << 30, 4, PERIOD_S, RING_S) as srv:
        sid = srv.open(*st)
        lat = []
        for period, lag in enumerate((0.25, 0.0, None)):
            for k, (_, arr, n) in enumerate(parts[period * per:(period + 1) * per]):
                when = None if lag is None else [pcal.clock_s() - (lag if k == per - 1 else 0.0)]
                srv.submit_many([sid], [arr], [n], arrival_s=when)
            srv.drain(30)
            r = srv.poll(5.0)
            assert r is not None and r["period"] == period
            lat.append(r["latency_s"])
        with pytest.raises(pcal.PcalError):
            srv.submit_many([sid], [parts[0][1]], [parts[0][2]], arrival_s=[float("nan")])
    assert lat[0] >= 0.25 + lat[1] - 0.05 and lat[0] >= 0.25
    assert 0 < lat[1] < 0.2 and 0 < lat[2] < 0.2
