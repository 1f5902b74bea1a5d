"""The allocation-free finalize entry point, for callers that cannot allocate
GPU memory (a fixed pool or arena, a budget fixed at start-up, a stream under
graph capture).  Given exact per-(bin, code) counts it must give the FP64
oracle's phasors, amplitudes and delay within the stated tolerances (phasors
1e-5 of the largest, phase 1e-3 rad, delay 1e-3 sigma_td), on every finalize
route it can take -- the 16-CTA cluster (N <= 256, L <= 32768), and the
grid-wide fold and DFT kernels for more tones or longer periods, which here
evaluate their twiddles on the fly -- and the same as the plan-based finalize,
call after call.  This file is collected last."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

LEVELS = (-3.3359, -1.0, 1.0, 3.3359)

# (fs, f_comb, f_offset, samples): N 64 / L 6400 (cluster), N 512 / L 10240
# (more tones than a cluster finalize takes), N 1024 / L 102400 (longest
# comb, period beyond the cluster's bins)
CASES = [
    (64_000_000, 1_000_000, 10_000, 4 * 3_000_001),
    (512_000_000, 1_000_000, 50_000, 4 * 2_500_003),
    (1_024_000_000, 1_000_000, 10_000, 4 * 2_600_000),
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


def run_noalloc(pcal, fs, fc, fo, N, d_counts, n):
    import torch

    d_res = torch.full((5 * N + 3,), float("nan"), dtype=torch.float64, device="cuda")
    pcal.pcal_tones_from_counts_noalloc(fs, fc, fo, N, d_counts, n, LEVELS, d_res)
    torch.cuda.synchronize()
    return d_res.cpu().numpy()


@pytest.mark.parametrize("case", CASES, ids=[f"N{c[0] // c[1]}" for c in CASES])
def test_noalloc_matches_oracle_twice(pcal, case):
    import torch

    fs, fc, fo, n = case
    N = fs // fc
    L = oracle.plan(fs, fc, fo)["L"]
    host = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.05, td=7.5e-9, seed=77).bits2(0, n)
    counts = oracle.counts_2bit(host, 0, L)
    ref = oracle.tones_from_bins(oracle.decode_counts(counts, LEVELS), fs, fc, fo)
    pr = oracle.products(ref, n, fs, fc, fo)
    d_counts = torch.from_numpy(counts).cuda()
    scale = np.max(np.abs(ref))
    for call in range(2):
        res = run_noalloc(pcal, fs, fc, fo, N, d_counts, n)
        T = res[0:2 * N:2] + 1j * res[1:2 * N:2]
        assert np.max(np.abs(T - ref)) <= 1e-5 * scale, (call, np.max(np.abs(T - ref)) / scale)
        strong = np.abs(ref) > 1e-2 * scale  # phase is defined where the tone stands out
        assert np.max(np.abs(np.angle(T[strong] / ref[strong]))) <= 1e-3, call
        assert np.allclose(res[2 * N:3 * N], pr["amp"], rtol=1e-5), call
        assert abs(res[5 * N] - pr["td"]) <= 1e-3 * pr["sigma_td"], (call, abs(res[5 * N] - pr["td"]) / pr["sigma_td"])
        assert res[5 * N + 2] == n


def test_noalloc_matches_plan_finalize_twice(pcal):
    import torch

    fs, fc, fo = 64_000_000, 1_000_000, 10_000
    n = 4 * 3_000_001
    host = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.02, td=12.5e-9, seed=77).bits2(0, n)
    with pcal.Plan(fs, fc, fo, "2bit") as p:
        p.accumulate(torch.from_numpy(host).cuda(), n)
        counts = p.bins()
        T_ref = p.finalize()
        ref = p.results()
        N = p.N
    d_counts = torch.from_numpy(counts).cuda()
    for call in range(2):
        res = run_noalloc(pcal, fs, fc, fo, N, d_counts, n)
        T = res[0:2 * N:2] + 1j * res[1:2 * N:2]
        scale = np.max(np.abs(T_ref))
        assert np.max(np.abs(T - T_ref)) <= 1e-5 * scale, f"call {call}"
        assert np.max(np.abs(np.angle(T / T_ref))) <= 1e-3, f"call {call}"
        assert np.allclose(res[2 * N:3 * N], ref["amp"], rtol=1e-5)
        assert abs(res[5 * N] - ref["td"]) <= 1e-3 * ref["sigma_td"]
        assert res[5 * N + 2] == n


def test_noalloc_rejects_too_many_tones(pcal):
    import torch

    d = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(pcal.PcalError) as ei:
        pcal.pcal_tones_from_counts_noalloc(2048e6, 1e6, 10e3, 2048, d, 0, (-3, -1, 1, 3), d)
    assert ei.value.code == pcal.PCAL_ETOOLARGE
