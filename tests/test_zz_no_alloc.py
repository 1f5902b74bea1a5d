"""The allocation-free finalize entry point, for callers that cannot allocate
GPU memory (a fixed pool or arena, a budget fixed at start-up, a stream under
graph capture).  It must give the same phasors and delay as the plan-based
finalize, call after call.  This file is collected last."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_plan_finalize_twice():
    import torch

    from paper_2501_05993_gb300 import build as libbuild

    libbuild.build()
    import paper_2501_05993_gb300 as pcal

    torch.cuda.set_device(0)
    fs, fc, fo = 64_000_000, 1_000_000, 10_000
    n = 4 * 3_000_001
    host = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.02, td=12.5e-9, seed=77).bits2(0, n)
    levels = (-3.3359, -1.0, 1.0, 3.3359)
    with pcal.Plan(fs, fc, fo, "2bit") as p:
        p.accumulate(torch.from_numpy(host).cuda(), n)
        counts = p.bins()
        T_ref = p.finalize()
        ref = p.results()
        N = p.N
    d_counts = torch.from_numpy(counts).cuda()
    for call in range(2):
        d_res = torch.full((5 * N + 3,), float("nan"), dtype=torch.float64, device="cuda")
        pcal.pcal_tones_from_counts_noalloc(fs, fc, fo, N, d_counts, n, levels, d_res)
        torch.cuda.synchronize()
        res = d_res.cpu().numpy()
        T = res[0:2 * N:2] + 1j * res[1:2 * N:2]
        scale = np.max(np.abs(T_ref))
        assert np.max(np.abs(T - T_ref)) <= 1e-5 * scale, f"call {call}"
        assert np.max(np.abs(np.angle(T / T_ref))) <= 1e-3, f"call {call}"
        assert np.allclose(res[2 * N:3 * N], ref["amp"], rtol=1e-5)
        assert abs(res[5 * N] - ref["td"]) <= 1e-3 * ref["sigma_td"]
        assert res[5 * N + 2] == n


def test_noalloc_rejects_too_many_tones():
    import torch

    import paper_2501_05993_gb300 as pcal

    d = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(pcal.PcalError) as ei:
        pcal.pcal_tones_from_counts_noalloc(2048e6, 1e6, 10e3, 2048, d, 0, (-3, -1, 1, 3), d)
    assert ei.value.code == pcal.PCAL_ETOOLARGE
