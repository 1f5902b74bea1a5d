"""Long-period plans (pcal_rotplan_*): prime and non-integral comb offsets.

There is no fold period to exploit, so every sample is rotated; the phasors
must still match the oracle's direct definition (phases reduced exactly in
128-bit integers) within the stated tolerance, across calls and periods, and
the delay products must agree with the oracle's.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

PHASOR_RTOL = 1e-5

CASES = [
    # fs, f_comb, f_offset, format, samples
    (16_000_000, 1_000_000, 10_007.0, "i8", 400_011),       # prime offset: L = 16e6 > 2^20
    (16_000_000, 1_000_000, 10_007.25, "f32", 300_000),     # a quarter hertz
    (32_000_000, 1_000_000, 333.3125, "2bit", 4 * 100_003),  # 2-bit, binary fraction
    (64_000_000, 1_000_000, 499_999.5, "i8", 500_000),      # close to f_comb / 2
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


def _dev(host, offset):
    import torch

    raw = host.view(np.uint8)
    buf = torch.zeros(raw.size + 64, dtype=torch.uint8, device="cuda")
    buf[offset:offset + raw.size].copy_(torch.from_numpy(raw))
    return buf, buf.data_ptr() + offset


@pytest.mark.parametrize("case", CASES, ids=[f"{c[2]}-{c[3]}" for c in CASES])
def test_rotplan_matches_direct_definition(pcal, case):
    fs, fc, fo, fmt, n = case
    s = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.1, td=4e-9, seed=12)
    cut = (n // 3) // 4 * 4
    h1, h2 = s.samples(fmt, 0, cut), s.samples(fmt, cut, n - cut)
    with pcal.RotPlan(fs, fc, fo, fmt) as rp:
        k1, a1 = _dev(h1, 3 if fmt != "f32" else 4)
        k2, a2 = _dev(h2, 5 if fmt != "f32" else 8)
        rp.accumulate(a1, cut)
        rp.accumulate(a2, n - cut)  # continues the absolute index
        rp.finalize_device()
        r = rp.results()
        # second period: the rotator phase keeps counting from n
        h3 = s.samples(fmt, n, n)
        k3, a3 = _dev(h3, 0)
        rp.accumulate(a3, n)
        rp.finalize_device()
        r2 = rp.results()
    ref = oracle.direct_any(np.concatenate([h1, h2]), fmt, 0, fs, fc, fo)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(r["phasors"] - ref)) <= PHASOR_RTOL * scale, np.max(np.abs(r["phasors"] - ref)) / scale
    ref2 = oracle.direct_any(h3, fmt, n, fs, fc, fo)
    assert np.max(np.abs(r2["phasors"] - ref2)) <= PHASOR_RTOL * np.max(np.abs(ref2))
    pr = oracle.products(ref, n, fs, fc, fo)
    assert np.allclose(r["amp"], pr["amp"], rtol=1e-5, atol=1e-5 * np.max(pr["amp"]))
    assert abs(r["td"] - pr["td"]) <= 1e-3 * pr["sigma_td"]
    assert abs(r["td_peak"] - pr["td_peak"]) <= 1e-3 / fs


def test_rotplan_rejects_bad_plans(pcal):
    for args, code in [((16e6, 1e6, 1.5e6, "i8"), pcal.PCAL_EINVAL),   # f_offset >= f_comb
                       ((16.5e6, 1e6, 10.0, "i8"), pcal.PCAL_EINVAL),   # fs not a multiple of f_comb
                       ((2048e6, 1e6, 10.0, "i8"), pcal.PCAL_ETOOLARGE)]:
        with pytest.raises(pcal.PcalError) as ei:
            pcal.RotPlan(*args)
        assert ei.value.code == code
