"""The seeded input generator: Philox known-answer vectors, chunk invariance,
and the statistics of each quantiser."""
import math

import numpy as np
import pytest

import synth

# Known-answer vectors published with the Philox4x32-10 reference code.
KAT = [
    ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
    ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
    ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
     [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
]


@pytest.mark.parametrize("ctr,key,out", KAT)
def test_philox_kat(ctr, key, out):
    assert synth.philox4x32(ctr, key) == out


@pytest.mark.parametrize("fmt", ["f32", "i8", "2bit"])
def test_chunking_is_invisible(fmt):
    s = synth.Stream(fs=64000, fc=1000, fo=10, amp=0.1, td=1e-6, seed=7, stream=3)
    whole = s.samples(fmt, 1000, 4 * 3000)
    parts = np.concatenate([s.samples(fmt, 1000, 4 * 1000), s.samples(fmt, 1000 + 4 * 1000, 4 * 2000)])
    assert np.array_equal(whole, parts)


def test_streams_and_seeds_differ():
    a = synth.Stream(fs=64000, fc=1000, fo=10, amp=0.0, td=0.0, seed=1, stream=0).real(0, 1000)
    b = synth.Stream(fs=64000, fc=1000, fo=10, amp=0.0, td=0.0, seed=1, stream=1).real(0, 1000)
    c = synth.Stream(fs=64000, fc=1000, fo=10, amp=0.0, td=0.0, seed=2, stream=0).real(0, 1000)
    assert not np.allclose(a, b) and not np.allclose(a, c)


def test_noise_statistics_and_quantisers():
    s = synth.Stream(fs=64000, fc=1000, fo=10, amp=0.0, td=0.0, seed=12)
    x = s.real(0, 400_000)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1) < 0.01
    q = s.bits2(0, 400_000)
    codes = ((q[:, None] >> (2 * np.arange(4))) & 3).reshape(-1)
    # thresholds 0 and +-0.98 sigma: P(|x| >= 0.98) = erfc(0.98/sqrt 2)
    p_outer = math.erfc(0.98 / math.sqrt(2))
    frac = np.bincount(codes, minlength=4) / codes.size
    assert abs(frac[0] + frac[3] - p_outer) < 0.005 and abs(frac[2] + frac[3] - 0.5) < 0.005
    # the 2-bit code follows the unquantised sample exactly
    expect = np.where(x >= 0, np.where(x >= 0.98, 3, 2), np.where(x >= -0.98, 1, 0))
    assert np.array_equal(codes, expect)
    i8 = s.i8(0, 400_000)
    assert np.array_equal(i8, np.clip(np.rint(20 * x), -128, 127).astype(np.int8))
    assert np.array_equal(s.f32(0, 1000), x[:1000].astype(np.float32))
