"""Precision study kernels (pcal_rotfold_*): the paper's FP32 rotate-then-fold.

The GPU accumulators must equal, bit for bit, a host emulation of the same
FP32 operations in the same order (so each variant computes what it claims),
and the phasors must agree with the FP64 oracle within what FP32 allows.
The emulation itself is pinned to the oracle on the CPU.
"""
import numpy as np
import pytest

import oracle
import synth
from rotfold_emulation import emulate, phasors

FS, FC, FO = 16_000_000, 1_000_000, 10_000  # N 16, N_rot 1600
N, LANES = 16, 4


def make(n0, n, fmt="i8", seed=8):
    s = synth.Stream(fs=FS, fc=FC, fo=FO, amp=0.2, td=3e-9, seed=seed)
    return s.samples(fmt, n0, n)


@pytest.mark.parametrize("variant", ["table", "table_kahan", "dfr"])
def test_emulation_matches_oracle(variant):
    """CPU: the emulated FP32 route gives the oracle's phasors to FP32 accuracy."""
    x = make(0, 40_000)
    acc = emulate(x, 0, FS, FO, N, LANES, variant)
    T = phasors(acc)
    ref = oracle.direct(x, "i8", 0, FS, FC, FO)
    assert np.max(np.abs(T - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_emulation_catches_a_wrong_rotation_sign():
    """CPU: a conjugated rotator (the sign mistake of the paper's listings) is far off."""
    x = make(0, 20_000)
    acc = emulate(x, 0, FS, FS - FO, N, LANES, "table")  # exp(+j w_o n)
    ref = oracle.direct(x, "i8", 0, FS, FC, FO)
    assert np.max(np.abs(phasors(acc) - ref)) > 0.1 * np.max(np.abs(ref))


@pytest.fixture(scope="module")
def pcal():
    import torch

    from paper_2501_05993_gb300 import build as libbuild

    libbuild.build()
    import paper_2501_05993_gb300 as pkg

    pkg.load()
    torch.cuda.set_device(0)
    return pkg


@pytest.mark.gpu
@pytest.mark.parametrize("variant", ["table", "table_kahan", "dfr"])
@pytest.mark.parametrize("fmt", ["i8", "f32"])
def test_rotfold_bit_exact_with_emulation(pcal, variant, fmt):
    import torch

    n1, n2 = 30_011, 20_000
    x1, x2 = make(0, n1, fmt), make(n1, n2, fmt)
    with pcal.RotFold(FS, FC, FO, fmt, variant, lanes=LANES) as r:
        d1, d2 = torch.from_numpy(x1).cuda(), torch.from_numpy(x2).cuda()
        r.accumulate(d1, n1)
        r.accumulate(d2, n2)  # continues the absolute index
        torch.cuda.synchronize()
        got = r.acc()
        want = emulate(x2, n1, FS, FO, N, LANES, variant, emulate(x1, 0, FS, FO, N, LANES, variant))
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), \
            np.argwhere(got != want)[:4].tolist()
        T = r.finalize()
    ref = oracle.direct(np.concatenate([x1, x2]), fmt, 0, FS, FC, FO)
    assert np.max(np.abs(T - ref)) <= 1e-4 * np.max(np.abs(ref))
