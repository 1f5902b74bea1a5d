"""Batched tone DFT (pcal_dft_*): CUDA-core FP32 and tensor-core (tcgen05) split-TF32 / split-BF16 modes
against the DFT definition T_i = sum_b P[b] e^{-j 2 pi i b / N} in FP64 (numpy's FFT evaluates exactly that
sum), within the phasor tolerance of 1e-5 of the largest phasor; the tensor-core modes, whose chunk sums are
added on CUDA cores in FP32, are held to the tighter bound of an FP32 sum."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# max |T - T_ref| / max |T_ref| per channel: the phasor tolerance for the CUDA-core FP32 sums (sequential over
# N terms, ~3e-6 measured at N = 1024); the tensor-core modes keep 2^-22 (split TF32) or 2^-26 (split BF16) of
# each operand and add FP32 chunk sums rounded to nearest
BOUND = {"fp32": 1e-5, "tf32x3": 2e-6, "bf16x6": 2e-6}
MODES = ["fp32", "tf32x3", "bf16x6"]
SHAPES = [(1, 16), (5, 50), (130, 64), (300, 256), (129, 1024), (64, 200)]


@pytest.fixture(scope="module")
def pcal():
    import torch

    from paper_2501_05993_gb300 import build as libbuild

    libbuild.build()
    import paper_2501_05993_gb300 as pkg

    pkg.load()
    torch.cuda.set_device(0)
    return pkg


def run(pcal, mode, P):
    import torch

    C, N = P.shape
    dP = torch.from_numpy(P.astype(np.complex64)).cuda()
    dT = torch.full((max(C, 1), N), complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")
    with pcal.Dft(N, mode) as d:
        d.execute(dP, C, dT)
        assert d.check() == 0
    return dT.cpu().numpy()[:C]


def rel_err(T, ref):
    return np.max(np.abs(T - ref), axis=1) / np.max(np.abs(ref), axis=1)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", SHAPES, ids=[f"C{c}-N{n}" for c, n in SHAPES])
def test_dft_matches_definition(pcal, mode, shape):
    C, N = shape
    rng = np.random.default_rng(C * 1000 + N)
    P = (rng.standard_normal((C, N)) + 1j * rng.standard_normal((C, N))) * 10.0 ** rng.uniform(-3, 6, (C, 1))
    P += 3 * np.sqrt(N) * np.exp(2j * np.pi * rng.integers(0, N, (C, 1)) * np.arange(N) / N)  # a pulse
    T = run(pcal, mode, P)
    ref = np.fft.fft(P.astype(np.complex64).astype(np.complex128), axis=1)
    err = rel_err(T, ref)
    assert np.all(np.isfinite(T))
    assert err.max() <= BOUND[mode], (mode, shape, err.max())


@pytest.mark.parametrize("mode", MODES)
def test_pure_tone_closed_form(pcal, mode):
    """P[b] = e^{j 2 pi i0 b / N}: T = N at i0, 0 elsewhere."""
    N = 256
    i0 = np.arange(20) * 13 % N
    P = np.exp(2j * np.pi * i0[:, None] * np.arange(N)[None, :] / N)
    T = run(pcal, mode, P)
    ref = np.zeros_like(P)
    ref[np.arange(20), i0] = N
    assert rel_err(T, ref).max() <= BOUND[mode]


@pytest.mark.parametrize("mode", ["tf32x3", "bf16x6"])
def test_channel_result_does_not_depend_on_the_batch(pcal, mode):
    """Rows of the contraction are independent: a channel's tones are bit-identical alone and in a batch."""
    rng = np.random.default_rng(5)
    P = rng.standard_normal((200, 64)) + 1j * rng.standard_normal((200, 64))
    T_all = run(pcal, mode, P)
    for c in (0, 127, 128, 199):
        T_one = run(pcal, mode, P[c:c + 1])
        assert np.array_equal(T_one[0], T_all[c])


def test_empty_batch_and_bad_arguments(pcal):
    T = run(pcal, "tf32x3", np.zeros((0, 64), np.complex64))
    assert T.shape == (0, 64)
    for N, mode in [(0, "tf32x3"), (1025, "fp32")]:
        with pytest.raises(pcal.PcalError):
            pcal.Dft(N, mode)
