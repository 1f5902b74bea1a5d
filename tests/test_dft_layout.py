"""Host checks of the tensor-core DFT's weight tiles (no GPU).

The tiles hold W^T of the real form of the tone DFT, T = [Re P | Im P] . W with
Re T_i and Im T_i in output columns 2i and 2i + 1 (angles 2 pi (i b mod N) / N),
each value split in two parts of the MMA type.  Decoding a tile with the no-swizzle K-major layout
(8-row x 16-byte core matrices, K-neighbours rows/8 * 128 bytes apart, 8-row
bands 128 bytes apart) must give back the matrix entries to the precision of the
split, and zeros in the padding.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import paper_2501_05993_gb300 as pcal

ESIZE = {"tf32x3": 4, "bf16x3": 2}
TILE = {"tf32x3": 128, "bf16x3": 256}  # output columns per tile


@pytest.fixture(scope="module")
def lib():
    from paper_2501_05993_gb300 import build as libbuild

    libbuild.build()
    return pcal.load()


def decode(tile: np.ndarray, rows: int, esize: int) -> np.ndarray:
    """rows x (128 / esize) values of a tile image, as float64."""
    kc = 128 // esize
    out = np.zeros((rows, kc))
    for r in range(rows):
        for k in range(kc):
            kb = k * esize
            o = ((kb // 16) * (rows // 8) + r // 8) * 128 + (r % 8) * 16 + kb % 16
            if esize == 4:
                out[r, k] = tile[o:o + 4].view(np.float32)[0]
            else:  # bf16: the high half of a float32
                out[r, k] = np.array([int(tile[o]) << 16 | int(tile[o + 1]) << 24], np.uint32).view(np.float32)[0]
    return out


def expected(N: int, n: np.ndarray, k: np.ndarray) -> np.ndarray:
    """W^T[n, k] of the real-form DFT (output column 2i = Re T_i, 2i + 1 = Im T_i; contraction index k < N for
    Re P[k], k >= N for Im P[k - N]), with zeros outside 2N x 2N."""
    i = n // 2
    b = np.where(k < N, k, k - N)
    th = 2 * np.pi * ((i * b) % N) / N
    c, s = np.cos(th), -np.sin(th)  # e^{-j th} = c + j s
    w = np.where(n % 2 == 0, np.where(k < N, c, -s), np.where(k < N, s, c))
    return np.where((n < 2 * N) & (k < 2 * N), w, 0.0)


@pytest.mark.parametrize("mode", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("N", [16, 50, 64, 200, 1024])
def test_weight_tiles_decode_to_the_dft_matrix(lib, mode, N):
    es = ESIZE[mode]
    kcv = 128 // es
    n_cols = (2 * N + 15) // 16 * 16
    NT = TILE[mode]
    tiles = (n_cols + NT - 1) // NT
    chunks = (2 * N + kcv - 1) // kcv
    tol = 2.0 ** -21 if mode == "tf32x3" else 2.0 ** -16
    for t in sorted({0, tiles - 1}):
        for c in sorted({0, chunks // 2, chunks - 1}):
            hi, lo, rows = pcal.pcal_dft_weights_host(N, mode, t, c)
            assert rows == min(NT, n_cols - NT * t) and rows % 16 == 0
            h, l = decode(hi, rows, es), decode(lo, rows, es)
            n = NT * t + np.arange(rows)[:, None]
            k = c * kcv + np.arange(kcv)[None, :]
            w = expected(N, n, k)
            assert np.max(np.abs(h + l - w)) <= tol, (t, c)
            assert np.all((h == 0) & (l == 0) | (w != 0) | ((n < 2 * N) & (k < 2 * N)))
            pad = (n >= 2 * N) | (k >= 2 * N)
            assert np.all(h[pad] == 0) and np.all(l[pad] == 0)
            if mode == "tf32x3":  # the parts are TF32 values: 13 low mantissa bits clear
                assert np.all(hi.view(np.uint32)[: rows * 32] & 0x1FFF == 0)
                assert np.all(lo.view(np.uint32)[: rows * 32] & 0x1FFF == 0)


def test_weights_reject_bad_arguments(lib):
    for args in [(0, "tf32x3", 0, 0), (1025, "tf32x3", 0, 0), (64, "tf32x3", 1, 0), (64, "bf16x3", 0, 2),
                 (200, "tf32x3", 4, 0), (200, "bf16x3", 2, 0),
                 (64, "fp32", 0, 0)]:  # the CUDA-core mode has no weight tiles
        with pytest.raises(pcal.PcalError):
            pcal.pcal_dft_weights_host(*args)


def test_operand_split_matches_the_tile_layout(tmp_path):
    """The split kernel's per-thread words (its loop body run on the host)
    equal the element-wise split of [Re P | Im P] into the tile layout, for
    ragged C and N and 8-byte-aligned P, and each mode's thread -> word map is
    a bijection on a tile (tests/host/dft_split_check.cu)."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    exe = tmp_path / "dft_split_check"
    subprocess.check_call([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                           "-I", os.path.join(root, "paper_2501_05993_gb300", "csrc"), "-I", os.path.join(root, "include"),
                           os.path.join(root, "tests", "host", "dft_split_check.cu"), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("OK")
