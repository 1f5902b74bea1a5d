"""Host checks of the tensor-core DFT's weight tiles (no GPU).

The tiles hold W^T of the real form of the tone DFT, T = [Re P | Im P] . W with
Re T_i and Im T_i in output columns 2i and 2i + 1 (angles 2 pi (i b mod N) / N),
each value split into parts of the MMA type (two TF32 parts, or three BF16
parts).  Decoding a tile with the no-swizzle K-major layout
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

ESIZE = {"tf32x3": 4, "bf16x6": 2}
PARTS = {"tf32x3": 2, "bf16x6": 3}
TILE = {"tf32x3": 256, "bf16x6": 256}  # output columns per tile
CHUNK = {"tf32x3": 128, "bf16x6": 64}  # bytes of K per tile row


@pytest.fixture(scope="module")
def lib():
    from paper_2501_05993_gb300 import build as libbuild

    libbuild.build()
    return pcal.load()


def decode(tile: np.ndarray, rows: int, esize: int, chunk: int) -> np.ndarray:
    """rows x (chunk / esize) values of a tile image, as float64."""
    kc = chunk // esize
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


@pytest.mark.parametrize("mode", ["tf32x3", "bf16x6"])
@pytest.mark.parametrize("N", [16, 50, 64, 200, 1024])
def test_weight_tiles_decode_to_the_dft_matrix(lib, mode, N):
    es = ESIZE[mode]
    kcv = CHUNK[mode] // es
    n_cols = (2 * N + 15) // 16 * 16
    tile = TILE[mode]
    tiles = (n_cols + tile - 1) // tile
    chunks = (2 * N + kcv - 1) // kcv
    # the sum of the parts carries the float32-rounded weight: 2^-22 of it left out by two TF32 parts, 2^-26 by
    # three BF16 parts, plus the float32 rounding (2^-24)
    tol = 2.0 ** -21 if mode == "tf32x3" else 2.0 ** -23
    for t in sorted({0, tiles - 1}):
        for c in sorted({0, chunks // 2, chunks - 1}):
            parts, rows = pcal.pcal_dft_weights_host(N, mode, t, c)
            assert len(parts) == PARTS[mode]
            assert rows == min(tile, n_cols - tile * t) and rows % 16 == 0
            vals = [decode(p, rows, es, CHUNK[mode]) for p in parts]
            n = tile * t + np.arange(rows)[:, None]
            k = c * kcv + np.arange(kcv)[None, :]
            w = expected(N, n, k)
            assert np.max(np.abs(sum(vals) - w)) <= tol, (t, c)
            # each part is at most half an ulp of the one before it (round to nearest at every step)
            for a, b in zip(vals, vals[1:]):
                assert np.all(np.abs(b) <= np.abs(a) * 2.0 ** -(8 if mode == "bf16x6" else 11) + 1e-300)
            pad = (n >= 2 * N) | (k >= 2 * N)
            assert all(np.all(v[pad] == 0) for v in vals)
            if mode == "tf32x3":  # the parts are TF32 values: 13 low mantissa bits clear
                assert all(np.all(p.view(np.uint32)[: rows * CHUNK[mode] // 4] & 0x1FFF == 0) for p in parts)


def test_weights_reject_bad_arguments(lib):
    for args in [(0, "tf32x3", 0, 0), (1025, "tf32x3", 0, 0), (64, "tf32x3", 1, 0), (64, "bf16x6", 0, 4),
                 (200, "tf32x3", 4, 0), (200, "bf16x6", 4, 0),
                 (64, "fp32", 0, 0)]:  # the CUDA-core mode has no weight tiles
        with pytest.raises(pcal.PcalError):
            pcal.pcal_dft_weights_host(*args)


def test_operand_split_matches_the_tile_layout(tmp_path):
    """The split kernel's per-thread words (its loop body run on the host)
    equal the element-wise split of [Re P | Im P] into each part's tile image, for
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
