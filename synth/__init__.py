"""Seeded synthetic comb-plus-noise baseband streams (inputs only).

This package makes the inputs that both the CPU oracle tests and the GPU path
consume; it contains none of the extraction arithmetic.  The signal is the
paper's Eq. 1 model (Sec. 2): Gaussian noise plus N equal-amplitude comb tones
at frequencies i*fc + fo whose phases come from one instrumental delay td.
Random numbers come from a Philox4x32-10 counter-based generator written from
its published definition (Salmon et al., SC'11), so a stream is reproducible
from (seed, stream id, absolute sample index) alone, in any chunking.

Quantisers: float32; int8 = clamp(round-half-even(scale*x)); 2-bit with
thresholds 0 and +-t, codes 0..3 = (h<<1)|l, four samples per byte, least
significant pair first.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_OUT = os.path.join(_HERE, "_build", "libsynth.so")
_lib = None

FMT_F32, FMT_I8, FMT_2BIT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile synth.c into a shared library next to it (in _build/)."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, u64, u32, dbl, vp = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_void_p
        lib.synth_philox4x32.argtypes = [ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.c_int, ctypes.POINTER(u32)]
        lib.synth_philox4x32.restype = None
        lib.synth_real.argtypes = [u64, u32, i64, i64, dbl, i64, i64, i64, i64, dbl, dbl, vp]
        lib.synth_real.restype = ctypes.c_int
        lib.synth_quantized.argtypes = [u64, u32, i64, i64, dbl, i64, i64, i64, i64, dbl, dbl, ctypes.c_int, dbl, vp]
        lib.synth_quantized.restype = ctypes.c_int
        ci = ctypes.c_int
        lib.synth_real_dy.argtypes = [u64, u32, i64, i64, dbl, i64, i64, i64, ci, i64, dbl, dbl, vp]
        lib.synth_real_dy.restype = ci
        lib.synth_quantized_dy.argtypes = [u64, u32, i64, i64, dbl, i64, i64, i64, ci, i64, dbl, dbl, ci, dbl, vp]
        lib.synth_quantized_dy.restype = ci
        _lib = lib
    return _lib


def philox4x32(ctr, key, rounds: int = 10):
    """Philox4x32-R block function: 4 x u32 counter, 2 x u32 key -> 4 x u32."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.synth_philox4x32(c, k, rounds, o)
    return [int(v) for v in o]


TABLE_MAX_L = 1 << 22  # longer comb periods are evaluated sample by sample


def dyadic(f) -> tuple[int, int]:
    """(num, shift) with f = num / 2**shift exactly (any finite binary float >= 0)."""
    num, den = float(f).as_integer_ratio()
    shift = den.bit_length() - 1
    if den != 1 << shift or num < 0:
        raise ValueError(f"offset {f!r} is not a non-negative binary fraction")
    return num, shift


@dataclass(frozen=True)
class Stream:
    """One synthetic baseband channel: integral fs and fc; fo integral, or any
    binary fraction of a hertz (then, or when the comb period is longer than
    TABLE_MAX_L, the comb is evaluated sample by sample)."""

    fs: int
    fc: int
    fo: float
    amp: float          # tone amplitude A in units of the noise sigma
    td: float           # injected instrumental delay in seconds
    sigma: float = 1.0  # noise standard deviation (0 gives the noise-free comb)
    seed: int = 2501059930
    stream: int = 0
    n_tones: int | None = None  # default N = fs / fc tones (Eq. 1 literally)

    @property
    def N(self) -> int:
        return self.fs // self.fc if self.n_tones is None else self.n_tones

    def _args(self, n0: int, count: int):
        return (self.seed, self.stream, int(n0), int(count), float(self.sigma), int(self.fs), int(self.fc),
                int(self.fo), int(self.N), float(self.amp), float(self.td))

    def _direct(self) -> bool:
        if float(self.fo) != int(self.fo):
            return True
        import math

        return self.fs // math.gcd(math.gcd(int(self.fs), int(self.fc)), int(self.fo)) > TABLE_MAX_L

    def _args_dy(self, n0: int, count: int):
        num, shift = dyadic(self.fo)
        return (self.seed, self.stream, int(n0), int(count), float(self.sigma), int(self.fs), int(self.fc), num,
                shift, int(self.N), float(self.amp), float(self.td))

    def _quantized(self, n0, count, fmt, param, out):
        lib = _load()
        if self._direct():
            rc = lib.synth_quantized_dy(*self._args_dy(n0, count), fmt, float(param), out.ctypes.data)
        else:
            rc = lib.synth_quantized(*self._args(n0, count), fmt, float(param), out.ctypes.data)
        if rc != 0:
            raise ValueError("synth_quantized: bad arguments")
        return out

    def real(self, n0: int, count: int) -> np.ndarray:
        """Unquantised FP64 samples for absolute indices n0 .. n0+count-1."""
        out = np.empty(int(count), dtype=np.float64)
        lib = _load()
        rc = (lib.synth_real_dy(*self._args_dy(n0, count), out.ctypes.data) if self._direct()
              else lib.synth_real(*self._args(n0, count), out.ctypes.data))
        if rc != 0:
            raise ValueError("synth_real: bad arguments")
        return out

    def f32(self, n0: int, count: int) -> np.ndarray:
        return self._quantized(n0, count, FMT_F32, 0.0, np.empty(int(count), dtype=np.float32))

    def i8(self, n0: int, count: int, scale: float = 20.0) -> np.ndarray:
        return self._quantized(n0, count, FMT_I8, scale, np.empty(int(count), dtype=np.int8))

    def bits2(self, n0: int, count: int, threshold: float = 0.98) -> np.ndarray:
        """2-bit packed bytes; count must be a multiple of 4."""
        if count % 4:
            raise ValueError("2-bit streams hold whole bytes: count must be a multiple of 4")
        return self._quantized(n0, count, FMT_2BIT, threshold, np.empty(int(count) // 4, dtype=np.uint8))

    def samples(self, fmt: str, n0: int, count: int) -> np.ndarray:
        if fmt == "f32":
            return self.f32(n0, count)
        if fmt == "i8":
            return self.i8(n0, count)
        if fmt == "2bit":
            return self.bits2(n0, count)
        raise ValueError(f"unknown sample format {fmt!r}")


# Levels of the 2-bit codes 0..3 (sign/magnitude, magnitude ratio 3.3359).
LEVELS_2BIT = (-3.3359, -1.0, 1.0, 3.3359)
