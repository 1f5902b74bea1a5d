"""FP64 CPU oracle for multi-tone phase-calibration (PCal) extraction.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference leg of ``bench.py`` may import this package; the
product path never does.  It shares no code with the CUDA library.

Functions and the passages they follow (paper Sec. 2 unless stated):

* ``plan``            Eq. 4 (N_rotator) and N = fs/f_comb (text after Eq. 1);
                      the combined fold period L = lcm(N, N_rotator).
* ``direct``          The definition the method reaches: T_i = sum_n x[n]
                      exp(-j theta_i n), theta_i = i*w_comb + w_offset (Eq. 1,
                      Eq. 3 and DFT(P)), n the absolute sample index.
* ``fold_real`` / ``tones_from_bins``  fold modulo L (Eq. 2 with the period of
                      Eq. 4), then the direct sum over the L bins.
* ``rotate_fold_dft`` the paper's own route: rotate (Eq. 3), fold to N_bins
                      (Eq. 2), N-point DFT of P.
* ``counts_2bit`` / ``sums_i8`` / ``decode_counts``  exact integer bins.
* ``products``        amplitude 2|T|/M, tone phase arg(T)+pi/2 (sin model of
                      Eq. 1), unwrapping along the comb, and the instrumental
                      delay as the |T|^2-weighted least-squares slope of phase
                      versus tone frequency (phi_i = 2*pi*f_i*t_d, Eq. 1).
* ``brute_force``     pure-Python loops for tiny inputs.

Readings of points the paper leaves open are listed in the C source header.
"""
from __future__ import annotations

import cmath
import contextlib
import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcal_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

FORMATS = {"f32": 0, "i8": 1, "2bit": 2, "f64": 3}
# Reading of the 2-bit levels (Sec. 1 fixes only a sample width of 2 bits or more): codes
# 0..3 = {-v, -1, +1, +v} with the customary magnitude ratio v = 3.3359.
DEFAULT_LEVELS = (-3.3359, -1.0, 1.0, 3.3359)
# The tone phase of the sin() model of Eq. 1 is arg(T) + pi/2.
PHASE_REFERENCE = math.pi / 2


def build(force: bool = False) -> str:
    """Compile the C oracle (plain -O2, single thread) into oracle/_build/."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, vp, ci = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
        lib.orc_set_mutation.argtypes = [ci]
        lib.orc_get_mutation.restype = ci
        lib.orc_plan.argtypes = [i64, i64, i64, vp, vp, vp, vp]
        lib.orc_direct.argtypes = [vp, ci, vp, i64, i64, i64, i64, i64, i64, vp]
        lib.orc_direct_dy.argtypes = [vp, ci, vp, i64, i64, i64, i64, i64, ci, i64, vp]
        lib.orc_fold_real.argtypes = [vp, ci, vp, i64, i64, i64, vp]
        lib.orc_tones_from_bins.argtypes = [vp, i64, i64, i64, i64, vp]
        lib.orc_rotate_fold_dft.argtypes = [vp, i64, i64, i64, vp]
        lib.orc_counts_2bit.argtypes = [vp, i64, i64, i64, vp]
        lib.orc_sums_i8.argtypes = [vp, i64, i64, i64, vp]
        lib.orc_decode_counts.argtypes = [vp, i64, vp, vp]
        for f in ("orc_plan", "orc_direct", "orc_fold_real", "orc_tones_from_bins", "orc_rotate_fold_dft",
                  "orc_counts_2bit", "orc_sums_i8", "orc_decode_counts"):
            getattr(lib, f).restype = ci
        _lib = lib
    return _lib


@contextlib.contextmanager
def mutation(code: int):
    """Plant a known mistake in the C oracle for the duration of a block."""
    lib = _load()
    lib.orc_set_mutation(int(code))
    try:
        yield
    finally:
        lib.orc_set_mutation(0)


def plan(fs: int, fc: int, fo: int) -> dict:
    """Eq. 4: N_rotator = fs/gcd(fs, fo); N = fs/fc; L = lcm(N, N_rotator)."""
    if fs <= 0 or fc <= 0 or fo < 0 or fs % fc:
        raise ValueError("need integral fs, fc > 0, fo >= 0 and fc dividing fs")
    n_bins = fs // fc
    n_rot = fs // math.gcd(fs, fo)
    L = n_bins * n_rot // math.gcd(n_bins, n_rot)
    return {"N": n_bins, "N_rot": n_rot, "L": L}


def _levels(levels) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(levels, dtype=np.float64).reshape(4))


def _samples(samples, fmt: str):
    a = np.ascontiguousarray(samples)
    want = {"f32": np.float32, "i8": np.int8, "2bit": np.uint8, "f64": np.float64}[fmt]
    if a.dtype != want:
        raise TypeError(f"{fmt} samples must be {np.dtype(want).name}, got {a.dtype}")
    return a


def _count(a: np.ndarray, fmt: str, M: int | None) -> int:
    full = a.size * 4 if fmt == "2bit" else a.size
    return full if M is None else int(M)


def direct(samples, fmt: str, n0: int, fs: int, fc: int, fo: int, n_tones: int | None = None,
           levels=DEFAULT_LEVELS, M: int | None = None) -> np.ndarray:
    """T_i = sum_t x[t] exp(-j theta_i (n0+t)) for i < n_tones (default N)."""
    a = _samples(samples, fmt)
    M = _count(a, fmt, M)
    n_tones = fs // fc if n_tones is None else int(n_tones)
    out = np.zeros(2 * n_tones, dtype=np.float64)
    lev = _levels(levels)
    rc = _load().orc_direct(a.ctypes.data, FORMATS[fmt], lev.ctypes.data, M, int(n0), fs, fc, fo, n_tones,
                            out.ctypes.data)
    if rc:
        raise ValueError(f"orc_direct failed ({rc})")
    return out[0::2] + 1j * out[1::2]


def direct_any(samples, fmt: str, n0: int, fs: int, fc: int, fo: float, n_tones: int | None = None,
               levels=DEFAULT_LEVELS, M: int | None = None) -> np.ndarray:
    """The direct definition for an offset that is any binary fraction of a
    hertz (fo = num / 2**shift exactly): prime or non-integral offsets."""
    num, den = float(fo).as_integer_ratio()
    shift = den.bit_length() - 1
    if den != 1 << shift or num < 0:
        raise ValueError("offset must be a non-negative binary fraction")
    a = _samples(samples, fmt)
    M = _count(a, fmt, M)
    n_tones = fs // fc if n_tones is None else int(n_tones)
    out = np.zeros(2 * n_tones, dtype=np.float64)
    lev = _levels(levels)
    rc = _load().orc_direct_dy(a.ctypes.data, FORMATS[fmt], lev.ctypes.data, M, int(n0), fs, fc, num, shift,
                               n_tones, out.ctypes.data)
    if rc:
        raise ValueError(f"orc_direct_dy failed ({rc})")
    return out[0::2] + 1j * out[1::2]


def fold_real(samples, fmt: str, n0: int, L: int, levels=DEFAULT_LEVELS, M: int | None = None) -> np.ndarray:
    """S[k] = sum over samples with (n0+t) mod L == k (Eq. 2, period L)."""
    a = _samples(samples, fmt)
    M = _count(a, fmt, M)
    S = np.zeros(int(L), dtype=np.float64)
    lev = _levels(levels)
    if _load().orc_fold_real(a.ctypes.data, FORMATS[fmt], lev.ctypes.data, M, int(n0), int(L), S.ctypes.data):
        raise ValueError("orc_fold_real failed")
    return S


def tones_from_bins(S, fs: int, fc: int, fo: int, n_tones: int | None = None) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.float64)
    n_tones = fs // fc if n_tones is None else int(n_tones)
    out = np.zeros(2 * n_tones, dtype=np.float64)
    if _load().orc_tones_from_bins(S.ctypes.data, fs, fc, fo, n_tones, out.ctypes.data):
        raise ValueError("orc_tones_from_bins failed")
    return out[0::2] + 1j * out[1::2]


def rotate_fold_dft(S, fs: int, fc: int, fo: int) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.float64)
    out = np.zeros(2 * (fs // fc), dtype=np.float64)
    if _load().orc_rotate_fold_dft(S.ctypes.data, fs, fc, fo, out.ctypes.data):
        raise ValueError("orc_rotate_fold_dft failed")
    return out[0::2] + 1j * out[1::2]


def counts_2bit(packed, n0: int, L: int, M: int | None = None) -> np.ndarray:
    """Exact per-(bin, code) counts, shape (L, 4), int64."""
    a = _samples(packed, "2bit")
    M = _count(a, "2bit", M)
    out = np.zeros((int(L), 4), dtype=np.int64)
    if _load().orc_counts_2bit(a.ctypes.data, M, int(n0), int(L), out.ctypes.data):
        raise ValueError("orc_counts_2bit failed")
    return out


def sums_i8(x, n0: int, L: int) -> np.ndarray:
    a = _samples(x, "i8")
    out = np.zeros(int(L), dtype=np.int64)
    if _load().orc_sums_i8(a.ctypes.data, a.size, int(n0), int(L), out.ctypes.data):
        raise ValueError("orc_sums_i8 failed")
    return out


def sums_f32(x, n0: int, L: int) -> np.ndarray:
    return fold_real(x, "f32", n0, L)


def decode_counts(counts, levels=DEFAULT_LEVELS) -> np.ndarray:
    c = np.ascontiguousarray(counts, dtype=np.int64)
    S = np.zeros(c.shape[0], dtype=np.float64)
    lev = _levels(levels)
    _load().orc_decode_counts(c.ctypes.data, c.shape[0], lev.ctypes.data, S.ctypes.data)
    return S


def bins(samples, fmt: str, n0: int, L: int, levels=DEFAULT_LEVELS) -> np.ndarray:
    """Real FP64 bins of any format (2-bit through its exact counts)."""
    if fmt == "2bit":
        return decode_counts(counts_2bit(samples, n0, L), levels)
    if fmt == "i8":
        return sums_i8(samples, n0, L).astype(np.float64)
    return sums_f32(samples, n0, L)


def fold(samples, fmt: str, n0: int, fs: int, fc: int, fo: int, levels=DEFAULT_LEVELS) -> np.ndarray:
    """Fold mode: exact/compensated bins over n mod L, then the bin sum."""
    L = plan(fs, fc, fo)["L"]
    return tones_from_bins(bins(samples, fmt, n0, L, levels), fs, fc, fo)


def wrap(a):
    """Wrap angles into [-pi, pi)."""
    return (np.asarray(a) + np.pi) % (2 * np.pi) - np.pi


def products(T, M: int, fs: int, fc: int, fo: int) -> dict:
    """Amplitude, phase, unwrapped phase and the delay fit of N tone phasors."""
    T = np.asarray(T, dtype=np.complex128)
    N = T.size
    amp = 2.0 * np.abs(T) / float(M) if M > 0 else np.zeros(N)
    psi = wrap(np.angle(T) + PHASE_REFERENCE)
    unwrapped = psi.copy()
    if N > 1:
        unwrapped[1:] = psi[0] + np.cumsum(wrap(np.diff(psi)))
    f = np.arange(N, dtype=np.float64) * fc + fo
    w = np.abs(T) ** 2
    out = {"amp": amp, "phase": psi, "unwrapped": unwrapped, "td": float("nan"), "sigma_td": float("nan"),
           "bandpass_phase": np.full(N, np.nan), "td_peak": peak_delay(T, fs)}
    W = w.sum()
    if N >= 2 and W > 0:
        fbar = (w * f).sum() / W
        pbar = (w * unwrapped).sum() / W
        sff = (w * (f - fbar) ** 2).sum()
        sfp = (w * (f - fbar) * (unwrapped - pbar)).sum()
        if sff > 0:
            slope = sfp / sff
            resid = unwrapped - pbar - slope * (f - fbar)
            out["bandpass_phase"] = resid  # phase after removing the fitted delay (Sec. 3's corrected bandpass)
            out["td"] = slope / (2 * np.pi)
            if N > 2:
                # weighted LS slope variance; invariant to the scale of w
                out["sigma_td"] = math.sqrt(((w * resid ** 2).sum() / (N - 2)) / sff) / (2 * np.pi)
    return out


def peak_delay(T, fs: int) -> float:
    """Delay from the time-domain pulse (Sec. 2: the largest bin of P and a
    three-point interpolation across its neighbours).  P = IDFT(T), the inverse
    of T_i = sum_b P[b] exp(-2 pi j i b / N); a delay t_d puts the pulse at
    b = -t_d fs (mod N).  The vertex of the parabola through |P| at the
    largest bin and its two neighbours refines the position; the result is
    wrapped into [-N/(2 fs), N/(2 fs))."""
    T = np.asarray(T, dtype=np.complex128)
    N = T.size
    if N == 0 or not np.any(T):
        return float("nan")
    b = np.arange(N)
    P = np.array([np.sum(T * np.exp(2j * np.pi * np.arange(N) * k / N)) for k in b]) / N
    mag = np.abs(P)
    k = int(np.argmax(mag))
    ym, y0, yp = mag[(k - 1) % N], mag[k], mag[(k + 1) % N]
    den = ym - 2.0 * y0 + yp
    delta = 0.5 * (ym - yp) / den if den != 0 else 0.0
    t = -(k + delta) / fs
    half = N / (2.0 * fs)
    return float((t + half) % (2.0 * half) - half)


def brute_force(x, n0: int, fs: int, fc: int, fo: int, n_tones: int | None = None):
    """Pure-Python T_i = sum_t x[t] exp(-2 pi j ((i fc + fo)(n0+t) mod fs)/fs)."""
    n_tones = fs // fc if n_tones is None else n_tones
    out = []
    for i in range(n_tones):
        acc = 0j
        for t, v in enumerate(x):
            r = ((i * fc + fo) * (n0 + t)) % fs
            acc += float(v) * cmath.exp(-2j * math.pi * r / fs)
        out.append(acc)
    return np.array(out, dtype=np.complex128)
