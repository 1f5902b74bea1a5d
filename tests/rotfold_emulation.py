"""Host emulation of the FP32 rotate-then-fold variants (test infrastructure).

It repeats, in numpy float32 with one rounding per operation, the exact
sequence of FP32 operations that pcal_rotfold_* performs for each (lane, bin)
thread, so the GPU accumulators can be compared bit for bit.  The rotator
values come from FP64 cos/sin rounded to FP32, as on the device.
"""
import math

import numpy as np


def _phasor(f: int, m: int, fs: int) -> complex:
    r = (f * m) % fs
    a = 2.0 * math.pi * r / fs
    return complex(math.cos(a), -math.sin(a))


def emulate(x: np.ndarray, n0: int, fs: int, fo: int, N: int, lanes: int, variant: str,
            acc: np.ndarray | None = None) -> np.ndarray:
    """Accumulators float32 [lanes][N][4] after folding x (samples n0 ...),
    starting from `acc` (zeros when None)."""
    f32 = np.float32
    out = np.zeros((lanes, N, 4), dtype=f32) if acc is None else acc.copy()
    g = math.gcd(fs, fo) if fo else fs
    n_rot = fs // g
    r_step = (fo // g) % n_rot
    period = N * lanes
    n = x.size
    xs = x.astype(f32)
    if variant != "dfr":
        m = np.arange(n_rot)
        table_re = np.cos(2.0 * np.pi * m / n_rot).astype(f32)
        table_im = (-np.sin(2.0 * np.pi * m / n_rot)).astype(f32)
    for lane in range(lanes):
        for b in range(N):
            want = lane * N + b
            i0 = (want - n0) % period
            if i0 >= n:
                continue
            idx = np.arange(i0, n, period)
            s = out[lane, b].copy()
            if variant == "dfr":
                p0 = _phasor(fo, n0 + i0, fs)
                p1 = _phasor(fo, n0 + i0 + period, fs)
                pd = _phasor(fo, period, fs)
                coef = f32(2.0 * pd.real)
                y0 = [f32(p0.real), f32(p0.imag)]
                y1 = [f32(p1.real), f32(p1.imag)]
                for i in idx:
                    xv = xs[i]
                    s[0] = f32(s[0] + f32(xv * y0[0]))
                    s[1] = f32(s[1] + f32(xv * y0[1]))
                    y2 = [f32(f32(coef * y1[0]) - y0[0]), f32(f32(coef * y1[1]) - y0[1])]
                    y0, y1 = y1, y2
            else:
                rot = ((n0 + idx) * r_step) % n_rot
                pr = (xs[idx] * table_re[rot]).astype(f32)
                pi = (xs[idx] * table_im[rot]).astype(f32)
                if variant == "table":
                    for k in range(idx.size):
                        s[0] = f32(s[0] + pr[k])
                        s[1] = f32(s[1] + pi[k])
                else:
                    for k in range(idx.size):
                        yr = f32(pr[k] - s[2])
                        yi = f32(pi[k] - s[3])
                        tr = f32(s[0] + yr)
                        ti = f32(s[1] + yi)
                        s[2] = f32(f32(tr - s[0]) - yr)
                        s[3] = f32(f32(ti - s[1]) - yi)
                        s[0], s[1] = tr, ti
            out[lane, b] = s
    return out


def phasors(acc: np.ndarray) -> np.ndarray:
    """Lanes added in FP64 (sum minus compensation), then the N-point DFT in FP64."""
    P = (acc[..., 0].astype(np.float64) - acc[..., 2]).sum(axis=0) + \
        1j * (acc[..., 1].astype(np.float64) - acc[..., 3]).sum(axis=0)
    N = P.size
    k = np.arange(N)
    W = np.exp(-2j * np.pi * np.outer(k, k) / N)
    return W @ P
