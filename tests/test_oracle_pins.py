"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-type the oracle's own loop: each compares it with a closed
form (a noise-free comb from Eq. 1, the geometric-series sum for partial
periods), a library routine (numpy's FFT evaluated at the tone bins), a
pure-Python brute force with a different phase reduction (mod fs instead of
mod L), values the paper prints (tests/golden/paper_constants.json), or
invariants.  test_planted_mistakes shows that each plausible mistake planted
in the oracle breaks at least one pin.
"""
import cmath
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def comb_closed_form(fs, fc, fo, amp, td, n0, M, n_tones=None):
    """Exact T_i of the noise-free comb of Eq. 1 over absolute samples
    n0..n0+M-1, by the geometric series of each complex exponential of
    sin(u) = (e^{ju} - e^{-ju}) / 2j.  Phases are reduced in integers mod fs."""
    N = fs // fc
    n_tones = N if n_tones is None else n_tones
    f = np.arange(N, dtype=np.int64) * fc + fo
    phi = 2 * np.pi * np.mod(f.astype(np.float64) * td, 1.0)

    def geo(a_int):
        # sum_{t<M} exp(j*2*pi*a*(n0+t)/fs) for integer a, exact reduction
        a = int(a_int) % fs
        start = np.exp(2j * np.pi * ((a * n0) % fs) / fs)
        if a == 0:
            return start * M
        z = np.exp(2j * np.pi * a / fs)
        zM = np.exp(2j * np.pi * ((a * M) % fs) / fs)
        return start * (1 - zM) / (1 - z)

    out = np.zeros(n_tones, dtype=np.complex128)
    for i in range(n_tones):
        fi = i * fc + fo
        acc = 0j
        for k in range(N):
            fk = int(f[k])
            acc += amp / 2j * (np.exp(1j * phi[k]) * geo(fk - fi) - np.exp(-1j * phi[k]) * geo(-fk - fi))
        out[i] = acc
    return out


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(np.asarray(b))), 1e-300))


# ---------------------------------------------------------------- plan (Eq. 4)

def test_plan_matches_paper_printed_values():
    g = json.load(open(GOLD))
    fs, fo, fc = g["fs_hz"]["value"], g["f_offset_hz"]["value"], g["f_comb_hz"]["value"]
    p = oracle.plan(fs, fc, fo)
    assert p["N_rot"] == g["N_rotator"]["value"] == 1600
    assert p["N"] == g["N_bins"]["value"] == 16
    assert p["L"] == 1600
    assert math.isclose(2 * math.pi * fo / fs, g["w_offset_rad_per_sample"]["value"], rel_tol=1e-14)


@pytest.mark.parametrize("fs,fc,fo,N,L", [
    (16_000_000, 1_000_000, 10_000, 16, 1600),
    (64_000_000, 1_000_000, 10_000, 64, 6400),
    (1_024_000_000, 1_000_000, 10_000, 1024, 102400),
    (32_000_000, 1_000_000, 0, 32, 32),
    (32_000_000, 1_000_000, 500_000, 32, 64),
    (16, 4, 1, 4, 16),
])
def test_plan_combined_period(fs, fc, fo, N, L):
    p = oracle.plan(fs, fc, fo)
    assert (p["N"], p["L"]) == (N, L)
    # L is the least common period of the comb (N) and the rotator (Eq. 4)
    assert p["L"] % p["N"] == 0 and p["L"] % p["N_rot"] == 0
    assert all(p["L"] % d or d == p["L"] for d in range(1, p["L"]) if d % p["N"] == 0 and d % p["N_rot"] == 0)


# ---------------------------------------------------------- closed forms

@pytest.mark.parametrize("fs,fc,fo,periods", [(16000, 1000, 10, 3), (64000, 1000, 10, 2), (48000, 4000, 60, 5)])
def test_closed_form_full_periods(fs, fc, fo, periods):
    """Noise-free comb, M a multiple of L: T_i = (A M / 2) e^{j(phi_i - pi/2)}."""
    amp, td = 0.02, 3.7e-5
    L = oracle.plan(fs, fc, fo)["L"]
    M, n0 = periods * L, 0
    x = synth.Stream(fs=fs, fc=fc, fo=fo, amp=amp, td=td, sigma=0.0).real(n0, M)
    T = oracle.direct(x, "f64", n0, fs, fc, fo)
    N = fs // fc
    phi = 2 * np.pi * (np.arange(N) * fc + fo) * td
    expect = amp * M / 2 * np.exp(1j * (phi - np.pi / 2))
    assert rel(T, expect) < 1e-9


@pytest.mark.parametrize("n0,M", [(0, 1234), (777, 2900), (12345, 999)])
def test_closed_form_partial_periods(n0, M):
    """M not a multiple of L and n0 != 0: the exact geometric-series sum."""
    fs, fc, fo, amp, td = 16000, 1000, 10, 0.5, 2.1e-5
    x = synth.Stream(fs=fs, fc=fc, fo=fo, amp=amp, td=td, sigma=0.0).real(n0, M)
    T = oracle.direct(x, "f64", n0, fs, fc, fo)
    assert rel(T, comb_closed_form(fs, fc, fo, amp, td, n0, M)) < 1e-9


def test_products_closed_form():
    """Amplitude 2|T|/M = A, phase = phi_i, delay fit = t_d exactly (no noise)."""
    fs, fc, fo, amp, td = 64000, 1000, 10, 0.01, 1.25e-5
    L = oracle.plan(fs, fc, fo)["L"]
    M = 3 * L
    x = synth.Stream(fs=fs, fc=fc, fo=fo, amp=amp, td=td, sigma=0.0).real(0, M)
    pr = oracle.products(oracle.direct(x, "f64", 0, fs, fc, fo), M, fs, fc, fo)
    N = fs // fc
    assert np.allclose(pr["amp"], amp, rtol=1e-9)
    phi = oracle.wrap(2 * np.pi * (np.arange(N) * fc + fo) * td)
    assert np.max(np.abs(oracle.wrap(pr["phase"] - phi))) < 1e-9
    assert abs(pr["td"] - td) < 1e-12 * td + 1e-18


@pytest.mark.parametrize("shift", [3, 11, 62])
def test_peak_delay_integer_shift(shift):
    """A noise-free comb whose delay is a whole number of samples puts the
    whole pulse in one bin of P: the peak estimate is the delay exactly
    (wrapped into one comb period), and the corrected bandpass is flat."""
    fs, fc, fo, amp = 64000, 1000, 10, 0.01
    td = shift / fs
    L = oracle.plan(fs, fc, fo)["L"]
    M = 2 * L
    x = synth.Stream(fs=fs, fc=fc, fo=fo, amp=amp, td=td, sigma=0.0).real(0, M)
    pr = oracle.products(oracle.direct(x, "f64", 0, fs, fc, fo), M, fs, fc, fo)
    N = fs // fc
    want = ((td + N / (2 * fs)) % (N / fs)) - N / (2 * fs)
    assert abs(pr["td_peak"] - want) < 1e-12
    assert np.max(np.abs(pr["bandpass_phase"])) < 1e-9


def test_peak_delay_fractional_shift():
    """Between samples the three-point estimate lands within a quarter sample."""
    fs, fc, fo, amp = 64000, 1000, 10, 0.01
    L = oracle.plan(fs, fc, fo)["L"]
    for frac in (0.2, 0.5, 0.8):
        td = (5 + frac) / fs
        x = synth.Stream(fs=fs, fc=fc, fo=fo, amp=amp, td=td, sigma=0.0).real(0, L)
        pr = oracle.products(oracle.direct(x, "f64", 0, fs, fc, fo), L, fs, fc, fo)
        assert abs(pr["td_peak"] - td) < 0.25 / fs, (frac, pr["td_peak"] * fs)


# ---------------------------------------------------------- library routine

@pytest.mark.parametrize("fmt", ["f32", "i8", "2bit", "f64"])
@pytest.mark.parametrize("n0", [0, 4 * 1001])
def test_fft_pin(fmt, n0):
    """T_i equals numpy's M-point FFT at bin (i fc + fo) M / fs (shifted by
    e^{-j theta_i n0}) when M is a multiple of L."""
    fs, fc, fo = 16000, 1000, 10
    L = oracle.plan(fs, fc, fo)["L"]
    M = 5 * L
    s = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.3, td=1e-5, sigma=1.0, seed=11)
    if fmt == "f64":
        raw, xv = s.real(n0, M), None
        xv = raw
    else:
        raw = s.samples(fmt, n0, M)
        if fmt == "2bit":
            codes = (raw[:, None] >> (2 * np.arange(4))) & 3
            xv = np.take(np.array(oracle.DEFAULT_LEVELS), codes.reshape(-1))
        else:
            xv = raw.astype(np.float64)
    T = oracle.direct(raw, fmt, n0, fs, fc, fo)
    X = np.fft.fft(xv)
    N = fs // fc
    f = np.arange(N) * fc + fo
    shift = np.exp(-2j * np.pi * ((f * n0) % fs) / fs)
    assert rel(T, X[(f * M) // fs] * shift) < 1e-10


def test_fo_zero_reduces_to_fold_plus_dft():
    """f_offset = 0: T = DFT(P) with P the Eq. 2 fold over N_bins."""
    fs, fc = 32000, 1000
    N = fs // fc
    x = synth.Stream(fs=fs, fc=fc, fo=0, amp=0.1, td=2e-5, seed=5).real(0, 40 * N)
    P = x.reshape(-1, N).sum(axis=0)
    assert rel(oracle.direct(x, "f64", 0, fs, fc, 0), np.fft.fft(P)) < 1e-11


# ---------------------------------------------------------- brute force

@pytest.mark.parametrize("fmt", ["f32", "i8", "2bit"])
@pytest.mark.parametrize("n0,M", [(0, 64), (5, 400), (1001, 1024)])
def test_brute_force_tiny(fmt, n0, M):
    fs, fc, fo = 16, 4, 1
    s = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.4, td=0.01, seed=3)
    raw = s.samples(fmt, n0, M)
    if fmt == "2bit":
        codes = ((raw[:, None] >> (2 * np.arange(4))) & 3).reshape(-1)
        xv = [oracle.DEFAULT_LEVELS[c] for c in codes]
    else:
        xv = raw.astype(np.float64).tolist()
    bf = oracle.brute_force(xv, n0, fs, fc, fo)
    assert rel(oracle.direct(raw, fmt, n0, fs, fc, fo), bf) < 1e-12
    L = oracle.plan(fs, fc, fo)["L"]
    # bins: brute-force dictionary fold
    bins = np.zeros(L)
    for t, v in enumerate(xv):
        bins[(n0 + t) % L] += v
    assert np.allclose(oracle.bins(raw, fmt, n0, L), bins, rtol=0, atol=1e-12)


# ---------------------------------------------------------- identities

@pytest.mark.parametrize("fmt", ["f32", "i8", "2bit"])
def test_fold_identity(fmt):
    """direct == fold (bins then bin sum) == rotate / fold to N / DFT."""
    fs, fc, fo = 64000, 1000, 30
    L = oracle.plan(fs, fc, fo)["L"]
    n0, M = 333, 3 * L + 4 * 77
    raw = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.05, td=4e-6, seed=9).samples(fmt, n0, M)
    T_direct = oracle.direct(raw, fmt, n0, fs, fc, fo)
    S = oracle.bins(raw, fmt, n0, L)
    assert rel(oracle.tones_from_bins(S, fs, fc, fo), T_direct) < 1e-11
    assert rel(oracle.rotate_fold_dft(S, fs, fc, fo), T_direct) < 1e-11


def test_two_bit_linearity_pin4():
    """levels {-v,-1,+1,+v} on codes (h<<1)|l decode to v(h+l-1) + (h-l)."""
    v = 3.3359
    for c in range(4):
        h, l = c >> 1, c & 1
        assert math.isclose(oracle.DEFAULT_LEVELS[c], v * (h + l - 1) + (h - l), abs_tol=1e-15)
    # and count-decoded bins equal the FP64 fold of the decoded samples
    raw = synth.Stream(fs=64, fc=4, fo=1, amp=0.2, td=0.0, seed=1).bits2(0, 4096)
    L = oracle.plan(64, 4, 1)["L"]
    via_counts = oracle.decode_counts(oracle.counts_2bit(raw, 0, L))
    assert np.allclose(via_counts, oracle.fold_real(raw, "2bit", 0, L), rtol=0, atol=1e-9)


def expected_bin_count(n0, M, L):
    k = np.arange(L)
    r = (k - n0) % L
    return M // L + (r < M % L)


@pytest.mark.parametrize("n0,M", [(0, 4096), (13, 4000), (6399, 64004)])
def test_counts_invariants(n0, M):
    L = 6400 if M > 10000 else 100
    raw = synth.Stream(fs=64_000, fc=1000, fo=10, amp=0.01, td=0.0, seed=2).bits2(n0, M)
    cnt = oracle.counts_2bit(raw, n0, L)
    assert np.array_equal(cnt.sum(axis=1), expected_bin_count(n0, M, L))


def test_counts_known_pattern():
    """Bytes 0xE4 hold codes 0,1,2,3 in sample order: with L = 4 and n0 = 0
    every bin k sees only code k."""
    nbytes = 1000
    cnt = oracle.counts_2bit(np.full(nbytes, 0xE4, dtype=np.uint8), 0, 4)
    assert np.array_equal(cnt, np.eye(4, dtype=np.int64) * nbytes)
    cnt = oracle.counts_2bit(np.full(nbytes, 0xE4, dtype=np.uint8), 1, 4)
    assert np.array_equal(cnt, np.roll(np.eye(4, dtype=np.int64), 1, axis=0) * nbytes)


@pytest.mark.parametrize("fmt", ["i8", "2bit", "f32"])
def test_chunk_split_invariance(fmt):
    fs, fc, fo = 64000, 1000, 10
    L = oracle.plan(fs, fc, fo)["L"]
    s = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.05, td=0.0, seed=4)
    n0, cuts = 100, [0, 4 * 37, 4 * 1700, 4 * 5000, 4 * 9001]
    f = (lambda raw, n: oracle.counts_2bit(raw, n, L)) if fmt == "2bit" else (lambda raw, n: oracle.bins(raw, fmt, n, L))
    whole = f(s.samples(fmt, n0, cuts[-1]), n0)
    parts = sum(f(s.samples(fmt, n0 + a, b - a), n0 + a) for a, b in zip(cuts[:-1], cuts[1:]))
    if fmt == "f32":
        assert np.allclose(parts, whole, rtol=0, atol=1e-9)
    else:
        assert np.array_equal(parts, whole)


# ---------------------------------------------------------- physics: delay

def test_delay_recovery_c1():
    """Config-1 shape at full size: t_d recovered within 5 sigma_td."""
    fs, fc, fo, amp, td, M = 16_000_000, 1_000_000, 10_000, 0.02, 3.7e-9, 16_000_000
    x = synth.Stream(fs=fs, fc=fc, fo=fo, amp=amp, td=td, seed=2501059931).f32(0, M)
    pr = oracle.products(oracle.fold(x, "f32", 0, fs, fc, fo), M, fs, fc, fo)
    # expected sigma_td ~ sqrt(2/M)/A / (2 pi fc sqrt(N(N^2-1)/12)) = 0.15 ns
    assert 0.03e-9 < pr["sigma_td"] < 0.5e-9
    assert abs(pr["td"] - td) < 5 * pr["sigma_td"]
    assert np.allclose(pr["amp"], amp, rtol=0.5)


def test_delay_recovery_two_bit():
    """2-bit, fs = 64 MHz, N = 64, t_d = 12.5 ns (phases wrap along the comb)."""
    fs, fc, fo, amp, td, M = 64_000_000, 1_000_000, 10_000, 0.01, 12.5e-9, 64_000_000
    raw = synth.Stream(fs=fs, fc=fc, fo=fo, amp=amp, td=td, seed=2501059932).bits2(0, M)
    pr = oracle.products(oracle.fold(raw, "2bit", 0, fs, fc, fo), M, fs, fc, fo)
    assert pr["sigma_td"] < 60e-12
    assert abs(pr["td"] - td) < 5 * pr["sigma_td"]


def test_phase_residuals_chi_square_c1():
    """Per-tone phase residuals after the delay fit are consistent with the
    expected phase noise: for a tone of amplitude A in unit noise over M
    samples, sigma_phi = sqrt(2/M)/A, so sum(resid^2)/sigma_phi^2 over the N
    tones follows chi^2 with N - 2 degrees of freedom.  Checked over several
    seeds (bounds hold with probability > 0.999 each)."""
    fs, fc, fo, amp, td, M = 16_000_000, 1_000_000, 10_000, 0.02, 3.7e-9, 4_000_000
    N = fs // fc
    sigma_phi = math.sqrt(2.0 / M) / amp
    stats = []
    for seed in range(5):
        x = synth.Stream(fs=fs, fc=fc, fo=fo, amp=amp, td=td, seed=9100 + seed).f32(0, M)
        pr = oracle.products(oracle.fold(x, "f32", 0, fs, fc, fo), M, fs, fc, fo)
        stats.append(float(np.sum((pr["bandpass_phase"] / sigma_phi) ** 2)))
    dof = N - 2
    for chi2 in stats:
        assert 0.15 * dof < chi2 < 3.0 * dof, stats
    assert 0.5 * dof < np.mean(stats) < 1.6 * dof, stats


def test_sigma_td_matches_delay_scatter_over_seeds():
    """sigma_td pinned by the statistics of the fit, not by its own formula.
    Over n = 60 independent noise realisations of a config-1-shaped stream
    (M a whole number of periods, so the tones and their images are
    orthogonal), the fitted delays scatter with a sample variance s^2 whose
    ratio (n-1) s^2 / sigma^2 follows chi^2 with n-1 degrees of freedom when
    sigma is the true standard deviation of the estimator.  The reported
    sigma_td (averaged over the seeds) must be that sigma: s / mean(sigma_td)
    inside the two-sided 0.1 % chi^2 band, widened by the 2.5 % sampling
    error of the mean.  It must also agree with the closed form for equal
    tone weights, sigma_phi / (2 pi f_comb sqrt(N (N^2 - 1) / 12)) with
    sigma_phi = sqrt(2/M)/A per tone in unit noise (Eq. 1 with phi_i =
    2 pi f_i t_d: the slope's variance is sigma_phi^2 / sum (f_i - f_bar)^2),
    and the delays must be unbiased.  A dropped 1/(N-2), a square root taken
    twice or a missing 1/(2 pi) moves sigma_td by a factor of 3.7 or more."""
    from scipy import stats as st

    fs, fc, fo, amp, td, M = 16_000_000, 1_000_000, 10_000, 0.02, 3.7e-9, 1_600_000
    N, n = fs // fc, 60
    tds, sig = [], []
    for seed in range(n):
        x = synth.Stream(fs=fs, fc=fc, fo=fo, amp=amp, td=td, seed=31000 + seed).f32(0, M)
        pr = oracle.products(oracle.fold(x, "f32", 0, fs, fc, fo), M, fs, fc, fo)
        tds.append(pr["td"])
        sig.append(pr["sigma_td"])
    tds, sig = np.array(tds), np.array(sig)
    s = np.std(tds, ddof=1)
    lo, hi = np.sqrt(st.chi2.ppf([0.0005, 0.9995], n - 1) / (n - 1))
    ratio = s / np.mean(sig)
    assert 0.975 * lo < ratio < 1.025 * hi, (ratio, lo, hi)
    closed = math.sqrt(2.0 / M) / amp / (2 * math.pi * fc * math.sqrt(N * (N * N - 1) / 12.0))
    assert 0.88 < np.mean(sig) / closed < 1.08, np.mean(sig) / closed
    assert abs(np.mean(tds) - td) < 4 * closed / math.sqrt(n)


# ---------------------------------------------------------- planted mistakes

def _pin_battery():
    """A compact battery of the pins above; returns the names that fail."""
    failed = []
    fs, fc, fo, amp, td = 16000, 1000, 10, 0.5, 2.1e-5
    n0, M = 777, 2900
    x = synth.Stream(fs=fs, fc=fc, fo=fo, amp=amp, td=td, sigma=0.0).real(n0, M)
    if rel(oracle.direct(x, "f64", n0, fs, fc, fo), comb_closed_form(fs, fc, fo, amp, td, n0, M)) > 1e-9:
        failed.append("closed_form")
    L = oracle.plan(fs, fc, fo)["L"]
    S = oracle.fold_real(x, "f64", n0, L)
    if rel(oracle.rotate_fold_dft(S, fs, fc, fo), comb_closed_form(fs, fc, fo, amp, td, n0, M)) > 1e-9:
        failed.append("route")
    cnt = oracle.counts_2bit(np.full(64, 0xE4, dtype=np.uint8), 0, 4)
    if not np.array_equal(cnt, np.eye(4, dtype=np.int64) * 64):
        failed.append("known_pattern")
    raw = synth.Stream(fs=64, fc=4, fo=1, amp=0.3, td=0.0, seed=1).bits2(8, 400)
    Lb = oracle.plan(64, 4, 1)["L"]
    if not np.array_equal(oracle.counts_2bit(raw, 8, Lb).sum(axis=1), expected_bin_count(8, 400, Lb)):
        failed.append("count_invariant")
    codes = ((raw[:, None] >> (2 * np.arange(4))) & 3).reshape(-1)
    xv = np.take(np.array(oracle.DEFAULT_LEVELS), codes)
    bins = np.zeros(Lb)
    np.add.at(bins, (8 + np.arange(codes.size)) % Lb, xv)
    if not np.allclose(oracle.bins(raw, "2bit", 8, Lb), bins, atol=1e-9):
        failed.append("brute_bins")
    return failed


def test_pin_battery_clean():
    assert _pin_battery() == []


@pytest.mark.parametrize("code", [1, 2, 3, 4, 5, 6])
def test_planted_mistakes(code):
    """Each planted oracle mistake is caught by at least one pin."""
    with oracle.mutation(code):
        failed = _pin_battery()
    assert failed, f"mutation {code} went unnoticed"


# ---------------------------------------------------------- offsets beyond the fold

def comb_closed_form_dyadic(fs, fc, num, shift, amp, td, n0, M):
    """Exact T_i of the noise-free comb for f_offset = num / 2**shift, by the
    geometric series of each exponential with its phase reduced in integers
    modulo fs * 2**shift."""
    N = fs // fc
    mod = fs << shift
    out = np.zeros(N, dtype=np.complex128)

    def geo(a):
        a %= mod
        start = np.exp(2j * np.pi * ((a * n0) % mod) / mod)
        if a == 0:
            return start * M
        z = np.exp(2j * np.pi * a / mod)
        zM = np.exp(2j * np.pi * ((a * M) % mod) / mod)
        return start * (1 - zM) / (1 - z)

    for i in range(N):
        ai = (i * fc << shift) + num                 # f_i * 2**shift
        phi = 2 * np.pi * math.fmod(ai / (1 << shift) * td, 1.0)
        acc = 0j
        for k in range(N):
            ak = (k * fc << shift) + num
            phik = 2 * np.pi * math.fmod(ak / (1 << shift) * td, 1.0)
            # sin(u) = (e^{ju} - e^{-ju}) / 2j, summed against e^{-j theta_i n}
            acc += amp / 2j * (np.exp(1j * phik) * geo(ak - ai) - np.exp(-1j * phik) * geo(-ak - ai))
        out[i] = acc
    return out


@pytest.mark.parametrize("fo", [10007.0, 10007.25, 333.125])
def test_direct_any_closed_form(fo):
    """A prime and two fractional offsets: the oracle's direct definition equals
    the exact geometric-series sum of the noise-free comb."""
    fs, fc, amp, td, n0, M = 64000, 8000, 0.3, 2.5e-6, 777, 20011
    num, den = float(fo).as_integer_ratio()
    shift = den.bit_length() - 1
    x = synth.Stream(fs=fs, fc=fc, fo=fo, amp=amp, td=td, sigma=0.0).real(n0, M)
    T = oracle.direct_any(x, "f64", n0, fs, fc, fo)
    assert rel(T, comb_closed_form_dyadic(fs, fc, num, shift, amp, td, n0, M)) < 1e-9


def test_direct_any_brute_force_exact_rationals():
    """Tiny input: pure Python with exact rational phases."""
    from fractions import Fraction

    fs, fc, fo = 32, 8, 3.375
    x = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.5, td=0.01, seed=4).real(5, 300)
    N = fs // fc
    ref = []
    for i in range(N):
        f = Fraction(i * fc) + Fraction(fo)
        acc = 0j
        for t, v in enumerate(x):
            cyc = (f * (5 + t) / fs) % 1
            acc += v * cmath.exp(-2j * math.pi * float(cyc))
        ref.append(acc)
    assert rel(oracle.direct_any(x, "f64", 5, fs, fc, fo), np.array(ref)) < 1e-12


def test_direct_any_integral_offset_is_the_definition():
    """For an integral offset with a short period both routes of the oracle
    evaluate the same sum."""
    fs, fc, fo = 16000, 1000, 10
    x = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.2, td=1e-5, seed=6).i8(3, 40000)
    assert rel(oracle.direct_any(x, "i8", 3, fs, fc, fo), oracle.direct(x, "i8", 3, fs, fc, fo)) < 1e-11


@pytest.mark.parametrize("code", [1, 2, 3])
def test_direct_any_planted_mistakes(code):
    fs, fc, amp, td, n0, M, fo = 64000, 8000, 0.3, 2.5e-6, 777, 20011, 10007.25
    num, den = float(fo).as_integer_ratio()
    x = synth.Stream(fs=fs, fc=fc, fo=fo, amp=amp, td=td, sigma=0.0).real(n0, M)
    want = comb_closed_form_dyadic(fs, fc, num, den.bit_length() - 1, amp, td, n0, M)
    with oracle.mutation(code):
        T = oracle.direct_any(x, "f64", n0, fs, fc, fo)
    assert rel(T, want) > 1e-3
