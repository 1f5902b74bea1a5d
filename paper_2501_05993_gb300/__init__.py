"""Python binding of libpcal: multi-tone phase-calibration extraction on GB300.

Argument marshalling only.  Every step of the extraction runs in libpcal's
CUDA kernels behind the C ABI declared in include/pcal.h; this module loads
``_build/libpcal.so`` (built by ``build.build()``) and raises if it is absent.
Device buffers may be given as torch CUDA tensors or raw device addresses;
streams as torch streams, raw ``cudaStream_t`` integers or ``None``.

The functions named like the C entry points (``pcal_plan_create`` ...) are
direct wrappers; :class:`Plan` is the convenience object built on them.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpcal.so")

PCAL_OK, PCAL_EINVAL, PCAL_ENOMEM, PCAL_ECUDA, PCAL_EBUSY, PCAL_ETOOLARGE, PCAL_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
PCAL_F32, PCAL_I8, PCAL_2BIT = 0, 1, 2
FORMATS = {"f32": PCAL_F32, "i8": PCAL_I8, "2bit": PCAL_2BIT}
PCAL_MAX_L, PCAL_MAX_N = 1048576, 8192


class Geometry(ctypes.Structure):
    _fields_ = [("fs", ctypes.c_int64), ("f_comb", ctypes.c_int64), ("f_offset", ctypes.c_int64),
                ("N", ctypes.c_int64), ("N_rot", ctypes.c_int64), ("L", ctypes.c_int64),
                ("step_comb", ctypes.c_int64), ("step_offset", ctypes.c_int64), ("format", ctypes.c_int32),
                ("samples_per_byte_x4", ctypes.c_int32), ("row_samples", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("n_abs", ctypes.c_int64), ("n_period", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("bulk_launches", ctypes.c_int64), ("bytes_folded", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tiling(ctypes.Structure):
    _fields_ = [("cols_total", ctypes.c_int32), ("col_width", ctypes.c_int32), ("col_groups", ctypes.c_int32),
                ("replicas", ctypes.c_int32), ("box_rows", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("row_groups", ctypes.c_int64), ("rows_per_cta", ctypes.c_int64), ("upper_planes", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("smem_bytes", ctypes.c_int64), ("total_boxes", ctypes.c_int32),
                ("static_boxes", ctypes.c_int32), ("max_boxes", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ChannelDesc(ctypes.Structure):
    _fields_ = [("fs", ctypes.c_double), ("f_comb", ctypes.c_double), ("f_offset", ctypes.c_double),
                ("N", ctypes.c_int), ("sample_format", ctypes.c_int)]


PCAL_SCHED_BUCKETS = 8


class Schedule(ctypes.Structure):
    _fields_ = [("ctas", ctypes.c_int), ("box_rows", ctypes.c_int), ("stages", ctypes.c_int),
                ("static_pct", ctypes.c_int), ("min_chunk", ctypes.c_int), ("col_cap", ctypes.c_int),
                ("col_cap_bucket", ctypes.c_int * PCAL_SCHED_BUCKETS)]

    def as_dict(self) -> dict:
        return {k: (list(getattr(self, k)) if k == "col_cap_bucket" else getattr(self, k)) for k, _ in self._fields_}


PCAL_MAX_BATCH, PCAL_BATCH_MAX_N = 4096, 1024


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_streams", ctypes.c_int), ("period_s", ctypes.c_double),
                ("ring_s", ctypes.c_double)]


class ServerResult(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_int32), ("n_tones", ctypes.c_int32), ("period", ctypes.c_int64),
                ("n_samples", ctypes.c_int64), ("td_s", ctypes.c_double), ("sigma_td_s", ctypes.c_double),
                ("latency_s", ctypes.c_double), ("td_peak_s", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_int64), ("queued", ctypes.c_int64), ("active", ctypes.c_int64),
                ("periods", ctypes.c_int64), ("samples", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("bytes_h2d", ctypes.c_int64), ("hbm_in_use", ctypes.c_int64), ("hbm_budget", ctypes.c_int64),
                ("p50_latency_s", ctypes.c_double), ("p99_latency_s", ctypes.c_double),
                ("max_latency_s", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PcalError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


_lib = None


def load(path: str | None = None):
    """Load libpcal.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libpcal is not built ({path} missing): run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    vp, i64, ci, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "pcal_plan_geometry": ([dbl, dbl, dbl, ci, ci, P(Geometry)], ci),
        "pcal_plan_create": ([dbl, dbl, dbl, ci, ci, P(vp)], ci),
        "pcal_plan_destroy": ([vp], ci),
        "pcal_plan_get_geometry": ([vp, P(Geometry)], ci),
        "pcal_plan_set_levels": ([vp, P(dbl)], ci),
        "pcal_accumulate": ([vp, vp, i64, vp], ci),
        "pcal_accumulate_host": ([vp, vp, i64, vp], ci),
        "pcal_accumulate_host_async": ([vp, vp, i64, vp], ci),
        "pcal_finalize_async": ([vp, vp], ci),
        "pcal_read_async_results": ([vp, ci, vp, vp, vp, vp, vp, vp], ci),
        "pcal_finalize_device": ([vp, vp], ci),
        "pcal_finalize": ([vp, vp], ci),
        "pcal_read_results": ([vp, vp, vp, vp, vp, vp, vp], ci),
        "pcal_get_delay": ([vp, P(dbl), P(dbl)], ci),
        "pcal_read_post": ([vp, vp, vp, vp], ci),
        "pcal_result_device": ([vp], vp),
        "pcal_get_bins": ([vp, vp], ci),
        "pcal_get_stats": ([vp, P(Stats)], ci),
        "pcal_strerror": ([ci], ctypes.c_char_p),
        "pcal_bulk_tiling": ([dbl, dbl, dbl, ci, ci, ci, i64, P(Tiling)], ci),
        "pcal_tones_from_counts_noalloc": ([dbl, dbl, dbl, ci, vp, i64, P(dbl), vp, vp], ci),
        "pcal_batch_create": ([P(ChannelDesc), ci, P(vp)], ci),
        "pcal_batch_destroy": ([vp], ci),
        "pcal_batch_get_geometry": ([vp, ci, P(Geometry)], ci),
        "pcal_batch_set_schedule": ([vp, P(Schedule)], ci),
        "pcal_batch_get_schedule": ([vp, P(Schedule)], ci),
        "pcal_batch_channel_tiling": ([vp, ci, P(ci), P(ci), P(ci)], ci),
        "pcal_batch_accumulate": ([vp, P(vp), P(i64), vp], ci),
        "pcal_batch_finalize_device": ([vp, vp], ci),
        "pcal_batch_step_graph": ([vp, P(vp), P(i64), vp], ci),
        "pcal_batch_read_results": ([vp, ci, vp, vp, vp, vp, vp, vp], ci),
        "pcal_batch_result_device": ([vp, ci, P(vp)], ci),
        "pcal_batch_read_post": ([vp, ci, vp, vp, vp], ci),
        "pcal_batch_get_bins": ([vp, ci, vp], ci),
        "pcal_batch_get_stats": ([vp, P(Stats)], ci),
        "pcal_batch_autotune": ([vp, P(vp), P(i64), vp, P(Schedule)], ci),
        "pcal_server_stream_bytes": ([P(ServerConfig), P(ChannelDesc), P(i64)], ci),
        "pcal_rotfold_create": ([dbl, dbl, dbl, ci, ci, ci, ci, P(vp)], ci),
        "pcal_rotfold_destroy": ([vp], ci),
        "pcal_rotfold_accumulate": ([vp, vp, i64, vp], ci),
        "pcal_rotfold_finalize": ([vp, vp, vp], ci),
        "pcal_rotfold_get_acc": ([vp, vp], ci),
        "pcal_selftest_wait_timeout": ([dbl, P(ctypes.c_uint)], ci),
        "pcal_dft_create": ([ci, ci, P(vp)], ci),
        "pcal_batch_set_dft": ([vp, ci], ci),
        "pcal_dft_destroy": ([vp], ci),
        "pcal_dft_execute": ([vp, vp, i64, vp, vp], ci),
        "pcal_dft_check": ([vp, P(ctypes.c_uint)], ci),
        "pcal_dft_weights_host": ([ci, ci, ci, ci, vp, P(ci), P(ci)], ci),
        "pcal_rotplan_create": ([dbl, dbl, dbl, ci, ci, P(vp)], ci),
        "pcal_rotplan_destroy": ([vp], ci),
        "pcal_rotplan_set_levels": ([vp, P(dbl)], ci),
        "pcal_rotplan_accumulate": ([vp, vp, i64, vp], ci),
        "pcal_rotplan_finalize_device": ([vp, vp], ci),
        "pcal_rotplan_read_results": ([vp, vp, vp, vp, vp, vp, vp, vp, vp], ci),
        "pcal_server_create": ([P(ServerConfig), P(vp)], ci),
        "pcal_server_destroy": ([vp], ci),
        "pcal_server_open": ([vp, P(ChannelDesc), P(ci)], ci),
        "pcal_server_submit": ([vp, ci, vp, i64], ci),
        "pcal_server_submit_many": ([vp, ci, P(ci), P(vp), P(i64)], ci),
        "pcal_server_submit_many_at": ([vp, ci, P(ci), P(vp), P(i64), P(dbl)], ci),
        "pcal_clock_s": ([], dbl),
        "pcal_server_close": ([vp, ci], ci),
        "pcal_server_poll": ([vp, P(ServerResult), vp, ci, dbl], ci),
        "pcal_server_drain": ([vp, dbl], ci),
        "pcal_server_get_stats": ([vp, P(ServerStats)], ci),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().pcal_strerror(int(code)).decode()


def _check(rc: int, where: str):
    if rc != PCAL_OK:
        raise PcalError(rc, where)


def _ptr(x) -> int:
    """Device address of a torch tensor or an integer address."""
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    return int(x)


def _stream(s) -> int:
    if s is None:
        return 0
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    return int(s)


# ---- thin wrappers with the C names ------------------------------------------------

def pcal_plan_geometry(fs, f_comb, f_offset, N, sample_format) -> Geometry:
    g = Geometry()
    _check(load().pcal_plan_geometry(float(fs), float(f_comb), float(f_offset), int(N), int(sample_format),
                                     ctypes.byref(g)), "pcal_plan_geometry")
    return g


def pcal_plan_create(fs, f_comb, f_offset, N, sample_format) -> int:
    h = ctypes.c_void_p()
    _check(load().pcal_plan_create(float(fs), float(f_comb), float(f_offset), int(N), int(sample_format),
                                   ctypes.byref(h)), "pcal_plan_create")
    return h.value


def pcal_plan_destroy(plan: int) -> None:
    _check(load().pcal_plan_destroy(plan), "pcal_plan_destroy")


def pcal_plan_set_levels(plan: int, levels) -> None:
    lv = (ctypes.c_double * 4)(*[float(v) for v in levels])
    _check(load().pcal_plan_set_levels(plan, lv), "pcal_plan_set_levels")


def device_sample_count(samples, fmt: str, n: int | None) -> int:
    """Samples to fold from `samples`: n, or all a tensor holds.  A tensor must
    be a contiguous CUDA tensor with elements of the format's size (1 byte for
    "2bit" and "i8", 4 for "f32"), and n may not exceed what it holds; an
    integer address needs an explicit n.  Raises ValueError otherwise."""
    if not hasattr(samples, "data_ptr"):
        if n is None:
            raise ValueError("an address needs an explicit sample count n")
        return int(n)
    if not samples.is_cuda:
        raise ValueError("samples must be a CUDA tensor (host arrays go through accumulate_host)")
    if not samples.is_contiguous():
        raise ValueError("samples must be contiguous")
    esize = 4 if fmt == "f32" else 1
    if samples.element_size() != esize:
        raise ValueError(f"{fmt} samples are {esize}-byte elements, got {samples.element_size()}-byte ones")
    held = samples.numel() * (4 if fmt == "2bit" else 1)
    if n is None:
        return held
    if int(n) > held:
        raise ValueError(f"n = {int(n)} exceeds the {held} samples the tensor holds")
    return int(n)


def host_sample_count(host: np.ndarray, fmt: str, n: int | None) -> int:
    """Samples to take from a host array: n, or all it holds.  The array must
    be C-contiguous with elements of the format's size (1 byte for "2bit" and
    "i8", 4 for "f32"), and n may not exceed what it holds.  Raises ValueError
    otherwise."""
    if not host.flags.c_contiguous:
        raise ValueError("host samples must be C-contiguous")
    esize = 4 if fmt == "f32" else 1
    if host.itemsize != esize:
        raise ValueError(f"{fmt} samples are {esize}-byte elements, got {host.itemsize}-byte ones")
    held = host.size * (4 if fmt == "2bit" else 1)
    if n is None:
        return held
    if int(n) > held:
        raise ValueError(f"n = {int(n)} exceeds the {held} samples the array holds")
    return int(n)


def pcal_accumulate(plan: int, samples, n: int, stream=None) -> None:
    _check(load().pcal_accumulate(plan, _ptr(samples), int(n), _stream(stream)), "pcal_accumulate")


def pcal_accumulate_host(plan: int, host: np.ndarray, n: int, stream=None) -> None:
    if not host.flags.c_contiguous:
        raise ValueError("host samples must be C-contiguous")
    _check(load().pcal_accumulate_host(plan, host.ctypes.data, int(n), _stream(stream)), "pcal_accumulate_host")


def pcal_accumulate_host_async(plan: int, host: np.ndarray, n: int, stream=None) -> None:
    """As pcal_accumulate_host without waiting for the copies: `host` must stay unchanged until the
    stream has passed this call's folds."""
    if not host.flags.c_contiguous:
        raise ValueError("host samples must be C-contiguous")
    _check(load().pcal_accumulate_host_async(plan, host.ctypes.data, int(n), _stream(stream)),
           "pcal_accumulate_host_async")


def pcal_finalize_async(plan: int, stream=None) -> None:
    _check(load().pcal_finalize_async(plan, _stream(stream)), "pcal_finalize_async")


def pcal_read_async_results(plan: int, n_tones: int, age: int = 0) -> dict:
    ph = np.zeros(2 * n_tones)
    amp, phase, un = np.zeros(n_tones), np.zeros(n_tones), np.zeros(n_tones)
    td, sg = ctypes.c_double(), ctypes.c_double()
    _check(load().pcal_read_async_results(plan, int(age), ph.ctypes.data, amp.ctypes.data, phase.ctypes.data,
                                          un.ctypes.data, ctypes.addressof(td), ctypes.addressof(sg)),
           "pcal_read_async_results")
    return {"phasors": ph[0::2] + 1j * ph[1::2], "amp": amp, "phase": phase, "unwrapped": un, "td": td.value,
            "sigma_td": sg.value}


def pcal_finalize_device(plan: int, stream=None) -> None:
    _check(load().pcal_finalize_device(plan, _stream(stream)), "pcal_finalize_device")


def pcal_finalize(plan: int, n_tones: int) -> np.ndarray:
    out = np.zeros(2 * n_tones, dtype=np.float64)
    _check(load().pcal_finalize(plan, out.ctypes.data), "pcal_finalize")
    return out[0::2] + 1j * out[1::2]


def pcal_read_results(plan: int, n_tones: int) -> dict:
    ph = np.zeros(2 * n_tones)
    amp, phase, un = np.zeros(n_tones), np.zeros(n_tones), np.zeros(n_tones)
    td, sg = ctypes.c_double(), ctypes.c_double()
    _check(load().pcal_read_results(plan, ph.ctypes.data, amp.ctypes.data, phase.ctypes.data, un.ctypes.data,
                                    ctypes.addressof(td), ctypes.addressof(sg)), "pcal_read_results")
    return {"phasors": ph[0::2] + 1j * ph[1::2], "amp": amp, "phase": phase, "unwrapped": un, "td": td.value,
            "sigma_td": sg.value}


def pcal_get_delay(plan: int) -> tuple[float, float]:
    td, sg = ctypes.c_double(), ctypes.c_double()
    _check(load().pcal_get_delay(plan, ctypes.byref(td), ctypes.byref(sg)), "pcal_get_delay")
    return td.value, sg.value


def pcal_read_post(plan: int, n_tones: int) -> dict:
    tp, pb = ctypes.c_double(), ctypes.c_double()
    bp = np.empty(n_tones)
    _check(load().pcal_read_post(plan, ctypes.addressof(tp), ctypes.addressof(pb), bp.ctypes.data), "pcal_read_post")
    return {"td_peak": tp.value, "peak_bin": pb.value, "bandpass_phase": bp}


def pcal_batch_read_post(batch: int, channel: int, n_tones: int) -> dict:
    tp, pb = ctypes.c_double(), ctypes.c_double()
    bp = np.empty(n_tones)
    _check(load().pcal_batch_read_post(batch, channel, ctypes.addressof(tp), ctypes.addressof(pb), bp.ctypes.data),
           "pcal_batch_read_post")
    return {"td_peak": tp.value, "peak_bin": pb.value, "bandpass_phase": bp}


def pcal_result_device(plan: int) -> int:
    return int(load().pcal_result_device(plan) or 0)


def pcal_get_bins(plan: int, geometry: Geometry) -> np.ndarray:
    L = int(geometry.L)
    if geometry.format == PCAL_2BIT:
        out = np.zeros((L, 4), dtype=np.int64)
    elif geometry.format == PCAL_I8:
        out = np.zeros(L, dtype=np.int64)
    else:
        out = np.zeros(L, dtype=np.float64)
    _check(load().pcal_get_bins(plan, out.ctypes.data), "pcal_get_bins")
    return out


def pcal_bulk_tiling(fs, f_comb, f_offset, N, sample_format, num_sms, n_rows) -> Tiling:
    t = Tiling()
    _check(load().pcal_bulk_tiling(float(fs), float(f_comb), float(f_offset), int(N), int(sample_format),
                                   int(num_sms), int(n_rows), ctypes.byref(t)), "pcal_bulk_tiling")
    return t


def pcal_tones_from_counts_noalloc(fs, f_comb, f_offset, N, d_counts, n_samples, levels, d_results,
                                   stream=None) -> None:
    """Finalize from device counts [L][4] into a device result buffer of
    5N+3 doubles, without any allocation (see include/pcal.h)."""
    lv = (ctypes.c_double * 4)(*[float(v) for v in levels])
    _check(load().pcal_tones_from_counts_noalloc(float(fs), float(f_comb), float(f_offset), int(N), _ptr(d_counts),
                                                 int(n_samples), lv, _ptr(d_results), _stream(stream)),
           "pcal_tones_from_counts_noalloc")


def pcal_get_stats(plan: int) -> Stats:
    s = Stats()
    _check(load().pcal_get_stats(plan, ctypes.byref(s)), "pcal_get_stats")
    return s


# ---- convenience object ---------------------------------------------------------------

class Plan:
    """One extraction plan (one baseband channel) on the current CUDA device."""

    def __init__(self, fs: int, f_comb: int, f_offset: int, fmt: str = "2bit", N: int | None = None):
        N = int(fs) // int(f_comb) if N is None else int(N)
        self.fmt = fmt
        self.handle = pcal_plan_create(fs, f_comb, f_offset, N, FORMATS[fmt])
        g = Geometry()
        _check(load().pcal_plan_get_geometry(self.handle, ctypes.byref(g)), "pcal_plan_get_geometry")
        self.geometry = g
        self.N, self.L = int(g.N), int(g.L)

    def close(self):
        if getattr(self, "handle", None):
            pcal_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_levels(self, levels):
        pcal_plan_set_levels(self.handle, levels)

    def accumulate(self, samples, n: int | None = None, stream=None):
        """Fold device samples (a torch CUDA tensor of the plan's format, or
        an address with an explicit n)."""
        pcal_accumulate(self.handle, samples, device_sample_count(samples, self.fmt, n), stream)

    def accumulate_host(self, host: np.ndarray, n: int | None = None, stream=None):
        pcal_accumulate_host(self.handle, host, host_sample_count(host, self.fmt, n), stream)

    def accumulate_host_async(self, host: np.ndarray, n: int | None = None, stream=None):
        pcal_accumulate_host_async(self.handle, host, host_sample_count(host, self.fmt, n), stream)

    def finalize_device(self, stream=None):
        pcal_finalize_device(self.handle, stream)

    def finalize_async(self, stream=None):
        pcal_finalize_async(self.handle, stream)

    def read_async(self, age: int = 0) -> dict:
        return pcal_read_async_results(self.handle, self.N, age)

    def finalize(self) -> np.ndarray:
        return pcal_finalize(self.handle, self.N)

    def results(self) -> dict:
        return pcal_read_results(self.handle, self.N)

    def bins(self) -> np.ndarray:
        return pcal_get_bins(self.handle, self.geometry)

    def post(self) -> dict:
        """Peak delay and corrected bandpass of the last finalize."""
        return pcal_read_post(self.handle, self.N)

    def stats(self) -> dict:
        return pcal_get_stats(self.handle).as_dict()

    @property
    def result_device_ptr(self) -> int:
        return pcal_result_device(self.handle)


# ---- batches ------------------------------------------------------------------------


def _ptr_array(samples, count: int):
    arr = (ctypes.c_void_p * count)(*[_ptr(x) or None for x in samples])
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), arr


def _n_array(n, count: int):
    arr = (ctypes.c_int64 * count)(*[int(v) for v in n])
    return arr


def pcal_batch_create(channels) -> int:
    """channels: sequence of (fs, f_comb, f_offset, fmt) or (fs, f_comb, f_offset, fmt, N)."""
    descs = (ChannelDesc * len(channels))()
    for d, ch in zip(descs, channels):
        fs, fc, fo, fmt = ch[:4]
        d.fs, d.f_comb, d.f_offset = float(fs), float(fc), float(fo)
        d.N = int(ch[4]) if len(ch) > 4 else int(round(fs / fc))
        d.sample_format = FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
    h = ctypes.c_void_p()
    _check(load().pcal_batch_create(descs, len(channels), ctypes.byref(h)), "pcal_batch_create")
    return h.value


def pcal_batch_destroy(batch: int) -> None:
    _check(load().pcal_batch_destroy(batch), "pcal_batch_destroy")


def pcal_batch_get_geometry(batch: int, channel: int) -> Geometry:
    g = Geometry()
    _check(load().pcal_batch_get_geometry(batch, channel, ctypes.byref(g)), "pcal_batch_get_geometry")
    return g


def pcal_batch_set_schedule(batch: int, sched: Schedule) -> None:
    _check(load().pcal_batch_set_schedule(batch, ctypes.byref(sched)), "pcal_batch_set_schedule")


def pcal_batch_get_schedule(batch: int) -> Schedule:
    s = Schedule()
    _check(load().pcal_batch_get_schedule(batch, ctypes.byref(s)), "pcal_batch_get_schedule")
    return s


def pcal_batch_accumulate(batch: int, samples, n, stream=None) -> None:
    pp, keep = _ptr_array(samples, len(samples))
    _check(load().pcal_batch_accumulate(batch, pp, _n_array(n, len(samples)), _stream(stream)),
           "pcal_batch_accumulate")


def pcal_batch_finalize_device(batch: int, stream=None) -> None:
    _check(load().pcal_batch_finalize_device(batch, _stream(stream)), "pcal_batch_finalize_device")


def pcal_batch_step_graph(batch: int, samples, n, stream=None) -> None:
    pp, keep = _ptr_array(samples, len(samples))
    _check(load().pcal_batch_step_graph(batch, pp, _n_array(n, len(samples)), _stream(stream)),
           "pcal_batch_step_graph")


def pcal_batch_read_results(batch: int, channel: int, n_tones: int) -> dict:
    ph = np.empty(2 * n_tones)
    amp, phase, unw = np.empty(n_tones), np.empty(n_tones), np.empty(n_tones)
    td, sig = ctypes.c_double(), ctypes.c_double()
    _check(load().pcal_batch_read_results(batch, channel, ph.ctypes.data, amp.ctypes.data, phase.ctypes.data,
                                          unw.ctypes.data, ctypes.addressof(td), ctypes.addressof(sig)),
           "pcal_batch_read_results")
    return {"phasors": ph[0::2] + 1j * ph[1::2], "amp": amp, "phase": phase, "unwrapped": unw,
            "td": td.value, "sigma_td": sig.value}


def pcal_batch_result_device(batch: int, channel: int) -> int:
    out = ctypes.c_void_p()
    _check(load().pcal_batch_result_device(batch, channel, ctypes.byref(out)), "pcal_batch_result_device")
    return out.value


def pcal_batch_get_bins(batch: int, channel: int, geometry: Geometry) -> np.ndarray:
    if geometry.format == PCAL_2BIT:
        out = np.empty((geometry.L, 4), dtype=np.int64)
    else:
        out = np.empty(geometry.L, dtype=np.int64)
    _check(load().pcal_batch_get_bins(batch, channel, out.ctypes.data), "pcal_batch_get_bins")
    return out


def pcal_batch_get_stats(batch: int) -> Stats:
    st = Stats()
    _check(load().pcal_batch_get_stats(batch, ctypes.byref(st)), "pcal_batch_get_stats")
    return st


def pcal_batch_autotune(batch: int, samples, n, stream=None) -> Schedule:
    pp, keep = _ptr_array(samples, len(samples))
    s = Schedule()
    _check(load().pcal_batch_autotune(batch, pp, _n_array(n, len(samples)), _stream(stream), ctypes.byref(s)),
           "pcal_batch_autotune")
    return s


class Batch:
    """Many channels (2-bit or int8) folded by one persistent launch per call."""

    def __init__(self, channels):
        self.channels = [tuple(c) for c in channels]
        self.handle = pcal_batch_create(self.channels)
        self.geometry = [pcal_batch_get_geometry(self.handle, c) for c in range(len(self.channels))]

    def close(self):
        if getattr(self, "handle", None):
            pcal_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __len__(self):
        return len(self.channels)

    def _check_tensors(self, samples, n):
        names = {v: k for k, v in FORMATS.items()}
        for c, x in enumerate(samples):
            if hasattr(x, "data_ptr") and c < len(self.channels):
                fmt = self.channels[c][3]
                device_sample_count(x, fmt if isinstance(fmt, str) else names[int(fmt)], n[c])

    def accumulate(self, samples, n, stream=None):
        self._check_tensors(samples, n)
        pcal_batch_accumulate(self.handle, samples, n, stream)

    def finalize_device(self, stream=None):
        pcal_batch_finalize_device(self.handle, stream)

    def step_graph(self, samples, n, stream=None):
        self._check_tensors(samples, n)
        pcal_batch_step_graph(self.handle, samples, n, stream)

    def results(self, channel: int) -> dict:
        return pcal_batch_read_results(self.handle, channel, int(self.geometry[channel].N))

    def bins(self, channel: int) -> np.ndarray:
        return pcal_batch_get_bins(self.handle, channel, self.geometry[channel])

    def post(self, channel: int) -> dict:
        return pcal_batch_read_post(self.handle, channel, int(self.geometry[channel].N))

    def stats(self) -> dict:
        return pcal_batch_get_stats(self.handle).as_dict()

    @property
    def schedule(self) -> dict:
        return pcal_batch_get_schedule(self.handle).as_dict()

    def set_schedule(self, **kw):
        s = pcal_batch_get_schedule(self.handle)
        for k, v in kw.items():
            if k == "col_cap_bucket":
                if len(v) != PCAL_SCHED_BUCKETS:
                    raise ValueError(f"col_cap_bucket takes {PCAL_SCHED_BUCKETS} caps")
                for i, x in enumerate(v):
                    s.col_cap_bucket[i] = int(x)
            else:
                setattr(s, k, int(v))
        pcal_batch_set_schedule(self.handle, s)

    def channel_tiling(self, channel: int) -> dict:
        """The bucket, column-group width (32-bit words) and group count of a channel's rows."""
        bk, cw, gc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().pcal_batch_channel_tiling(self.handle, int(channel), ctypes.byref(bk), ctypes.byref(cw),
                                                ctypes.byref(gc)), "pcal_batch_channel_tiling")
        return {"bucket": bk.value, "col_width": cw.value, "col_groups": gc.value}

    def set_dft(self, mode: str):
        """Tone DFT of the finalize: "fp32" (inside each channel's cluster), "tf32x3" or "bf16x6"
        (one tensor-core contraction per distinct N)."""
        _check(load().pcal_batch_set_dft(self.handle, DFT_MODES[mode]), "pcal_batch_set_dft")

    def autotune(self, samples, n, stream=None) -> dict:
        return pcal_batch_autotune(self.handle, samples, n, stream).as_dict()


# ---- serving --------------------------------------------------------------------------


def clock_s() -> float:
    """The library's monotonic clock (seconds), the clock of serving arrival times and latencies."""
    return load().pcal_clock_s()


def pcal_server_stream_bytes(fs, f_comb, f_offset, fmt, period_s=1.0, ring_s=0.1, N=None) -> int:
    cfg = ServerConfig(1, 1, float(period_s), float(ring_s))
    d = ChannelDesc(float(fs), float(f_comb), float(f_offset), int(N if N is not None else round(fs / f_comb)),
                    FORMATS[fmt] if isinstance(fmt, str) else int(fmt))
    out = ctypes.c_int64()
    _check(load().pcal_server_stream_bytes(ctypes.byref(cfg), ctypes.byref(d), ctypes.byref(out)),
           "pcal_server_stream_bytes")
    return out.value


class Server:
    """Live streams folded by continuous batching (see pcal_server_* in pcal.h)."""

    def __init__(self, hbm_budget_bytes: int, max_streams: int, period_s: float = 1.0, ring_s: float = 0.1):
        cfg = ServerConfig(int(hbm_budget_bytes), int(max_streams), float(period_s), float(ring_s))
        h = ctypes.c_void_p()
        _check(load().pcal_server_create(ctypes.byref(cfg), ctypes.byref(h)), "pcal_server_create")
        self.handle = h.value
        self.n_tones = {}
        self.fmts = {}

    def close(self):
        if getattr(self, "handle", None):
            _check(load().pcal_server_destroy(self.handle), "pcal_server_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def open(self, fs, f_comb, f_offset, fmt, N=None) -> int:
        d = ChannelDesc(float(fs), float(f_comb), float(f_offset), int(N if N is not None else round(fs / f_comb)),
                        FORMATS[fmt] if isinstance(fmt, str) else int(fmt))
        sid = ctypes.c_int()
        _check(load().pcal_server_open(self.handle, ctypes.byref(d), ctypes.byref(sid)), "pcal_server_open")
        self.n_tones[sid.value] = d.N
        self.fmts[sid.value] = {v: k for k, v in FORMATS.items()}[d.sample_format]
        return sid.value

    def _host_n(self, stream: int, host: np.ndarray, n: int) -> int:
        fmt = self.fmts.get(int(stream))
        if fmt is None:  # not opened here: the library checks the stream id
            if not host.flags.c_contiguous:
                raise ValueError("host samples must be C-contiguous")
            return int(n)
        return host_sample_count(host, fmt, n)

    def submit(self, stream: int, host: np.ndarray, n: int):
        n = self._host_n(stream, host, n)
        _check(load().pcal_server_submit(self.handle, int(stream), host.ctypes.data, n), "pcal_server_submit")

    def submit_many(self, streams, hosts, ns, arrival_s=None):
        """One chunk per stream; arrival_s: the chunks' arrival times on pcal_clock_s (None: now)."""
        k = len(streams)
        ids = (ctypes.c_int * k)(*[int(x) for x in streams])
        ptrs = (ctypes.c_void_p * k)(*[h.ctypes.data for h in hosts])
        nn = (ctypes.c_int64 * k)(*[self._host_n(x, h, m) for x, h, m in zip(streams, hosts, ns)])
        arr = None
        if arrival_s is not None:
            if len(arrival_s) != k:
                raise ValueError("one arrival time per chunk")
            arr = (ctypes.c_double * k)(*[float(t) for t in arrival_s])
        _check(load().pcal_server_submit_many_at(self.handle, k, ids,
                                                 ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p)), nn, arr),
               "pcal_server_submit_many_at")

    def close_stream(self, stream: int):
        _check(load().pcal_server_close(self.handle, int(stream)), "pcal_server_close")

    def poll(self, timeout_s: float = 0.0, max_tones: int = PCAL_BATCH_MAX_N):
        r = ServerResult()
        ph = np.empty(2 * max_tones)
        rc = load().pcal_server_poll(self.handle, ctypes.byref(r), ph.ctypes.data, int(max_tones), float(timeout_s))
        if rc < 0:
            raise PcalError(rc, "pcal_server_poll")
        if rc == 0:
            return None
        n = r.n_tones
        return {"stream": r.stream, "period": r.period, "n_samples": r.n_samples, "td": r.td_s,
                "sigma_td": r.sigma_td_s, "latency_s": r.latency_s, "td_peak": r.td_peak_s,
                "phasors": ph[0:2 * n:2] + 1j * ph[1:2 * n:2]}

    def drain(self, timeout_s: float = 60.0):
        _check(load().pcal_server_drain(self.handle, float(timeout_s)), "pcal_server_drain")

    def stats(self) -> dict:
        st = ServerStats()
        _check(load().pcal_server_get_stats(self.handle, ctypes.byref(st)), "pcal_server_get_stats")
        return st.as_dict()


# ---- precision study: the paper's per-sample rotation in FP32 -------------------------

PCAL_ROT_TABLE, PCAL_ROT_TABLE_KAHAN, PCAL_ROT_DFR = 0, 1, 2
ROT_VARIANTS = {"table": PCAL_ROT_TABLE, "table_kahan": PCAL_ROT_TABLE_KAHAN, "dfr": PCAL_ROT_DFR}


class RotFold:
    """Rotate-then-fold in FP32 (the paper's route), for the precision study."""

    def __init__(self, fs, f_comb, f_offset, fmt: str, variant: str, lanes: int = 128, N=None):
        self.N = int(N if N is not None else round(fs / f_comb))
        self.lanes = int(lanes)
        h = ctypes.c_void_p()
        _check(load().pcal_rotfold_create(float(fs), float(f_comb), float(f_offset), self.N, FORMATS[fmt],
                                          ROT_VARIANTS[variant], self.lanes, ctypes.byref(h)), "pcal_rotfold_create")
        self.handle = h.value
        self.fmt = fmt

    def close(self):
        if getattr(self, "handle", None):
            load().pcal_rotfold_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def accumulate(self, samples, n: int, stream=None):
        n = device_sample_count(samples, self.fmt, n)
        _check(load().pcal_rotfold_accumulate(self.handle, _ptr(samples), n, _stream(stream)),
               "pcal_rotfold_accumulate")

    def acc(self) -> np.ndarray:
        out = np.empty((self.lanes, self.N, 4), dtype=np.float32)
        _check(load().pcal_rotfold_get_acc(self.handle, out.ctypes.data), "pcal_rotfold_get_acc")
        return out

    def finalize(self, stream=None) -> np.ndarray:
        out = np.empty(2 * self.N)
        _check(load().pcal_rotfold_finalize(self.handle, out.ctypes.data, _stream(stream)), "pcal_rotfold_finalize")
        return out[0::2] + 1j * out[1::2]


# ---- long-period plans: offsets that cannot be folded ---------------------------------


class RotPlan:
    """Per-sample double-float rotation for prime or non-integral offsets."""

    def __init__(self, fs, f_comb, f_offset, fmt: str = "i8", N=None):
        self.N = int(N if N is not None else round(fs / f_comb))
        h = ctypes.c_void_p()
        _check(load().pcal_rotplan_create(float(fs), float(f_comb), float(f_offset), self.N, FORMATS[fmt],
                                          ctypes.byref(h)), "pcal_rotplan_create")
        self.handle = h.value
        self.fmt = fmt

    def close(self):
        if getattr(self, "handle", None):
            load().pcal_rotplan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def accumulate(self, samples, n: int, stream=None):
        n = device_sample_count(samples, self.fmt, n)
        _check(load().pcal_rotplan_accumulate(self.handle, _ptr(samples), n, _stream(stream)),
               "pcal_rotplan_accumulate")

    def finalize_device(self, stream=None):
        _check(load().pcal_rotplan_finalize_device(self.handle, _stream(stream)), "pcal_rotplan_finalize_device")

    def results(self) -> dict:
        N = self.N
        ph, amp, phase, unw, bp = np.empty(2 * N), np.empty(N), np.empty(N), np.empty(N), np.empty(N)
        td, sig, tp = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(load().pcal_rotplan_read_results(self.handle, ph.ctypes.data, amp.ctypes.data, phase.ctypes.data,
                                                unw.ctypes.data, ctypes.addressof(td), ctypes.addressof(sig),
                                                ctypes.addressof(tp), bp.ctypes.data), "pcal_rotplan_read_results")
        return {"phasors": ph[0::2] + 1j * ph[1::2], "amp": amp, "phase": phase, "unwrapped": unw,
                "td": td.value, "sigma_td": sig.value, "td_peak": tp.value, "bandpass_phase": bp}

    def finalize(self) -> np.ndarray:
        self.finalize_device()
        return self.results()["phasors"]


# ---- batched tone DFT ---------------------------------------------------------------

PCAL_DFT_FP32, PCAL_DFT_TC_TF32X3, PCAL_DFT_TC_BF16X6 = 0, 1, 2
DFT_MODES = {"fp32": PCAL_DFT_FP32, "tf32x3": PCAL_DFT_TC_TF32X3, "bf16x6": PCAL_DFT_TC_BF16X6}
DFT_TILE_COLS = {"tf32x3": 256, "bf16x6": 256}  # output columns per weight tile (pcal.h)
DFT_CHUNK_BYTES = {"tf32x3": 128, "bf16x6": 64}  # bytes of K per weight tile row (pcal.h)


class Dft:
    """Batched N-point tone DFT of C channels: T[c, i] = sum_b P[c, b] e^{-j 2 pi i b / N}
    (device complex64 arrays [C][N]); mode "fp32" (CUDA cores), "tf32x3" or "bf16x6" (tensor cores)."""

    def __init__(self, N: int, mode: str = "tf32x3"):
        self.N, self.mode = int(N), mode
        h = ctypes.c_void_p()
        _check(load().pcal_dft_create(self.N, DFT_MODES[mode], ctypes.byref(h)), "pcal_dft_create")
        self.handle = h.value

    def close(self):
        if getattr(self, "handle", None):
            load().pcal_dft_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def execute(self, P, C: int, T, stream=None):
        """T[:C] = the tone DFT of P[:C] (C x N complex64, CUDA tensors or addresses)."""
        for name, x in (("P", P), ("T", T)):
            if hasattr(x, "data_ptr"):
                if not x.is_cuda or not x.is_contiguous() or x.element_size() != 8:
                    raise ValueError(f"{name} must be a contiguous complex64 CUDA tensor")
                if x.numel() < int(C) * self.N:
                    raise ValueError(f"{name} holds {x.numel()} values, fewer than C x N = {int(C) * self.N}")
        _check(load().pcal_dft_execute(self.handle, _ptr(P), int(C), _ptr(T), _stream(stream)), "pcal_dft_execute")

    def check(self) -> int:
        flags = ctypes.c_uint()
        _check(load().pcal_dft_check(self.handle, ctypes.byref(flags)), "pcal_dft_check")
        return flags.value


def pcal_dft_weights_host(N: int, mode: str, tile: int, chunk: int) -> tuple[list, int]:
    """Host copy of weight tile (tile, chunk) of a tensor-core mode: its parts (2 or 3 byte arrays of
    DFT_TILE_COLS[mode] x DFT_CHUNK_BYTES[mode] bytes, the tile image of each part) and its rows."""
    stride = DFT_TILE_COLS.get(mode, 128) * DFT_CHUNK_BYTES.get(mode, 128)
    buf = np.zeros(3 * stride, np.uint8)
    rows, n_parts = ctypes.c_int(), ctypes.c_int()
    _check(load().pcal_dft_weights_host(int(N), DFT_MODES[mode], int(tile), int(chunk), buf.ctypes.data,
                                        ctypes.byref(rows), ctypes.byref(n_parts)), "pcal_dft_weights_host")
    return [buf[stride * p:stride * (p + 1)] for p in range(n_parts.value)], rows.value


def pcal_selftest_wait_timeout(limit_s: float) -> tuple[int, int]:
    """(status, device error bits) of a bounded wait that is made to run out."""
    flags = ctypes.c_uint()
    rc = load().pcal_selftest_wait_timeout(float(limit_s), ctypes.byref(flags))
    return rc, flags.value
