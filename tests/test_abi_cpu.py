"""The C ABI without a GPU: the library loads, exports every entry point the
header declares, validates plans on the host, and fails cleanly without a
device.  Also the host check of the 2-bit kernel's bit-sliced arithmetic."""
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2501_05993_gb300 as pcal
from paper_2501_05993_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pcal.h")


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return pcal.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pcal_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_core_entry_points():
    names = declared_functions()
    for core in ("pcal_plan_create", "pcal_accumulate", "pcal_finalize"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", pcal.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pcal_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


@pytest.mark.parametrize("fs,fc,fo,fmt,N,L", [
    (16e6, 1e6, 10e3, pcal.PCAL_F32, 16, 1600),
    (64e6, 1e6, 10e3, pcal.PCAL_2BIT, 64, 6400),
    (1024e6, 1e6, 10e3, pcal.PCAL_I8, 1024, 102400),
    (32e6, 1e6, 0, pcal.PCAL_2BIT, 32, 32),
    (16, 4, 1, pcal.PCAL_2BIT, 4, 16),
    (48e6, 1e6, 30e3, pcal.PCAL_I8, 48, 4800),
])
def test_geometry(lib, fs, fc, fo, fmt, N, L):
    g = pcal.pcal_plan_geometry(fs, fc, fo, N, fmt)
    assert (g.N, g.L) == (N, L)
    assert g.N_rot == int(fs) // __import__("math").gcd(int(fs), int(fo))
    spw = {pcal.PCAL_F32: 1, pcal.PCAL_I8: 4, pcal.PCAL_2BIT: 16}[fmt]
    assert g.samples_per_byte_x4 == spw
    row_bytes = g.row_samples * 4 // spw
    assert g.row_samples % L == 0 and g.row_samples % (4 * spw) == 0 and row_bytes >= 256


@pytest.mark.parametrize("args,code", [
    ((16e6, 1e6, 10e3, 15, pcal.PCAL_F32), pcal.PCAL_EINVAL),      # N != fs/fc
    ((16e6, 1e6, 1e6, 16, pcal.PCAL_F32), pcal.PCAL_EINVAL),       # f_offset >= f_comb
    ((16e6 + 0.5, 1e6, 10e3, 16, pcal.PCAL_F32), pcal.PCAL_EINVAL),  # non-integral Hz
    ((16e6, 1e6, -1.0, 16, pcal.PCAL_F32), pcal.PCAL_EINVAL),
    ((16e6, 3e6, 10e3, 5, pcal.PCAL_F32), pcal.PCAL_EINVAL),       # f_comb does not divide fs
    ((16e6, 1e6, 10e3, 16, 7), pcal.PCAL_EINVAL),                  # unknown format
    ((1024e6, 1e6, 7.0, 1024, pcal.PCAL_I8), pcal.PCAL_ETOOLARGE),  # L = fs / gcd = 1.024e9
    ((16384e6, 1e6, 0.0, 16384, pcal.PCAL_I8), pcal.PCAL_ETOOLARGE),  # N above the cap
])
def test_geometry_errors(lib, args, code):
    with pytest.raises(pcal.PcalError) as ei:
        pcal.pcal_plan_geometry(*args)
    assert ei.value.code == code


def test_strerror(lib):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert pcal.strerror(code) and pcal.strerror(code) != "unknown pcal status"
    assert pcal.strerror(-99) == "unknown pcal status"


def test_plan_create_without_a_device_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pcal.PcalError) as ei:
        pcal.pcal_plan_create(64e6, 1e6, 10e3, 64, pcal.PCAL_2BIT)
    assert ei.value.code in (pcal.PCAL_ECUDA, pcal.PCAL_ENOMEM)


def test_null_arguments_are_rejected(lib):
    assert lib.pcal_accumulate(None, None, 4, None) == pcal.PCAL_EINVAL
    assert lib.pcal_finalize(None, None) == pcal.PCAL_EINVAL
    assert lib.pcal_plan_destroy(None) == pcal.PCAL_OK
    assert lib.pcal_get_bins(None, None) == pcal.PCAL_EINVAL


def test_bitplane_arithmetic_on_host(tmp_path):
    exe = tmp_path / "bitplane_check"
    src = os.path.join(ROOT, "tests", "host", "bitplane_check.cpp")
    inc = os.path.join(ROOT, "paper_2501_05993_gb300", "csrc")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", inc, src, "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("OK")


TILING_CASES = [(fs, fc, fo, fmt) for fmt in (pcal.PCAL_2BIT, pcal.PCAL_I8, pcal.PCAL_F32)
                for fs, fc, fo in [(64e6, 1e6, 10e3), (16e6, 1e6, 10e3), (16, 4, 1), (32e6, 1e6, 5e5),
                                   (1024e6, 1e6, 10e3), (48e6, 1e6, 30e3), (256e6, 1e6, 10e3), (128e6, 1e6, 7e4),
                                   (32e6, 1e6, 0)]]


@pytest.mark.parametrize("fs,fc,fo,fmt", TILING_CASES)
@pytest.mark.parametrize("num_sms", [152, 148, 1])
@pytest.mark.parametrize("n_rows", [1, 17, 5000, 80000, 3_000_000])
def test_bulk_tiling_invariants(lib, fs, fc, fo, fmt, num_sms, n_rows):
    """Host check of every bulk launch's shape: the kernel relies on each of
    these properties (bounds of the TMA boxes and shared memory, the 16-bit
    per-CTA counters, whole 32-row 2-bit blocks, one consumer group per
    pipeline stage, full coverage of the rows)."""
    N = int(fs) // int(fc)
    g = pcal.pcal_plan_geometry(fs, fc, fo, N, fmt)
    try:
        t = pcal.pcal_bulk_tiling(fs, fc, fo, N, fmt, num_sms, n_rows)
    except pcal.PcalError:
        pytest.fail("no tile plan")
    spw = g.samples_per_byte_x4
    assert t.cols_total == g.row_samples // spw
    assert t.col_width % 8 == 0 and 8 <= t.col_width <= 256          # TMA box: <= 256, 32-byte rows
    assert t.col_groups * t.col_width >= t.cols_total > (t.col_groups - 1) * t.col_width
    assert 1 <= t.box_rows <= 256
    if fmt == pcal.PCAL_2BIT:
        assert t.box_rows % 32 == 0                                  # whole add32 blocks
        rows_per_thread = -(-t.max_boxes // t.replicas) * t.box_rows
        assert rows_per_thread // 32 < (1 << t.upper_planes) or t.upper_planes == 0 and rows_per_thread < 32
        assert t.upper_planes <= 11
        ms = (t.col_width + 31) // 32 * 32 + 2
        assert t.replicas * t.col_width * 128 + 128 * ms <= t.stages * ((t.box_rows * t.col_width * 4 + 1023) // 1024 * 1024)
    assert t.stages % t.replicas == 0 and t.stages >= 3             # one consumer group per stage
    assert t.rows_per_cta == t.max_boxes * t.box_rows <= 65535       # 16-bit per-CTA counts
    assert t.total_boxes == -(-n_rows // t.box_rows)
    # every box is taken: static shares, then the counter, within the caps
    assert t.row_groups * t.max_boxes >= t.total_boxes
    assert t.static_boxes <= t.max_boxes and t.row_groups * t.static_boxes <= t.total_boxes
    wpr = (t.col_width + 31) // 32
    assert t.threads == (wpr * t.replicas + 1) * 32 <= 640
    assert t.smem_bytes + 1024 <= 227 * 1024


def test_server_arena_on_host(tmp_path):
    """The serving runtime's HBM arena (first fit, coalescing free blocks)
    against a brute-force per-unit model on random alloc / release sequences."""
    exe = tmp_path / "arena_check"
    src = os.path.join(ROOT, "tests", "host", "arena_check.cpp")
    inc = os.path.join(ROOT, "paper_2501_05993_gb300", "csrc")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", inc, src, "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("OK")


def test_double_float_arithmetic_on_host(tmp_path):
    exe = tmp_path / "df64_check"
    src = os.path.join(ROOT, "tests", "host", "df64_check.cpp")
    inc = os.path.join(ROOT, "paper_2501_05993_gb300", "csrc")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", inc, src, "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("OK")


class _FakeDeviceTensor:
    """The attributes Plan.accumulate reads from a torch CUDA tensor."""

    def __init__(self, numel, esize, cuda=True, contiguous=True):
        self._numel, self._esize, self.is_cuda, self._contig = numel, esize, cuda, contiguous

    def data_ptr(self):
        return 4096

    def numel(self):
        return self._numel

    def element_size(self):
        return self._esize

    def is_contiguous(self):
        return self._contig


def test_device_sample_count_checks_the_tensor():
    count = pcal.device_sample_count
    assert count(_FakeDeviceTensor(100, 1), "2bit", None) == 400
    assert count(_FakeDeviceTensor(100, 1), "2bit", 396) == 396
    assert count(_FakeDeviceTensor(100, 1), "i8", None) == 100
    assert count(_FakeDeviceTensor(100, 4), "f32", None) == 100
    assert count(12345, "f32", 7) == 7  # an address with an explicit count
    bad = [(_FakeDeviceTensor(100, 1), "2bit", 404),           # more than the tensor holds
           (_FakeDeviceTensor(100, 4), "i8", None),            # float32 data for an int8 plan
           (_FakeDeviceTensor(100, 1), "f32", None),           # bytes for a float32 plan
           (_FakeDeviceTensor(100, 1, contiguous=False), "i8", None),
           (_FakeDeviceTensor(100, 1, cuda=False), "i8", None),  # host data
           (12345, "i8", None)]                                  # an address without a count
    for args in bad:
        with pytest.raises(ValueError):
            count(*args)
    import torch
    with pytest.raises(ValueError):
        count(torch.zeros(16, dtype=torch.uint8), "2bit", None)  # a real CPU tensor


def test_dft_and_batch_wrappers_check_tensors():
    """Dft.execute and Batch.accumulate refuse tensors they would misread,
    before any library call (a stand-in object in place of a live handle)."""
    import types

    dft = types.SimpleNamespace(N=64, handle=None)
    good = _FakeDeviceTensor(4 * 64, 8)
    for P, T, C in [(_FakeDeviceTensor(4 * 64, 4), good, 4),          # float32, not complex64
                    (good, _FakeDeviceTensor(4 * 64, 8, cuda=False), 4),
                    (good, _FakeDeviceTensor(4 * 64, 8, contiguous=False), 4),
                    (good, good, 5)]:                                # C x N beyond the tensors
        with pytest.raises(ValueError):
            pcal.Dft.execute(dft, P, C, T)
    batch = types.SimpleNamespace(channels=[(64e6, 1e6, 1e4, "2bit"), (64e6, 1e6, 1e4, pcal.PCAL_I8)])
    pcal.Batch._check_tensors(batch, [_FakeDeviceTensor(100, 1), 12345], [400, 7])   # fine
    for samples, n in [([_FakeDeviceTensor(100, 1), 0], [404, 0]),                  # beyond the 2-bit tensor
                       ([0, _FakeDeviceTensor(100, 4)], [0, 100])]:                  # float32 for an int8 channel
        with pytest.raises(ValueError):
            pcal.Batch._check_tensors(batch, samples, n)


def test_host_sample_count_checks_the_array():
    count = pcal.host_sample_count
    assert count(np.zeros(100, np.uint8), "2bit", None) == 400
    assert count(np.zeros(100, np.int8), "i8", 60) == 60
    assert count(np.zeros(100, np.float32), "f32", None) == 100
    for host, fmt, n in [(np.zeros(100, np.uint8), "2bit", 404),
                         (np.zeros(100, np.float32), "i8", None),
                         (np.zeros(100, np.int8), "f32", None),
                         (np.zeros((10, 20), np.int8)[:, ::2], "i8", None)]:  # not contiguous
        with pytest.raises(ValueError):
            count(host, fmt, n)
    import types

    srv = types.SimpleNamespace(fmts={3: "i8"})
    assert pcal.Server._host_n(srv, 3, np.zeros(10, np.int8), 10) == 10
    assert pcal.Server._host_n(srv, 9, np.zeros(10, np.int8), 99) == 99  # unknown stream: the library decides
    with pytest.raises(ValueError):
        pcal.Server._host_n(srv, 3, np.zeros(10, np.int8), 11)
