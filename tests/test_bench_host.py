"""bench.py's host-side helpers without a GPU: the nvidia-smi clock record it
attaches to every line, and the rule that roofline.traffic is reported only
while the kernel source still matches the one the ncu summary was taken on."""
import os
import shutil

import pytest

import bench

ROW = "0, {sm}, 2070, 900.5, 0x{mask}, {hw}, {hwt}, {swt}, {pcap}"


def test_clock_record_median_max_and_reasons():
    rows = [ROW.format(sm=2070, mask="0", hw="Not Active", hwt="Not Active", swt="Not Active", pcap="Not Active"),
            ROW.format(sm=1980, mask="4", hw="Not Active", hwt="Not Active", swt="Not Active", pcap="Active"),
            "garbage line",
            "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active",
            ROW.format(sm=2055, mask="0", hw="Not Active", hwt="Not Active", swt="Not Active", pcap="Not Active")]
    r = bench.ClockSampler.parse("\n".join(rows))
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2055 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_record_flags_slowdowns():
    rows = [ROW.format(sm=1500, mask="8", hw="Active", hwt="Not Active", swt="Active", pcap="Not Active")]
    r = bench.ClockSampler.parse("\n".join(rows))
    assert r["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler.parse("")["sm_mhz"] is None


@pytest.mark.parametrize("name", ["fold2bit_c2_dram.txt", "fold_f32_c1_dram.txt"])
def test_traffic_only_while_the_source_matches(tmp_path, monkeypatch, name):
    """A summary stamped with the kernel source's sha256 yields its DRAM bytes; any change to the source
    withdraws them (the committed summary is checked against the committed source the same way)."""
    import hashlib

    summary = open(os.path.join(bench.ROOT, "profiles", name)).read()
    recorded = int(summary.split("dram_bytes_per_launch=")[1].split()[0])
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(bench.ROOT, "profiles"), root / "profiles")
    csrc = root / "paper_2501_05993_gb300" / "csrc"
    csrc.mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "paper_2501_05993_gb300", "csrc", "fold_bulk.cu"), csrc / "fold_bulk.cu")
    sha = hashlib.sha256((csrc / "fold_bulk.cu").read_bytes()).hexdigest()
    lines = [f"source_sha256={sha}" if l.startswith("source_sha256=") else l for l in summary.splitlines()]
    (root / "profiles" / name).write_text("\n".join(lines) + "\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.read_traffic("fold_bulk.cu", name) == recorded  # same source: the recorded figure
    with open(csrc / "fold_bulk.cu", "a") as f:
        f.write("\n// changed\n")
    assert bench.read_traffic("fold_bulk.cu", name) is None


def test_clock_sampler_stop_reads_and_removes_its_file(tmp_path):
    class FakeProc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    path = tmp_path / "clocks.csv"
    path.write_text(ROW.format(sm=2070, mask="0", hw="Not Active", hwt="Not Active", swt="Not Active",
                               pcap="Not Active") + "\n")
    s = bench.ClockSampler(0)
    s.proc, s.path = FakeProc(), str(path)
    r = s.stop()
    assert r["sm_mhz"] == 2070 and r["reasons"] == [] and r["samples"] == 1
    assert not path.exists()
