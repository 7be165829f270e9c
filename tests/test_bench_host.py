"""Host-side logic of bench.py (CPU only): the unit conversion of the
metric, the clock-sample summary that decides whether a run is kept, and
the lookup of the pair kernel's measured DRAM traffic, which must be
withheld once the kernel source differs from the captured one."""
import hashlib
import os

import pytest

import bench


def test_walker_ns_per_day():
    # 16 walkers x 200 steps of 1 fs in 0.0864 s: 3.2 walker-ns per 86.4 ms
    assert bench.walker_ns_per_day(16, 200, 0.001, 0.0864) == pytest.approx(3200.0, rel=1e-12)


def test_clock_summary(tmp_path):
    p = tmp_path / "clocks.csv"
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "1, 1200, 2070, 300.0, 0x0, Active, Not Active, Not Active, Not Active",  # another GPU
        "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    p.write_text("\n".join(rows) + "\n")
    s = bench.ClockSampler(str(p)).summary(0)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    s1 = bench.ClockSampler(str(p)).summary(1)
    assert s1["reasons"] == ["hw_slowdown"] and s1["sm_mhz"] == 1200.0
    assert bench.ClockSampler(str(tmp_path / "none.csv")).summary()["reasons"] == ["unavailable"]


def _fake_tree(root, k_pairs_src):
    csrc = root / "paper_2307_08006_gb300" / "csrc"
    csrc.mkdir(parents=True)
    srcs = {"k_pairs.cu": k_pairs_src, "labf_internal.cuh": b"struct Dev {};", "labf_dyn.cuh": b"// dyn"}
    for name, body in srcs.items():
        (csrc / name).write_bytes(body)
    h = hashlib.sha256()
    for name in ("k_pairs.cu", "labf_internal.cuh", "labf_dyn.cuh"):
        h.update(srcs[name])
    return h.hexdigest()[:16]


def test_measured_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    sha = _fake_tree(tmp_path, b"__global__ void k_pairs() {}")
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k_pairs_solvation16.md").write_text(
        "summary\n"
        f"traffic_bytes_per_launch: variant=0 form=fused dram_bytes=50877440 source_sha256={sha}\n"
        f"traffic_bytes_per_launch: variant=0 form=single dram_bytes=49861727 source_sha256={sha}\n"
        f"traffic_bytes_per_launch: variant=3 form=single dram_bytes=49878420 source_sha256={sha}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic(0)[0] == 50877440  # the fused capture first
    assert bench.measured_traffic(3)[0] == 49878420  # else the variant's one-task capture
    assert bench.measured_traffic(4) == (None, "no capture of pair_variant=4")
    # any change to the kernel source withholds the number
    (tmp_path / "paper_2307_08006_gb300" / "csrc" / "k_pairs.cu").write_bytes(b"__global__ void k_pairs() {;}")
    assert bench.measured_traffic(0) == (None, "kernel source changed since the capture")
    os.remove(tmp_path / "profiles" / "k_pairs_solvation16.md")
    assert bench.measured_traffic(0) == (None, "no capture")


def test_workload_name_carries_the_list_parameters():
    w = bench.workload_name(0.2, 0.075)
    assert "list skin 0.2 nm" in w and "pruning margin 0.075 nm" in w and "12300 atoms" in w
    assert bench.workload_name() == bench.workload_name(bench.SKIN_NM, bench.PRUNE_NM)
