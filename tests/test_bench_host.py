"""Host-side pieces of bench.py: the DRAM-traffic lookup behind the roofline's `traffic`
field, and the roofline classification.  No GPU."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _profile(tmp_root, kind, fpi, dram, src_rel, sha):
    os.makedirs(os.path.join(tmp_root, "profiles"), exist_ok=True)
    with open(os.path.join(tmp_root, "profiles", "k_test.md"), "w") as f:
        f.write("# test\n\n```\n"
                f"traffic_kind: {kind}\ntraffic_flops_per_instance: {fpi}\n"
                f"traffic_dram_bytes_per_instance: {dram}\ntraffic_kernel_source: {src_rel}\n"
                f"traffic_kernel_source_sha1: {sha}\n```\n")


def test_traffic_lookup_scales_a_matching_capture(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("// kernel source\n")
    sha = hashlib.sha1(src.read_bytes()).hexdigest()
    _profile(str(tmp_path), 5, 1000, 370, "kernel.cu", sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic(5, 64 * 1000) == 64 * 370      # 64 instances of the capture
    assert bench.measured_traffic(4, 64 * 1000) is None          # another kernel kind
    assert bench.measured_traffic(5, 1500) is None               # not a whole number of instances
    src.write_text("// kernel source, changed\n")                 # the kernel changed since
    assert bench.measured_traffic(5, 64 * 1000) is None


def test_committed_traffic_capture_matches_the_current_kernel_source():
    """The committed capture of the dominant kernel is the current source's: its traffic per
    64-instance launch of the 30-qubit workload is about 1.04 x the algorithmic bytes."""
    flops = 64 * 8 * 2 ** 36
    traffic = bench.measured_traffic(5, flops)
    assert traffic is not None
    algorithmic = 64 * (2 ** 26 + 2 ** 22 + 2 ** 24) * 4
    assert 1.0 <= traffic / algorithmic <= 1.1


@pytest.mark.parametrize("kind,flops,nbytes,bound", [(5, 1e12, 1e9, "tensor"), (5, 1e9, 1e9, "hbm"),
                                                     (0, 1e12, 1e9, "alu"), (7, 1e9, 1e9, "hbm")])
def test_roofline_bound_follows_intensity_and_kernel_class(kind, flops, nbytes, bound):
    peaks = {"hbm_gbs": 6788.3, "bf16_tflops": 1912.1, "bf16_tflops_sustained": 1717.8, "sm_max_mhz": 2070.0,
             "_source": "test"}
    r = bench.roofline_of(kind, flops, nbytes, 1.0, peaks)
    assert r["bound"] == bound
    assert r["frac"] > 0
