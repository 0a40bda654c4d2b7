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


PEAKS = {"hbm_gbs": 6765.0, "bf16_tflops": 1940.0, "bf16_tflops_sustained": 1725.0, "sm_max_mhz": 2070.0}


def test_tf32_roofline_counts_three_products_per_real_product():
    """On the 3xTF32 kernel (kind 4) each real product is three TF32 products: achieved is 3x
    the algorithmic rate against the TF32 peak; other kinds fall back to roofline_of."""
    flops, nbytes, ms, tf32 = 8.0 * 2 ** 36, 4.0 * 2 ** 26, 10.0, 1000.0
    r = bench.roofline_tf32(4, flops, nbytes, ms, tf32, PEAKS)
    assert r["bound"] == "tensor" and r["peak"] == tf32
    assert r["achieved"] == pytest.approx(3 * flops / 1e-2 / 1e12)
    assert r["complex_tflops"] == pytest.approx(flops / 1e-2 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / tf32)
    # low intensity: bound by HBM at the copy rate
    r = bench.roofline_tf32(4, 1e6, 1e9, ms, tf32, PEAKS)
    assert r["bound"] == "hbm" and r["achieved"] == pytest.approx(1e9 / 1e-2 / 1e9)
    assert bench.roofline_tf32(0, flops, nbytes, ms, tf32, PEAKS) == bench.roofline_of(0, flops, nbytes, ms, PEAKS)


def test_alu_roofline_peak_is_the_fp32_lanes():
    r = bench.roofline_of(0, 1e15, 1e9, 1000.0, PEAKS)
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)


@pytest.mark.parametrize("m,k,n", [(2, 24, 2), (4, 16, 16), (14, 12, 10), (12, 12, 12)])
def test_sweep_layouts(m, k, n):
    """Sweep labels: every layout is a permutation of its label set, seeded and repeatable;
    arranged GEPDOT operands lead with the common labels in one order; arranged tensor-core
    operands lead with the K tile labels, C with three tile columns then the tile rows."""
    for layout in ("arranged", "random"):
        la, lb, lc = bench.sweep_labels(m, k, n, layout, seed=5)
        assert (la, lb, lc) == bench.sweep_labels(m, k, n, layout, seed=5)
        ms, ks, ns = set(range(m)), set(range(100, 100 + k)), set(range(200, 200 + n))
        assert sorted(la) == sorted(ms | ks) and sorted(lb) == sorted(ks | ns) and sorted(lc) == sorted(ms | ns)
    la, lb, lc = bench.sweep_labels(m, k, n, "arranged", seed=5)
    if m + n <= 10 and k >= 12:
        assert la[:k] == lb[:k] == list(range(100, 100 + k))
    elif m >= 7 and n >= 6:
        kt = 5 if k >= 5 else 4
        assert la[:kt] == lb[:kt] == list(range(100, 100 + kt))
        assert lc[:3] == [200, 201, 202] and lc[3:10] == list(range(7))


def test_oracle_slice_cuts_need_no_product_library(monkeypatch):
    """The reference arm's slicing comes from the oracle alone: with the product library made
    unloadable, the 30-qubit workload still gets its six cuts, each a (qubit, segment) wire
    label of the oracle's network."""
    from inputs import grid_circuit, subcube_spec
    from paper_2504_09186_gb300 import tnc as T

    monkeypatch.setattr(T, "load_library", lambda *a, **k: (_ for _ in ()).throw(RuntimeError("no library")))
    circ = grid_circuit(5, 6, 14, seed=1)
    fixed, open_q = subcube_spec(30, 10, seed=2)
    cuts = bench.oracle_slice_cuts(circ, fixed, open_q, 6, 23)
    assert len(cuts) == 6 and len(set(cuts)) == 6
    assert all(0 <= q < 30 and j >= 0 for q, j in cuts)
