"""Host-side checks of bench.py's bookkeeping (no GPU): DRAM traffic is reported only for the
kernel instantiation and fiber count it was captured on, every profiled scope the bench reads
exists in the library's list, and every traffic figure has its ncu summary in profiles/."""
import json
import os

import bench
from paper_1912_11494_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_only_for_the_captured_instantiation_and_size():
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    n = t["fibers"]
    assert n == 4_145_000  # the bench workload
    assert bench.traffic_for("k_exact_blocks", "gemm_bf16", n) == t["k_exact_blocks@gemm_bf16"]
    assert bench.traffic_for("k_gemm_screen", "gemm_bf16", n) == t["k_gemm_screen@gemm_bf16"]
    assert bench.traffic_for("k_label_plain", "plain", n) == t["k_label_plain"]
    assert bench.traffic_for("k_fused", "culled_fused", n) == t["k_fused@culled_fused"]
    # other template instantiations and other sizes were not captured
    assert bench.traffic_for("k_gemm_screen", "gemm_inv_tf32", n) is None
    assert bench.traffic_for("k_exact_blocks", "gemm_tf32", n) is None
    assert bench.traffic_for("k_label_plain", "plain", 1_000_000) is None


def test_traffic_is_marked_with_its_capture_size():
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert t["captured_fibers"] == 1_000_000
    assert "extrapolated" in bench.traffic_source() and "1,000,000" in bench.traffic_source()


def test_profiled_scopes_exist_in_the_library():
    for slot in bench.LAUNCH_SLOTS:
        assert slot in binding.PROFILED_KERNELS
        assert bench.KERNELS_PER_SLOT[slot] >= 1
    for slot in bench.KERNEL_NAME:
        assert slot in bench.LAUNCH_SLOTS


def test_every_traffic_figure_has_its_ncu_summary():
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    texts = [open(os.path.join(ROOT, "profiles", f)).read()
             for f in os.listdir(os.path.join(ROOT, "profiles")) if f.endswith(".md")]
    for key in t:
        if key.startswith("_") or key in ("fibers", "captured_fibers"):
            continue
        kernel = key.split("@")[0]
        assert any(kernel in x and "dram__bytes_read.sum" in x for x in texts), key
