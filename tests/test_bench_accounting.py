"""The bench's byte accounting and its ncu traffic table, on the CPU: the
algorithmic bytes per species-site update are 2 Q b (each population read
once and written once), plus the node density read and written by half
storage; and the default workload's traffic entry belongs to the current step
kernel sources, so that a kernel change without a new capture is noticed
here rather than reported with stale counters."""
import sys
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2504_07059_gb300 import workloads as W  # noqa: E402


def test_algorithmic_bytes_per_update():
    d3 = W.stratification_3d(n=8)
    d2 = W.loschmidt_ternary_gravity(nx=4, ny=16)
    assert bench.bytes_per_ssu(d3, "fp32") == 152
    assert bench.bytes_per_ssu(d3, "fp64") == 304
    assert bench.bytes_per_ssu(d3, "fp16") == 80
    assert bench.bytes_per_ssu(d2, "fp32") == 72
    assert bench.bytes_per_ssu(d2, "fp16") == 40


def test_traffic_entry_matches_the_current_kernel_sources():
    digest = bench.kernel_digest()
    for prec in ("fp32", "fp16"):
        t = bench.NCU_TRAFFIC.get((digest, "stratification", 256, prec))
        assert t is not None, (digest, prec)
        algorithmic = bench.bytes_per_ssu(W.stratification_3d(n=8), prec) * 3 * 256 ** 3
        assert 0.9 < t / algorithmic < 1.1   # within 10 % of the algorithmic bytes
