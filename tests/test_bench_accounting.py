"""The bench's byte accounting and its ncu traffic table, on the CPU: the
algorithmic bytes per species-site update are 2 Q b (each population read
once and written once), plus the node density read and written by half
storage; and the ncu traffic entries are keyed to the step kernel sources
they were captured from, so that a changed kernel reports no traffic rather
than stale counters."""
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


def test_traffic_entries_are_plausible_and_keyed_to_kernel_sources():
    """Every captured traffic entry is within 10 % of the algorithmic bytes of
    its workload (the 256^3 box, or the batched sweep: 2 Q b per
    species-site update of every tube), and the lookup the bench makes gives
    nothing for sources that were not captured (a changed kernel reports
    traffic null)."""
    assert bench.NCU_TRAFFIC
    for (digest, workload, size, prec), t in bench.NCU_TRAFFIC.items():
        assert len(digest) == 16 and workload in ("stratification", "tubes")
        if workload == "stratification":
            algorithmic = bench.bytes_per_ssu(W.stratification_3d(n=8), prec) * 3 * size ** 3
        else:
            per = bench.bytes_per_ssu(W.loschmidt_binary(nx=4, ny=16), prec)   # D2Q9: 2 x 9 x b
            algorithmic = sum(ns * 32 * L * per for L, ns in (W.tube_length_and_species(k) for k in range(size)))
        assert 0.9 < t / algorithmic < 1.1, (digest, workload, prec, t / algorithmic)
    assert bench.traffic_for("0" * 16, "stratification", 256, "fp32") is None
    assert len(bench.kernel_digest()) == 16
    assert len(bench.kernel_digest(bench.BATCH_SOURCES)) == 16


def test_tube_shapes_match_the_sweep():
    """The shape helper draws the same lengths and species counts as the sweep."""
    tubes = W.batched_tubes(count=12)
    for k, t in enumerate(tubes):
        assert W.tube_length_and_species(k) == (t.shape[1], t.ns)
