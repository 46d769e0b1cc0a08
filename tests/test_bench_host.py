"""Host-side pieces of the benchmark that need no GPU: the clock summary, the committed ncu
traffic figure, and the algorithmic-bytes model of the roofline."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import pytest  # noqa: E402

import bench  # noqa: E402
from paper_2012_13133_gb300 import inputs as I  # noqa: E402


def test_clock_summary_reads_median_max_and_active_reasons():
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "0, 2070, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, [N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]\n",
        "garbage\n",
    ]
    c = bench.ClockSampler.summarise(lines)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 4
    hot = bench.ClockSampler.summarise(["0, 1500, 2070, 1400, 0x8, Active, Active, Not Active, Not Active\n"])
    assert hot["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    assert bench.ClockSampler.summarise([]) is None


def test_committed_ncu_traffic_matches_the_current_kernel_sources():
    """The ncu summary carries the hash of the kernel sources it was taken on; the bench reports
    its traffic only while that hash matches (null otherwise, until the profile is retaken)."""
    t = bench.read_traffic()
    if t is None:
        pytest.skip("the committed ncu summary was taken on other kernel sources")
    w = I.WORKLOADS["grid1024"]
    model = bench.model_bytes_per_vector(w.n1, w.n2, 2 * w.n1, 2 * w.n2, 524288)
    lam = 4.0 * (2 * w.n1) * (2 * w.n2)
    for nv, b in t:
        # the measured DRAM bytes stay within 25% of the model (no wholesale re-reads)
        assert nv >= 1 and 0.75 * (model * nv + lam) <= b <= 1.25 * (model * nv + lam), (nv, b)
    # the traffic at a captured width is the captured value, and it grows with the width
    assert bench.traffic_at(t, t[0][0]) == pytest.approx(t[0][1])
    assert bench.traffic_at(t, t[-1][0]) == pytest.approx(t[-1][1])
    assert bench.traffic_at(t, 2 * t[-1][0]) > t[-1][1]


def test_traffic_interpolation_between_two_batch_widths():
    pts = [(4, 180.0), (64, 2480.0)]
    assert bench.traffic_at(pts, 4) == 180.0 and bench.traffic_at(pts, 64) == 2480.0
    # a launch mix of 4- and 64-vector launches: the mean traffic is the line at the mean width
    mix = [4] * 9 + [64]
    mean_nv = sum(mix) / len(mix)
    assert bench.traffic_at(pts, mean_nv) == pytest.approx(sum(bench.traffic_at(pts, v) for v in mix) / len(mix))
    assert bench.traffic_at([(64, 2560.0)], 32) == 1280.0


def test_model_bytes_per_vector_of_the_grid1024_matvec():
    # slab written once and read/written/read by the three passes (16 n1 M2) plus 16 p for the
    # vector read, nugget re-read, output write and index lists: 33.6 + 8.4 MB
    assert bench.model_bytes_per_vector(1024, 1024, 2048, 2048, 524288) == 16 * 1024 * 2048 + 16 * 524288
