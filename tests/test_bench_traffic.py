"""The benchmark reports the DRAM traffic of the kernel it timed from a table of ncu captures;
the table covers every launch configuration the autotuner can pick on the two workloads it is
read for (the headline pipe, both schemes, and the larger-than-L2 aneurysm, twist)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2101_11107_gb300 import lbm  # noqa: E402

NAMES = lbm.LAUNCH_CONFIG_NAMES
# configurations the autotuner times: every one for the FP32 twist, the one-cell ones for A-B
TWIST = NAMES
AB = [n for n in NAMES if not n.startswith("2c") and not n.startswith("pipe")]


def test_headline_pipe_has_a_capture_for_every_choice():
    for scheme, names in (("esoteric", TWIST), ("ab", AB)):
        for name in names:
            assert ("womersley", "fp32", scheme, name) in bench.K_STEP_TRAFFIC, (scheme, name)


def test_larger_than_l2_anchor_has_a_capture_for_every_choice():
    for name in TWIST:
        assert ("aneurysm512", "fp32", "esoteric", name) in bench.K_STEP_TRAFFIC, name


def test_traffic_entries_are_plausible():
    for key, (traffic, kernel) in bench.K_STEP_TRAFFIC.items():
        assert isinstance(traffic, int) and traffic > 0, key
        assert kernel.startswith("k_step"), key
        workload, storage, scheme, name = key
        assert name in NAMES and scheme in ("esoteric", "ab") and storage == "fp32", key
