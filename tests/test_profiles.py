"""The stored ncu DRAM traffic of the interior kernel (profiles/interior_traffic.json),
which bench.py reports as the roofline's `traffic`, against the kernel sources and
the per-node byte counts.

The capture is keyed by a hash of the interior kernel's sources and compiler flags:
a kernel that changed since the capture would make the bench report no traffic, so
the key must match the sources as committed.  The captured bytes per interior node
must lie between the algorithmic bytes (the 27 distributions and 4 c_i u values
read and written once) less what stays in L2 at kernel end, and the storage layout's
bytes plus the halo re-reads; far above that would mean wasted re-reads.
"""
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _stored():
    with open(os.path.join(ROOT, "profiles", "interior_traffic.json")) as f:
        return json.load(f)


def test_stored_traffic_is_keyed_to_the_current_sources():
    assert _stored()["csrc_sha256"] == bench.kernel_source_hash()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_stored_traffic_per_node_is_near_the_algorithmic_bytes(precision):
    e = _stored()[precision]
    per_node = e["dram_bytes"] / e["interior_nodes"]
    # part of the writes is still in L2 when the kernel ends: a few % below
    assert per_node >= 0.95 * bench.bytes_per_node(precision)
    # halo rows and node classes: within 10% above what the layout moves
    assert per_node <= 1.10 * bench.storage_bytes_per_node(precision)


def test_measured_traffic_scales_with_the_units():
    d = _stored()["fp32"]
    full = bench.measured_traffic("fp32", d["interior_nodes"])
    assert full == d["dram_bytes"]
    assert bench.measured_traffic("fp32", d["interior_nodes"] // 2) == round(d["dram_bytes"] / 2)
    assert bench.measured_traffic("fp8", 10) is None
