"""CPU checks of the benchmark's roofline bookkeeping (no GPU, nothing launched).

The DRAM traffic that bench.py reports for the pivoted-QR panel kernel comes from an
ncu capture of one kernel revision at one bond dimension; it must be reported only
for that revision and size, and be null otherwise."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_panel_capture_describes_the_committed_kernel():
    """The committed capture (profiles/qr_panel_kernel_chi4096.md) was taken on the
    panel kernel as it is in csrc/qr.cu."""
    import hashlib

    sha = hashlib.sha256(bench.panel_kernel_source().encode()).hexdigest()
    assert sha == bench.PANEL_NCU["kernel_sha256"]
    r = bench.PANEL_NCU["dram_over_algorithmic"]
    assert 0 < r <= 1.0
    assert bench.panel_traffic(1e10, bench.PANEL_NCU["chi"]) == r * 1e10


def test_panel_traffic_is_null_for_another_size_or_source(monkeypatch):
    assert bench.panel_traffic(1e10, 2048) is None
    src = bench.panel_kernel_source()
    monkeypatch.setattr(bench, "panel_kernel_source", lambda: src + "// changed\n")
    assert bench.panel_traffic(1e10, bench.PANEL_NCU["chi"]) is None
