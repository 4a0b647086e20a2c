"""Host-side logic of bench.py's roofline: the algorithmic bytes per hop and
the gate that reports measured walk traffic only for the sources it was
measured on.  CPU only."""
import numpy as np
import pytest

import bench
import workloads as W


def test_committed_walk_profiles_match_the_walk_sources():
    # the bench line carries `traffic` only while profiles/k_walk_<workload>.md
    # was taken on the walk sources as they are; a kernel change without a new
    # capture would silently drop it from the line
    for tag in ("grid3d27pt_128cube", "grid3d7pt_64cube"):
        per_hop, path = bench._walk_traffic_per_hop(tag)
        assert per_hop is not None and per_hop > 0.0, tag
        assert path.startswith("profiles")


def test_walk_traffic_gate_rejects_other_sources(monkeypatch):
    # a different source set hashes to another digest: no traffic is reported
    monkeypatch.setattr(bench, "WALK_SOURCES", bench.WALK_SOURCES + ["bench.py"])
    assert bench._walk_traffic_per_hop("grid3d27pt_128cube") == (None, None)
    assert bench._walk_traffic_per_hop("no_such_workload") == (None, None)


def test_walk_bytes_per_hop_closed_forms():
    # header + ceil(4 (deg + 1) / 32) threshold sectors + one successor sector:
    # every node of degree <= 7 needs one threshold sector, so 5- and 7-point
    # grids give exactly 3 x 32 B whatever the weights
    rng = np.random.default_rng(0)
    # (a weighted mean: equal up to its rounding)
    assert bench.walk_bytes_per_hop(W.grid2d_5pt(9, 7)) == pytest.approx(96.0, rel=1e-12)
    assert bench.walk_bytes_per_hop(W.grid3d(6, 5, 4, 7, rng, excess_frac_hi=1e-3)) == pytest.approx(96.0, rel=1e-12)
    # 27-point: interior nodes (degree 26) need four threshold sectors, 192 B;
    # boundary nodes fewer, so the stationary mean lies below 192 and rises
    # toward it with the grid size
    small = bench.walk_bytes_per_hop(W.grid3d(6, 6, 6, 27, rng, excess_frac=1e-4))
    large = bench.walk_bytes_per_hop(W.grid3d(16, 16, 16, 27, rng, excess_frac=1e-4))
    assert 96.0 < small < large < 192.0
