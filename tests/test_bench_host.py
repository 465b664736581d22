"""Host-side logic of bench.py (no GPU): the valid-DOF count behind the metric against the
oracle's valid regions, the source-hash gate on the stored ncu traffic figures, and the
parsing of the clock samples that decides whether a run was throttled."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle.hierarchy import Hierarchy as OH  # noqa: E402
from paper_2506_02663_gb300 import workloads as wl  # noqa: E402


def test_valid_dof_matches_oracle_valid_regions():
    """DOF = valid cells of every level (Eq. validRegion): level-0 cells minus the coarsened
    fine box, plus every fine cell."""
    for name in ("bumps2d", "bumps3d"):
        dim, n0, boxes = wl.hierarchy_boxes(name)
        H = OH(dim, n0, boxes, bc=[0] * (2 * dim))
        want = int(sum(int(np.sum(lev.valid)) for lev in H.levels))
        assert bench.valid_dof(n0, boxes) == want, name


def test_traffic_figure_only_for_matching_sources(tmp_path, monkeypatch):
    """A stored DRAM figure is reported only while the hash of the kernel's own source files
    (the entry's ``sources``) matches the one recorded at capture time."""
    os.makedirs(tmp_path / "profiles")
    h = bench._kernel_source_hash(("sweep3d.cuh",))
    json.dump({"a_w": {"dram_bytes_per_launch": 123.0, "sources": ["sweep3d.cuh"], "source_hash": h},
               "b_w": {"dram_bytes_per_launch": 456.0, "sources": ["sweep3d.cuh"], "source_hash": "0" * 16}},
              open(tmp_path / "profiles" / "traffic.json", "w"))
    real = bench._kernel_source_hash
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda files=None: h if tuple(files) == ("sweep3d.cuh",) else real(files))
    assert bench._traffic("a_w") == 123.0
    assert bench._traffic("b_w") is None   # taken on other kernel sources
    assert bench._traffic("c_w") is None   # not captured


def test_clock_samples_parsed_with_throttle_reasons(tmp_path):
    """Median SM clock under load, the maximum, and every throttle reason seen Active."""
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")

    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s = bench.ClockSampler(0)
    s.proc = _Proc()
    s.fh = open(path, "a")
    s.path = str(path)
    out = s.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
