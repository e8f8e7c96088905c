"""bench.py's roofline inputs on the host: the DRAM traffic it reports is read from
the committed ncu summaries under profiles/, and those files agree with each other."""
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PROFILES = os.path.join(ROOT, "profiles")


def test_traffic_file_has_the_bench_keys():
    t = bench.read_traffic(os.path.join(PROFILES, "ncu_traffic.txt"))
    for key in ("k_smooth_level0 traffic_bytes_per_launch", "k_smooth_level0 cold_ms_per_launch",
                "step traffic_bytes_per_step"):
        assert key in t and t[key] is not None and t[key] > 0, key
    assert bench.read_traffic(os.path.join(PROFILES, "no_such_file.txt")) == {}


def test_smooth_traffic_is_the_mean_of_the_summarised_launches():
    t = bench.read_traffic(os.path.join(PROFILES, "ncu_traffic.txt"))
    md = open(os.path.join(PROFILES, "k_smooth_level0_heat1024.md")).read()
    rows = re.findall(r"^\| (\d+) \| (\d+) \| (\d+) \| (\d+) \|$", md, flags=re.M)
    assert len(rows) == 2, rows
    traffic = sum(int(r[1]) + int(r[2]) for r in rows) / len(rows)
    cold_ms = sum(int(r[3]) for r in rows) / len(rows) * 1e-6
    assert t["k_smooth_level0 traffic_bytes_per_launch"] == pytest.approx(traffic, abs=1.0)
    assert t["k_smooth_level0 cold_ms_per_launch"] == pytest.approx(cold_ms, rel=1e-9)


def test_step_traffic_matches_the_launch_list_total():
    t = bench.read_traffic(os.path.join(PROFILES, "ncu_traffic.txt"))
    md = open(os.path.join(PROFILES, "step_traffic_heat1024_radau5_LD_f32amg.md")).read()
    m = re.search(r"^\| \*\*total\*\* \| (\d+) \| [\d.]+ \| 100% \| ([\d.]+) \|$", md, flags=re.M)
    assert m, "total row"
    assert t["step traffic_bytes_per_step"] / 1e9 == pytest.approx(float(m.group(2)), abs=0.006)
    head = re.search(r"\*\*DRAM traffic per step: ([\d.]+) GB\*\*", md)
    assert head and float(head.group(1)) == pytest.approx(float(m.group(2)), abs=0.006)
