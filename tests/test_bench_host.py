"""CPU checks of bench.py's host-side rules (no GPU).

* The DRAM traffic reported with the roofline comes from the committed ncu
  record only while that record's kernel hash matches the hop sources; a
  change to either source file makes it null.
* The job's value is the slowest rank's time over the solves of all ranks.
* The workload description names the benchmark lattice and tolerance.
"""
import json
import os
import shutil

import pytest

import bench


def test_traffic_record_matches_current_kernel_sources():
    rec = bench.ncu_traffic()
    if rec is None:
        pytest.skip("profiles/hop_traffic.json was taken on other kernel sources: the bench reports null")
    assert rec["kernel_hash"] == bench.kernel_hash()
    per_kind = rec["f32_bytes_per_kind"]
    assert abs(sum(per_kind) / len(per_kind) - rec["f32_bytes_per_launch"]) <= 1


def test_traffic_is_dropped_when_the_kernel_changes(tmp_path, monkeypatch):
    # a copy of the repository's kernel sources and record, then one byte more
    root = tmp_path
    for rel in bench.KERNEL_SOURCES + ["profiles/hop_traffic.json"]:
        dst = root / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, rel), dst)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.ncu_traffic() is not None
    with open(root / bench.KERNEL_SOURCES[0], "a") as f:
        f.write("\n")
    assert bench.ncu_traffic() is None
    # and a record written for the new sources is taken again
    rec = json.load(open(root / "profiles/hop_traffic.json"))
    rec["kernel_hash"] = bench.kernel_hash()
    json.dump(rec, open(root / "profiles/hop_traffic.json", "w"))
    assert bench.ncu_traffic() is not None


@pytest.mark.parametrize("ws,steps", [(1, 5), (2, 3), (8, 10)])
def test_whole_job_value(ws, steps):
    assert bench.whole_job_value(3.0, steps, ws) == pytest.approx(3.0 / (steps * ws))
    assert bench.max_over_ranks(2.5, 1, "cpu") == 2.5


def test_workload_description():
    d = bench.workload_desc("f32")
    assert "16x16x16x32" in d and "Ls=16" in d and "1e-10" in d and "f32 inner" in d
