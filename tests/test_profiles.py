"""The committed ncu summary of the stage kernel belongs to the current stage-kernel
code (its source hash ignores comments), so the bench line's `traffic` and `issue`
figures, which come from it, describe the kernel that runs."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_stage_profile_matches_the_code():
    text = open(os.path.join(ROOT, "profiles", "stage_kernel_4096x2048.md")).read()
    tile = re.search(r"- tile: `([^`]+)`", text).group(1)
    assert re.search(r"source_sha256: `([0-9a-f]+)`", text).group(1) == bench.stage_source_hash()
    assert bench.profiled(tile, "4096x2048", "dram_bytes_per_launch_avg") > 0
    assert bench.profiled(tile, "4096x2048", "warp_inst_per_launch") > 0


def test_profile_summaries_name_their_commands():
    for f in ("stage_kernel_4096x2048.md", "launches_4096x2048.md", "k_residual64_4096x2048.md"):
        text = open(os.path.join(ROOT, "profiles", f)).read()
        assert "ncu " in text and "--clock-control none" in text and "bench.py" in text, f
