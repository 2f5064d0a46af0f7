"""The committed ncu summaries stay tied to the kernel source they measured: the bench
reads the fine-level sweep's DRAM traffic from `profiles/k_jacobi_tp_ecs_1024.md` only
while the recorded source hash matches, so a kernel change without a new capture shows
up here instead of as a silent null in the bench line."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_source_hash_is_stable_hex():
    h = bench.kernel_source_sha()
    assert re.fullmatch(r"[0-9a-f]{16}", h)
    assert bench.kernel_source_sha() == h


def test_jacobi_profile_matches_current_kernel_source():
    traffic = bench.profiled_traffic("k_jacobi", "tp_ecs_1024")
    assert traffic is not None, "profiles/k_jacobi_tp_ecs_1024.md records another source hash"
    # three compulsory complex128 arrays of the 1023^2 interior, within a few percent
    assert 0.9 * 3 * 16 * 1023 ** 2 <= traffic <= 1.1 * 4 * 16 * 1023 ** 2


def test_every_profile_names_its_command():
    for name in sorted(os.listdir(os.path.join(ROOT, "profiles"))):
        text = open(os.path.join(ROOT, "profiles", name)).read()
        assert "ncu " in text and "--clock-control none" in text, name
        assert "python bench.py" in text, name
