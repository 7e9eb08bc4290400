"""Host-side pieces of bench.py that need no GPU: the kernel-source hash that
ties a committed ncu summary to the source it was taken on, and the reading of
that summary's DRAM traffic (none unless the hashes match)."""
import os

import bench


def test_kernel_hash_ignores_comments_and_blank_lines(tmp_path, monkeypatch):
    src = tmp_path / "paper_2512_23037_gb300" / "csrc"
    src.mkdir(parents=True)
    names = ("kernels.cu", "kernels.cuh", "program.h", "device_common.cuh", "lanes.cu", "shot_common.cuh")
    for n in names:
        (src / n).write_text("int a = 1;  // one\n\n// a comment line\nint b = 2;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h1 = bench.kernel_hash()
    assert len(h1) == 16 and int(h1, 16) >= 0
    for n in names:  # other comments and blank lines: the same code
        (src / n).write_text("  int a = 1;  // another comment\nint b = 2;\n\n")
    assert bench.kernel_hash() == h1
    (src / "lanes.cu").write_text("int a = 1;\nint b = 3;\n")  # one changed token
    assert bench.kernel_hash() != h1


def test_profile_traffic_only_for_the_matching_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "lane_kernel_x.md").write_text("# x\n\nkernel_source_sha256: 0123456789abcdef\n\ndram_bytes_per_shot: 75.5\n")
    (prof / "shot_kernel_x.md").write_text("kernel_source_sha256: 0123456789abcdef\ndram_bytes_per_launch_full: 1.5e9\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("0123456789abcdef", "lane_kernel_x.md", 1000) == 75.5 * 1000
    assert bench.profile_traffic("0123456789abcdef", "shot_kernel_x.md", 1000) == 1.5e9
    assert bench.profile_traffic("fedcba9876543210", "lane_kernel_x.md", 1000) is None
    assert bench.profile_traffic("0123456789abcdef", "missing.md", 1000) is None


def test_committed_profiles_name_a_source_hash():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for n in ("lane_kernel_w42.md", "lane_kernel_w97.md"):
        txt = open(os.path.join(root, "profiles", n)).read()
        assert "kernel_source_sha256:" in txt and "dram_bytes_per_shot:" in txt, n
