"""Host-side helpers of bench.py (no GPU): the radix-pass plan it reports,
the kernel-source digest that keys the committed DRAM-traffic figures, and
the lookup of those figures."""
import os
import shutil

import bench


def test_sort_passes_plan():
    # (passes, widest digit of the kernels) for key widths and digit caps
    assert bench.sort_passes(27, 8) == (4, 8)     # 7, 7, 7, 6 bits on the 8-bit kernels
    assert bench.sort_passes(22, 8) == (3, 8)     # 8, 7, 7
    assert bench.sort_passes(18, 8) == (3, 8)     # 6, 6, 6
    assert bench.sort_passes(27, 9) == (3, 9)     # 9, 9, 9
    assert bench.sort_passes(31, 11) == (3, 11)   # 11, 10, 10
    assert bench.sort_passes(1, 8) == (1, 8)
    assert bench.sort_passes(0, 8) == (0, 8)


def _tree(tmp_path, kernels_src, traffic_lines):
    root = tmp_path / "repo"
    (root / "paper_2403_10647_gb300" / "csrc").mkdir(parents=True)
    (root / "profiles").mkdir()
    (root / "paper_2403_10647_gb300" / "csrc" / "kernels.cu").write_text(kernels_src)
    (root / "profiles" / "dram_traffic.txt").write_text("# header\n" + "\n".join(traffic_lines) + "\n")
    return str(root)


def test_digest_ignores_comments_and_whitespace(tmp_path, monkeypatch):
    src = "int f(int a) {\n    return a + 1;   // one more\n}\n"
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path, src, []))
    d0 = bench.kernels_digest()
    p = os.path.join(bench.ROOT, "paper_2403_10647_gb300", "csrc", "kernels.cu")
    with open(p, "w") as f:
        f.write("/* a block\n comment */\nint f(int a)\n{\n  return a + 1; // changed note\n}\n")
    assert bench.kernels_digest() == d0
    with open(p, "w") as f:
        f.write("int f(int a) {\n    return a + 2;\n}\n")
    d1 = bench.kernels_digest()
    assert d1 != d0
    # a launch-shape constant in the kernels' header changes the code too
    h = os.path.join(bench.ROOT, "paper_2403_10647_gb300", "csrc", "kernels.h")
    with open(h, "w") as f:
        f.write("#define BLOCKS 5\n")
    assert bench.kernels_digest() != d1


def test_traffic_lookup_needs_the_current_digest(tmp_path, monkeypatch):
    src = "int g() { return 7; }\n"
    root = _tree(tmp_path, src, [])
    monkeypatch.setattr(bench, "ROOT", root)
    digest = bench.kernels_digest()
    lines = [f"downsweep 8 15.0 {digest}", "downsweep 8 99.0 0000000000000000", f"upsweep 9 4.0 {digest}"]
    with open(os.path.join(root, "profiles", "dram_traffic.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    assert bench.traffic_from_profiles("downsweep", 8, 1000) == 15000.0
    assert bench.traffic_from_profiles("downsweep", 9, 1000) is None      # other digit width
    assert bench.traffic_from_profiles("upsweep", 9, 10) == 40.0
    assert bench.traffic_from_profiles("extract", 8, 10) is None           # no line
    shutil.rmtree(os.path.join(root, "profiles"))
    assert bench.traffic_from_profiles("downsweep", 8, 1000) is None      # no file


def test_committed_traffic_lines_are_well_formed():
    """Every committed line names a kernel, a digit width, bytes per pair and
    a 16-hex-digit digest."""
    path = os.path.join(bench.ROOT, "profiles", "dram_traffic.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert rows
    for r in rows:
        assert len(r) == 4 and r[1].isdigit() and float(r[2]) > 0 and len(r[3]) == 16
        int(r[3], 16)
