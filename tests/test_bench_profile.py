"""The benchmark's link to its committed profile (host logic, no GPU).

The benchmark reports the graph kernel's DRAM traffic from the committed ncu
summary only while the query path's code is the code that was captured: the
summary records a hash of the sources, taken without their comments and with
white space collapsed, so an edited comment keeps the figure and an edited
statement drops it."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_comments_are_removed_and_strings_kept():
    src = 'int a = 1; // one\n/* two\n lines */ const char *s = "x // y /* z */";\n'
    out = bench.strip_comments(src)
    assert "one" not in out and "two" not in out and "lines" not in out
    assert '"x // y /* z */"' in out
    assert "int a = 1;" in out and "const char *s =" in out


def test_hash_ignores_comments_only(tmp_path, monkeypatch):
    f = tmp_path / "k.cuh"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "QUERY_SOURCES", ["k.cuh"])
    f.write_text("int f(int x) { return x + 1; }  // add one\n")
    h0 = bench.kernel_source_hash()
    f.write_text("// a new comment\nint f(int x) { return x + 1; }  /* add one */\n")
    assert bench.kernel_source_hash() == h0
    f.write_text("int f(int x) { return x + 2; }\n")
    assert bench.kernel_source_hash() != h0


def test_profile_traffic_only_for_the_captured_sources(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "query_kernel_label_1m.md").write_text(
        "source_hash: 0123456789abcdef (...)\ntraffic_bytes_per_full_launch: 1228405456\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("0123456789abcdef") == 1228405456.0
    assert bench.profile_traffic("fedcba9876543210") is None
