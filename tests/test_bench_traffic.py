"""Host logic of bench.py's roofline traffic on CPU: the DRAM bytes of one ncu
capture are reported only while the captured kernel's code is unchanged, and
the code key ignores comments and blank lines (so documentation edits keep
the capture) but nothing else."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_key_ignores_comments_and_blank_lines_only():
    a = "int f(int x) {\n  return x + 1;   // add one\n}\n"
    b = "// a new header comment\n\nint f(int x) {\n  return x + 1;\n\n}\n"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench.code_sha256(a) == bench.code_sha256(b)
    assert bench.code_sha256(a) != bench.code_sha256(c)


def test_traffic_reported_only_for_the_captured_code(monkeypatch):
    current = bench.kernel_code_sha256()
    monkeypatch.setitem(bench.TRAFFIC_CAPTURE, "code_sha256", current)
    assert bench.traffic_bytes() == bench.TRAFFIC_CAPTURE["bytes_per_launch"]
    assert bench.captured("tensor_pipe_active_pct") == bench.TRAFFIC_CAPTURE["tensor_pipe_active_pct"]
    monkeypatch.setitem(bench.TRAFFIC_CAPTURE, "code_sha256", "0" * 64)
    assert bench.traffic_bytes() is None
    assert bench.captured("tensor_pipe_active_pct") is None


def test_committed_tensor_pipe_share_matches_the_profile_summary():
    """The figure in the bench line is the one the committed ncu summary of the
    same code reports."""
    text = open(os.path.join(ROOT, "profiles", "query_tc16_body_scale_1M.txt")).read()
    assert bench.TRAFFIC_CAPTURE["code_sha256"] in text
    line = [l for l in text.splitlines() if l.strip().startswith("tensor pipe active")][0]
    assert float(line.split()[-2]) == bench.TRAFFIC_CAPTURE["tensor_pipe_active_pct"]


def test_committed_capture_is_plausible_for_the_workload():
    # the capture's bytes are those of one 1M-point launch: at least the
    # algorithmic I/O (49 B per query), and at most what the slope scratch
    # could move (every slope written and read from HBM: 7 layers x 512
    # columns x 2 B x 2 per query) plus that I/O
    n = 1 << 20
    lo = 49 * n
    hi = n * (7 * 512 * 2 * 2 + 49)
    assert lo <= bench.TRAFFIC_CAPTURE["bytes_per_launch"] <= hi
