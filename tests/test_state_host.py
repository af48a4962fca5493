"""Host-side checks of the saved serving-state file format (no GPU): a bit-exact round trip
and rejection of corrupted, truncated, padded, foreign and missing files, compiled from the
library's own header with the host C++ compiler."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2504_13445_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "native", "state_io_check.cpp")


def test_state_file_format(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "state_io_check")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-I", CSRC, SRC, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe, str(tmp_path)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
