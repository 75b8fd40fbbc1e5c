"""Host scheduling rules of the persistent tensor-core launch, checked on the CPU:
the tail split's part count is allowed and optimal (brute force), and the
overlapped download's column bands cover every tile once, keep mirrored
column tiles together and end at wave boundaries (tests/sched_check.cpp,
compiled against the library's own scheduling header)."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_schedule_rules():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "sched_check")
        subprocess.run(["g++", "-std=c++17", "-O1", "-o", exe, os.path.join(HERE, "sched_check.cpp")], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
