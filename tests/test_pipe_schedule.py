"""The pipelined middle passes' dispenser order, checked on the host.

The kernel's CTAs only ever wait for items handed out before their own, so
the order must (i) hand out every (kind, plane, tile) item exactly once and
(ii) put each plane's row-forward items before its middle items and those
before its row-inverse items.  tests/pipe_schedule_check.cu compiles the
kernel header's own make_pipe_sched / pipe_decode for the host and checks
both over 405 schedule shapes (up to 16448 planes).
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_pipe_dispenser_order(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "pipe_schedule_check")
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include"),
                        os.path.join(HERE, "pipe_schedule_check.cu"), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "cases 405 bad 0"
