"""The pair schedule on the CPU: tests/native/schedule_check.cu compiles the
library's own run builder and item decoding (csrc/hk_sched.cuh) for the host
and checks, for block counts 1..130 and several larger ones, batches of
uneven sets sharing a launch, and slot caps from 1 to unlimited, that every
pair of blocks is visited exactly once, that blocks and slots stay in range,
and that no slot is written twice in a phase (the invariants the pair
kernels' one-writer slots rest on)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))


def test_pair_schedule_invariants():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "schedule_check")
        subprocess.run([nvcc, "-std=c++17", "-O1", "-x", "cu",
                        "-I" + os.path.join(ROOT, "paper_2010_02994_gb300", "csrc"), "-I" + os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "native", "schedule_check.cu"), "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
