"""Host-side check of the integer-pipe FP32 <-> FP64 conversions that the
mixed-precision stage-2 update uses (csrc/fpsplit.cuh): the same header,
compiled for the CPU, must give the compiler's own conversions bit for bit
(every float for widen; boundaries, rounding ties and carries and random
encodings for split).  The GPU parity tests cover the device build."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2507_20461_gb300", "csrc")


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_conversions_match_hardware_rounding(tmp_path):
    exe = str(tmp_path / "fpsplit_check")
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "fpsplit_check.cpp"), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
