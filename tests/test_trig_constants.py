"""Compile-time twiddle constants of the composite FFT butterflies (trig::cos2pi/sin2pi in
tf_fft.cuh), built into a host program with nvcc and compared with the mathematical
values cos(2 pi m / R), sin(2 pi m / R) computed to 30 digits (mpmath) -- no GPU needed."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_twiddle_constants_match_the_circle(tmp_path):
    mpmath = pytest.importorskip("mpmath")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "trig_table"
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-o", str(exe),
                    os.path.join(HERE, "c_abi", "trig_table.cu")], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    mpmath.mp.dps = 30
    rows = [line.split() for line in out.splitlines()]
    assert len(rows) == 3 + 5 + 7 + 8 + 14 + 16 + 20 + 25 + 28 + 32 + 49 + 64
    worst = 0.0
    for R, m, c, s in rows:
        R, m = int(R), int(m)
        ang = 2 * mpmath.pi * m / R
        worst = max(worst, abs(float(c) - float(mpmath.cos(ang))),
                    abs(float(s) - float(mpmath.sin(ang))))
    assert worst <= 2.5e-16, worst
