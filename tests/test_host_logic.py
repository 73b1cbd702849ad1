"""Host-side logic of the library, compiled for the CPU (no GPU needed).

The fixed-point unit 2^-s of the consumption sums (kp::mass_shift) must keep
every entry's mass at most 2^30 units (one 32-bit conversion per entry) and
every per-knapsack sum below 2^62, and be the largest such s up to 40.
"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("host") / "mass_shift_probe")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CUDA_INC, os.path.join(HERE, "host", "mass_shift_probe.cpp"),
                    "-o", exe], check=True, capture_output=True)
    return exe


def _shifts(exe, pairs):
    text = "".join(f"{c!r} {m!r}\n" for c, m in pairs)
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
    return [int(v) for v in out.split()]


def test_mass_shift_bounds_and_maximality(probe):
    counts = [1.0, 20.0, 1e6, 2e9, 1e12]
    maxbs = [np.float32(v) for v in (1e-30, 2.0 ** -41, 1e-6, 2.0 ** -10, 0.37, 1.0, 3.0, 1e6, 1e20)]
    pairs = [(c, float(m)) for c in counts for m in maxbs]
    for (c, m), s in zip(pairs, _shifts(probe, pairs)):
        assert -120 <= s <= 40
        if s > -120:
            assert m * 2.0 ** s <= 2.0 ** 30, (c, m, s)
            assert (c * m + 1) * 2.0 ** s <= 2.0 ** 62, (c, m, s)
        if -120 < s < 40:  # one more bit breaks one of the two bounds the shift keeps
            assert m * 2.0 ** (s + 1) > 2.0 ** 30 or (c * m + 1) * 2.0 ** (s + 1) > 2.0 ** 62, (c, m, s)


def test_mass_shift_unit_scale_instance(probe):
    # b ~ U[0,1] with 2e9 entries (the 1e8-user workload): 30 bits per entry
    (s,) = _shifts(probe, [(2e9, float(np.float32(0.99999994)))])
    assert s == 30
    assert 2e9 * 2.0 ** 30 < 2.0 ** 62
    assert math.isclose(2.0 ** -s, 2.0 ** -30)
