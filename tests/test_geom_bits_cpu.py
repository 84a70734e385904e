"""The bit-field FP64 helpers of the tensor-core element set-up, run on the
host (the same source, compiled by nvcc for the CPU) against exact rational
arithmetic and numpy's FP64 -> FP32 rounding:

  split_f64_bits(x)  x as hi + lo to 2^-47 of |x|, flagged outside
                     [2^-60, 2^60) (0 excepted)
  f64_to_f32_bits(x) FP64 -> FP32 rounded to nearest even, bit for bit
                     (normal, overflow, subnormal, zero, NaN)
"""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("geom_bits") / "geom_bits")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"), "-I",
                    os.path.join(ROOT, "paper_1310_1194_gb300", "csrc"), os.path.join(ROOT, "tests", "geom_bits_host.cu"),
                    "-o", exe], check=True, capture_output=True)

    def run(mode, xs, ys=None):
        ys = np.zeros_like(xs) if ys is None else ys
        lines = "".join(f"{mode} {int(a):x} {int(b):x}\n" for a, b in zip(np.asarray(xs, np.float64).view(np.uint64),
                                                                          np.asarray(ys, np.float64).view(np.uint64)))
        out = subprocess.run([exe], input=lines, capture_output=True, text=True, check=True).stdout.split()
        a = np.array(out, dtype=object).reshape(-1, 3)
        ok = a[:, 0].astype(int).astype(bool)
        hi = np.array([int(v, 16) for v in a[:, 1]], dtype=np.uint32).view(np.float32)
        lo = np.array([int(v, 16) for v in a[:, 2]], dtype=np.uint32).view(np.float32)
        return ok, hi, lo
    return run


def test_split_f64_bits_against_exact_values(harness):
    rng = np.random.default_rng(11)
    x = rng.uniform(-1, 1, 3000) * 10.0 ** rng.integers(-25, 25, 3000)
    x = np.concatenate([x, [0.0, -0.0, 2.0 ** -60, 2.0 ** 60, -(2.0 ** 60) * (1 - 2 ** -53), 1e-300]])
    ok, hi, lo = harness(1, x)
    for i in range(len(x)):
        v = Fraction(float(x[i]))
        in_range = v == 0 or Fraction(2) ** -60 <= abs(v) < Fraction(2) ** 60
        assert ok[i] == in_range, x[i]
        if in_range:
            got = Fraction(float(hi[i])) + Fraction(float(lo[i]))
            assert abs(got - v) <= abs(v) * Fraction(1, 2 ** 47), x[i]


def test_f64_to_f32_bits_rounds_like_numpy(harness):
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, 3000) * 10.0 ** rng.integers(-50, 50, 3000)
    # halfway cases (ties to even), the largest finite values, overflow, subnormals
    f = np.float32(1.5).view(np.uint32)
    ties = [float(np.uint32(f + k).view(np.float32)) + 2.0 ** -24 for k in range(4)]
    edge = [3.4028234663852886e38, 3.4028235677973366e38, 3.5e38, -3.5e38, 1e-39, -1e-45, 1.1754943508222875e-38,
            0.0, -0.0, 1e300]
    # subnormal FP32 results across the whole range, with halfway cases
    sub = rng.uniform(0, 1.2e-38, 2000) * rng.choice([-1, 1], 2000)
    tiny = np.array([2.0 ** -149, 2.0 ** -150, 3 * 2.0 ** -151, 2.0 ** -151, 1.5 * 2.0 ** -149, 2.5 * 2.0 ** -149,
                     (1 - 2.0 ** -25) * 2.0 ** -126, -(2.0 ** -126) * (1 - 2.0 ** -24), 1e-320, -1e-300])
    x = np.concatenate([x, ties, edge, sub, tiny])
    ok, got, _ = harness(2, x)
    with np.errstate(over="ignore", under="ignore"):
        want = x.astype(np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    # NaN stays NaN
    ok, got, _ = harness(2, np.array([np.nan, -np.inf, np.inf]))
    assert np.isnan(got[0]) and got[1] == -np.inf and got[2] == np.inf
